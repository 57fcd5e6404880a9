// Accuracy of the library's double-float arithmetic (tt_df.cuh) against FP64
// on seeded random inputs: sin/cos over several periods, the reciprocal, and
// the Kerr flow and Hamiltonian against the FP64 flow of the same state, and
// the logarithm of the tabulated metric's radial coordinate.
// Prints one line per quantity: name, max error, error measure.  H is a sum of
// terms that cancel, so its error is measured against the size of those terms.
#include <cmath>
#include <cstdio>
#include <vector>

#include "tt_df.cuh"

using namespace tt;

__global__ void k_accuracy(int n, const double* in, double* out) {
    df_sincos_table(s_df_tab);
    df_log_table(s_df_ln);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* p = in + 8 * i;
    const double a = p[0], r = p[1], th = p[2], pr = p[3], pth = p[4], pt = p[5], pph = p[6], x = p[7];
    const KerrK k = make_kerr(1.0, a);
    const RayConst R = make_ray_const(a, pt, pph);
    const State y{r, th, pr, pth};
    State f;
    double H;
    kerr_flow64(k, R, y, f, H);
    const StateDF yd{df_of(r), df_of(th), df_of(pr), df_of(pth)};
    StateDF fd;
    DF Hd;
    kerr_flow_df(make_kerr_df(k), make_ray_df(R), yd, fd, Hd);
    DF s, c;
    df_sincos(df_of(th), s, c);
    double* o = out + 20 * i;
    o[0] = f.r;   o[1] = df_to64(fd.r);
    o[2] = f.th;  o[3] = df_to64(fd.th);
    o[4] = f.pr;  o[5] = df_to64(fd.pr);
    o[6] = f.pth; o[7] = df_to64(fd.pth);
    o[8] = H;     o[9] = df_to64(Hd);
    o[10] = sin(th); o[11] = df_to64(s);
    o[12] = cos(th); o[13] = df_to64(c);
    o[14] = 1.0 / x; o[15] = df_to64(df_rcp(df_of(x)));
    o[16] = log(x);  o[17] = df_to64(df_log(df_of(x)));
    // the terms of 2 Sigma H: Delta pr^2, pth^2, (pph + a sin^2 pt)^2 / sin^2, ((r^2 + a^2) pt + a pph)^2 / Delta
    const double sn = sin(th), cs = cos(th), s2 = sn * sn;
    const double Sig = r * r + a * a * cs * cs, Del = r * r - 2.0 * r + a * a;
    const double t3 = (pph + a * s2 * pt), t4 = (r * r + a * a) * pt + a * pph;
    o[18] = (Del * pr * pr + pth * pth + t3 * t3 / s2 + t4 * t4 / fabs(Del)) / (2.0 * Sig);
}

int main() {
    const int n = 8192;
    std::vector<double> in(8 * n), out(20 * n);
    unsigned long long st = 2609;
    auto rnd = [&]() {
        st = st * 6364136223846793005ULL + 1442695040888963407ULL;
        return (double)(st >> 11) / 9007199254740992.0;
    };
    for (int i = 0; i < n; ++i) {
        double* p = &in[8 * i];
        p[0] = (i % 4 == 0) ? 0.0 : 0.998 * (2 * rnd() - 1);
        const double rp = 1.0 + std::sqrt(1.0 - p[0] * p[0]);
        p[1] = (i % 3 == 0) ? 500 + 600 * rnd() : rp * (1.01 + 20 * rnd());   // outside the horizon
        p[2] = (i % 5 == 0) ? -4.0 + 12.0 * rnd() : 0.02 + 3.1 * rnd();     // some beyond (0, pi)
        p[3] = 2 * rnd() - 1;
        p[4] = 10 * (2 * rnd() - 1);
        p[5] = 1.0;
        p[6] = 10 * (2 * rnd() - 1);
        p[7] = std::ldexp(0.5 + rnd(), (int)(60 * rnd()) - 30);
    }
    double *din = nullptr, *dout = nullptr;
    if (cudaMalloc(&din, in.size() * 8) != cudaSuccess || cudaMalloc(&dout, out.size() * 8) != cudaSuccess) {
        std::printf("alloc failed\n");
        return 1;
    }
    cudaMemcpy(din, in.data(), in.size() * 8, cudaMemcpyHostToDevice);
    k_accuracy<<<(n + 127) / 128, 128>>>(n, din, dout);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::printf("cuda error %s\n", cudaGetErrorString(e));
        return 1;
    }
    cudaMemcpy(out.data(), dout, out.size() * 8, cudaMemcpyDeviceToHost);
    cudaFree(din);
    cudaFree(dout);
    // relative error for the flow components and the reciprocal, absolute for
    // sin, cos and log, and for H relative to the size of its terms
    const char* names[] = {"flow_r", "flow_th", "flow_pr", "flow_pth", "H", "sin", "cos", "rcp", "log"};
    for (int q = 0; q < 9; ++q) {
        double worst = 0.0;
        for (int i = 0; i < n; ++i) {
            const double a = out[20 * i + 2 * q], b = out[20 * i + 2 * q + 1];
            double d = std::fabs(a - b);
            if (q < 4 || q == 7) d /= std::fabs(a) + 1e-300;
            if (q == 4) d /= out[20 * i + 18];
            if (d > worst) worst = d;
        }
        std::printf("%s %.6e %s\n", names[q], worst, (q == 4) ? "rel_terms" : (q < 4 || q == 7) ? "rel" : "abs");
    }
    return 0;
}

// Accuracy of the library's double-float arithmetic (tt_df.cuh) against FP64
// on seeded random inputs: sin/cos over several periods, the reciprocal, and
// the Kerr flow and Hamiltonian against the FP64 flow of the same state, and
// the logarithm of the tabulated metric's radial coordinate and its patches.
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

// The tabulated-metric patches: double-float against FP64 at the same points,
// on a random coefficient table (8 x 6 cells).  Per point: the 15 FP64 values,
// the 15 double-float ones and the scale of each (the sum of its terms' sizes).
__global__ void k_table(int n, const double* pts, ImageDesc d, double* out) {
    df_log_table(s_df_ln);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = pts[2 * i], th = pts[2 * i + 1];
    double f[5], fr[5], ft[5];
    table_fields64(d, r, th, f, fr, ft);
    DF g[5], gr[5], gt[5];
    table_fields_df(d, df_of(r), df_of(th), g, gr, gt);
    // the cell and unit coordinates (as table_fields64 takes them)
    const double tu = (log(r) - d.u0) / d.du, tw = th / d.dth;
    const int k = min(max((int)floor(tu), 0), d.nr - 2), j = min(max((int)floor(tw), 0), d.nth - 2);
    const double t = fabs(tu - k), w = fabs(tw - j);
    const double* c = d.table + ((size_t)j * (d.nr - 1) + k) * kTableCoef;
    double* o = out + 45 * i;
    for (int fi = 0; fi < 5; ++fi) {
        double sv = 0.0, st = 0.0, sw = 0.0;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                const double m = fabs(c[16 * fi + 4 * a + b]);
                sv += m * pow(t, a) * pow(w, b);
                st += m * a * pow(t, a > 0 ? a - 1 : 0) * pow(w, b);
                sw += m * b * pow(t, a) * pow(w, b > 0 ? b - 1 : 0);
            }
        const double* q[3] = {f, fr, ft};
        const DF* qd[3] = {g, gr, gt};
        const double sc[3] = {sv, st / (d.du * r), sw / d.dth};
        for (int m = 0; m < 3; ++m) {
            o[15 * 0 + 3 * fi + m] = q[m][fi];
            o[15 * 1 + 3 * fi + m] = df_to64(qd[m][fi]);
            o[15 * 2 + 3 * fi + m] = sc[m];
        }
    }
}

static float2 split2(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
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

    // tabulated metric: 9 x 7 nodes, r in [1.5, 50], random coefficients of
    // magnitude up to 10^fi for field fi; points inside and just outside
    const int nr = 9, nth = 7, nt = 4096;
    const size_t ncoef = (size_t)(nr - 1) * (nth - 1) * kTableCoef;
    std::vector<double> cf(ncoef);
    std::vector<float2> cdf(ncoef);
    for (size_t q = 0; q < ncoef; ++q) {
        const int fi = (int)((q % kTableCoef) / 16);
        cf[q] = (2 * rnd() - 1) * std::pow(10.0, fi);
        cdf[q] = split2(cf[q]);
    }
    std::vector<double> pts(2 * nt), tout(45 * nt);
    for (int q = 0; q < nt; ++q) {
        pts[2 * q] = 1.45 * std::pow(55.0 / 1.45, rnd());
        pts[2 * q + 1] = -0.1 + (M_PI + 0.2) * rnd();
    }
    ImageDesc d{};
    d.nr = nr;
    d.nth = nth;
    d.u0 = std::log(1.5);
    d.du = (std::log(50.0) - d.u0) / (nr - 1);
    d.dth = M_PI / (nth - 1);
    d.u0_df = split2(d.u0);
    d.idu_df = split2(1.0 / d.du);
    d.idth_df = split2(1.0 / d.dth);
    double *dc = nullptr, *dp = nullptr, *dto = nullptr;
    float2* dcd = nullptr;
    if (cudaMalloc(&dc, ncoef * 8) != cudaSuccess || cudaMalloc(&dcd, ncoef * 8) != cudaSuccess ||
        cudaMalloc(&dp, pts.size() * 8) != cudaSuccess || cudaMalloc(&dto, tout.size() * 8) != cudaSuccess) {
        std::printf("alloc failed\n");
        return 1;
    }
    cudaMemcpy(dc, cf.data(), ncoef * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dcd, cdf.data(), ncoef * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(dp, pts.data(), pts.size() * 8, cudaMemcpyHostToDevice);
    d.table = dc;
    d.table_df = dcd;
    k_table<<<(nt + 127) / 128, 128>>>(nt, dp, d, dto);
    const cudaError_t e2 = cudaDeviceSynchronize();
    if (e2 != cudaSuccess) {
        std::printf("cuda error %s\n", cudaGetErrorString(e2));
        return 1;
    }
    cudaMemcpy(tout.data(), dto, tout.size() * 8, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dcd);
    cudaFree(dp);
    cudaFree(dto);
    const char* tnames[3] = {"table_value", "table_dr", "table_dth"};
    for (int m = 0; m < 3; ++m) {
        double worst = 0.0;
        for (int q = 0; q < nt; ++q)
            for (int fi = 0; fi < 5; ++fi) {
                const double* o = &tout[45 * q];
                const double dd = std::fabs(o[3 * fi + m] - o[15 + 3 * fi + m]) / o[30 + 3 * fi + m];
                if (dd > worst) worst = dd;
            }
        std::printf("%s %.6e rel_terms\n", tnames[m], worst);
    }
    return 0;
}

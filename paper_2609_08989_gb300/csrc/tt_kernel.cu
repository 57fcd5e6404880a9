// tt_kernel.cu -- persistent ray-tracing kernel (sm_103a).
//
// One ray per thread, warps pull rays from a shared queue (one atomicAdd per
// warp refill).  A lane whose ray terminates writes its outputs and goes idle;
// idle lanes are refilled together once enough of the warp is idle, so the
// warp keeps stepping full instead of idling behind its slowest ray.  Every
// loop is bounded: a lane takes at most max_steps steps per ray and each warp
// iteration either steps a ray or consumes queue entries, so no thread waits
// on another.
#include <cstdint>
#include <cuda_runtime.h>

#include "tt_device.cuh"
#include "tt_internal.h"

namespace tt {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// One Dormand-Prince step in FP64 (paper Sec. 3.2): returns the fifth-order
// point yn, its flow kn (first-same-as-last) and H there, and the error vector.
// ---------------------------------------------------------------------------
template <int METRIC>
__device__ __forceinline__ void dp5_step64(const ImageDesc& d, double M, double a, const RayConst& R,
                                           const State& y, const State& k1, double h, State& yn,
                                           State& kn, double& Hn, State& err) {
    using namespace dp;
    State k2, k3, k4, k5, k6, ys;
    double Hs;
#define TT_STAGE(dst, expr_r, expr_t, expr_p, expr_q)                                \
    ys.r = fma(h, (expr_r), y.r);                                                    \
    ys.th = fma(h, (expr_t), y.th);                                                  \
    ys.pr = fma(h, (expr_p), y.pr);                                                  \
    ys.pth = fma(h, (expr_q), y.pth);                                                \
    flow64<METRIC>(d, M, a, R, ys, dst, Hs);
#define TT_C2(f) (a21 * k1.f)
#define TT_C3(f) fma(a32, k2.f, a31 * k1.f)
#define TT_C4(f) fma(a43, k3.f, fma(a42, k2.f, a41 * k1.f))
#define TT_C5(f) fma(a54, k4.f, fma(a53, k3.f, fma(a52, k2.f, a51 * k1.f)))
#define TT_C6(f) fma(a65, k5.f, fma(a64, k4.f, fma(a63, k3.f, fma(a62, k2.f, a61 * k1.f))))
#define TT_C7(f) fma(b6, k6.f, fma(b5, k5.f, fma(b4, k4.f, fma(b3, k3.f, b1 * k1.f))))
    TT_STAGE(k2, TT_C2(r), TT_C2(th), TT_C2(pr), TT_C2(pth))
    TT_STAGE(k3, TT_C3(r), TT_C3(th), TT_C3(pr), TT_C3(pth))
    TT_STAGE(k4, TT_C4(r), TT_C4(th), TT_C4(pr), TT_C4(pth))
    TT_STAGE(k5, TT_C5(r), TT_C5(th), TT_C5(pr), TT_C5(pth))
    TT_STAGE(k6, TT_C6(r), TT_C6(th), TT_C6(pr), TT_C6(pth))
    yn.r = fma(h, TT_C7(r), y.r);
    yn.th = fma(h, TT_C7(th), y.th);
    yn.pr = fma(h, TT_C7(pr), y.pr);
    yn.pth = fma(h, TT_C7(pth), y.pth);
    flow64<METRIC>(d, M, a, R, yn, kn, Hn);
#define TT_E(f) h * fma(e7, kn.f, fma(e6, k6.f, fma(e5, k5.f, fma(e4, k4.f, fma(e3, k3.f, e1 * k1.f)))))
    err.r = TT_E(r);
    err.th = TT_E(th);
    err.pr = TT_E(pr);
    err.pth = TT_E(pth);
#undef TT_E
#undef TT_STAGE
#undef TT_C2
#undef TT_C3
#undef TT_C4
#undef TT_C5
#undef TT_C6
#undef TT_C7
}

__device__ __forceinline__ double sq_ratio(double e, double y, double yn, double atol, double rtol) {
    double sc = fma(rtol, fmax(fabs(y), fabs(yn)), atol);
    double q = e / sc;
    return q * q;
}

// Mean-square error norm over (r, theta, p_r, p_theta).
__device__ __forceinline__ double err_norm2(const State& y, const State& yn, const State& e,
                                            double atol, double rtol) {
    double s = sq_ratio(e.r, y.r, yn.r, atol, rtol);
    s += sq_ratio(e.th, y.th, yn.th, atol, rtol);
    s += sq_ratio(e.pr, y.pr, yn.pr, atol, rtol);
    s += sq_ratio(e.pth, y.pth, yn.pth, atol, rtol);
    return 0.25 * s;
}

// ---------------------------------------------------------------------------
// Crossing refinement.
// Henon's exact step: integrate dz/dtheta = f / (dtheta/dlambda) for
// z = (r, p_r, p_th) from the start of the accepted step to theta = pi/2 with
// Dormand-Prince in 2^m equal sub-steps, m = 0..6, taking the first m whose
// largest sub-step error norm (over r, p_r, p_th) is <= 1.
// ---------------------------------------------------------------------------
template <int METRIC>
__device__ __forceinline__ void theta_flow64(const ImageDesc& d, double M, double a, const RayConst& R,
                                             const State& y, State& g) {
    State f;
    double H;
    flow64<METRIC>(d, M, a, R, y, f, H);
    double it = rcp64(f.th);
    g.r = f.r * it;
    g.th = 1.0;
    g.pr = f.pr * it;
    g.pth = f.pth * it;
}

template <int METRIC>
__device__ double refine_henon64(const ImageDesc& d, double M, double a, const RayConst& R,
                                 const State& y0, const State& f0, double atol, double rtol) {
    using namespace dp;
    const double dth_all = kHalfPi - y0.th;
    const double it0 = rcp64(f0.th);
    State g0;
    g0.r = f0.r * it0;
    g0.pr = f0.pr * it0;
    g0.pth = f0.pth * it0;
    double r_out = y0.r;
    for (int m = 0; m <= 6; ++m) {
        const int nsub = 1 << m;
        const double dl = dth_all / (double)nsub;
        State z = y0, g = g0;
        double worst = 0.0;
        for (int q = 0; q < nsub; ++q) {
            State k2, k3, k4, k5, k6, k7, zs;
            const double th0 = z.th;
#define TT_HS(dst, cc, er, ep, eq)                        \
    zs.r = fma(dl, (er), z.r);                            \
    zs.pr = fma(dl, (ep), z.pr);                          \
    zs.pth = fma(dl, (eq), z.pth);                        \
    zs.th = fma(dl, (cc), th0);                           \
    theta_flow64<METRIC>(d, M, a, R, zs, dst);
#define TT_C2(f) (a21 * g.f)
#define TT_C3(f) fma(a32, k2.f, a31 * g.f)
#define TT_C4(f) fma(a43, k3.f, fma(a42, k2.f, a41 * g.f))
#define TT_C5(f) fma(a54, k4.f, fma(a53, k3.f, fma(a52, k2.f, a51 * g.f)))
#define TT_C6(f) fma(a65, k5.f, fma(a64, k4.f, fma(a63, k3.f, fma(a62, k2.f, a61 * g.f))))
#define TT_C7(f) fma(b6, k6.f, fma(b5, k5.f, fma(b4, k4.f, fma(b3, k3.f, b1 * g.f))))
            TT_HS(k2, c2, TT_C2(r), TT_C2(pr), TT_C2(pth))
            TT_HS(k3, c3, TT_C3(r), TT_C3(pr), TT_C3(pth))
            TT_HS(k4, c4, TT_C4(r), TT_C4(pr), TT_C4(pth))
            TT_HS(k5, c5, TT_C5(r), TT_C5(pr), TT_C5(pth))
            TT_HS(k6, 1.0, TT_C6(r), TT_C6(pr), TT_C6(pth))
            State zn;
            zn.r = fma(dl, TT_C7(r), z.r);
            zn.pr = fma(dl, TT_C7(pr), z.pr);
            zn.pth = fma(dl, TT_C7(pth), z.pth);
            zn.th = th0 + dl;
            theta_flow64<METRIC>(d, M, a, R, zn, k7);
#define TT_E(f) dl * fma(e7, k7.f, fma(e6, k6.f, fma(e5, k5.f, fma(e4, k4.f, fma(e3, k3.f, e1 * g.f)))))
            double s = sq_ratio(TT_E(r), z.r, zn.r, atol, rtol);
            s += sq_ratio(TT_E(pr), z.pr, zn.pr, atol, rtol);
            s += sq_ratio(TT_E(pth), z.pth, zn.pth, atol, rtol);
#undef TT_E
#undef TT_HS
#undef TT_C2
#undef TT_C3
#undef TT_C4
#undef TT_C5
#undef TT_C6
#undef TT_C7
            s *= (1.0 / 3.0);
            if (!(s <= worst)) worst = s;
            z = zn;
            g = k7;
        }
        r_out = z.r;
        if (worst <= 1.0) break;
    }
    return r_out;
}

// Paper's method (Sec. 3.2): bisection of theta(lambda) - pi/2 on the cubic-
// Hermite interpolant of the accepted step, to 1e-12 in lambda.
__device__ double refine_hermite64(const State& y0, const State& f0, const State& y1,
                                   const State& f1, double h) {
    double lo = 0.0, hi = 1.0;
    const bool s0 = y0.th <= kHalfPi;
    for (int it = 0; it < 200 && (hi - lo) * h > 1e-12; ++it) {
        double mid = 0.5 * (lo + hi);
        double B[4], dB[4];
        hermite4(mid, B, dB);
        double th = B[0] * y0.th + B[1] * h * f0.th + B[2] * y1.th + B[3] * h * f1.th;
        if ((th <= kHalfPi) == s0) lo = mid;
        else hi = mid;
    }
    double sc = 0.5 * (lo + hi);
    double B[4], dB[4];
    hermite4(sc, B, dB);
    return B[0] * y0.r + B[1] * h * f0.r + B[2] * y1.r + B[3] * h * f1.r;
}

// Hairer-Norsett-Wanner starting step (embedded order 4), four-component norm.
template <int METRIC>
__device__ double initial_step64(const ImageDesc& d, double M, double a, const RayConst& R,
                                 const State& y0, const State& f0, double atol, double rtol) {
    double sr = fma(rtol, fabs(y0.r), atol), st = fma(rtol, fabs(y0.th), atol);
    double sp = fma(rtol, fabs(y0.pr), atol), sq = fma(rtol, fabs(y0.pth), atol);
    double d0 = sqrt(0.25 * ((y0.r / sr) * (y0.r / sr) + (y0.th / st) * (y0.th / st) +
                             (y0.pr / sp) * (y0.pr / sp) + (y0.pth / sq) * (y0.pth / sq)));
    double d1 = sqrt(0.25 * ((f0.r / sr) * (f0.r / sr) + (f0.th / st) * (f0.th / st) +
                             (f0.pr / sp) * (f0.pr / sp) + (f0.pth / sq) * (f0.pth / sq)));
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
    State y1, f1;
    y1.r = y0.r + h0 * f0.r;
    y1.th = y0.th + h0 * f0.th;
    y1.pr = y0.pr + h0 * f0.pr;
    y1.pth = y0.pth + h0 * f0.pth;
    double H1;
    flow64<METRIC>(d, M, a, R, y1, f1, H1);
    double q0 = (f1.r - f0.r) / sr, q1 = (f1.th - f0.th) / st;
    double q2 = (f1.pr - f0.pr) / sp, q3 = (f1.pth - f0.pth) / sq;
    double d2 = sqrt(0.25 * (q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3)) / h0;
    double dm = fmax(d1, d2);
    double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 0.2);
    return fmin(100.0 * h0, h1);
}

// ---------------------------------------------------------------------------
// Per-lane ray record.
// ---------------------------------------------------------------------------
struct Lane {
    const ImageDesc* d;
    long long q;            // output index within the image
    State y, k1;            // state and its flow (first-same-as-last)
    RayConst R;
    double M, a;
    double h, lam, hmax, inten;
    int steps, rejects, ncross, nrec;
    bool last_rej;
};

__device__ __forceinline__ void write_final(const Lane& L, int code) {
    const ImageDesc& d = *L.d;
    const long long q = L.q, n = d.pix_count;
    d.code[q] = (int8_t)code;
    d.n_cross[q] = (int8_t)min(L.ncross, 127);
    d.intensity[q] = L.inten;
    d.h_max[q] = L.hmax;
    d.steps[q] = L.steps;
    d.rejects[q] = L.rejects;
    for (int k = L.nrec; k < kMaxCross; ++k) {
        d.r_cross[k * n + q] = 0.0;
        d.g[k * n + q] = 0.0;
        d.I_cross[k * n + q] = 0.0;
    }
}

// Initial data from the ZAMO tetrad (paper Sec. 2.2), time-reversed. Returns
// false (and writes a BADPIXEL record) if the pixel is outside the sky.
template <int METRIC>
__device__ bool init_ray(Lane& L, const ImageDesc* d_ptr, long long q, const SolverDesc& sol) {
    const ImageDesc& d = *d_ptr;
    L.d = d_ptr;
    L.q = q;
    L.M = d.M;
    L.a = d.a;
    L.steps = 0;
    L.rejects = 0;
    L.ncross = 0;
    L.nrec = 0;
    L.inten = 0.0;
    L.hmax = 0.0;
    L.lam = 0.0;
    L.last_rej = false;
    const long long p = d.pix_begin + q;
    const long long i = p % d.nx, j = p / d.nx;
    const double alpha = d.alpha_min + ((double)i + 0.5) * d.dalpha;
    const double beta = d.beta_min + ((double)j + 0.5) * d.dbeta;
    const double D = d.r_obs, th = d.theta_obs;
    const double rho2 = alpha * alpha + beta * beta;
    if (!isfinite(alpha) || !isfinite(beta) || !(rho2 < D * D)) {
        write_final(L, 5);
        return false;
    }
    double g[5];
    lower64<METRIC>(d, D, th, g);
    const double gtt = g[0], gtp = g[1], grr = g[2], gthth = g[3], gpp = g[4];
    const double omega = -gtp / gpp;
    const double N = sqrt(-gtt + omega * omega * gpp);
    const double pl_r = sqrt(1.0 - rho2 / (D * D));
    const double pu_t = 1.0 / N;
    const double pu_r = pl_r / sqrt(grr);
    const double pu_th = (beta / D) / sqrt(gthth);
    const double pu_ph = omega / N + (-alpha / D) / sqrt(gpp);
    const double p_t = gtt * pu_t + gtp * pu_ph;
    const double p_r = grr * pu_r;
    const double p_th = gthth * pu_th;
    const double p_ph = gtp * pu_t + gpp * pu_ph;
    L.y.r = D;
    L.y.th = th;
    L.y.pr = -p_r;
    L.y.pth = -p_th;
    L.R = make_ray_const(d.a, -p_t, -p_ph);
    double H0;
    flow64<METRIC>(d, L.M, L.a, L.R, L.y, L.k1, H0);
    L.hmax = fabs(H0);
    L.h = (sol.h0 > 0.0) ? sol.h0 : initial_step64<METRIC>(d, L.M, L.a, L.R, L.y, L.k1, sol.atol, sol.rtol);
    return true;
}

// One step attempt; returns the termination code or -1 if the ray continues.
template <int METRIC>
__device__ int step_ray64(Lane& L, const SolverDesc& sol) {
    const ImageDesc& d = *L.d;
    if ((long long)L.steps + (long long)L.rejects >= sol.max_steps) return 2;
    const double hmin = (sol.h_min > 0.0) ? sol.h_min : 1e-14 * fmax(1.0, fabs(L.lam));
    if (L.h < hmin) return 3;
    State yn, kn, e;
    double Hn;
    dp5_step64<METRIC>(d, L.M, L.a, L.R, L.y, L.k1, L.h, yn, kn, Hn, e);
    const double err2 = err_norm2(L.y, yn, e, sol.atol, sol.rtol);
    if (isnan(err2) || !isfinite(yn.r) || !isfinite(yn.th) || !isfinite(yn.pr) || !isfinite(yn.pth))
        return 4;
    if (err2 <= 1.0) {
        L.steps++;
        if (d.disk && ((L.y.th <= kHalfPi) != (yn.th <= kHalfPi))) {
            const double rc = (sol.refine == 1)
                                  ? refine_hermite64(L.y, L.k1, yn, kn, L.h)
                                  : refine_henon64<METRIC>(d, L.M, L.a, L.R, L.y, L.k1, sol.atol, sol.rtol);
            if (rc >= d.r_in && rc <= d.r_out) {
                if (L.nrec < d.max_cross) {
                    const double gf = redshift64<METRIC>(d, rc, L.R.pt, L.R.pph);
                    const double F = flux64(d, rc);
                    const double g2 = gf * gf;
                    const double I = g2 * g2 * F;
                    const long long n = d.pix_count, q = L.q;
                    d.r_cross[L.nrec * n + q] = rc;
                    d.g[L.nrec * n + q] = gf;
                    d.I_cross[L.nrec * n + q] = I;
                    L.inten += I;
                    L.nrec++;
                }
                L.ncross++;
            }
        }
        L.lam += L.h;
        L.y = yn;
        L.k1 = kn;
        L.hmax = fmax(L.hmax, fabs(Hn));
        if (yn.r < d.r_capture) return 1;
        if (yn.r > d.r_escape) return 0;
        double fac = (err2 == 0.0) ? 10.0 : 0.9 * pow(err2, -0.1);
        fac = fmin(L.last_rej ? 1.0 : 10.0, fmax(0.2, fac));
        L.h *= fac;
        L.last_rej = false;
    } else {
        L.rejects++;
        L.h *= fmax(0.2, 0.9 * pow(err2, -0.1));
        L.last_rej = true;
    }
    return -1;
}

__device__ __forceinline__ int find_image(const ImageDesc* descs, int n, long long rid) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (descs[mid].ray_begin <= rid) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int METRIC>
__device__ __forceinline__ void trace_loop(const ImageDesc* descs, int n_desc, long long total,
                                           const SolverDesc& sol, int refill, unsigned long long* queue) {
    const int lane = threadIdx.x & 31;
    Lane L;
    bool active = false;
    bool drained = false;
    for (;;) {
        const unsigned idle = __ballot_sync(kFull, !active);
        const int n_idle = __popc(idle);
        if (!drained && n_idle > 0 && (n_idle >= refill || n_idle == 32)) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(queue, (unsigned long long)n_idle);
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned long long)n_idle >= (unsigned long long)total) drained = true;
            if (!active) {
                const long long rid = (long long)base + __popc(idle & ((1u << lane) - 1u));
                if (rid < total) {
                    const int im = (n_desc == 1) ? 0 : find_image(descs, n_desc, rid);
                    active = init_ray<METRIC>(L, descs + im, rid - descs[im].ray_begin, sol);
                }
            }
        }
        if (!__any_sync(kFull, active)) {
            if (drained) break;
            continue;
        }
        if (active) {
            const int code = step_ray64<METRIC>(L, sol);
            if (code >= 0) {
                write_final(L, code);
                active = false;
            }
        }
    }
}

template <int METRIC, int N>
__global__ void __launch_bounds__(128) trace_kernel64(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC>(p.desc, p.n_desc, p.total, p.sol, p.refill, p.queue);
}

template <int METRIC, int N>
__global__ void __launch_bounds__(256) trace_kernel64_b256(const __grid_constant__ LaunchParams<N> p) {
    trace_loop<METRIC>(p.desc, p.n_desc, p.total, p.sol, p.refill, p.queue);
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <int N, typename K>
static cudaError_t launch_persistent(K kern, int block, int blocks_per_sm, const LaunchParams<N>& p,
                                     cudaStream_t st) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    int bps = blocks_per_sm > 0 ? min(blocks_per_sm, occ) : occ;
    long long warps_needed = (p.total + 31) / 32;
    long long grid = (long long)bps * sm_count();
    long long grid_cap = (warps_needed * 32 + block - 1) / block;
    if (grid > grid_cap) grid = grid_cap;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, block, 0, st>>>(p);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_n(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                            const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream) {
    LaunchParams<N> p;
    p.sol = sol;
    p.n_desc = n;
    p.refill = shape.refill > 0 ? shape.refill : 8;
    p.total = total;
    p.queue = queue;
    for (int i = 0; i < n; ++i) p.desc[i] = descs[i];
    const int bps = shape.blocks_per_sm;
#define TT_LAUNCH(KERN, BLOCK) return launch_persistent<N>(KERN, BLOCK, bps, p, stream)
    if (shape.block == 256) {
        if (metric_mode == 0) TT_LAUNCH((trace_kernel64_b256<0, N>), 256);
        if (metric_mode == 1) TT_LAUNCH((trace_kernel64_b256<1, N>), 256);
        TT_LAUNCH((trace_kernel64_b256<2, N>), 256);
    }
    if (metric_mode == 0) TT_LAUNCH((trace_kernel64<0, N>), 128);
    if (metric_mode == 1) TT_LAUNCH((trace_kernel64<1, N>), 128);
    TT_LAUNCH((trace_kernel64<2, N>), 128);
#undef TT_LAUNCH
}

cudaError_t launch_trace(const ImageDesc* descs, int n, long long total_rays, int metric_mode,
                         const SolverDesc& sol, const LaunchShape& shape, unsigned long long* queue,
                         cudaStream_t stream) {
    if (n < 1 || n > kMaxImagesPerLaunch) return cudaErrorInvalidValue;
    if (n == 1) return launch_n<1>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
    return launch_n<kMaxImagesPerLaunch>(descs, n, total_rays, metric_mode, sol, shape, queue, stream);
}

}  // namespace tt

// tt_trace.cuh -- device code of the persistent ray-tracing kernels (sm_103a).
//
// One ray per thread; warps pull rays from a shared queue (one atomicAdd per
// warp refill).  On GB300 an FP64 instruction issues at 1/64 of the FP32 rate
// and a warp pays for its inactive lanes, so per-ray side work outside the
// regular step (initial data, crossing refinement and emission, the final
// record, the mixed path's extended-precision steps and |H| checks) runs in
// warp-uniform phases in which every lane that needs it takes part at once:
//
//   refill phase  : when >= `refill` lanes are done or idle (or none runs):
//                   pending crossings are refined, finished rays are written,
//                   idle lanes take new rays and build their initial data;
//   steps         : FP64 and double-float paths: every running lane.  Mixed
//                   paths: lanes near the horizon (r < r_fp64) or the axis
//                   (within the pole angle) take a double-float step once
//                   `fp64_batch` of them (or every running lane) need one, or
//                   they have waited `fp64_wait` iterations; the others an
//                   FP32 step;
//   crossings     : once >= `crossing_batch` lanes have a crossing pending;
//   |H| check     : mixed paths, every `monitor_period` iterations, in FP64.
//
// Every loop is bounded: a lane takes at most max_steps steps per ray and each
// warp iteration either steps rays or consumes queue entries; nothing waits on
// another thread.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tt_device.cuh"
#include "tt_df.cuh"
#include "tt_internal.h"

namespace tt {

constexpr unsigned kFull = 0xffffffffu;

// x^(-1/10) for the step-size factor: the SFU's single-precision power refined
// by one Newton step of y^-10 = x, y <- y (1.1 - 0.1 x y^10), which squares the
// relative error (~1e-7 -> ~1e-13).  Callers handle x < 1e-30 themselves.
__device__ __forceinline__ double pow_m01(double x) {
    double y = (double)__powf((float)x, -0.1f);
    double y2 = y * y, y4 = y2 * y2, y10 = y4 * y4 * y2;
    return y * fma(-0.1 * x, y10, 1.1);
}

// Step-size factor 0.9 err^(-1/5) from err^2 (large when err^2 is tiny or 0).
__device__ __forceinline__ double step_factor(double err2) {
    return lt_pos(err2, 1e-30) ? 1e30 : 0.9 * pow_m01(err2);
}

// ---------------------------------------------------------------------------
// One step of an embedded 5(4) pair in FP64 (paper Sec. 3.2): returns the
// fifth-order point yn, the flow kn and H there, and the error vector divided
// by h.  For
// Dormand-Prince kn is the seventh stage (first same as last); for Cash-Karp
// and Fehlberg it is evaluated after the six stages.
// ---------------------------------------------------------------------------
// On the closed-form metric (METRIC 0) the stages take sin and cos of theta
// from (s0, c0) of the step start by angle addition, and the new point's are
// returned in (sn, cn) for the next step (first same as last).
template <int METRIC>
__device__ __forceinline__ void flow64_near(const ImageDesc& d, const KerrK& kk, const RayConst& R, const State& y,
                                            double th0, double s0, double c0, State& f, double& H, double& s,
                                            double& c) {
    if constexpr (METRIC == 0) {
        sincos_near(y.th, th0, s0, c0, s, c);
        kerr_flow64_sc(kk, R, y, s, c, f, H);
    } else {
        flow64<METRIC>(d, kk, R, y, f, H);
    }
}

template <int METRIC, int METHOD = 0>
__device__ __forceinline__ void rk_step64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
                                           const State& y, const State& k1, double h, State& yn,
                                           State& kn, double& Hn, State& err, double s0 = 0.0, double c0 = 1.0,
                                           double* sn = nullptr, double* cn = nullptr) {
    using T = RK<METHOD>;
    State k2, k3, k4, k5, k6, ys;
    double Hs, ss = s0, cs = c0;
#define TT_STAGE(dst, expr_r, expr_t, expr_p, expr_q)                                \
    ys.r = fma(h, (expr_r), y.r);                                                    \
    ys.th = fma(h, (expr_t), y.th);                                                  \
    ys.pr = fma(h, (expr_p), y.pr);                                                  \
    ys.pth = fma(h, (expr_q), y.pth);                                                \
    flow64_near<METRIC>(d, kk, R, ys, y.th, s0, c0, dst, Hs, ss, cs);
// stages 2-4: coefficients pre-multiplied by h (one multiply each, shared by
// the four components), the stage point an FMA chain from y
#define TT_PSTAGE(dst, EXPR)                                                         \
    ys.r = EXPR(r);                                                                  \
    ys.th = EXPR(th);                                                                \
    ys.pr = EXPR(pr);                                                                \
    ys.pth = EXPR(pth);                                                              \
    flow64_near<METRIC>(d, kk, R, ys, y.th, s0, c0, dst, Hs, ss, cs);
    const double h21 = h * T::a21, h31 = h * T::a31, h32 = h * T::a32;
    const double h41 = h * T::a41, h42 = h * T::a42, h43 = h * T::a43;
#define TT_P2(f) fma(h21, k1.f, y.f)
#define TT_P3(f) fma(h32, k2.f, fma(h31, k1.f, y.f))
#define TT_P4(f) fma(h43, k3.f, fma(h42, k2.f, fma(h41, k1.f, y.f)))
#define TT_C5(f) fma(T::a54, k4.f, fma(T::a53, k3.f, fma(T::a52, k2.f, T::a51 * k1.f)))
#define TT_C6(f) fma(T::a65, k5.f, fma(T::a64, k4.f, fma(T::a63, k3.f, fma(T::a62, k2.f, T::a61 * k1.f))))
#define TT_C7(f) fma(T::b6, k6.f, TT_MAC(T::b5, k5.f, fma(T::b4, k4.f, fma(T::b3, k3.f, T::b1 * k1.f))))
    TT_PSTAGE(k2, TT_P2)
    TT_PSTAGE(k3, TT_P3)
    TT_PSTAGE(k4, TT_P4)
    TT_STAGE(k5, TT_C5(r), TT_C5(th), TT_C5(pr), TT_C5(pth))
    TT_STAGE(k6, TT_C6(r), TT_C6(th), TT_C6(pr), TT_C6(pth))
    yn.r = fma(h, TT_C7(r), y.r);
    yn.th = fma(h, TT_C7(th), y.th);
    yn.pr = fma(h, TT_C7(pr), y.pr);
    yn.pth = fma(h, TT_C7(pth), y.pth);
    flow64_near<METRIC>(d, kk, R, yn, y.th, s0, c0, kn, Hn, ss, cs);
    if (sn) {
        *sn = ss;
        *cn = cs;
    }
// the error vector without its factor h (err_norm2 applies it once)
#define TT_E(f) \
    TT_MAC(T::e7, kn.f, fma(T::e6, k6.f, fma(T::e5, k5.f, fma(T::e4, k4.f, fma(T::e3, k3.f, T::e1 * k1.f)))))
    err.r = TT_E(r);
    err.th = TT_E(th);
    err.pr = TT_E(pr);
    err.pth = TT_E(pth);
#undef TT_E
#undef TT_STAGE
#undef TT_PSTAGE
#undef TT_P2
#undef TT_P3
#undef TT_P4
#undef TT_C5
#undef TT_C6
#undef TT_C7
}

// ---------------------------------------------------------------------------
// Gragg-Bulirsch-Stoer macro-step in FP64 (paper Sec. 3.2): Gragg's modified
// midpoint rule with n_j = 2j sub-steps (j = 1..kGbsK, no smoothing step), each
// result extrapolated to sub-step 0 in (H/n_j)^2 by Aitken-Neville; the
// solution is the diagonal entry T_kk and the error T_kk - T_k,k-1.  Chain and
// extrapolation run on the increment z - y (so the rounding in the error
// estimate, a small difference of extrapolated values, scales with the step's
// change rather than with |y|).  The table row lives in registers (the j and l
// loops unroll, so each weight 1 / ((j / (j - l))^2 - 1) is a constant).
// ---------------------------------------------------------------------------
constexpr int kGbsK = 6;

__device__ __forceinline__ State axpy(double a, const State& x, const State& y) {
    return State{fma(a, x.r, y.r), fma(a, x.th, y.th), fma(a, x.pr, y.pr), fma(a, x.pth, y.pth)};
}

__device__ __forceinline__ State sub(const State& x, const State& y) {
    return State{x.r - y.r, x.th - y.th, x.pr - y.pr, x.pth - y.pth};
}

__device__ __forceinline__ State add(const State& x, const State& y) {
    return State{x.r + y.r, x.th + y.th, x.pr + y.pr, x.pth + y.pth};
}

// dT = T_kk - y, err = T_kk - T_k,k-1 for dz/dx = flow(z) from (y, f0 = flow(y)) over H.
template <class Flow>
__device__ __forceinline__ void gbs_core(const State& y, const State& f0, double H, Flow&& flow, State& dT,
                                         State& err) {
    State T[kGbsK];
#pragma unroll
    for (int j = 1; j <= kGbsK; ++j) {
        const double h = H / (double)(2 * j);
        State d0 = State{0.0, 0.0, 0.0, 0.0};
        State d1 = State{h * f0.r, h * f0.th, h * f0.pr, h * f0.pth};
        for (int m = 1; m < 2 * j; ++m) {
            State fz;
            flow(add(y, d1), fz);
            const State d2 = axpy(2.0 * h, fz, d0);
            d0 = d1;
            d1 = d2;
        }
        if (j == 1) {
            T[0] = d1;
        } else {
            State prev = T[0];                  // T_{j-1,1}
            T[0] = d1;
#pragma unroll
            for (int l = 1; l < j; ++l) {
                // 1 / ((j / (j - l))^2 - 1) as one quotient of integers (rounded alike
                // whether or not the loop unrolls into constants)
                const double w = (double)((j - l) * (j - l)) / (double)(l * (2 * j - l));
                const State old = T[l];         // T_{j-1,l+1}
                T[l] = axpy(w, sub(T[l - 1], prev), T[l - 1]);
                prev = old;
            }
        }
    }
    dT = T[kGbsK - 1];
    err = sub(T[kGbsK - 1], T[kGbsK - 2]);
}

template <int METRIC>
__device__ __forceinline__ void gbs_step64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
                                           const State& y, const State& f0, double H, State& yn, State& kn,
                                           double& Hn, State& err) {
    State dT;
    gbs_core(y, f0, H, [&](const State& z, State& fz) {
        double Hs;
        flow64<METRIC>(d, kk, R, z, fz, Hs);
    }, dT, err);
    yn = add(y, dT);
    flow64<METRIC>(d, kk, R, yn, kn, Hn);
}

// Step factor of the extrapolator: 0.94 (0.65 / err)^(1/(2k-1)) from err^2.
__device__ __forceinline__ double gbs_factor(double err2) {
    return (err2 == 0.0) ? 4.0 : 0.94 * pow(err2 / (0.65 * 0.65), -0.5 / (2.0 * kGbsK - 1.0));
}

// ---------------------------------------------------------------------------
// Stormer-Verlet for the Hamiltonian H(q, p), q = (r, theta), p = (p_r, p_theta)
// (paper Sec. 3.2; the generalised leapfrog of Hairer, Lubich & Wanner):
//   p+ = p - h/2 dH/dq(q, p+),  Q = q + h/2 [dH/dp(q, p+) + dH/dp(Q, p+)],
//   P = p+ - h/2 dH/dq(Q, p+),
// both implicit equations solved by fixed-point iteration from the explicit
// guess until no component moves by more than 1e-15 max(1, |value|), at most
// kVerletIt iterations.  The flow gives (dH/dp, -dH/dq) = (r', theta', p_r', p_theta').
// ---------------------------------------------------------------------------
constexpr int kVerletIt = 50;

__device__ __forceinline__ bool moved2(double a0, double b0, double a1, double b1) {
    return fabs(a0 - b0) > 1e-15 * fmax(1.0, fabs(b0)) || fabs(a1 - b1) > 1e-15 * fmax(1.0, fabs(b1));
}

template <int METRIC>
__device__ __forceinline__ void verlet_step64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
                                              const State& y, const State& f0, double h, State& yn, State& kn,
                                              double& Hn) {
    const double hh = 0.5 * h;
    State w = y, g;
    double Hs;
    w.pr = fma(hh, f0.pr, y.pr);
    w.pth = fma(hh, f0.pth, y.pth);
    for (int it = 0; it < kVerletIt; ++it) {
        flow64<METRIC>(d, kk, R, w, g, Hs);
        const double npr = fma(hh, g.pr, y.pr), npth = fma(hh, g.pth, y.pth);
        const bool mv = moved2(npr, w.pr, npth, w.pth);
        w.pr = npr;
        w.pth = npth;
        if (!mv) break;
    }
    flow64<METRIC>(d, kk, R, w, g, Hs);         // w = (q, p+)
    const double ar = g.r, ath = g.th;
    w.r = fma(h, ar, y.r);
    w.th = fma(h, ath, y.th);
    for (int it = 0; it < kVerletIt; ++it) {
        flow64<METRIC>(d, kk, R, w, g, Hs);
        const double nr = fma(hh, ar + g.r, y.r), nth = fma(hh, ath + g.th, y.th);
        const bool mv = moved2(nr, w.r, nth, w.th);
        w.r = nr;
        w.th = nth;
        if (!mv) break;
    }
    flow64<METRIC>(d, kk, R, w, g, Hs);         // w = (Q, p+)
    yn = State{w.r, w.th, fma(hh, g.pr, w.pr), fma(hh, g.pth, w.pth)};
    flow64<METRIC>(d, kk, R, yn, kn, Hn);
}

// e / (atol + rtol max(|y|, |yn|)); callers square and sum with explicit FMAs
// (never left to the compiler's contraction, so every build rounds alike).
__device__ __forceinline__ double err_ratio(double e, double y, double yn, double atol, double rtol) {
    const double sc = fma(rtol, fmax(fabs(y), fabs(yn)), atol);
    return e * rcp64(sc);
}

__device__ __forceinline__ double sq3(double a, double b, double c) {
    return fma(c, c, fma(b, b, a * a));
}

// Mean-square error norm over (r, theta, p_r, p_theta).  The four scale
// factors share one reciprocal: 1/sc_0 = sc_1 sc_2 sc_3 / (sc_0 sc_1 sc_2 sc_3),
// refined by a single Newton step (~1e-14 relative: the norm only decides
// err <= 1 and scales the step).  A product outside the normal range (tolerances
// near 1e-75 or 1e75) takes the per-component reciprocals instead.
// The error vector is he * e (he = h for the Runge-Kutta pairs, whose e omits
// the step's factor h; 1 otherwise).
__device__ __forceinline__ double err_norm2(const State& y, const State& yn, const State& e,
                                            double atol, double rtol, double he) {
    const double s0 = fma(rtol, fmax(fabs(y.r), fabs(yn.r)), atol);
    const double s1 = fma(rtol, fmax(fabs(y.th), fabs(yn.th)), atol);
    const double s2 = fma(rtol, fmax(fabs(y.pr), fabs(yn.pr)), atol);
    const double s3 = fma(rtol, fmax(fabs(y.pth), fabs(yn.pth)), atol);
    const double p01 = s0 * s1, p23 = s2 * s3;
    const double pp = p01 * p23;
    // outside [2^-930, 2^930] (the exponent field, on the integer pipe)
    const int ex = (__double2hiint(pp) >> 20) & 0x7ff;
    if (ex < 1023 - 930 || ex > 1023 + 930) {
        const double q3 = err_ratio(he * e.pth, y.pth, yn.pth, atol, rtol);
        return 0.25 * fma(q3, q3, sq3(err_ratio(he * e.r, y.r, yn.r, atol, rtol),
                                      err_ratio(he * e.th, y.th, yn.th, atol, rtol),
                                      err_ratio(he * e.pr, y.pr, yn.pr, atol, rtol)));
    }
    double inv;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(inv) : "d"(pp));
    inv = fma(inv, fma(-pp, inv, 1.0), inv) * he;
    const double i01 = inv * p23, i23 = inv * p01;   // he/(s0 s1), he/(s2 s3)
    const double q0 = (e.r * s1) * i01, q1 = (e.th * s0) * i01;
    const double q2 = (e.pr * s3) * i23, q3 = (e.pth * s2) * i23;
    return 0.25 * fma(q3, q3, fma(q2, q2, fma(q1, q1, q0 * q0)));
}

// Non-finite tests on the exponent bits (integer pipe, not the FP64 pipe).
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}

__device__ __forceinline__ bool nan_bits(double x) {
    const int hi = __double2hiint(x);
    return (hi & 0x7ff00000) == 0x7ff00000 && (((hi & 0x000fffff) | __double2loint(x)) != 0);
}

// ---------------------------------------------------------------------------
// Crossing refinement.
// Henon's exact step: integrate dz/dtheta = f / (dtheta/dlambda) for
// z = (r, p_r, p_th) from the start of the accepted step to theta = pi/2 with
// the ray's 5(4) pair in 2^m equal sub-steps, m = 0..6, taking the first m whose
// largest sub-step error norm (over r, p_r, p_th) is <= 1.
// ---------------------------------------------------------------------------
template <int METRIC>
__device__ __forceinline__ void theta_flow64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
                                             const State& y, State& g) {
    State f;
    double H;
    flow64<METRIC>(d, kk, R, y, f, H);
    double it = rcp64(f.th);
    g.r = f.r * it;
    g.th = 1.0;
    g.pr = f.pr * it;
    g.pth = f.pth * it;
}

template <int METRIC, int METHOD = 0>
__device__ double refine_henon64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
                                 const State& y0, const State& f0, double atol, double rtol) {
    using T = RK<METHOD>;
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
    theta_flow64<METRIC>(d, kk, R, zs, dst);
#define TT_C2(f) (T::a21 * g.f)
#define TT_C3(f) fma(T::a32, k2.f, T::a31 * g.f)
#define TT_C4(f) fma(T::a43, k3.f, fma(T::a42, k2.f, T::a41 * g.f))
#define TT_C5(f) fma(T::a54, k4.f, fma(T::a53, k3.f, fma(T::a52, k2.f, T::a51 * g.f)))
#define TT_C6(f) fma(T::a65, k5.f, fma(T::a64, k4.f, fma(T::a63, k3.f, fma(T::a62, k2.f, T::a61 * g.f))))
#define TT_C7(f) fma(T::b6, k6.f, TT_MAC(T::b5, k5.f, fma(T::b4, k4.f, fma(T::b3, k3.f, T::b1 * g.f))))
            TT_HS(k2, T::c2, TT_C2(r), TT_C2(pr), TT_C2(pth))
            TT_HS(k3, T::c3, TT_C3(r), TT_C3(pr), TT_C3(pth))
            TT_HS(k4, T::c4, TT_C4(r), TT_C4(pr), TT_C4(pth))
            TT_HS(k5, T::c5, TT_C5(r), TT_C5(pr), TT_C5(pth))
            TT_HS(k6, T::c6, TT_C6(r), TT_C6(pr), TT_C6(pth))
            State zn;
            zn.r = fma(dl, TT_C7(r), z.r);
            zn.pr = fma(dl, TT_C7(pr), z.pr);
            zn.pth = fma(dl, TT_C7(pth), z.pth);
            zn.th = th0 + dl;
            theta_flow64<METRIC>(d, kk, R, zn, k7);
#define TT_E(f) \
    dl * TT_MAC(T::e7, k7.f, fma(T::e6, k6.f, fma(T::e5, k5.f, fma(T::e4, k4.f, fma(T::e3, k3.f, T::e1 * g.f)))))
            double s = sq3(err_ratio(TT_E(r), z.r, zn.r, atol, rtol), err_ratio(TT_E(pr), z.pr, zn.pr, atol, rtol),
                           err_ratio(TT_E(pth), z.pth, zn.pth, atol, rtol));
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

// Henon's exact step for Gragg-Bulirsch-Stoer rays: the same sub-stepping and
// error rule as refine_henon64, each sub-step one extrapolation macro-step of
// the theta-system (theta integrated as a component, as its own derivative 1).
template <int METRIC>
__device__ double refine_henon_gbs64(const ImageDesc& d, const KerrK& kk, const RayConst& R, const State& y0,
                                     const State& f0, double atol, double rtol) {
    const double dth_all = kHalfPi - y0.th;
    const double it0 = rcp64(f0.th);
    const State g0 = State{f0.r * it0, 1.0, f0.pr * it0, f0.pth * it0};
    auto tflow = [&](const State& z, State& g) { theta_flow64<METRIC>(d, kk, R, z, g); };
    double r_out = y0.r;
    for (int m = 0; m <= 6; ++m) {
        const int nsub = 1 << m;
        const double dl = dth_all / (double)nsub;
        State z = y0, g = g0;
        double worst = 0.0;
        for (int q = 0; q < nsub; ++q) {
            State dz, e;
            gbs_core(z, g, dl, tflow, dz, e);
            const State zn = add(z, dz);
            double s = sq3(err_ratio(e.r, z.r, zn.r, atol, rtol), err_ratio(e.pr, z.pr, zn.pr, atol, rtol),
                           err_ratio(e.pth, z.pth, zn.pth, atol, rtol));
            s *= (1.0 / 3.0);
            if (!(s <= worst)) worst = s;
            z = zn;
            tflow(z, g);
        }
        r_out = z.r;
        if (worst <= 1.0) break;
    }
    return r_out;
}

// Paper's method (Sec. 3.2): bisection of theta(lambda) - pi/2 on the cubic-
// Hermite interpolant of the accepted step, to 1e-12 in lambda.
static __device__ double refine_hermite64(const State& y0, const State& f0, const State& y1,
                                   const State& f1, double h) {
    double lo = 0.0, hi = 1.0;
    const bool s0 = y0.th <= kHalfPi;
    for (int it = 0; it < 200 && (hi - lo) * h > 1e-12; ++it) {
        double mid = 0.5 * (lo + hi);
        double B[4], dB[4];
        hermite4(mid, B, dB);
        double th = fma(B[3] * h, f1.th, fma(B[2], y1.th, fma(B[1] * h, f0.th, B[0] * y0.th)));
        if ((th <= kHalfPi) == s0) lo = mid;
        else hi = mid;
    }
    double sc = 0.5 * (lo + hi);
    double B[4], dB[4];
    hermite4(sc, B, dB);
    return fma(B[3] * h, f1.r, fma(B[2], y1.r, fma(B[1] * h, f0.r, B[0] * y0.r)));
}

// Hairer-Norsett-Wanner starting step (embedded order 4), four-component norm.
template <int METRIC>
__device__ double initial_step64(const ImageDesc& d, const KerrK& kk, const RayConst& R,
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
    flow64<METRIC>(d, kk, R, y1, f1, H1);
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
    State y, k1;            // FP64 state and its flow (first-same-as-last, valid if k64_ok)
    double s0, c0;          // sin and cos of y.th (FP64 path, closed-form metric)
    RayConst R;
    KerrK kk;
    double h, lam, hmax, inten;
    int steps, rejects, ncross, nrec, code;
    bool last_rej;
    // a disk crossing waiting for its (batched) refinement: the start of its step
    bool pend;
    State yc;
    // mixed precision
    StateF k1f;             // FP32 flow at the state (valid if k32_ok)
    StateF lo;              // low parts of the compensated FP32-pair state
    RayConstF Rf;
    float Mf, a2f, rpmf;    // M, a^2, r_+ - r_-
    float rph, rpl;         // r_+ as an FP32 pair
    float caph, capl;       // capture radius as an FP32 pair
    float escf, fp64f;      // escape radius, extended-precision-step radius
    float thpf;             // extended-precision steps within this angle of the axis
    float hf, lamf;         // step size and affine parameter of the FP32 steps
    bool k64_ok, k32_ok;
    // double-float steps: low parts of the flow at the state (valid with k1f if
    // kdf_ok), the spacetime and ray constants, and the running max of |H|
    StateF k1lo;
    bool kdf_ok;
    float hmaxf;
    KerrDF kdf;
    RayDF rdf;
    // mixed paths: a near-critical ray, traced in double-float
    bool crit;
};

// Output stores.  The bounds-checking build (TT_BOUNDS_CHECK) tests every index
// against its buffer's length and, instead of a store outside it, counts a
// fault in the solver's counter (read back by tartarus_debug_faults); nothing
// traps.  Otherwise the plain store.
#ifdef TT_BOUNDS_CHECK
#define TT_STORE(d, arr, idx, len, val)                                        \
    do {                                                                       \
        const long long i_ = (idx);                                            \
        if (i_ >= 0 && i_ < (len)) (d).arr[i_] = (val);                        \
        else if (sol.faults) atomicAdd(sol.faults, 1ull);                      \
    } while (0)
#else
#define TT_STORE(d, arr, idx, len, val) ((d).arr[(idx)] = (val))
#endif

__device__ __forceinline__ void write_final(const Lane& L, int code, const SolverDesc& sol) {
    const ImageDesc& d = *L.d;
    const long long q = L.q, n = d.pix_count;
    TT_STORE(d, code, q, n, (int8_t)code);
    TT_STORE(d, n_cross, q, n, (int8_t)min(L.ncross, 127));
    TT_STORE(d, intensity, q, n, L.inten);
    TT_STORE(d, h_max, q, n, fmax(L.hmax, (double)L.hmaxf));
    TT_STORE(d, steps, q, n, L.steps);
    TT_STORE(d, rejects, q, n, L.rejects);
    for (int k = L.nrec; k < kMaxCross; ++k) {
        TT_STORE(d, r_cross, k * n + q, kMaxCross * n, 0.0);
        TT_STORE(d, g, k * n + q, kMaxCross * n, 0.0);
        TT_STORE(d, I_cross, k * n + q, kMaxCross * n, 0.0);
    }
}

__device__ __forceinline__ void split_pair(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

__device__ __forceinline__ State pair_to64(const StateF& hi, const StateF& lo) {
    return State{(double)hi.r + (double)lo.r, (double)hi.th + (double)lo.th, (double)hi.pr + (double)lo.pr,
                 (double)hi.pth + (double)lo.pth};
}

__device__ __forceinline__ void split_state(const State& y, StateF& hi, StateF& lo) {
    split_pair(y.r, hi.r, lo.r);
    split_pair(y.th, hi.th, lo.th);
    split_pair(y.pr, hi.pr, lo.pr);
    split_pair(y.pth, hi.pth, lo.pth);
}

// The Hairer-Norsett-Wanner starting step in FP32 for the mixed paths, from the
// FP32 flow k1f at yf (already in L); the flow takes theta as dth0 = theta - m pi
// (see step_ray32).
static __device__ float initial_step32(const Lane& L, const StateF& y0, float dr0, float dth0, float atol,
                                       float rtol) {
    const StateF f0 = L.k1f;
    const float sr = fmaf(rtol, fabsf(y0.r), atol), st = fmaf(rtol, fabsf(y0.th), atol);
    const float sp = fmaf(rtol, fabsf(y0.pr), atol), sq = fmaf(rtol, fabsf(y0.pth), atol);
    auto n4 = [&](float a, float b, float c, float e) {
        return sqrtf(0.25f * (a / sr * (a / sr) + b / st * (b / st) + c / sp * (c / sp) + e / sq * (e / sq)));
    };
    const float d0 = n4(y0.r, y0.th, y0.pr, y0.pth);
    const float d1 = n4(f0.r, f0.th, f0.pr, f0.pth);
    const float h0 = (d0 < 1e-5f || d1 < 1e-5f) ? 1e-6f : 0.01f * d0 / d1;
    const StateF y1 = {fmaf(h0, f0.r, y0.r), fmaf(h0, f0.th, y0.th), fmaf(h0, f0.pr, y0.pr), fmaf(h0, f0.pth, y0.pth)};
    StateF f1;
    float H1;
    kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, StateF{y1.r, fmaf(h0, f0.th, dth0), y1.pr, y1.pth}, fmaf(h0, f0.r, dr0),
                f1, H1);
    const float d2 = n4(f1.r - f0.r, f1.th - f0.th, f1.pr - f0.pr, f1.pth - f0.pth) / h0;
    const float dm = fmaxf(d1, d2);
    const float h1 = (dm <= 1e-15f) ? fmaxf(1e-6f, h0 * 1e-3f) : __powf(0.01f / dm, 0.2f);
    return fminf(100.0f * h0, h1);
}

// An image (or a pixel range of whole rows) whose width is a multiple of 8 and
// whose row count is a multiple of 4 is handed out in 8 x 4 pixel tiles (32
// consecutive queue entries per tile), so that the rays a warp takes together
// start close on the sky and stay in step: the queue entry q of such a range
// traces the tile's pixel returned here (relative to the range's first pixel).
// Outputs are per pixel either way.
__device__ __forceinline__ long long tile_pixel(const ImageDesc& d, long long q) {
    const long long band = 4LL * d.nx;
    if ((d.nx & 7) == 0 && d.pix_begin % band == 0 && d.pix_count % band == 0) {
        const long long tile = q >> 5, tiles_x = d.nx >> 3;
        const long long ty = tile / tiles_x, tx = tile - ty * tiles_x;
        const int lane = (int)(q & 31);
        q = (ty * 4 + (lane >> 3)) * d.nx + tx * 8 + (lane & 7);
    }
    return q;
}

// ---------------------------------------------------------------------------
// Near-critical rays (mixed paths, closed-form Kerr).  With the photon's
// constants of motion xi = L/E and eta = Q/E^2 (Q Carter's constant) the
// radial motion obeys (Sigma dr/dlambda)^2 = E^2 R(r),
//   R(r) = r^4 + (a^2 - xi^2 - eta) r^2 + 2 M (eta + (xi - a)^2) r - a^2 eta.
// A ray on the critical curve (the shadow's edge) has a double root of R at a
// spherical photon orbit r_m; a nearby ray lingers there for ~ln(1/delta)
// circuits, each multiplying a perturbation by ~e^pi.  r_m is taken as the
// largest root of R'(r) / 4 = r^3 + P r + C, P = (a^2 - xi^2 - eta)/2,
// C = M (eta + (xi - a)^2)/2 (the local minimum of R; trigonometric form of
// the cubic's three real roots), and R(r_m) / (2 r_m^2 b), b^2 = xi^2 + eta,
// estimates the ray's distance from the critical curve in impact parameter
// (dR/db = -2 b r^2 when xi and eta scale together).  Evaluated in FP32 (the
// band, ~0.15 M, is ~10^6 times its rounding) from the observer's tetrad as in
// init_ray; the same code classifies a ray in the scan and in the main pass,
// so every ray is traced exactly once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool near_critical(const ImageDesc& d, long long q, float band) {
    const long long p = d.pix_begin + q;
    const long long i = p % d.nx, j = p / d.nx;
    const float al = (float)d.alpha_min + ((float)i + 0.5f) * (float)d.dalpha;
    const float be = (float)d.beta_min + ((float)j + 0.5f) * (float)d.dbeta;
    const float D = (float)d.r_obs;
    if (!isfinite(al) || !isfinite(be) || !(fmaf(al, al, be * be) < D * D)) return false;
    // physical momentum at the observer (ZAMO tetrad, as in init_ray)
    const float iN = (float)d.obs_iN, omN = (float)d.obs_omN;
    const float pu_th = (be / D) * (float)d.obs_ith;
    const float pu_ph = fmaf(-al / D, (float)d.obs_iph, omN);
    const float gtt = (float)d.obs_g[0], gtp = (float)d.obs_g[1], gthth = (float)d.obs_g[3], gpp = (float)d.obs_g[4];
    const float E = -fmaf(gtt, iN, gtp * pu_ph);
    const float Lz = fmaf(gtp, iN, gpp * pu_ph);
    const float pth = gthth * pu_th;
    float so, co;
    sincosf((float)d.theta_obs, &so, &co);
    const float a = (float)d.a, M = (float)d.M, a2 = a * a;
    const float Q = fmaf(pth, pth, co * co * (Lz * Lz / (so * so) - a2 * E * E));
    const float xi = Lz / E, eta = Q / (E * E);
    const float P = 0.5f * (a2 - xi * xi - eta);
    const float C = 0.5f * M * (eta + (xi - a) * (xi - a));
    if (!(P < 0.0f) || !(4.0f * P * P * P + 27.0f * C * C < 0.0f)) return false;     // one real root: no minimum
    const float m = 2.0f * sqrtf(-P * (1.0f / 3.0f));
    const float cs = fminf(1.0f, fmaxf(-1.0f, 3.0f * C / (P * m)));
    const float rm = m * cosf(acosf(cs) * (1.0f / 3.0f));
    if (!(rm > (float)d.r_plus)) return false;
    const float R = fmaf(fmaf(fmaf(rm, rm, 2.0f * P), rm, 4.0f * C), rm, -a2 * eta);
    const float b = sqrtf(fmaxf(fmaf(xi, xi, eta), 1e-12f));
    return fabsf(R) < band * M * (2.0f * rm * rm * b);
}

// Initial data from the ZAMO tetrad (paper Sec. 2.2), time-reversed, for the
// pixel q (after tile_pixel).  Returns false (and writes a BADPIXEL record) if
// the pixel is outside the sky.  df_init: set the ray up for double-float steps
// (the double-float path, and near-critical rays of the mixed paths).
template <int METRIC>
__device__ bool init_ray(Lane& L, const ImageDesc* d_ptr, long long q, const SolverDesc& sol,
                         bool df_init = false) {
    const ImageDesc& d = *d_ptr;
    L.d = d_ptr;
    L.q = q;
    L.kk = make_kerr(d.M, d.a);
    L.steps = 0;
    L.rejects = 0;
    L.ncross = 0;
    L.nrec = 0;
    L.code = -1;
    L.inten = 0.0;
    L.hmax = 0.0;
    L.lam = 0.0;
    L.last_rej = false;
    L.pend = false;
    const long long p = d.pix_begin + q;
    const long long i = p % d.nx, j = p / d.nx;
    const double alpha = d.alpha_min + ((double)i + 0.5) * d.dalpha;
    const double beta = d.beta_min + ((double)j + 0.5) * d.dbeta;
    const double D = d.r_obs, th = d.theta_obs;
    const double rho2 = alpha * alpha + beta * beta;
    if (!isfinite(alpha) || !isfinite(beta) || !(rho2 < D * D)) {
        write_final(L, 5, sol);
        return false;
    }
    // ZAMO tetrad at the observer: e_(t) = (1/N)(dt + omega dphi), e_(i) = d_i / sqrt(g_ii)
    double g[5], omN, iN, ir, ith, iph;
    if (d.obs_ready) {
        for (int k = 0; k < 5; ++k) g[k] = d.obs_g[k];
        omN = d.obs_omN;
        iN = d.obs_iN;
        ir = d.obs_ir;
        ith = d.obs_ith;
        iph = d.obs_iph;
    } else {
        lower64<METRIC>(d, D, th, g);
        const double omega = -g[1] / g[4];
        const double N = sqrt(-g[0] + omega * omega * g[4]);
        iN = 1.0 / N;
        omN = omega * iN;
        ir = 1.0 / sqrt(g[2]);
        ith = 1.0 / sqrt(g[3]);
        iph = 1.0 / sqrt(g[4]);
    }
    const double gtt = g[0], gtp = g[1], grr = g[2], gthth = g[3], gpp = g[4];
    const double pl_r = sqrt(1.0 - rho2 / (D * D));
    const double pu_t = iN;
    const double pu_r = pl_r * ir;
    const double pu_th = (beta / D) * ith;
    const double pu_ph = omN + (-alpha / D) * iph;
    const double p_t = gtt * pu_t + gtp * pu_ph;
    const double p_r = grr * pu_r;
    const double p_th = gthth * pu_th;
    const double p_ph = gtp * pu_t + gpp * pu_ph;
    L.y.r = D;
    L.y.th = th;
    L.y.pr = -p_r;
    L.y.pth = -p_th;
    L.R = make_ray_const(d.a, -p_t, -p_ph);
    L.k32_ok = false;
    L.kdf_ok = false;
    L.hmaxf = 0.0f;
    if (sol.precision == 0 && !df_init) {
        double H0;
        flow64<METRIC>(d, L.kk, L.R, L.y, L.k1, H0);
        sincos(L.y.th, &L.s0, &L.c0);
        L.hmax = fabs(H0);
        L.h = (sol.h0 > 0.0) ? sol.h0 : initial_step64<METRIC>(d, L.kk, L.R, L.y, L.k1, sol.atol, sol.rtol);
        L.k64_ok = true;
    } else {
        // mixed paths: FP32 flow and starting step, |H(y0)| (~1e-16) not sampled;
        // double-float path: the FP64 flow and starting step
        L.k64_ok = false;
        L.Rf = to_float(L.R, d.M);
        L.Mf = (float)d.M;
        L.a2f = (float)(d.a * d.a);
        L.rpmf = (float)(d.r_plus - d.r_minus);
        split_pair(d.r_plus, L.rph, L.rpl);
        split_pair(d.r_capture, L.caph, L.capl);
        L.escf = (float)d.r_escape;
        L.fp64f = (float)d.r_fp64;
        L.thpf = (float)d.th_pole;
        L.lamf = 0.0f;
        if (sol.precision == 3 || df_init) {
            // double-float steps: the FP64 path's starting step (once per ray), so
            // that both begin the same step sequence
            L.kdf = make_kerr_df(L.kk);
            L.rdf = make_ray_df(L.R);
            double H64;
            flow64<METRIC>(d, L.kk, L.R, L.y, L.k1, H64);
            L.hmax = fabs(H64);
            L.hf = (float)((sol.h0 > 0.0) ? sol.h0
                                         : initial_step64<METRIC>(d, L.kk, L.R, L.y, L.k1, sol.atol, sol.rtol));
        } else {
            const StateF yf = {(float)L.y.r, (float)L.y.th, (float)L.y.pr, (float)L.y.pth};
            const float dr0 = (float)(L.y.r - d.r_plus);
            const float dth0 = (float)(L.y.th - rint(L.y.th * 0.3183098861837907) * 3.141592653589793);
            float H0;
            kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, StateF{yf.r, dth0, yf.pr, yf.pth}, dr0, L.k1f, H0);
            L.k32_ok = true;
            L.hf = (sol.h0 > 0.0) ? (float)sol.h0
                                  : initial_step32(L, yf, dr0, dth0, (float)sol.atol, (float)sol.rtol);
        }
        L.h = (double)L.hf;
    }
    return true;
}

// Emission at a refined crossing radius (paper Sec. 2.3-2.4): counted if on the
// disk, stored (r, g, g^4 F) while slots remain.
template <int METRIC>
__device__ __forceinline__ void record_crossing(Lane& L, double rc, const SolverDesc& sol) {
    const ImageDesc& d = *L.d;
    if (rc >= d.r_in && rc <= d.r_out) {
        if (L.nrec < d.max_cross) {
            const double gf = redshift64<METRIC>(d, rc, L.R.pt, L.R.pph);
            const double F = flux64(d, rc);
            const double g2 = gf * gf;
            const double I = g2 * g2 * F;
            const long long n = d.pix_count, q = L.q;
            TT_STORE(d, r_cross, L.nrec * n + q, kMaxCross * n, rc);
            TT_STORE(d, g, L.nrec * n + q, kMaxCross * n, gf);
            TT_STORE(d, I_cross, L.nrec * n + q, kMaxCross * n, I);
            L.inten += I;
            L.nrec++;
        }
        L.ncross++;
    }
}

__device__ __forceinline__ float sq_ratio32(float e, float y, float yn, float atol, float rtol) {
    float sc = fmaf(rtol, fmaxf(fabsf(y), fabsf(yn)), atol);
    float q = __fdividef(e, sc);
    return q * q;
}

// Henon's exact step with FP32 stages (mixed paths): the same sub-stepping and
// error rule as refine_henon64, the theta-system evaluated with the FP32 flow
// at stage points formed from the FP64 sub-step start, and the sub-step
// results accumulated in FP64.
__device__ __forceinline__ void theta_flow32(const Lane& L, const StateF& y, float dr, StateF& g) {
    StateF f;
    float H;
    kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, y, dr, f, H);
    const float it = __frcp_rn(f.th);
    g.r = f.r * it;
    g.th = 1.0f;
    g.pr = f.pr * it;
    g.pth = f.pth * it;
}

static __device__ double refine_henon32(const Lane& L, const State& y0, double r_plus, float atol, float rtol) {
    using namespace dp;
    const double dth_all = kHalfPi - y0.th;
    double r_out = y0.r;
    StateF g0;
    theta_flow32(L, StateF{(float)y0.r, (float)y0.th, (float)y0.pr, (float)y0.pth}, (float)(y0.r - r_plus), g0);
    for (int m = 0; m <= 6; ++m) {
        const int nsub = 1 << m;
        const double dl64 = dth_all / (double)nsub;
        const float dl = (float)dl64;
        State z = y0;
        StateF g = g0;
        float worst = 0.0f;
        for (int q = 0; q < nsub; ++q) {
            const StateF zf = {(float)z.r, (float)z.th, (float)z.pr, (float)z.pth};
            const float dr0 = (float)(z.r - r_plus);
            StateF k2, k3, k4, k5, k6, k7, zs;
#define TT_HS(dst, cc, er, ep, eq)                        \
    zs.r = fmaf(dl, (er), zf.r);                          \
    zs.pr = fmaf(dl, (ep), zf.pr);                        \
    zs.pth = fmaf(dl, (eq), zf.pth);                      \
    zs.th = fmaf(dl, (float)(cc), zf.th);                 \
    theta_flow32(L, zs, fmaf(dl, (er), dr0), dst);
#define TT_C2(f) ((float)a21 * g.f)
#define TT_C3(f) fmaf((float)a32, k2.f, (float)a31 * g.f)
#define TT_C4(f) fmaf((float)a43, k3.f, fmaf((float)a42, k2.f, (float)a41 * g.f))
#define TT_C5(f) fmaf((float)a54, k4.f, fmaf((float)a53, k3.f, fmaf((float)a52, k2.f, (float)a51 * g.f)))
#define TT_C6(f) \
    fmaf((float)a65, k5.f, fmaf((float)a64, k4.f, fmaf((float)a63, k3.f, fmaf((float)a62, k2.f, (float)a61 * g.f))))
#define TT_C7(f) \
    fmaf((float)b6, k6.f, fmaf((float)b5, k5.f, fmaf((float)b4, k4.f, fmaf((float)b3, k3.f, (float)b1 * g.f))))
            TT_HS(k2, c2, TT_C2(r), TT_C2(pr), TT_C2(pth))
            TT_HS(k3, c3, TT_C3(r), TT_C3(pr), TT_C3(pth))
            TT_HS(k4, c4, TT_C4(r), TT_C4(pr), TT_C4(pth))
            TT_HS(k5, c5, TT_C5(r), TT_C5(pr), TT_C5(pth))
            TT_HS(k6, 1.0, TT_C6(r), TT_C6(pr), TT_C6(pth))
            const StateF inc = {dl * TT_C7(r), dl, dl * TT_C7(pr), dl * TT_C7(pth)};
            const StateF zn = {zf.r + inc.r, zf.th + dl, zf.pr + inc.pr, zf.pth + inc.pth};
            theta_flow32(L, zn, dr0 + inc.r, k7);
#define TT_E(f) dl * fmaf((float)e7, k7.f, fmaf((float)e6, k6.f, fmaf((float)e5, k5.f, \
                fmaf((float)e4, k4.f, fmaf((float)e3, k3.f, (float)e1 * g.f)))))
            float s = sq_ratio32(TT_E(r), zf.r, zn.r, atol, rtol);
            s += sq_ratio32(TT_E(pr), zf.pr, zn.pr, atol, rtol);
            s += sq_ratio32(TT_E(pth), zf.pth, zn.pth, atol, rtol);
#undef TT_E
#undef TT_HS
#undef TT_C2
#undef TT_C3
#undef TT_C4
#undef TT_C5
#undef TT_C6
#undef TT_C7
            s *= (1.0f / 3.0f);
            if (!(s <= worst)) worst = s;
            z.r += (double)inc.r;
            z.th = y0.th + (double)(q + 1) * dl64;
            z.pr += (double)inc.pr;
            z.pth += (double)inc.pth;
            g = k7;
        }
        r_out = z.r;
        if (worst <= 1.0f) break;
    }
    return r_out;
}

// Refine the pending crossing from the start of its step and record it.
// PREC 0: FP64 Henon.  Mixed paths: Henon with FP32 stages, or in FP64 when
// the solver asks for it (refine 2); emission is evaluated in FP64 either way.
template <int METRIC, int PREC, int METHOD = 0>
__device__ void refine_pending(Lane& L, const SolverDesc& sol) {
    const ImageDesc& d = *L.d;
    double rc;
    if ((PREC == 1 || PREC == 2) && sol.refine != 2) {
        rc = refine_henon32(L, L.yc, d.r_plus, (float)sol.atol, (float)sol.rtol);
    } else {
        State f0;
        double H0;
        flow64<METRIC>(d, L.kk, L.R, L.yc, f0, H0);
        L.hmax = fmax(L.hmax, fabs(H0));
        // the pairs and the extrapolator use their own steps, Verlet Dormand-Prince
        if constexpr (METHOD == 3)
            rc = refine_henon_gbs64<METRIC>(d, L.kk, L.R, L.yc, f0, sol.atol, sol.rtol);
        else
            rc = refine_henon64<METRIC, (METHOD <= 2 ? METHOD : 0)>(d, L.kk, L.R, L.yc, f0, sol.atol, sol.rtol);
    }
    record_crossing<METRIC>(L, rc, sol);
    L.pend = false;
}

// A crossing was found in the step that starts at y (FP64).  Henon refinement
// is deferred to a batched phase; crossings stay in order along the ray.
template <int METRIC, int PREC, int METHOD = 0>
__device__ __forceinline__ void note_crossing(Lane& L, const State& y, const SolverDesc& sol) {
    if (L.pend) refine_pending<METRIC, PREC, METHOD>(L, sol);
    L.yc = y;
    L.pend = true;
}

// One FP64 step attempt; returns the termination code or -1 if the ray continues.
template <int METRIC, int PREC, int METHOD = 0>
__device__ int step_ray64(Lane& L, const SolverDesc& sol) {
    const ImageDesc& d = *L.d;
    if ((long long)L.steps + (long long)L.rejects >= sol.max_steps) return 2;
    const double hmin = (sol.h_min > 0.0) ? sol.h_min : 1e-14 * fmax(1.0, fabs(L.lam));
    if (lt_pos(L.h, hmin)) return 3;
    State yn, kn, e;
    double Hn, sn = L.s0, cn = L.c0;
    if constexpr (METHOD == 4) {
        verlet_step64<METRIC>(d, L.kk, L.R, L.y, L.k1, L.h, yn, kn, Hn);
    } else if constexpr (METHOD == 3) {
        gbs_step64<METRIC>(d, L.kk, L.R, L.y, L.k1, L.h, yn, kn, Hn, e);
    } else {
        rk_step64<METRIC, METHOD>(d, L.kk, L.R, L.y, L.k1, L.h, yn, kn, Hn, e, L.s0, L.c0, &sn, &cn);
    }
    // Verlet: fixed step, always accepted
    const double err2 = (METHOD == 4) ? 0.0 : err_norm2(L.y, yn, e, sol.atol, sol.rtol, METHOD == 3 ? 1.0 : L.h);
    if (nan_bits(err2) | nonfinite_bits(yn.r) | nonfinite_bits(yn.th) | nonfinite_bits(yn.pr) |
        nonfinite_bits(yn.pth))
        return 4;
    if (le_pos(err2, 1.0)) {
        L.steps++;
        if (d.disk && (le_pos(L.y.th, kHalfPi) != le_pos(yn.th, kHalfPi))) {
            if (sol.refine == 1) {
                const double rc = refine_hermite64(L.y, L.k1, yn, kn, L.h);
                if (L.pend) refine_pending<METRIC, PREC, METHOD>(L, sol);
                record_crossing<METRIC>(L, rc, sol);
            } else {
                note_crossing<METRIC, PREC, METHOD>(L, L.y, sol);
            }
        }
        L.lam += L.h;
        L.y = yn;
        L.k1 = kn;
        L.s0 = sn;
        L.c0 = cn;
        L.hmax = fmax(L.hmax, fabs(Hn));
        if (lt_pos(yn.r, d.r_capture)) return 1;
        if (lt_pos(d.r_escape, yn.r)) return 0;
        if constexpr (METHOD == 3) {
            L.h *= fmin(L.last_rej ? 1.0 : 4.0, fmax(0.02, gbs_factor(err2)));
        } else if constexpr (METHOD != 4) {
            L.h *= fmin(L.last_rej ? 1.0 : 10.0, fmax(0.2, step_factor(err2)));
        }
        L.last_rej = false;
    } else {
        L.rejects++;
        if constexpr (METHOD == 3) {
            L.h *= fmin(1.0, fmax(0.02, gbs_factor(err2)));
        } else {
            L.h *= fmax(0.2, step_factor(err2));
        }
        L.last_rej = true;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// Mixed precision (closed-form Kerr).  The seven stages, the flow and the error
// estimate run in FP32.  PREC 1 and 2: the error norm and the step-size control
// in FP32 too; the state accumulated in FP64 (PREC 1: y_new = y + (double)(h
// sum b_i k_i)) or as a compensated FP32 pair (PREC 2: hi + lo with TwoSum,
// ~48 bits), which needs no FP64 instruction in the step.  PREC 4 (the
// prescribed split): FP64 state, and the error norm and step control in FP64
// from the FP32 error terms.  Steps in the zones near the horizon and the axis
// are taken by the caller (double-float, or FP64 for PREC 4).
// ---------------------------------------------------------------------------

// hi + lo <- hi + lo + x (Knuth's TwoSum, then renormalised).
__device__ __forceinline__ void pair_add(float& hi, float& lo, float x) {
    float s = hi + x;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (x - bb);
    float l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
}

// sign of (hi + lo) - (ch + cl), exact enough whenever the difference exceeds ~1e-14 relative
__device__ __forceinline__ bool pair_below(float hi, float lo, float ch, float cl) {
    return ((hi - ch) + (lo - cl)) < 0.0f;
}

template <int PREC>
__device__ int step_ray32(Lane& L, StateF& yhi, const SolverDesc& sol) {
    constexpr int ACC = (PREC == 2) ? 1 : 0;
    const ImageDesc& d = *L.d;
    if ((long long)L.steps + (long long)L.rejects >= sol.max_steps) return 2;
    const float h = L.hf;
    const float hmin = (sol.h_min > 0.0) ? (float)sol.h_min : 1e-14f * fmaxf(1.0f, L.lamf);
    if (h < hmin) return 3;
    using namespace dp;
    StateF y;
    float dr0, dth0;
    // The flow depends on theta only through sin^2, cos^2 and sin cos, which are
    // the same at delta = theta - m pi (m the nearest integer to theta / pi): the
    // stages take delta, formed from the high-precision state, so that near
    // theta = pi (where an FP32 theta resolves pi - theta, and so sin theta,
    // only to ~2.4e-7 absolute) sin theta keeps FP32's relative precision, as it
    // does near theta = 0.
    if (ACC == 0) {
        y = StateF{(float)L.y.r, (float)L.y.th, (float)L.y.pr, (float)L.y.pth};
        dr0 = (float)(L.y.r - d.r_plus);
        const float m = rintf(y.th * 0.318309886f);
        dth0 = (float)fma(-(double)m, 3.141592653589793, L.y.th);
    } else {
        y = yhi;
        dr0 = (y.r - L.rph) + (L.lo.r - L.rpl);
        const float m = rintf(y.th * 0.318309886f);
        dth0 = fmaf(-m, 3.14159274f, y.th) + fmaf(m, 8.74227766e-8f, L.lo.th);
    }
    float Hs;
    if (!L.k32_ok) {
        kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, StateF{y.r, dth0, y.pr, y.pth}, dr0, L.k1f, Hs);
        L.k32_ok = true;
    }
    const StateF k1 = L.k1f;
    StateF k2, k3, k4, k5, k6, k7, ys;
#define TT_FS(dst, er, et, ep, eq)                         \
    ys.r = fmaf(h, (er), y.r);                             \
    ys.th = fmaf(h, (et), dth0);                           \
    ys.pr = fmaf(h, (ep), y.pr);                           \
    ys.pth = fmaf(h, (eq), y.pth);                         \
    kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, ys, fmaf(h, (er), dr0), dst, Hs);
#define TT_C2(f) ((float)a21 * k1.f)
#define TT_C3(f) fmaf((float)a32, k2.f, (float)a31 * k1.f)
#define TT_C4(f) fmaf((float)a43, k3.f, fmaf((float)a42, k2.f, (float)a41 * k1.f))
#define TT_C5(f) fmaf((float)a54, k4.f, fmaf((float)a53, k3.f, fmaf((float)a52, k2.f, (float)a51 * k1.f)))
#define TT_C6(f) \
    fmaf((float)a65, k5.f, fmaf((float)a64, k4.f, fmaf((float)a63, k3.f, fmaf((float)a62, k2.f, (float)a61 * k1.f))))
#define TT_C7(f) \
    fmaf((float)b6, k6.f, fmaf((float)b5, k5.f, fmaf((float)b4, k4.f, fmaf((float)b3, k3.f, (float)b1 * k1.f))))
    TT_FS(k2, TT_C2(r), TT_C2(th), TT_C2(pr), TT_C2(pth))
    TT_FS(k3, TT_C3(r), TT_C3(th), TT_C3(pr), TT_C3(pth))
    TT_FS(k4, TT_C4(r), TT_C4(th), TT_C4(pr), TT_C4(pth))
    TT_FS(k5, TT_C5(r), TT_C5(th), TT_C5(pr), TT_C5(pth))
    TT_FS(k6, TT_C6(r), TT_C6(th), TT_C6(pr), TT_C6(pth))
    StateF inc;
    inc.r = h * TT_C7(r);
    inc.th = h * TT_C7(th);
    inc.pr = h * TT_C7(pr);
    inc.pth = h * TT_C7(pth);
    StateF yn = {y.r + inc.r, y.th + inc.th, y.pr + inc.pr, y.pth + inc.pth};
    float Hn;
    kerr_flow32(L.Mf, L.a2f, L.rpmf, L.Rf, StateF{yn.r, dth0 + inc.th, yn.pr, yn.pth}, dr0 + inc.r, k7, Hn);
#define TT_E(f) \
    h * fmaf((float)e7, k7.f, fmaf((float)e6, k6.f, fmaf((float)e5, k5.f, fmaf((float)e4, k4.f, \
             fmaf((float)e3, k3.f, (float)e1 * k1.f)))))
    float err2;
    double err64 = 0.0;
    State y64n;
    if constexpr (PREC == 4) {
        // FP64 norm from the FP32 error terms and the FP64 states
        y64n = State{L.y.r + (double)inc.r, L.y.th + (double)inc.th, L.y.pr + (double)inc.pr,
                     L.y.pth + (double)inc.pth};
        const State e64 = State{(double)TT_E(r), (double)TT_E(th), (double)TT_E(pr), (double)TT_E(pth)};
        err64 = err_norm2(L.y, y64n, e64, sol.atol, sol.rtol, 1.0);
        err2 = nan_bits(err64) ? __int_as_float(0x7fffffff) : (err64 <= 1.0 ? 0.0f : 2.0f);
    } else {
        const float atol = (float)sol.atol, rtol = (float)sol.rtol;
        err2 = sq_ratio32(TT_E(r), y.r, yn.r, atol, rtol);
        err2 += sq_ratio32(TT_E(th), y.th, yn.th, atol, rtol);
        err2 += sq_ratio32(TT_E(pr), y.pr, yn.pr, atol, rtol);
        err2 += sq_ratio32(TT_E(pth), y.pth, yn.pth, atol, rtol);
        err2 *= 0.25f;
    }
#undef TT_E
#undef TT_FS
#undef TT_C2
#undef TT_C3
#undef TT_C4
#undef TT_C5
#undef TT_C6
#undef TT_C7
    if (isnan(err2) || !isfinite(yn.r) || !isfinite(yn.th) || !isfinite(yn.pr) || !isfinite(yn.pth)) return 4;
    if (err2 <= 1.0f) {
        L.steps++;
        bool captured, escaped;
        if (ACC == 0) {
            if constexpr (PREC != 4) {
                y64n.r = L.y.r + (double)inc.r;
                y64n.th = L.y.th + (double)inc.th;
                y64n.pr = L.y.pr + (double)inc.pr;
                y64n.pth = L.y.pth + (double)inc.pth;
            }
            if (d.disk && ((L.y.th <= kHalfPi) != (y64n.th <= kHalfPi))) note_crossing<0, PREC>(L, L.y, sol);
            L.y = y64n;
            captured = y64n.r < d.r_capture;
            escaped = y64n.r > d.r_escape;
        } else {
            StateF hi = yhi, lo = L.lo;
            pair_add(hi.r, lo.r, inc.r);
            pair_add(hi.th, lo.th, inc.th);
            pair_add(hi.pr, lo.pr, inc.pr);
            pair_add(hi.pth, lo.pth, inc.pth);
            // pi/2 as an FP32 pair
            const float pi2h = 1.57079637f, pi2l = -4.37113883e-08f;
            const bool s0 = !pair_below(pi2h, pi2l, yhi.th, L.lo.th);     // theta <= pi/2 before
            const bool s1 = !pair_below(pi2h, pi2l, hi.th, lo.th);        // and after
            if (d.disk && s0 != s1) note_crossing<0, PREC>(L, pair_to64(yhi, L.lo), sol);
            yhi = hi;
            L.lo = lo;
            captured = pair_below(hi.r, lo.r, L.caph, L.capl);
            escaped = hi.r > L.escf;
        }
        L.lamf += h;
        L.k1f = k7;
        L.k64_ok = false;
        L.kdf_ok = false;
        if (captured) return 1;
        if (escaped) return 0;
        if constexpr (PREC == 4) {
            L.hf = (float)((double)h * fmin(L.last_rej ? 1.0 : 10.0, fmax(0.2, step_factor(err64))));
        } else {
            float fac = (err2 < 1e-30f) ? 10.0f : 0.9f * __powf(err2, -0.1f);
            fac = fminf(L.last_rej ? 1.0f : 10.0f, fmaxf(0.2f, fac));
            L.hf = h * fac;
        }
        L.last_rej = false;
    } else {
        L.rejects++;
        if constexpr (PREC == 4) L.hf = (float)((double)h * fmax(0.2, step_factor(err64)));
        else L.hf = h * fmaxf(0.2f, 0.9f * __powf(err2, -0.1f));
        L.last_rej = true;
    }
    return -1;
}

// A zone step of the prescribed split (PREC 4): the FP64 Dormand-Prince step
// from the FP64 state, with the FSAL flow, sin and cos taken afresh after FP32
// steps; the step size and affine parameter are carried over from and back to
// the FP32 steps.
__device__ __forceinline__ int step_zone64_split(Lane& L, const SolverDesc& sol) {
    if (!L.k64_ok) {
        double H;
        flow64<0>(*L.d, L.kk, L.R, L.y, L.k1, H);
        sincos(L.y.th, &L.s0, &L.c0);
        L.k64_ok = true;
    }
    L.h = (double)L.hf;
    L.lam = (double)L.lamf;
    const int code = step_ray64<0, 4>(L, sol);
    L.hf = (float)L.h;
    L.lamf = (float)L.lam;
    L.k32_ok = false;
    L.kdf_ok = false;
    return code;
}

// ---------------------------------------------------------------------------
// One Dormand-Prince step in double-float (~48 bits) on the FP32 pipe: the
// mixed paths' steps near the horizon and the axis (FULL false), and every step
// of the double-float path (FULL true).  The flow is always evaluated in
// double-float at stage points held in double-float, and the new state is
// accumulated in double-float.  FULL forms the stage sums sum_j a_ij k_j in
// double-float with double-float coefficients; otherwise the (small) stage
// increments h sum_j a_ij k_j are formed in FP32 from the high parts and the
// fifth-order sum uses FP32 coefficients -- a perturbation of ~6e-8 of a step's
// change, far below the mixed paths' tolerance.  The error norm and the
// step-size control run in FP32.  ACC 0: the state is the FP64 L.y;
// ACC 1: the FP32 pair (yhi, L.lo).
// ---------------------------------------------------------------------------
template <int METRIC, int ACC, bool FULL>
__device__ int step_ray_df(Lane& L, StateF& yhi, const SolverDesc& sol) {
    constexpr int PREC = FULL ? 3 : ACC + 1;
    const ImageDesc& d = *L.d;
    if ((long long)L.steps + (long long)L.rejects >= sol.max_steps) return 2;
    const float h = L.hf;
    const float hmin = (sol.h_min > 0.0) ? (float)sol.h_min : 1e-14f * fmaxf(1.0f, L.lamf);
    if (h < hmin) return 3;
    using namespace dp;
    KerrDF kd;
    RayDF rd;
    if constexpr (FULL) {
        kd = L.kdf;
        rd = L.rdf;
    } else {
        kd = make_kerr_df(L.kk);
        rd = make_ray_df(L.R);
    }
    StateDF y;
    if constexpr (ACC == 0) {
        y = StateDF{df_of(L.y.r), df_of(L.y.th), df_of(L.y.pr), df_of(L.y.pth)};
    } else {
        y = StateDF{DF{yhi.r, L.lo.r}, DF{yhi.th, L.lo.th}, DF{yhi.pr, L.lo.pr}, DF{yhi.pth, L.lo.pth}};
    }
    DF Hs;
    StateDF k1;
    if (!L.kdf_ok) {
        flow_df<METRIC>(d, kd, rd, y, k1, Hs);
    } else {
        k1 = StateDF{DF{L.k1f.r, L.k1lo.r}, DF{L.k1f.th, L.k1lo.th}, DF{L.k1f.pr, L.k1lo.pr},
                     DF{L.k1f.pth, L.k1lo.pth}};
    }
    StateDF k2, k3, k4, k5, k6, k7, ys, yn;
#define TT_DS(dst, S)                                                                 \
    ys.r = S(r);                                                                      \
    ys.th = S(th);                                                                    \
    ys.pr = S(pr);                                                                    \
    ys.pth = S(pth);                                                                  \
    flow_df<METRIC>(d, kd, rd, ys, dst, Hs);
    if constexpr (FULL) {
        constexpr DF A21 = df_const(a21), A31 = df_const(a31), A32 = df_const(a32);
        constexpr DF A41 = df_const(a41), A42 = df_const(a42), A43 = df_const(a43);
        constexpr DF A51 = df_const(a51), A52 = df_const(a52), A53 = df_const(a53), A54 = df_const(a54);
        constexpr DF A61 = df_const(a61), A62 = df_const(a62), A63 = df_const(a63), A64 = df_const(a64),
                     A65 = df_const(a65);
        constexpr DF B1 = df_const(b1), B3 = df_const(b3), B4 = df_const(b4), B5 = df_const(b5), B6 = df_const(b6);
#define TT_F2(f) df_add(y.f, df_mul_f(df_mul(k1.f, A21), h))
#define TT_F3(f) df_add(y.f, df_mul_f(dot_end(dot_next(dot_first(A31, k1.f), A32, k2.f)), h))
#define TT_F4(f) \
    df_add(y.f, df_mul_f(dot_end(dot_next(dot_next(dot_first(A41, k1.f), A42, k2.f), A43, k3.f)), h))
#define TT_F5(f)                                                                                         \
    df_add(y.f, df_mul_f(dot_end(dot_next(dot_next(dot_next(dot_first(A51, k1.f), A52, k2.f), A53, k3.f), \
                                          A54, k4.f)), h))
#define TT_F6(f)                                                                                         \
    df_add(y.f, df_mul_f(dot_end(dot_next(dot_next(dot_next(dot_next(dot_first(A61, k1.f), A62, k2.f),   \
                                                            A63, k3.f), A64, k4.f), A65, k5.f)), h))
#define TT_F7(f)                                                                                         \
    df_add(y.f, df_mul_f(dot_end(dot_next(dot_next(dot_next(dot_next(dot_first(B1, k1.f), B3, k3.f),     \
                                                            B4, k4.f), B5, k5.f), B6, k6.f)), h))
        TT_DS(k2, TT_F2)
        TT_DS(k3, TT_F3)
        TT_DS(k4, TT_F4)
        TT_DS(k5, TT_F5)
        TT_DS(k6, TT_F6)
        yn = StateDF{TT_F7(r), TT_F7(th), TT_F7(pr), TT_F7(pth)};
#undef TT_F2
#undef TT_F3
#undef TT_F4
#undef TT_F5
#undef TT_F6
#undef TT_F7
    } else {
#define TT_G2(f) df_add_f(y.f, h * ((float)a21 * k1.f.hi))
#define TT_G3(f) df_add_f(y.f, h * fmaf((float)a32, k2.f.hi, (float)a31 * k1.f.hi))
#define TT_G4(f) df_add_f(y.f, h * fmaf((float)a43, k3.f.hi, fmaf((float)a42, k2.f.hi, (float)a41 * k1.f.hi)))
#define TT_G5(f)                                                                                         \
    df_add_f(y.f, h * fmaf((float)a54, k4.f.hi, fmaf((float)a53, k3.f.hi, fmaf((float)a52, k2.f.hi,       \
                                                                             (float)a51 * k1.f.hi))))
#define TT_G6(f)                                                                                         \
    df_add_f(y.f, h * fmaf((float)a65, k5.f.hi, fmaf((float)a64, k4.f.hi, fmaf((float)a63, k3.f.hi,      \
                                               fmaf((float)a62, k2.f.hi, (float)a61 * k1.f.hi)))))
#define TT_G7(f)                                                                                         \
    df_add(y.f, df_mul_f(df_add(df_mul_f(k6.f, (float)b6), df_add(df_mul_f(k5.f, (float)b5),             \
           df_add(df_mul_f(k4.f, (float)b4), df_add(df_mul_f(k3.f, (float)b3), df_mul_f(k1.f, (float)b1))))), h))
        TT_DS(k2, TT_G2)
        TT_DS(k3, TT_G3)
        TT_DS(k4, TT_G4)
        TT_DS(k5, TT_G5)
        TT_DS(k6, TT_G6)
        yn = StateDF{TT_G7(r), TT_G7(th), TT_G7(pr), TT_G7(pth)};
#undef TT_G2
#undef TT_G3
#undef TT_G4
#undef TT_G5
#undef TT_G6
#undef TT_G7
    }
#undef TT_DS
    DF Hn;
    flow_df<METRIC>(d, kd, rd, yn, k7, Hn);
    // The error estimate h sum_i e_i k_i is a small difference of nearly equal
    // stage flows (sum_i e_i = 0): at tolerances near 1e-10 it is formed in
    // double-float with double-float weights (FULL), else FP32 rounding noise in
    // it, not the truncation error, would set the step size.
#define TT_E32(f)                                                                                       \
    h * fmaf((float)e7, k7.f.hi, fmaf((float)e6, k6.f.hi, fmaf((float)e5, k5.f.hi, fmaf((float)e4, k4.f.hi, \
             fmaf((float)e3, k3.f.hi, (float)e1 * k1.f.hi)))))
#define TT_EDF(f)                                                                                       \
    (h * dot_end(dot_next(dot_next(dot_next(dot_next(dot_next(dot_first(E1, k1.f), E3, k3.f), E4, k4.f),   \
                                            E5, k5.f), E6, k6.f), E7, k7.f)).hi)
    float er, eth, epr, epth;
    if constexpr (FULL) {
        constexpr DF E1 = df_const(e1), E3 = df_const(e3), E4 = df_const(e4), E5 = df_const(e5),
                     E6 = df_const(e6), E7 = df_const(e7);
        er = TT_EDF(r);
        eth = TT_EDF(th);
        epr = TT_EDF(pr);
        epth = TT_EDF(pth);
    } else {
        er = TT_E32(r);
        eth = TT_E32(th);
        epr = TT_E32(pr);
        epth = TT_E32(pth);
    }
#undef TT_E32
#undef TT_EDF
    const float atol = (float)sol.atol, rtol = (float)sol.rtol;
    float err2 = sq_ratio32(er, y.r.hi, yn.r.hi, atol, rtol);
    err2 += sq_ratio32(eth, y.th.hi, yn.th.hi, atol, rtol);
    err2 += sq_ratio32(epr, y.pr.hi, yn.pr.hi, atol, rtol);
    err2 += sq_ratio32(epth, y.pth.hi, yn.pth.hi, atol, rtol);
    err2 *= 0.25f;
    if (isnan(err2) || !isfinite(yn.r.hi) || !isfinite(yn.th.hi) || !isfinite(yn.pr.hi) || !isfinite(yn.pth.hi))
        return 4;
    if (err2 <= 1.0f) {
        L.steps++;
        const float pi2h = 1.57079637f, pi2l = -4.37113883e-08f;      // pi/2 as an FP32 pair
        const bool s0 = !pair_below(pi2h, pi2l, y.th.hi, y.th.lo);      // theta <= pi/2 before
        const bool s1 = !pair_below(pi2h, pi2l, yn.th.hi, yn.th.lo);    // and after
        if (d.disk && s0 != s1) {
            const State yc = (ACC == 0) ? L.y : pair_to64(yhi, L.lo);
            note_crossing<METRIC, PREC>(L, yc, sol);
        }
        if constexpr (ACC == 0) {
            L.y = State{df_to64(yn.r), df_to64(yn.th), df_to64(yn.pr), df_to64(yn.pth)};
        } else {
            yhi = StateF{yn.r.hi, yn.th.hi, yn.pr.hi, yn.pth.hi};
            L.lo = StateF{yn.r.lo, yn.th.lo, yn.pr.lo, yn.pth.lo};
        }
        L.k1f = StateF{k7.r.hi, k7.th.hi, k7.pr.hi, k7.pth.hi};
        L.k1lo = StateF{k7.r.lo, k7.th.lo, k7.pr.lo, k7.pth.lo};
        L.kdf_ok = true;
        L.k32_ok = true;
        L.k64_ok = false;
        L.lamf += h;
        L.hmaxf = fmaxf(L.hmaxf, fabsf(Hn.hi));
        if (pair_below(yn.r.hi, yn.r.lo, L.caph, L.capl)) return 1;
        if (yn.r.hi > L.escf) return 0;
        float fac = (err2 < 1e-30f) ? 10.0f : 0.9f * __powf(err2, -0.1f);
        fac = fminf(L.last_rej ? 1.0f : 10.0f, fmaxf(0.2f, fac));
        L.hf = h * fac;
        L.last_rej = false;
    } else {
        L.rejects++;
        L.kdf_ok = true;                        // k1 still belongs to the unchanged state
        L.k32_ok = true;
        L.k1f = StateF{k1.r.hi, k1.th.hi, k1.pr.hi, k1.pth.hi};
        L.k1lo = StateF{k1.r.lo, k1.th.lo, k1.pr.lo, k1.pth.lo};
        L.hf = h * fmaxf(0.2f, 0.9f * __powf(err2, -0.1f));
        L.last_rej = true;
    }
    return -1;
}

// A double-float-path step near the horizon or the axis of a tabulated metric,
// in FP64: there the interpolated D = g_tt g_phiphi - g_tphi^2 (-Delta sin^2
// theta for Kerr) goes to zero, and W / D (and its derivatives) lose the
// double-float's digits in proportion; the FP32-pair state, step size and
// affine parameter are carried over exactly and back.
template <int METRIC>
__device__ int step_zone64(Lane& L, StateF& yhi, const SolverDesc& sol) {
    L.y = pair_to64(yhi, L.lo);
    if (!L.k64_ok) {
        double H;
        flow64<METRIC>(*L.d, L.kk, L.R, L.y, L.k1, H);
        L.k64_ok = true;
    }
    L.h = (double)L.hf;
    L.lam = (double)L.lamf;
    const int code = step_ray64<METRIC, 3>(L, sol);
    split_state(L.y, yhi, L.lo);
    L.hf = (float)L.h;
    L.lamf = (float)L.lam;
    L.kdf_ok = false;
    return code;
}

// Steps of the double-float table path that run in FP64 (the zones of the
// solver's fp64_radius_factor and fp64_pole_sin).
__device__ __forceinline__ bool in_zone(const Lane& L, const StateF& yhi) {
    const float axis = fabsf(fmaf(-rintf(yhi.th * 0.318309886f), 3.14159274f, yhi.th));
    return (yhi.r < L.fp64f) || (axis < L.thpf);
}

// FP64 |H| at the lane's current state (mixed-path monitor).
template <int ACC>
__device__ __forceinline__ void check_h64(Lane& L, const StateF& yhi) {
    const State y = (ACC == 0) ? L.y : pair_to64(yhi, L.lo);
    L.hmax = fmax(L.hmax, fabs(kerr_h64(L.kk, L.R, y)));
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

// Lane states of the warp loop.
enum : int { kIdle = 0, kRun = 1, kDone = 2 };


// PREC 0: FP64.  PREC 1: mixed with FP64 accumulation.  PREC 2: mixed with the
// compensated FP32-pair accumulation.  PREC 3: double-float.  PREC 4: mixed
// with the prescribed FP64 split (norm, zone steps, refinement).  METHOD (FP64
// only): 0 Dormand-Prince, 1 Cash-Karp, 2 Fehlberg, 3 Gragg-Bulirsch-Stoer,
// 4 Verlet.  solc: the solver settings of the mixed paths' near-critical rays.
//
// Mixed paths with a critical band: the warps of one SM in crit_stride scan the rays
// (queue[1]) for near-critical ones and traces those in double-float, with
// whole warps of them; the other warps take the rays from queue[0], skipping
// the near-critical ones (the same test picks them out).  A warp whose queue
// is drained takes the other one.  The long double-float rays thus start first
// and overlap with the bulk of the image.
template <int METRIC, int PREC, int METHOD = 0>
__device__ __forceinline__ void trace_loop(const ImageDesc* descs, int n_desc, long long total,
                                           const SolverDesc& sol, const SolverDesc& solc, const TuneParams& tp,
                                           unsigned long long* queue) {
    static_assert(PREC == 0 || METHOD == 0, "the mixed and double-float paths step with Dormand-Prince");
    constexpr int ACC = (PREC == 2 || PREC == 3) ? 1 : 0;
    constexpr bool MIX = (PREC == 1 || PREC == 2 || PREC == 4);
    if constexpr (PREC != 0) {
        df_sincos_table(s_df_tab);
        if constexpr (METRIC == 1) df_log_table(s_df_ln);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    Lane L;
    L.pend = false;
    L.crit = false;
    StateF yhi = {0.0f, 0.0f, 0.0f, 0.0f};   // pair accumulator: hi parts
    int st = kIdle;
    bool drained = false;
    // the warps of one SM in crit_stride start with the scan for near-critical
    // rays, the others with the bulk (so that an SM runs the double-float code
    // or the FP32 code, not both, and its instruction cache holds one of them);
    // a warp whose queue is drained and whose lanes are all written takes the
    // other queue, until both are drained (warp-uniform)
    const float band = (float)sol.crit_band;
    const bool use_crit = MIX && band > 0.0f;
    unsigned smid = 0;
    if (use_crit) asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    bool crit_phase = use_crit && (smid % (unsigned)tp.crit_stride) == 0;
    bool drained_c = !use_crit;
    int wait64 = 0;
    unsigned iter = 0;
    // crossings of near-critical rays are refined as on the double-float path
    auto refine = [&]() {
        if constexpr (MIX) {
            if (L.crit) {
                refine_pending<METRIC, 3>(L, solc);
                return;
            }
        }
        refine_pending<METRIC, PREC, METHOD>(L, sol);
    };
    for (;;) {
        // ---- refill phase: flush finished rays, start new ones -------------
        // (near-critical rays differ widely in length: their warps refill at a
        // threshold of their own)
        const int n_free = __popc(__ballot_sync(kFull, st != kRun));
        const bool more = crit_phase ? !drained_c : !drained;
        const int refill_at = crit_phase ? tp.crit_refill : tp.refill;
        if (n_free > 0 && (n_free >= refill_at || n_free == 32) && (more || __any_sync(kFull, st == kDone))) {
            if (st != kIdle && L.pend) refine();
            if (st == kDone) {
                if (MIX && !L.crit) check_h64<ACC>(L, yhi);
                write_final(L, L.code, sol);
                st = kIdle;
            }
            if (crit_phase) {
                // fill the idle lanes with near-critical rays: each round tests one
                // queue entry per idle lane (bounded: every round consumes entries)
                while (!drained_c) {
                    const unsigned idle = __ballot_sync(kFull, st == kIdle);
                    if (!idle) break;
                    const int n_idle = __popc(idle);
                    unsigned long long base = 0;
                    if (lane == 0) base = atomicAdd(queue + 1, (unsigned long long)n_idle);
                    base = __shfl_sync(kFull, base, 0);
                    if (base + (unsigned long long)n_idle >= (unsigned long long)total) drained_c = true;
                    if (st == kIdle) {
                        const long long rid = (long long)base + __popc(idle & ((1u << lane) - 1u));
                        if (rid < total) {
                            const int im = (n_desc == 1) ? 0 : find_image(descs, n_desc, rid);
                            const ImageDesc* dp = descs + im;
                            const long long q = tile_pixel(*dp, rid - dp->ray_begin);
                            if (near_critical(*dp, q, band) && init_ray<METRIC>(L, dp, q, solc, true)) {
                                st = kRun;
                                L.crit = true;
                                if (ACC == 1) split_state(L.y, yhi, L.lo);
                            }
                        }
                    }
                }
            } else if (!drained) {
                const unsigned idle = __ballot_sync(kFull, st == kIdle);
                const int n_idle = __popc(idle);
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(queue, (unsigned long long)n_idle);
                base = __shfl_sync(kFull, base, 0);
                if (base + (unsigned long long)n_idle >= (unsigned long long)total) drained = true;
                if (st == kIdle) {
                    const long long rid = (long long)base + __popc(idle & ((1u << lane) - 1u));
                    if (rid < total) {
                        const int im = (n_desc == 1) ? 0 : find_image(descs, n_desc, rid);
                        const ImageDesc* dp = descs + im;
                        const long long q = tile_pixel(*dp, rid - dp->ray_begin);
                        // near-critical rays were traced in the scan
                        const bool skip = MIX && band > 0.0f && near_critical(*dp, q, band);
                        if (!skip && init_ray<METRIC>(L, dp, q, sol)) {
                            st = kRun;
                            L.crit = false;
                            if (ACC == 1) split_state(L.y, yhi, L.lo);
                        }
                    }
                }
            }
        }
        const unsigned running = __ballot_sync(kFull, st == kRun);
        if (!running) {
            if (__any_sync(kFull, st == kDone)) continue;          // written by the next refill
            // every lane idle: once this queue is drained, take the other one
            if (drained && drained_c) break;
            if (crit_phase ? drained_c : drained) crit_phase = !crit_phase;
            continue;
        }
        ++iter;
        // ---- step phases ---------------------------------------------------
        if constexpr (PREC == 3 && METRIC == 1) {
            // FP64 zone steps, batched across the warp like the mixed paths'
            // extended-precision steps (a warp runs the FP64 step's code once for
            // all its zone lanes, not once per straggler)
            const bool want64 = (st == kRun) && in_zone(L, yhi);
            const unsigned w64 = __ballot_sync(kFull, want64);
            if (w64) {
                const bool run64 = (__popc(w64) >= tp.fp64_batch) || (w64 == running) || (wait64 >= tp.fp64_wait);
                wait64 = run64 ? 0 : wait64 + 1;
                if (run64 && want64) {
                    const int code = step_zone64<METRIC>(L, yhi, sol);
                    if (code >= 0) {
                        L.code = code;
                        st = kDone;
                    }
                }
            }
            if (st == kRun && !want64) {
                const int code = step_ray_df<METRIC, 1, true>(L, yhi, sol);
                if (code >= 0) {
                    L.code = code;
                    st = kDone;
                }
            }
        } else if constexpr (PREC == 3) {
            if (st == kRun) {
                const int code = step_ray_df<METRIC, 1, true>(L, yhi, sol);
                if (code >= 0) {
                    L.code = code;
                    st = kDone;
                }
            }
        } else if constexpr (PREC == 0) {
            if (st == kRun) {
                const int code = step_ray64<METRIC, 0, METHOD>(L, sol);
                if (code >= 0) {
                    L.code = code;
                    st = kDone;
                }
            }
        } else if (crit_phase) {
            // near-critical rays: every step in double-float, as on the double-float path
            if (st == kRun) {
                const int code = step_ray_df<METRIC, ACC, true>(L, yhi, solc);
                if (code >= 0) {
                    L.code = code;
                    st = kDone;
                }
            }
        } else {
            bool want64 = false;
            if (st == kRun) {
                // extended precision near the horizon and near the axis (the
                // coordinate singularities); the distance to the axis is
                // |theta - m pi| for the nearest integer m, since a ray through the
                // axis continues with theta outside (0, pi)
                const float thf = (ACC == 0) ? (float)L.y.th : yhi.th;
                const float rf = (ACC == 0) ? (float)L.y.r : yhi.r;
                const float axis = fabsf(fmaf(-rintf(thf * 0.318309886f), 3.14159274f, thf));
                want64 = (rf < L.fp64f) || (axis < L.thpf);
            }
            const unsigned w64 = __ballot_sync(kFull, want64);
            if (w64) {
                const bool run64 = (__popc(w64) >= tp.fp64_batch) || (w64 == running) || (wait64 >= tp.fp64_wait);
                wait64 = run64 ? 0 : wait64 + 1;
                if (run64 && want64) {
                    // the zone step: FP64 on the prescribed split, else double-float on
                    // the FP32 pipe
                    int code;
                    if constexpr (PREC == 4) code = step_zone64_split(L, sol);
                    else code = step_ray_df<METRIC, ACC, false>(L, yhi, sol);
                    if (code >= 0) {
                        L.code = code;
                        st = kDone;
                    }
                }
            }
            if (st == kRun && !want64) {
                const int code = step_ray32<PREC>(L, yhi, sol);
                if (code >= 0) {
                    L.code = code;
                    st = kDone;
                }
            }
        }
        // ---- batched crossing refinement -----------------------------------
        const unsigned pend = __ballot_sync(kFull, st == kRun && L.pend);
        if (pend && __popc(pend) >= tp.crossing_batch) {
            if (st == kRun && L.pend) refine();
        }
        // ---- FP64 |H| monitor (mixed) --------------------------------------
        if (MIX && (iter % (unsigned)tp.monitor_period) == 0) {
            if (st == kRun && !L.crit) check_h64<ACC>(L, yhi);
        }
    }
}

int sm_count();

// Persistent launch: as many blocks as fit (or blocks_per_sm) on every SM, no
// more than the rays need.
template <int N, typename K>
cudaError_t launch_persistent(K kern, int block, int blocks_per_sm, const LaunchParams<N>& p, cudaStream_t st) {
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

// Fill the launch parameters (defaults for zero tune fields).
template <int N>
void fill_params(LaunchParams<N>& p, const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                 const LaunchShape& shape, unsigned long long* queue) {
    p.sol = sol;
    p.solc = sol;                       // near-critical rays of the mixed paths
    p.solc.rtol = sol.crit_rtol;
    p.solc.atol = sol.crit_atol;
    p.n_desc = n;
    // defaults (the autotuner's choices on GB300): refill once every lane of the
    // warp is free (initial data and the final record then run with full lanes),
    // refine crossings in batches of 16 (FP64) or 32 lanes, and run the mixed
    // paths' zone steps once every running lane needs one (or after fp64_wait)
    const bool mixed = sol.precision != 0;
    p.tune.refill = shape.refill > 0 ? shape.refill : 32;
    p.tune.crossing_batch = shape.crossing_batch > 0 ? shape.crossing_batch : (mixed ? 32 : 16);
    // (the double-float table path's FP64 zone steps measured fastest unbatched)
    p.tune.fp64_batch = shape.fp64_batch > 0 ? shape.fp64_batch : (sol.precision == 3 ? 1 : 32);
    p.tune.monitor_period = shape.monitor_period > 0 ? shape.monitor_period : 32;
    p.tune.fp64_wait = shape.fp64_wait > 0 ? shape.fp64_wait : 64;
    p.tune.crit_stride = shape.crit_stride > 0 ? shape.crit_stride : 1;
    p.tune.crit_refill = shape.crit_refill > 0 ? shape.crit_refill : 32;
    p.total = total;
    p.queue = queue;
    for (int i = 0; i < n; ++i) p.desc[i] = descs[i];
}

// Mixed-precision launches (tt_kernel_mixed.cu, the prescribed split in
// tt_kernel_split.cu) and double-float launches (tt_kernel_df.cu).
cudaError_t launch_mixed(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                         const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream);
cudaError_t launch_split(const ImageDesc* descs, int n, long long total, const SolverDesc& sol,
                         const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream);
cudaError_t launch_df(const ImageDesc* descs, int n, long long total, int metric_mode, const SolverDesc& sol,
                      const LaunchShape& shape, unsigned long long* queue, cudaStream_t stream);

}  // namespace tt

// tt_device.cuh -- device arithmetic of the geodesic tracer (sm_103a).
//
// One ray per thread.  The state carried through the integrator is the
// dynamical core (r, theta, p_r, p_theta) of the paper's 8-dimensional
// phase-space array (Sec. 2.1): p_t and p_phi are constants of the motion and
// t, phi never feed back into the flow, so they are not integrated.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tt_internal.h"

namespace tt {

constexpr double kHalfPi = 1.5707963267948966;   // binary64 pi/2

// Comparisons of doubles on the integer pipe (the FP64 pipe is the FP64
// path's bound, and a comparison there costs an issue slot like an FMA):
// IEEE-754 orders non-negative doubles as their bit patterns read as signed
// 64-bit integers, and every negative double reads as a negative integer, so
// x < y (x <= y) for y >= 0 and any non-NaN x is the integer comparison.
__device__ __forceinline__ bool lt_pos(double x, double y) { return __double_as_longlong(x) < __double_as_longlong(y); }
__device__ __forceinline__ bool le_pos(double x, double y) { return __double_as_longlong(x) <= __double_as_longlong(y); }
// |x| below a threshold given by the high 32 bits of a positive double.
__device__ __forceinline__ bool abs_below_hi(double x, int hi) { return (__double2hiint(x) & 0x7fffffff) < hi; }
constexpr int kHi0p01 = 0x3F847AE1;    // high word of 0.01 (the threshold is 0.01 - 3e-11)
constexpr int kHi0p1 = 0x3FB99999;     // high word of 0.1 (the threshold is 0.1 - 4e-10)

// ---------------------------------------------------------------------------
// Reciprocal: the SFU's approximate double reciprocal y refined by one step of
// the third-order (Halley-type) iteration y <- y (1 + e + e^2), e = 1 - x y:
// the result is (1/x)(1 - e^3), so the approximation's relative error cubes
// (two Newton-Raphson steps square it twice; this takes three fused
// multiply-adds instead of four) and it is within about one ulp of 1/x for
// normal x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rcp64(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// Per-ray constants of the (time-reversed) photon.
struct RayConst {
    double pt, pph;       // p_t, p_phi
    double apph;          // a p_phi
    double pph2;          // p_phi^2
    double a2pt2;         // a^2 p_t^2
    double c0;            // 2 a p_t p_phi
    double pt4;           // 4 p_t
    double pt2;           // 2 p_t
};

__device__ __forceinline__ RayConst make_ray_const(double a, double pt, double pph) {
    RayConst R;
    R.pt = pt;
    R.pph = pph;
    R.apph = a * pph;
    R.pph2 = pph * pph;
    R.a2pt2 = a * a * pt * pt;
    R.c0 = 2.0 * a * pt * pph;
    R.pt4 = 4.0 * pt;
    R.pt2 = 2.0 * pt;
    return R;
}

// Per-spacetime constants of the closed-form Kerr flow.
struct KerrK {
    double M, a, a2, twoM, fourA2;
};

__device__ __forceinline__ KerrK make_kerr(double M, double a) {
    KerrK k;
    k.M = M;
    k.a = a;
    k.a2 = a * a;
    k.twoM = 2.0 * M;
    k.fourA2 = 4.0 * a * a;
    return k;
}

struct State {
    double r, th, pr, pth;
};

// ---------------------------------------------------------------------------
// Kerr flow.  H = K / (2 Sigma) with Carter's separated form of g^{mu nu} p p,
//   K = Delta p_r^2 + p_th^2 + (p_phi + a p_t sin^2)^2 / sin^2
//       - ((r^2 + a^2) p_t + a p_phi)^2 / Delta,
// so dr = Delta p_r / Sigma, dth = p_th / Sigma and
//   dp_r  = -(dK/dr  - 4 r H) / (2 Sigma),
//   dp_th = -(dK/dth + 4 a^2 sin cos H) / (2 Sigma),
// Hamilton's equations of Sec. 2.1 exactly (the H terms keep the flow exact
// off the constraint surface).  With A = (r^2 + a^2) p_t + a p_phi and
// H2 = 2H = K / Sigma the two forces are evaluated as
//   dp_r  = [r (H2 + 2 p_t A/Delta) - (r - M)((A/Delta)^2 + p_r^2)] / Sigma,
//   dp_th = -sin cos [a^2 H2 + a^2 p_t^2 - p_phi^2 / sin^4] / Sigma
// (the same expressions regrouped: 4 fewer FP64 operations per evaluation).
// One reciprocal serves 1/Sigma, 1/Delta and 1/sin^2.
// ---------------------------------------------------------------------------
// The flow given s = sin(theta), c = cos(theta) of the state.
__device__ __forceinline__ void kerr_flow64_sc(const KerrK& k, const RayConst& R, const State& y, double s,
                                               double c, State& f, double& H) {
    const double r = y.r;
    const double s2 = s * s, c2 = c * c, sc = s * c;
    const double r2 = r * r;
    const double Sig = fma(k.a2, c2, r2);
    const double Del = fma(r, r - k.twoM, k.a2);
    const double A = fma(fma(r, r, k.a2), R.pt, R.apph);
    const double SD = Sig * Del;
    const double inv = rcp64(SD * s2);
    const double w = inv * s2;                       // 1 / (Sigma Delta)
    const double iS = w * Del;                       // 1 / Sigma
    const double iD = w * Sig;                       // 1 / Delta
    const double u = inv * SD;                       // 1 / sin^2
    const double pr2 = y.pr * y.pr;
    const double AiD = A * iD;
    double K = fma(R.a2pt2, s2, R.c0);
    K = fma(R.pph2, u, K);
    K = fma(y.pth, y.pth, K);
    K = fma(Del, pr2, K);
    K = fma(-A, AiD, K);
    const double H2 = K * iS;
    H = 0.5 * H2;
    const double q1 = fma(R.pt2, AiD, H2);
    const double q2 = fma(AiD, AiD, pr2);
    const double t1 = fma(-R.pph2, u * u, R.a2pt2);
    const double t2 = fma(k.a2, H2, t1);
    f.r = (Del * y.pr) * iS;
    f.th = y.pth * iS;
    f.pr = fma(r, q1, -((r - k.M) * q2)) * iS;
    f.pth = -(sc * iS) * t2;
}

__device__ __forceinline__ void kerr_flow64(const KerrK& k, const RayConst& R, const State& y, State& f,
                                            double& H) {
    double s, c;
    sincos(y.th, &s, &c);
    kerr_flow64_sc(k, R, y, s, c, f, H);
}

// sin and cos of theta from those of a nearby theta0 (the start of the step):
// angle addition with the Taylor series of d = theta - theta0 through d^9 and
// d^8, whose truncation is below 3e-18 for |d| < 0.1 -- ~20 FP64 instructions
// against ~28 for a full sincos (measured on GB300); through d^5 and d^6 for
// |d| < 0.01 (truncation below 2e-18, three fused multiply-adds fewer); farther
// away, sincos.  (The tier thresholds are compared on the integer pipe.)
__device__ __forceinline__ void sincos_near(double th, double th0, double s0, double c0, double& s, double& c) {
    const double d = th - th0;
    if (abs_below_hi(d, kHi0p01)) {
        const double d2 = d * d;
        const double sd = d * fma(d2, fma(d2, 1.0 / 120.0, -1.0 / 6.0), 1.0);
        const double cd = fma(d2, fma(d2, fma(d2, -1.0 / 720.0, 1.0 / 24.0), -0.5), 1.0);
        s = fma(s0, cd, c0 * sd);
        c = fma(c0, cd, -(s0 * sd));
    } else if (abs_below_hi(d, kHi0p1)) {
        const double d2 = d * d;
        const double sd =
            d * fma(d2, fma(d2, fma(d2, fma(d2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0);
        const double cd = fma(d2, fma(d2, fma(d2, fma(d2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
        s = fma(s0, cd, c0 * sd);
        c = fma(c0, cd, -(s0 * sd));
    } else {
        sincos(th, &s, &c);
    }
}

// ---------------------------------------------------------------------------
// FP32 Kerr flow for the mixed-precision stages.  Same Hamiltonian, arranged
// for single precision:
//  * Delta = (r - r_+)(r - r_-) from dr = r - r_+, which the caller forms from
//    the high-precision state, so the flow stays relatively accurate down to
//    the horizon event;
//  * the radial force uses the exact (off-shell) identity
//      dK/dr - 4 r H = [K C - Delta' T + 2 A Q / Delta] / Delta,
//      C = (2M (r^2 - a^2 cos^2) - 2 r a^2 sin^2) / Sigma,
//      T = p_th^2 + (p_phi + a p_t sin^2)^2 / sin^2,
//      Q = 2M (r^2 - a^2) p_t + (2r - 2M) a p_phi,
//    in which the O(r^3) terms that cancel in dK/dr are already cancelled
//    analytically; in the direct form FP32 loses ~r^2/b^2 of its precision
//    far from the hole (10^4 at r = 1000), which shows up as drift of H.
// ---------------------------------------------------------------------------
struct RayConstF {
    float pt, pph, apph, pph2, a2pt2, c0, twoMpt;
};

__device__ __forceinline__ RayConstF to_float(const RayConst& R, double M) {
    RayConstF F;
    F.pt = (float)R.pt;
    F.pph = (float)R.pph;
    F.apph = (float)R.apph;
    F.pph2 = (float)R.pph2;
    F.a2pt2 = (float)R.a2pt2;
    F.c0 = (float)R.c0;
    F.twoMpt = (float)(2.0 * M * R.pt);
    return F;
}

struct StateF {
    float r, th, pr, pth;
};

// M, a^2 and r_+ - r_- in FP32; dr = r - r_+.
__device__ __forceinline__ void kerr_flow32_body(float M, float a2, float rpm, const RayConstF& R, const StateF& y,
                                            float dr, StateF& f, float& H) {
    float s, c;
    sincosf(y.th, &s, &c);
    const float r = y.r;
    float s2 = s * s, c2 = c * c, sc = s * c;
    float r2 = r * r;
    float Sig = fmaf(a2, c2, r2);
    float Del = dr * (dr + rpm);
    float A = fmaf(r2 + a2, R.pt, R.apph);
    float SD = Sig * Del;
    float inv = __frcp_rn(SD * s2);
    float iS = inv * (Del * s2);
    float iD = inv * (Sig * s2);
    float u = inv * SD;
    float pr2 = y.pr * y.pr;
    float AiD = A * iD;
    float T = fmaf(y.pth, y.pth, fmaf(R.pph2, u, fmaf(R.a2pt2, s2, R.c0)));
    float K = fmaf(-A, AiD, fmaf(Del, pr2, T));
    float hiS = 0.5f * iS;
    H = K * hiS;
    float twoM = 2.0f * M;
    float Dr = fmaf(2.0f, r, -twoM);
    float C = fmaf(twoM, fmaf(-a2, c2, r2), -2.0f * r * a2 * s2) * iS;
    float Q = fmaf(R.twoMpt, r2 - a2, Dr * R.apph);
    float G = fmaf(K, C, fmaf(-Dr, T, 2.0f * AiD * Q));
    float dKt = 2.0f * sc * fmaf(-R.pph2, u * u, R.a2pt2);
    f.r = Del * iS * y.pr;
    f.th = y.pth * iS;
    f.pr = -G * iD * hiS;
    f.pth = -fmaf(4.0f * a2 * sc, H, dKt) * hiS;
}

// The FP32 flow as one shared out-of-line copy (arguments and results by
// value, so they travel in registers): the mixed kernels call it from many
// stages, and inlining it everywhere made instruction-cache misses, not
// arithmetic, their bound.
struct Flow32 {
    StateF f;
    float H;
};

static __device__ __noinline__ Flow32 kerr_flow32_call(float M, float a2, float rpm, RayConstF R, StateF y, float dr) {
    Flow32 o;
    kerr_flow32_body(M, a2, rpm, R, y, dr, o.f, o.H);
    return o;
}

__device__ __forceinline__ void kerr_flow32(float M, float a2, float rpm, const RayConstF& R, const StateF& y,
                                            float dr, StateF& f, float& H) {
    const Flow32 o = kerr_flow32_call(M, a2, rpm, R, y, dr);
    f = o.f;
    H = o.H;
}

// H alone (no derivatives), FP64: the mixed paths' constraint monitor.
__device__ __forceinline__ double kerr_h64(const KerrK& k, const RayConst& R, const State& y) {
    double s, c;
    sincos(y.th, &s, &c);
    const double r = y.r;
    double s2 = s * s, r2 = r * r;
    double Sig = fma(k.a2, c * c, r2);
    double Del = fma(r, r - k.twoM, k.a2);
    double A = fma(r2 + k.a2, R.pt, R.apph);
    double SD = Sig * Del;
    double inv = rcp64(SD * s2);
    double T = fma(y.pth, y.pth, fma(R.pph2, inv * SD, fma(R.a2pt2, s2, R.c0)));
    double K = fma(-A, A * (inv * Sig * s2), fma(Del, y.pr * y.pr, T));
    return 0.5 * K * (inv * Del * s2);
}

// Kerr g_tt, g_tphi, g_rr, g_thth, g_phiphi (Boyer-Lindquist).
__device__ __forceinline__ void kerr_lower64(double M, double a, double r, double th, double g[5]) {
    double s, c;
    sincos(th, &s, &c);
    double s2 = s * s;
    double Sig = r * r + a * a * c * c;
    double Del = r * r - 2.0 * M * r + a * a;
    g[0] = -(1.0 - 2.0 * M * r / Sig);
    g[1] = -2.0 * M * a * r * s2 / Sig;
    g[2] = Sig / Del;
    g[3] = Sig;
    g[4] = (r * r + a * a + 2.0 * M * a * a * r * s2 / Sig) * s2;
}

// ---------------------------------------------------------------------------
// Tabulated metric: bicubic Hermite patches in (u = ln r, theta), one per cell
// of the node grid, held on the device in the monomial basis of the cell's
// unit coordinates (t, w): per field, c_ij (i: power of t, j: power of w),
// evaluated with their t- and w-derivatives by Horner's rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void hermite4(double t, double h[4], double dh[4]) {
    // explicit FMAs only, so that every build rounds alike
    double t2 = t * t, omt = 1.0 - t;
    h[0] = fma(2.0, t, 1.0) * omt * omt;
    h[1] = t * omt * omt;
    h[2] = t2 * fma(-2.0, t, 3.0);
    h[3] = t2 * (t - 1.0);
    dh[0] = 6.0 * (t2 - t);
    dh[1] = fma(3.0, t2, fma(-4.0, t, 1.0));
    dh[2] = 6.0 * (t - t2);
    dh[3] = fma(3.0, t2, -2.0 * t);
}

// p = c0 + c1 x + c2 x^2 + c3 x^3 and dp = dp/dx
__device__ __forceinline__ void horner_d(double c0, double c1, double c2, double c3, double x, double& p,
                                         double& dp) {
    double q = fma(c3, x, c2);
    double d = fma(c3, x, q);
    q = fma(q, x, c1);
    d = fma(d, x, q);
    p = fma(q, x, c0);
    dp = d;
}

// All five fields (g_tt, g_tphi, g_thth, g_phiphi, g^rr) with d/dr and d/dth.
__device__ __forceinline__ void table_fields64(const ImageDesc& d, double r, double th,
                                               double f[5], double fr[5], double ft[5]) {
    double tu = (log(r) - d.u0) / d.du;
    double tw = th / d.dth;
    int k = (int)floor(tu), j = (int)floor(tw);
    k = min(max(k, 0), d.nr - 2);
    j = min(max(j, 0), d.nth - 2);
    const double t = tu - (double)k, w = tw - (double)j;
    const double* cell = d.table + ((size_t)j * (d.nr - 1) + k) * kTableCoef;
    const double inv_dur = 1.0 / (d.du * r), inv_dth = 1.0 / d.dth;
#pragma unroll
    for (int fi = 0; fi < 5; ++fi) {
        const double2* c = reinterpret_cast<const double2*>(cell + 16 * fi);
        double P[4], Q[4];        // sum_j c_ij w^j and its w-derivative, per power i of t
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 c01 = __ldg(c + 2 * i), c23 = __ldg(c + 2 * i + 1);
            horner_d(c01.x, c01.y, c23.x, c23.y, w, P[i], Q[i]);
        }
        double v, vt;
        horner_d(P[0], P[1], P[2], P[3], t, v, vt);
        const double vw = fma(fma(fma(Q[3], t, Q[2]), t, Q[1]), t, Q[0]);
        f[fi] = v;
        fr[fi] = vt * inv_dur;
        ft[fi] = vw * inv_dth;
    }
}

// Flow of H = 1/2 [W/D + g^rr p_r^2 + p_th^2 / g_thth], with the inverse of the
// (t, phi) block, D = g_tt g_phiphi - g_tphi^2,
// W = g_phiphi p_t^2 - 2 g_tphi p_t p_phi + g_tt p_phi^2.
__device__ __forceinline__ void table_flow64(const ImageDesc& d, const RayConst& R, const State& y,
                                             State& f, double& H) {
    double F[5], Fr[5], Ft[5];
    table_fields64(d, y.r, y.th, F, Fr, Ft);
    const double pt2 = R.pt * R.pt, ptp = 2.0 * R.pt * R.pph;
    double D = fma(F[0], F[3], -F[1] * F[1]);
    double iD = rcp64(D);
    double W = fma(F[3], pt2, fma(-F[1], ptp, F[0] * R.pph2));
    double WiD = W * iD;
    double ith = rcp64(F[2]);
    double pr2 = y.pr * y.pr, pth2 = y.pth * y.pth;
    H = 0.5 * (WiD + fma(F[4], pr2, pth2 * ith));
    double dW_r = fma(Fr[3], pt2, fma(-Fr[1], ptp, Fr[0] * R.pph2));
    double dD_r = fma(Fr[0], F[3], fma(F[0], Fr[3], -2.0 * F[1] * Fr[1]));
    double dW_t = fma(Ft[3], pt2, fma(-Ft[1], ptp, Ft[0] * R.pph2));
    double dD_t = fma(Ft[0], F[3], fma(F[0], Ft[3], -2.0 * F[1] * Ft[1]));
    double ith2 = ith * ith;
    double d2H_r = fma(fma(-WiD, dD_r, dW_r), iD, fma(Fr[4], pr2, -Fr[2] * ith2 * pth2));
    double d2H_t = fma(fma(-WiD, dD_t, dW_t), iD, fma(Ft[4], pr2, -Ft[2] * ith2 * pth2));
    f.r = F[4] * y.pr;
    f.th = y.pth * ith;
    f.pr = -0.5 * d2H_r;
    f.pth = -0.5 * d2H_t;
}

__device__ __forceinline__ void table_lower64(const ImageDesc& d, double r, double th, double g[5]) {
    double F[5], Fr[5], Ft[5];
    table_fields64(d, r, th, F, Fr, Ft);
    g[0] = F[0];
    g[1] = F[1];
    g[2] = 1.0 / F[4];
    g[3] = F[2];
    g[4] = F[3];
}

// The table flow as one out-of-line copy (descriptor by pointer, the rest by
// value): six stage evaluations and the refinement's inlined copies made the
// table kernels' instruction footprint, not their FP64 arithmetic, a bound.
struct FlowT64 {
    State f;
    double H;
};

static __device__ __noinline__ FlowT64 table_flow64_call(const ImageDesc* d, RayConst R, State y) {
    FlowT64 o;
    table_flow64(*d, R, y, o.f, o.H);
    return o;
}

// METRIC: 0 closed-form Kerr, 1 table, 2 chosen per image at run time.
template <int METRIC>
__device__ __forceinline__ void flow64(const ImageDesc& d, const KerrK& k, const RayConst& R,
                                       const State& y, State& f, double& H) {
    if (METRIC == 0 || (METRIC == 2 && d.kind == 0)) kerr_flow64(k, R, y, f, H);
    else {
        const FlowT64 o = table_flow64_call(&d, R, y);
        f = o.f;
        H = o.H;
    }
}

template <int METRIC>
__device__ __forceinline__ void lower64(const ImageDesc& d, double r, double th, double g[5]) {
    if (METRIC == 0 || (METRIC == 2 && d.kind == 0)) kerr_lower64(d.M, d.a, r, th, g);
    else table_lower64(d, r, th, g);
}

// ---------------------------------------------------------------------------
// Page-Thorne flux (paper Sec. 2.3, prefactor as printed) with the host-resolved
// roots and coefficients; zero inside the ISCO.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double flux64(const ImageDesc& d, double r) {
    double x = sqrt(r / d.M);
    if (x < d.fx0) return 0.0;
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        if (d.fcoef[i] != 0.0) sum = fma(d.fcoef[i], log(x - d.fxr[i]) - d.flog0[i], sum);
    double br = x - d.fx0 - 1.5 * d.fa * log(x / d.fx0) - sum;
    double x2 = x * x;
    double pref = 3.0 / (2.0 * x2 * x2 * (x2 * x - 3.0 * x + 2.0 * d.fa));
    return d.flux_scale * pref * br;
}

// Redshift g = p_t / (u^t (p_t + Omega p_phi)) of a prograde Keplerian emitter
// (paper Sec. 2.4); Doppler off: g = 1 / u^t.
template <int METRIC>
__device__ __forceinline__ double redshift64(const ImageDesc& d, double r, double pt, double pph) {
    double g[5];
    if (METRIC == 0 || (METRIC == 2 && d.kind == 0)) {
        double M = d.M, a = d.a;
        g[0] = -(1.0 - 2.0 * M / r);
        g[1] = -2.0 * M * a / r;
        g[4] = r * r + a * a + 2.0 * M * a * a / r;
    } else {
        lower64<METRIC>(d, r, kHalfPi, g);
    }
    double Om = d.sqrtM / (r * sqrt(r) + d.a * d.sqrtM);
    double ut = 1.0 / sqrt(-g[0] - 2.0 * Om * g[1] - Om * Om * g[4]);
    if (!d.doppler) return 1.0 / ut;
    return pt / (ut * (pt + Om * pph));
}

// ---------------------------------------------------------------------------
// Dormand-Prince 5(4) coefficients (Dormand & Prince 1980).
// ---------------------------------------------------------------------------
namespace dp {
constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 4.0 / 5.0, c5 = 8.0 / 9.0;
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                 a54 = -212.0 / 729.0;
constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                 a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                 b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
// e = b - bhat
constexpr double e1 = 35.0 / 384.0 - 5179.0 / 57600.0;
constexpr double e3 = 500.0 / 1113.0 - 7571.0 / 16695.0;
constexpr double e4 = 125.0 / 192.0 - 393.0 / 640.0;
constexpr double e5 = -2187.0 / 6784.0 + 92097.0 / 339200.0;
constexpr double e6 = 11.0 / 84.0 - 187.0 / 2100.0;
constexpr double e7 = -1.0 / 40.0;
}  // namespace dp

// Embedded 5(4) pairs of Sec. 3.2 for the FP64 stepper: stage nodes c_i,
// coefficients a_ij, fifth-order weights b_i (they advance the solution) and
// e_i = b_i - bhat_i (the error estimate).  b_2 = 0 and e_2 = 0 in all three.
// Dormand-Prince has seven stages, the seventh at the new point (first same as
// last, e_7 != 0); Cash-Karp and Fehlberg have six, and the flow at the new
// point is one extra evaluation that becomes the next step's first stage.
template <int METHOD>
struct RK;

template <>
struct RK<0> {   // Dormand & Prince (1980)
    static constexpr double c2 = dp::c2, c3 = dp::c3, c4 = dp::c4, c5 = dp::c5, c6 = 1.0;
    static constexpr double a21 = dp::a21, a31 = dp::a31, a32 = dp::a32, a41 = dp::a41, a42 = dp::a42,
                            a43 = dp::a43, a51 = dp::a51, a52 = dp::a52, a53 = dp::a53, a54 = dp::a54,
                            a61 = dp::a61, a62 = dp::a62, a63 = dp::a63, a64 = dp::a64, a65 = dp::a65;
    static constexpr double b1 = dp::b1, b3 = dp::b3, b4 = dp::b4, b5 = dp::b5, b6 = dp::b6;
    static constexpr double e1 = dp::e1, e3 = dp::e3, e4 = dp::e4, e5 = dp::e5, e6 = dp::e6, e7 = dp::e7;
};

template <>
struct RK<1> {   // Cash & Karp (1990)
    static constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 3.0 / 5.0, c5 = 1.0, c6 = 7.0 / 8.0;
    static constexpr double a21 = 1.0 / 5.0;
    static constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
    static constexpr double a41 = 3.0 / 10.0, a42 = -9.0 / 10.0, a43 = 6.0 / 5.0;
    static constexpr double a51 = -11.0 / 54.0, a52 = 5.0 / 2.0, a53 = -70.0 / 27.0, a54 = 35.0 / 27.0;
    static constexpr double a61 = 1631.0 / 55296.0, a62 = 175.0 / 512.0, a63 = 575.0 / 13824.0,
                            a64 = 44275.0 / 110592.0, a65 = 253.0 / 4096.0;
    static constexpr double b1 = 37.0 / 378.0, b3 = 250.0 / 621.0, b4 = 125.0 / 594.0, b5 = 0.0,
                            b6 = 512.0 / 1771.0;
    static constexpr double e1 = 37.0 / 378.0 - 2825.0 / 27648.0, e3 = 250.0 / 621.0 - 18575.0 / 48384.0,
                            e4 = 125.0 / 594.0 - 13525.0 / 55296.0, e5 = -277.0 / 14336.0,
                            e6 = 512.0 / 1771.0 - 1.0 / 4.0, e7 = 0.0;
};

template <>
struct RK<2> {   // Fehlberg (1969)
    static constexpr double c2 = 1.0 / 4.0, c3 = 3.0 / 8.0, c4 = 12.0 / 13.0, c5 = 1.0, c6 = 1.0 / 2.0;
    static constexpr double a21 = 1.0 / 4.0;
    static constexpr double a31 = 3.0 / 32.0, a32 = 9.0 / 32.0;
    static constexpr double a41 = 1932.0 / 2197.0, a42 = -7200.0 / 2197.0, a43 = 7296.0 / 2197.0;
    static constexpr double a51 = 439.0 / 216.0, a52 = -8.0, a53 = 3680.0 / 513.0, a54 = -845.0 / 4104.0;
    static constexpr double a61 = -8.0 / 27.0, a62 = 2.0, a63 = -3544.0 / 2565.0, a64 = 1859.0 / 4104.0,
                            a65 = -11.0 / 40.0;
    static constexpr double b1 = 16.0 / 135.0, b3 = 6656.0 / 12825.0, b4 = 28561.0 / 56430.0, b5 = -9.0 / 50.0,
                            b6 = 2.0 / 55.0;
    static constexpr double e1 = 16.0 / 135.0 - 25.0 / 216.0, e3 = 6656.0 / 12825.0 - 1408.0 / 2565.0,
                            e4 = 28561.0 / 56430.0 - 2197.0 / 4104.0, e5 = -9.0 / 50.0 + 1.0 / 5.0,
                            e6 = 2.0 / 55.0, e7 = 0.0;
};

// acc + w k, with the term dropped at compile time when the weight w is zero
#define TT_MAC(w, k, acc) (((w) == 0.0) ? (acc) : fma((w), (k), (acc)))

}  // namespace tt

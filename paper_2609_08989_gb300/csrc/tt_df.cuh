// tt_df.cuh -- double-float arithmetic (an unevaluated sum hi + lo of two FP32
// numbers, ~48 significant bits) for the FP32 pipe.
//
// GB300 issues FP64 at 1/64 of the FP32 rate, so the steps that need more than
// FP32 (near the horizon and the polar axis on the mixed paths, and every step
// of the double-float path) run in this format instead.  The building blocks are
// the classical error-free transformations: Knuth's TwoSum and Dekker's
// FastTwoSum for addition, and the FMA-based exact product (a b = p + e with
// e = fma(a, b, -p)); the compound operations follow the "sloppy" double-double
// algorithms (error relative to the operands, like FP64 addition itself).
#pragma once

#include <cuda_runtime.h>

#include "tt_device.cuh"

namespace tt {

struct DF {
    float hi, lo;
};

struct StateDF {
    DF r, th, pr, pth;
};

// exact split of a double into hi + lo (the nearest double-float)
__host__ __device__ constexpr DF df_const(double v) {
    return DF{(float)v, (float)(v - (double)(float)v)};
}

__device__ __forceinline__ DF df_of(double v) {
    const float h = (float)v;
    return DF{h, (float)(v - (double)h)};
}

__device__ __forceinline__ double df_to64(DF x) {
    return (double)x.hi + (double)x.lo;
}

// The primitives use the _rn intrinsics, which the compiler never contracts
// into FMAs: an error-free transformation is only exact if each operation is
// rounded exactly where it is written.

// |a| >= |b| (or a == 0): s + e = a + b exactly
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e = a + b exactly, any order of magnitude
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF df_add(DF x, DF y) {
    const DF s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ DF df_neg(DF x) {
    return DF{-x.hi, -x.lo};
}

__device__ __forceinline__ DF df_sub(DF x, DF y) {
    return df_add(x, df_neg(y));
}

__device__ __forceinline__ DF df_add_f(DF x, float y) {
    const DF s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

__device__ __forceinline__ DF df_mul(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_mul_f(DF x, float y) {
    const float p = __fmul_rn(x.hi, y);
    float e = fmaf(x.hi, y, -p);
    e = fmaf(x.lo, y, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_sqr(DF x) {
    const float p = __fmul_rn(x.hi, x.hi);
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(__fadd_rn(x.hi, x.hi), x.lo, e);
    return fast_two_sum(p, e);
}

// x * y + z, the product's error term carried straight into the sum (no
// intermediate renormalisation)
__device__ __forceinline__ DF df_fma(DF x, DF y, DF z) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const DF s = two_sum(p, z.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo)));
}

// "Lazy" forms: the same error-free parts without the closing renormalisation
// (FastTwoSum).  Their lo may exceed half an ulp of hi by a few bits, and an
// operation that takes such a value rounds x.lo y.hi in FP32: harmless after
// a product of renormalised values (lo within ~2 ulps), but after a sum that
// cancels lo can be a sizeable part of the value, and the product that takes
// it then keeps only ~2^-48 of the sum's operands, not of its result.  So the
// flows use lazy products of renormalised values and renormalise every sum;
// Horner chains (terms of one size, error measured against them) are lazy
// throughout.  A reciprocal's argument is renormalised.
__device__ __forceinline__ DF df_mul_lazy(DF x, DF y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return DF{p, e};
}

__device__ __forceinline__ DF df_sqr_lazy(DF x) {
    const float p = __fmul_rn(x.hi, x.hi);
    float e = fmaf(x.hi, x.hi, -p);
    e = fmaf(__fadd_rn(x.hi, x.hi), x.lo, e);
    return DF{p, e};
}

__device__ __forceinline__ DF df_add_lazy(DF x, DF y) {
    const DF s = two_sum(x.hi, y.hi);
    return DF{s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo))};
}

__device__ __forceinline__ DF df_sub_lazy(DF x, DF y) {
    return df_add_lazy(x, df_neg(y));
}

// x y + z
__device__ __forceinline__ DF df_fma_lazy(DF x, DF y, DF z) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    const DF s = two_sum(p, z.hi);
    return DF{s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo))};
}

__device__ __forceinline__ DF df_norm(DF x) {
    return two_sum(x.hi, x.lo);
}

// Dot products sum_j c_j k_j of double-float terms, in the style of Ogita,
// Rump & Oishi's Dot2: the high parts' products are accumulated exactly with
// TwoSum, and their rounding errors, the products' own errors (by FMA) and the
// cross terms hi*lo are summed in FP32 -- as accurate as chained double-float
// multiply-adds at ~3/4 of their instructions.
struct DotAcc {
    float s, t;
};

__device__ __forceinline__ float dot_err(DF c, DF k, float p) {
    return fmaf(c.hi, k.hi, -p) + fmaf(c.hi, k.lo, c.lo * k.hi);
}

__device__ __forceinline__ DotAcc dot_first(DF c, DF k) {
    const float p = __fmul_rn(c.hi, k.hi);
    return DotAcc{p, dot_err(c, k, p)};
}

__device__ __forceinline__ DotAcc dot_next(DotAcc d, DF c, DF k) {
    const float p = __fmul_rn(c.hi, k.hi);
    const DF s = two_sum(d.s, p);
    return DotAcc{s.hi, d.t + (s.lo + dot_err(c, k, p))};
}

// the final sum may be cancelled below the error terms: TwoSum, not FastTwoSum
__device__ __forceinline__ DF dot_end(DotAcc d) {
    const DF s = two_sum(d.s, d.t);
    return fast_two_sum(s.hi, s.lo);
}

// 1/x: the correctly rounded FP32 reciprocal r0 leaves the residual
// e = 1 - x_hi r0 exactly representable (one FMA); 1/x = r0 (1 + e + e^2 + ...),
// and the terms through e^2 (the last ~2^-48) restore double-float precision.
__device__ __forceinline__ DF df_rcp(DF x) {
    const float r0 = __frcp_rn(x.hi);
    float e = fmaf(-x.hi, r0, 1.0f);
    e = fmaf(-x.lo, r0, e);
    return fast_two_sum(r0, __fmul_rn(r0, fmaf(e, e, e)));
}

// ---------------------------------------------------------------------------
// sin and cos of theta in double-float, for any theta (a ray through the polar
// axis continues with theta outside (0, pi)).  theta = k pi/64 + d with
// |d| <= pi/128; sin and cos of k pi/64 come from a 128-entry table over one
// period (computed in FP64 when a block starts, see df_sincos_table), and of d
// from their Taylor series: the terms beyond d^3/6 and d^2/2 (< 3e-9 relative)
// in FP32, those before in double-float.  Angle addition then combines the two.
// ---------------------------------------------------------------------------
constexpr int kSinCosN = 128;                      // entries per period, step pi/64
constexpr double kPiOver64 = 0.04908738521234051935;

// the table, one copy per block of the kernels that step in double-float
static __shared__ float4 s_df_tab[kSinCosN];

// Fill tab[0..127] = (sin hi, sin lo, cos hi, cos lo) of k pi/64 (by the threads
// of one block; the caller synchronises the block afterwards).
__device__ __forceinline__ void df_sincos_table(float4* tab) {
    for (int k = threadIdx.x; k < kSinCosN; k += blockDim.x) {
        double s, c;
        sincos((double)k * kPiOver64, &s, &c);
        const DF sd = df_of(s), cd = df_of(c);
        tab[k] = make_float4(sd.hi, sd.lo, cd.hi, cd.lo);
    }
}

__device__ __forceinline__ void df_sincos(DF th, DF& s, DF& c) {
    constexpr float kInv = (float)(64.0 / 3.14159265358979323846);
    constexpr DF P = df_const(kPiOver64);
    constexpr float P2 = (float)(kPiOver64 - (double)P.hi - (double)P.lo);
    const int k = __float2int_rn(th.hi * kInv);    // |k| < 2^24 keeps k P_hi exact below
    const float kf = (float)k;
    // d = theta - k P: k P_hi exactly as p0 + e0 (FMA), k P_lo as p1 + e1
    const float p0 = __fmul_rn(kf, P.hi), e0 = fmaf(kf, P.hi, -p0);
    const float p1 = __fmul_rn(kf, P.lo), e1 = fmaf(kf, P.lo, -p1);
    const float d0 = __fsub_rn(th.hi, p0);         // exact (Sterbenz) for k != 0; theta_hi for k = 0
    const float tail = (th.lo - e0) - ((p1 + e1) + kf * P2);
    const DF d = fast_two_sum(d0, tail);
    const DF q = df_sqr(d);                         // d^2 <= 6.1e-4
    const float qf = q.hi;
    // sin d = d + d q (-1/6 + q (1/120 - q/5040))
    const float ws = qf * fmaf(-qf, 1.0f / 5040.0f, 1.0f / 120.0f);
    constexpr DF M6 = df_const(-1.0 / 6.0);
    const DF sd = df_add(d, df_mul(d, df_mul(q, df_add_f(M6, ws))));
    // cos d = 1 + q (-1/2 + q (1/24 - q/720))
    const float wc = qf * fmaf(-qf, 1.0f / 720.0f, 1.0f / 24.0f);
    const DF cd = df_add_f(df_mul(q, two_sum(-0.5f, wc)), 1.0f);
    const float4 t = s_df_tab[k & (kSinCosN - 1)];  // k mod 128 (two's complement)
    const DF sk = DF{t.x, t.y}, ck = DF{t.z, t.w};
    s = df_add(df_mul(sk, cd), df_mul(ck, sd));
    c = df_sub(df_mul(ck, cd), df_mul(sk, sd));
}

// ---------------------------------------------------------------------------
// Kerr flow in double-float: the expressions of kerr_flow64 (Carter's
// separated Hamiltonian, forces regrouped), term for term.
// ---------------------------------------------------------------------------
struct KerrDF {
    DF M, a2, twoM;
};

struct RayDF {
    DF pt, apph, pph2, a2pt2, c0, pt2;
    DF ptsq, ptp;           // p_t^2, 2 p_t p_phi (tabulated metric)
};

__device__ __forceinline__ KerrDF make_kerr_df(const KerrK& k) {
    return KerrDF{df_of(k.M), df_of(k.a2), df_of(k.twoM)};
}

__device__ __forceinline__ RayDF make_ray_df(const RayConst& R) {
    return RayDF{df_of(R.pt),    df_of(R.apph), df_of(R.pph2), df_of(R.a2pt2),
                 df_of(R.c0),    df_of(R.pt2),  df_of(R.pt * R.pt), df_of(2.0 * R.pt * R.pph)};
}

__device__ __forceinline__ void kerr_flow_df_body(const KerrDF& k, const RayDF& R, const StateDF& y, StateDF& f,
                                                  DF& H) {
    // products of renormalised values in the lazy form (their lo stays within
    // ~2 ulps of hi); every sum, which may cancel, renormalises, so that no
    // cancelled value carries a large lo into a product
    DF s, c;
    df_sincos(y.th, s, c);
    const DF r = y.r;
    const DF s2 = df_sqr_lazy(s), c2 = df_sqr_lazy(c), sc = df_mul_lazy(s, c);
    const DF r2 = df_sqr_lazy(r);
    const DF Sig = df_fma(k.a2, c2, r2);
    const DF Del = df_fma(r, df_sub(r, k.twoM), k.a2);
    const DF A = df_fma(df_add(r2, k.a2), R.pt, R.apph);
    const DF SD = df_mul_lazy(Sig, Del);
    const DF inv = df_rcp(df_norm(df_mul_lazy(SD, s2)));
    const DF iS = df_mul_lazy(inv, df_mul_lazy(Del, s2));
    const DF iD = df_mul_lazy(inv, df_mul_lazy(Sig, s2));
    const DF u = df_mul_lazy(inv, SD);
    const DF pr2 = df_sqr_lazy(y.pr);
    const DF AiD = df_mul(A, iD);
    DF K = df_fma(R.a2pt2, s2, R.c0);
    K = df_fma(R.pph2, u, K);
    K = df_add(K, df_sqr_lazy(y.pth));
    K = df_fma(Del, pr2, K);
    K = df_sub(K, df_mul_lazy(A, AiD));
    const DF H2 = df_mul(K, iS);
    H = DF{0.5f * H2.hi, 0.5f * H2.lo};
    const DF q1 = df_fma(R.pt2, AiD, H2);
    const DF q2 = df_add(df_sqr_lazy(AiD), pr2);
    const DF t1 = df_sub(R.a2pt2, df_mul_lazy(R.pph2, df_sqr_lazy(u)));
    const DF t2 = df_fma(k.a2, H2, t1);
    f.r = df_mul(df_mul_lazy(Del, y.pr), iS);
    f.th = df_mul(y.pth, iS);
    f.pr = df_mul(df_sub(df_mul_lazy(r, q1), df_mul_lazy(df_sub(r, k.M), q2)), iS);
    f.pth = df_neg(df_mul(df_mul_lazy(sc, iS), t2));
}

// One out-of-line copy, arguments and results by value (in registers).
struct FlowDF {
    StateDF f;
    DF H;
};

static __device__ __noinline__ FlowDF kerr_flow_df_call(KerrDF k, RayDF R, StateDF y) {
    FlowDF o;
    kerr_flow_df_body(k, R, y, o.f, o.H);
    return o;
}

__device__ __forceinline__ void kerr_flow_df(const KerrDF& k, const RayDF& R, const StateDF& y, StateDF& f, DF& H) {
    const FlowDF o = kerr_flow_df_call(k, R, y);
    f = o.f;
    H = o.H;
}

// ---------------------------------------------------------------------------
// Natural logarithm in double-float, table-driven in the manner of Tang (ACM
// TOMS 16, 1990): x = 2^e m with m in [1, 2) and c = 1 + k/32 the nearest
// table point, ln x = e ln 2 + ln c + 2 atanh s with s = (m - c)/(m + c),
// |s| <= 1/128.  The series 2 atanh s = 2 s + s^3 (2/3 + 2 s^2/5 + ...) keeps
// s and s^3 2/3 in double-float and the rest (< 1.2e-11) in FP32; its first
// omitted term is below 1e-24.  ln c comes from a 33-entry table computed in
// FP64 when a block starts.
// ---------------------------------------------------------------------------
constexpr int kLnN = 32;

// the table, one copy per block of the tabulated-metric double-float kernels
static __shared__ float2 s_df_ln[kLnN + 1];

// Fill tab[0..32] = ln(1 + k/32) (by the threads of one block; the caller
// synchronises the block afterwards).
__device__ __forceinline__ void df_log_table(float2* tab) {
    for (int k = threadIdx.x; k <= kLnN; k += blockDim.x) {
        const DF v = df_of(log1p((double)k / kLnN));
        tab[k] = make_float2(v.hi, v.lo);
    }
}

// ln x for x.hi positive and normal.
__device__ __forceinline__ DF df_log(DF x) {
    const int bits = __float_as_int(x.hi);
    const int e = ((bits >> 23) & 0xff) - 127;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);      // in [1, 2)
    const float ml = __fmul_rn(x.lo, __int_as_float((127 - e) << 23));     // x.lo 2^-e, exact
    const int k = __float2int_rn(__fmul_rn(__fsub_rn(m, 1.0f), (float)kLnN));
    const float c = fmaf((float)k, 1.0f / kLnN, 1.0f);                     // exact
    // m - c is exact (Sterbenz) and a multiple of 2^-23, so at least |ml| or zero
    const DF num = fast_two_sum(__fsub_rn(m, c), ml);
    const DF den = df_add_f(DF{m, ml}, c);
    const DF sv = df_mul(num, df_rcp(den));
    const DF s2 = df_sqr(sv);
    const float q = s2.hi;
    const float w = q * fmaf(q, fmaf(q, 2.0f / 9.0f, 2.0f / 7.0f), 2.0f / 5.0f);
    constexpr DF TWO3 = df_const(2.0 / 3.0);
    const DF lm = df_add(DF{2.0f * sv.hi, 2.0f * sv.lo}, df_mul(df_mul(s2, sv), df_add_f(TWO3, w)));
    // e ln 2 with ln 2 in three parts (hi and lo of the double-float and the
    // float nearest the rest), so that it carries the double ln 2's ~1e-17
    constexpr double kLn2 = 0.69314718055994530942;
    constexpr DF L2 = df_const(kLn2);
    constexpr float L3 = (float)(kLn2 - (double)L2.hi - (double)L2.lo);
    const float ef = (float)e;
    DF el = df_mul_f(L2, ef);
    el = df_add_f(el, ef * L3);
    const float2 lc = s_df_ln[k];
    return df_add(df_add(el, DF{lc.x, lc.y}), lm);
}

// ---------------------------------------------------------------------------
// Tabulated metric in double-float: the patches of table_fields64 (monomial
// coefficients per cell and field, Horner's rule for the value and both
// unit-cell derivatives) with double-float coefficients and arithmetic.
// ---------------------------------------------------------------------------
// p = c0 + c1 x + c2 x^2 + c3 x^3 and dp = dp/dx (both left unnormalised)
__device__ __forceinline__ void horner_d_df(DF c0, DF c1, DF c2, DF c3, DF x, DF& p, DF& dp) {
    DF q = df_fma_lazy(c3, x, c2);
    DF d = df_fma_lazy(c3, x, q);
    q = df_fma_lazy(q, x, c1);
    d = df_fma_lazy(d, x, q);
    p = df_fma_lazy(q, x, c0);
    dp = d;
}

// The 15 results pass through this thread's slots of s_df_out, so that the loop
// over the fields stays rolled: the flow is evaluated at every stage, and five
// unrolled copies of its patch evaluation overflowed the instruction cache.
// Slots are strided by the block size (distinct banks within a warp); the
// double-float kernels run 256-thread blocks.
constexpr int kDfBlock = 256;
static __shared__ float2 s_df_out[15 * kDfBlock];

// floor(x) clamped to [0, n_max] (NaN to 0), for a double-float x
__device__ __forceinline__ int df_cell(DF x, int n_max) {
    float f = floorf(x.hi);
    if (x.hi == f && x.lo < 0.0f) f -= 1.0f;
    return (int)fminf(fmaxf(f, 0.0f), (float)n_max);
}

// All five fields (g_tt, g_tphi, g_thth, g_phiphi, g^rr) with d/dr and d/dth.
__device__ __forceinline__ void table_fields_df(const ImageDesc& d, DF r, DF th, DF f[5], DF fr[5], DF ft[5]) {
    const DF u0 = DF{d.u0_df.x, d.u0_df.y}, idu = DF{d.idu_df.x, d.idu_df.y};
    const DF idth = DF{d.idth_df.x, d.idth_df.y};
    const DF tu = df_mul(df_sub(df_log(r), u0), idu);
    const DF tw = df_mul(th, idth);
    const int k = df_cell(tu, d.nr - 2), j = df_cell(tw, d.nth - 2);
    const DF t = df_add_f(tu, -(float)k), w = df_add_f(tw, -(float)j);
    const float2* cell = d.table_df + ((size_t)j * (d.nr - 1) + k) * kTableCoef;
    const DF inv_dur = df_mul(idu, df_rcp(r));                 // 1 / (du r)
    float2* out = s_df_out + threadIdx.x;
#pragma unroll 1
    for (int fi = 0; fi < 5; ++fi) {
        const float4* c = reinterpret_cast<const float4*>(cell + 16 * fi);
        DF P[4], Q[4];        // sum_j c_ij w^j and its w-derivative, per power i of t
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 a = __ldg(c + 2 * i), b = __ldg(c + 2 * i + 1);
            horner_d_df(DF{a.x, a.y}, DF{a.z, a.w}, DF{b.x, b.y}, DF{b.z, b.w}, w, P[i], Q[i]);
        }
        DF v, vt;
        horner_d_df(P[0], P[1], P[2], P[3], t, v, vt);
        const DF vw = df_fma_lazy(df_fma_lazy(df_fma_lazy(Q[3], t, Q[2]), t, Q[1]), t, Q[0]);
        v = df_norm(v);
        const DF vr = df_mul(df_norm(vt), inv_dur), vth = df_mul(df_norm(vw), idth);
        out[(3 * fi) * kDfBlock] = make_float2(v.hi, v.lo);
        out[(3 * fi + 1) * kDfBlock] = make_float2(vr.hi, vr.lo);
        out[(3 * fi + 2) * kDfBlock] = make_float2(vth.hi, vth.lo);
    }
#pragma unroll
    for (int fi = 0; fi < 5; ++fi) {
        const float2 a = out[(3 * fi) * kDfBlock], b = out[(3 * fi + 1) * kDfBlock], c = out[(3 * fi + 2) * kDfBlock];
        f[fi] = DF{a.x, a.y};
        fr[fi] = DF{b.x, b.y};
        ft[fi] = DF{c.x, c.y};
    }
}

// The flow of table_flow64 in double-float: H = 1/2 [W/D + g^rr p_r^2 +
// p_th^2 / g_thth] with D = g_tt g_phiphi - g_tphi^2 and
// W = g_phiphi p_t^2 - 2 g_tphi p_t p_phi + g_tt p_phi^2.
__device__ __forceinline__ void table_flow_df(const ImageDesc& d, const RayDF& R, const StateDF& y, StateDF& f,
                                              DF& H) {
    DF F[5], Fr[5], Ft[5];
    table_fields_df(d, y.r, y.th, F, Fr, Ft);
    const DF D = df_sub(df_mul(F[0], F[3]), df_sqr(F[1]));
    const DF iD = df_rcp(D);
    const DF W = dot_end(dot_next(dot_next(dot_first(F[3], R.ptsq), df_neg(F[1]), R.ptp), F[0], R.pph2));
    const DF WiD = df_mul(W, iD);
    const DF ith = df_rcp(F[2]);
    const DF pr2 = df_sqr(y.pr);
    const DF pthi = df_mul(y.pth, ith);                      // p_th / g_thth
    const DF pth2i = df_mul(y.pth, pthi);
    const DF H2 = df_add(WiD, df_fma(F[4], pr2, pth2i));
    H = DF{0.5f * H2.hi, 0.5f * H2.lo};
    const DF pthi2 = df_sqr(pthi);                           // p_th^2 / g_thth^2
    // d(2H)/dx = (dW - W/D dD)/D + d(g^rr) p_r^2 - d(g_thth) p_th^2 / g_thth^2
#define TT_D2H(G)                                                                                            \
    df_add(df_mul(df_sub(dot_end(dot_next(dot_next(dot_first(G[3], R.ptsq), df_neg(G[1]), R.ptp), G[0], R.pph2)), \
                         df_mul(WiD, dot_end(dot_next(dot_next(dot_first(G[0], F[3]), F[0], G[3]),                \
                                                      DF{-2.0f * F[1].hi, -2.0f * F[1].lo}, G[1])))),           \
                  iD),                                                                                         \
           df_sub(df_mul(G[4], pr2), df_mul(G[2], pthi2)))
    const DF d2H_r = TT_D2H(Fr);
    const DF d2H_t = TT_D2H(Ft);
#undef TT_D2H
    f.r = df_mul(F[4], y.pr);
    f.th = pthi;
    f.pr = DF{-0.5f * d2H_r.hi, -0.5f * d2H_r.lo};
    f.pth = DF{-0.5f * d2H_t.hi, -0.5f * d2H_t.lo};
}

// One out-of-line copy (descriptor by pointer, the rest by value).
static __device__ __noinline__ FlowDF table_flow_df_call(const ImageDesc* d, RayDF R, StateDF y) {
    FlowDF o;
    table_flow_df(*d, R, y, o.f, o.H);
    return o;
}

// METRIC 0: closed-form Kerr, 1: table.
template <int METRIC>
__device__ __forceinline__ void flow_df(const ImageDesc& d, const KerrDF& k, const RayDF& R, const StateDF& y,
                                        StateDF& f, DF& H) {
    static_assert(METRIC == 0 || METRIC == 1, "the double-float kernels take one metric kind per launch");
    if constexpr (METRIC == 0) {
        kerr_flow_df(k, R, y, f, H);
    } else {
        const FlowDF o = table_flow_df_call(&d, R, y);
        f = o.f;
        H = o.H;
    }
}

}  // namespace tt

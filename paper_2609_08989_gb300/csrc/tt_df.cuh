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
};

__device__ __forceinline__ KerrDF make_kerr_df(const KerrK& k) {
    return KerrDF{df_of(k.M), df_of(k.a2), df_of(k.twoM)};
}

__device__ __forceinline__ RayDF make_ray_df(const RayConst& R) {
    return RayDF{df_of(R.pt), df_of(R.apph), df_of(R.pph2), df_of(R.a2pt2), df_of(R.c0), df_of(R.pt2)};
}

__device__ __forceinline__ void kerr_flow_df_body(const KerrDF& k, const RayDF& R, const StateDF& y, StateDF& f,
                                                  DF& H) {
    DF s, c;
    df_sincos(y.th, s, c);
    const DF r = y.r;
    const DF s2 = df_sqr(s), c2 = df_sqr(c), sc = df_mul(s, c);
    const DF r2 = df_sqr(r);
    const DF Sig = df_fma(k.a2, c2, r2);
    const DF Del = df_fma(r, df_sub(r, k.twoM), k.a2);
    const DF A = df_fma(df_add(r2, k.a2), R.pt, R.apph);
    const DF SD = df_mul(Sig, Del);
    const DF inv = df_rcp(df_mul(SD, s2));
    const DF iS = df_mul(inv, df_mul(Del, s2));
    const DF iD = df_mul(inv, df_mul(Sig, s2));
    const DF u = df_mul(inv, SD);
    const DF pr2 = df_sqr(y.pr);
    const DF AiD = df_mul(A, iD);
    DF K = df_fma(R.a2pt2, s2, R.c0);
    K = df_fma(R.pph2, u, K);
    K = df_add(K, df_sqr(y.pth));
    K = df_fma(Del, pr2, K);
    K = df_sub(K, df_mul(A, AiD));
    const DF H2 = df_mul(K, iS);
    H = DF{0.5f * H2.hi, 0.5f * H2.lo};
    const DF q1 = df_fma(R.pt2, AiD, H2);
    const DF q2 = df_add(df_sqr(AiD), pr2);
    const DF t1 = df_sub(R.a2pt2, df_mul(R.pph2, df_sqr(u)));
    const DF t2 = df_fma(k.a2, H2, t1);
    f.r = df_mul(df_mul(Del, y.pr), iS);
    f.th = df_mul(y.pth, iS);
    f.pr = df_mul(df_sub(df_mul(r, q1), df_mul(df_sub(r, k.M), q2)), iS);
    f.pth = df_neg(df_mul(df_mul(sc, iS), t2));
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

}  // namespace tt

// arith.cuh -- arithmetic policies of the GB300 kernels.
//
// Three policies share one kernel source:
//   F64 : storage double, arithmetic double (native FP64; 1/72 of the FP32 rate on GB300).
//   F32 : storage float,  arithmetic float.
//   DW  : storage float2 {hi, lo}, arithmetic on double-word numbers (hi + lo, |lo| <= ulp(hi)/2)
//         built from error-free transformations on the FP32 units, giving about 2^-47 relative
//         accuracy per operation at a fraction of the cost of native FP64 on this part.
//         The algorithms are the published ones: TwoSum (Knuth, TAOCP vol. 2), Fast2Sum (Dekker
//         1971), TwoProd via FMA, and the double-word products of Joldes, Muller and Popescu,
//         "Tight and rigorous error bounds for basic building blocks of double-word arithmetic",
//         ACM TOMS 44(2), 2017 (DWTimesFP3 and DWTimesDW2). The sum is the "sloppy" double-word
//         sum (TwoSum of the high parts plus the low parts, renormalised): its error is bounded by
//         a few units of 2^-48 times |a| + |b|, the absolute accuracy a stencil sum needs.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpmg {

struct dw {
    float hi, lo;
};

// ---------------------------------------------------------------- error-free transformations
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dw dw_add(dw a, dw b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    dw z;
    fast_two_sum(s, e, z.hi, z.lo);
    return z;
}
__device__ __forceinline__ dw dw_neg(dw a) { return dw{-a.hi, -a.lo}; }
__device__ __forceinline__ dw dw_sub(dw a, dw b) { return dw_add(a, dw_neg(b)); }

// DWTimesFP3: double-word times float, with FMA.
__device__ __forceinline__ dw dw_mul_f(dw a, float b) {
    float ch = __fmul_rn(a.hi, b);
    float cl1 = __fmaf_rn(a.hi, b, -ch);
    float cl3 = __fmaf_rn(a.lo, b, cl1);
    dw z;
    fast_two_sum(ch, cl3, z.hi, z.lo);
    return z;
}
// DWTimesDW2: double-word times double-word, with FMA.
__device__ __forceinline__ dw dw_mul(dw a, dw b) {
    float ch = __fmul_rn(a.hi, b.hi);
    float cl1 = __fmaf_rn(a.hi, b.hi, -ch);
    float tl = __fmul_rn(a.hi, b.lo);
    float cl2 = __fmaf_rn(a.lo, b.hi, tl);
    float cl3 = __fadd_rn(cl1, cl2);
    dw z;
    fast_two_sum(ch, cl3, z.hi, z.lo);
    return z;
}
// a*b + c without renormalising the product: the exact product of the high parts (FMA TwoProd)
// plus the cross terms, added to c by TwoSum of the high parts and a float sum of the rest, then
// one Fast2Sum. The error is a few units of 2^-48 times |a*b| + |c|, like DWTimesDW2 followed by
// the sum, at 15 instead of 18 operations.
__device__ __forceinline__ dw dw_fma(dw a, dw b, dw c) {
    float ph = __fmul_rn(a.hi, b.hi);
    float pl = __fmaf_rn(a.hi, b.hi, -ph);
    pl = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pl));
    float s, e;
    two_sum(ph, c.hi, s, e);
    const float t = __fadd_rn(e, __fadd_rn(pl, c.lo));
    dw z;
    fast_two_sum(s, t, z.hi, z.lo);
    return z;
}
// (a + b) + (c + d): TwoSum on the high parts, all low parts and rounding errors summed in float,
// one Fast2Sum at the end (27 operations instead of 33 for three double-word sums)
__device__ __forceinline__ dw dw_sum4(dw a, dw b, dw c, dw d) {
    float s1, e1, s2, e2, s3, e3;
    two_sum(a.hi, b.hi, s1, e1);
    two_sum(c.hi, d.hi, s2, e2);
    two_sum(s1, s2, s3, e3);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(c.lo, d.lo)),
                               __fadd_rn(__fadd_rn(e1, e2), e3));
    dw z;
    fast_two_sum(s3, lo, z.hi, z.lo);
    return z;
}

// The same three operations without the final Fast2Sum: the result (s, t) is an unnormalised
// pair (|t| may exceed ulp(s)/2 by a few ulps of the low part) whose value hi + lo carries the same
// accuracy. Every operation above accepts such a pair as input (TwoSum needs no ordering; in the
// products the low part only enters the FP32 cross terms), so a chain renormalises once, at its
// end. Used inside the stencil and the forward elimination (three fewer operations each).
__device__ __forceinline__ dw dw_fma_u(dw a, dw b, dw c) {
    float ph = __fmul_rn(a.hi, b.hi);
    float pl = __fmaf_rn(a.hi, b.hi, -ph);
    pl = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pl));
    float s, e;
    two_sum(ph, c.hi, s, e);
    return dw{s, __fadd_rn(e, __fadd_rn(pl, c.lo))};
}
__device__ __forceinline__ dw dw_sum4_u(dw a, dw b, dw c, dw d) {
    float s1, e1, s2, e2, s3, e3;
    two_sum(a.hi, b.hi, s1, e1);
    two_sum(c.hi, d.hi, s2, e2);
    two_sum(s1, s2, s3, e3);
    return dw{s3, __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(c.lo, d.lo)), __fadd_rn(__fadd_rn(e1, e2), e3))};
}
__device__ __forceinline__ dw dw_mul_u(dw a, dw b) {
    float ch = __fmul_rn(a.hi, b.hi);
    float cl1 = __fmaf_rn(a.hi, b.hi, -ch);
    float tl = __fmul_rn(a.hi, b.lo);
    float cl2 = __fmaf_rn(a.lo, b.hi, tl);
    return dw{ch, __fadd_rn(cl1, cl2)};
}
__device__ __forceinline__ dw dw_add_u(dw a, dw b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return dw{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// 1/a: correctly rounded float reciprocal of the high part refined by one Newton step evaluated
// in double-word arithmetic: y = y0 + y0 (1 - a y0). Relative error about 2^-47.
__device__ __forceinline__ dw dw_rcp(dw a) {
    float y0 = __frcp_rn(a.hi);
    dw t = dw_mul_f(a, y0);                     // a*y0 = 1 - delta
    float e = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);  // 1 - t.hi is exact (Sterbenz)
    dw z;
    fast_two_sum(y0, __fmul_rn(y0, e), z.hi, z.lo);
    return z;
}

// ---------------------------------------------------------------- policy traits
// Each policy provides: storage type S, arithmetic type R, load/store, cst (from a double
// constant), to_d, to_f/from_f (to and from float, for the mixed-precision hand-over), add, sub,
// mul, fma, rcp, and acc_dot (accumulate a*b into a per-thread partial sum, read with acc_get).

struct PolF64 {
    typedef double S;
    typedef double R;
    static constexpr int id = 0;
    __device__ __forceinline__ static R ld(const S* p, size_t i) { return __ldg(p + i); }
    __device__ __forceinline__ static R ld_plain(const S* p, size_t i) { return p[i]; }
    __device__ __forceinline__ static void st(S* p, size_t i, R x) { p[i] = x; }
    // scratch store (never rounded to a storage format) and the storage rounding of a value
    __device__ __forceinline__ static void sts(S* p, size_t i, R x) { p[i] = x; }
    __device__ __forceinline__ static R rnd(R x) { return x; }
    __device__ __forceinline__ static R cst(double x) { return x; }
    // the same conversion on the host, for constants handed to kernels ready-made
    static R hcst(double x) { return x; }
    __device__ __forceinline__ static double to_d(R x) { return x; }
    __device__ __forceinline__ static R zero() { return 0.0; }
    __device__ __forceinline__ static R add(R a, R b) { return a + b; }
    __device__ __forceinline__ static R sub(R a, R b) { return a - b; }
    __device__ __forceinline__ static R mul(R a, R b) { return a * b; }
    // a*b + c
    __device__ __forceinline__ static R fma(R a, R b, R c) { return ::fma(a, b, c); }
    __device__ __forceinline__ static R sum4(R a, R b, R c, R d) { return (a + b) + (c + d); }
    // the unnormalised forms of double-word chains (the plain operations here)
    __device__ __forceinline__ static R fma_u(R a, R b, R c) { return ::fma(a, b, c); }
    __device__ __forceinline__ static R sum4_u(R a, R b, R c, R d) { return (a + b) + (c + d); }
    __device__ __forceinline__ static R add_u(R a, R b) { return a + b; }
    __device__ __forceinline__ static R mul_u(R a, R b) { return a * b; }
    __device__ __forceinline__ static R neg(R a) { return -a; }
    __device__ __forceinline__ static R rcp(R a) { return 1.0 / a; }
    // per-thread partial sum type for dot products and norms
    typedef double Acc;
    __device__ __forceinline__ static void acc_dot(Acc& s, Acc& c, R a, R b) { s = ::fma(a, b, s); }
    __device__ __forceinline__ static double acc_get(Acc s, Acc c) { return s; }
    __device__ __forceinline__ static float to_f(R x) { return __double2float_rn(x); }
    __device__ __forceinline__ static R from_f(float x) { return (double)x; }
};

struct PolF32 {
    typedef float S;
    typedef float R;
    static constexpr int id = 1;
    __device__ __forceinline__ static R ld(const S* p, size_t i) { return __ldg(p + i); }
    __device__ __forceinline__ static R ld_plain(const S* p, size_t i) { return p[i]; }
    __device__ __forceinline__ static void st(S* p, size_t i, R x) { p[i] = x; }
    __device__ __forceinline__ static void sts(S* p, size_t i, R x) { p[i] = x; }
    __device__ __forceinline__ static R rnd(R x) { return x; }
    __device__ __forceinline__ static R cst(double x) { return (float)x; }
    static R hcst(double x) { return (float)x; }  // round to nearest, as on the device
    __device__ __forceinline__ static double to_d(R x) { return (double)x; }
    __device__ __forceinline__ static R zero() { return 0.0f; }
    __device__ __forceinline__ static R add(R a, R b) { return a + b; }
    __device__ __forceinline__ static R sub(R a, R b) { return a - b; }
    __device__ __forceinline__ static R mul(R a, R b) { return a * b; }
    __device__ __forceinline__ static R fma(R a, R b, R c) { return fmaf(a, b, c); }
    __device__ __forceinline__ static R sum4(R a, R b, R c, R d) { return (a + b) + (c + d); }
    __device__ __forceinline__ static R fma_u(R a, R b, R c) { return fmaf(a, b, c); }
    __device__ __forceinline__ static R sum4_u(R a, R b, R c, R d) { return (a + b) + (c + d); }
    __device__ __forceinline__ static R add_u(R a, R b) { return a + b; }
    __device__ __forceinline__ static R mul_u(R a, R b) { return a * b; }
    __device__ __forceinline__ static R neg(R a) { return -a; }
    __device__ __forceinline__ static R rcp(R a) { return __frcp_rn(a); }
    // Kahan-compensated float partial sums (the FP32 pipe is the fast one on this part)
    typedef float Acc;
    __device__ __forceinline__ static void acc_dot(Acc& s, Acc& c, R a, R b) {
        float y = __fsub_rn(__fmul_rn(a, b), c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ static double acc_get(Acc s, Acc c) { return (double)s - (double)c; }
    __device__ __forceinline__ static float to_f(R x) { return x; }
    __device__ __forceinline__ static R from_f(float x) { return x; }
};

struct PolDW {
    typedef float2 S;
    typedef dw R;
    static constexpr int id = 2;
    __device__ __forceinline__ static R ld(const S* p, size_t i) {
        float2 v = __ldg(p + i);
        return dw{v.x, v.y};
    }
    __device__ __forceinline__ static R ld_plain(const S* p, size_t i) {
        float2 v = p[i];
        return dw{v.x, v.y};
    }
    __device__ __forceinline__ static void st(S* p, size_t i, R x) { p[i] = make_float2(x.hi, x.lo); }
    __device__ __forceinline__ static void sts(S* p, size_t i, R x) { p[i] = make_float2(x.hi, x.lo); }
    __device__ __forceinline__ static R rnd(R x) { return x; }
    __device__ __forceinline__ static R cst(double x) {
        float h = __double2float_rn(x);
        return dw{h, __double2float_rn(x - (double)h)};
    }
    // the same split on the host (x - h is exact in double; both roundings to nearest)
    static R hcst(double x) {
        const float h = (float)x;
        return dw{h, (float)(x - (double)h)};
    }
    __device__ __forceinline__ static double to_d(R x) { return (double)x.hi + (double)x.lo; }
    __device__ __forceinline__ static R zero() { return dw{0.0f, 0.0f}; }
    __device__ __forceinline__ static R add(R a, R b) { return dw_add(a, b); }
    __device__ __forceinline__ static R sub(R a, R b) { return dw_sub(a, b); }
    __device__ __forceinline__ static R mul(R a, R b) { return dw_mul(a, b); }
    __device__ __forceinline__ static R fma(R a, R b, R c) { return dw_fma(a, b, c); }
    __device__ __forceinline__ static R sum4(R a, R b, R c, R d) { return dw_sum4(a, b, c, d); }
    __device__ __forceinline__ static R fma_u(R a, R b, R c) { return dw_fma_u(a, b, c); }
    __device__ __forceinline__ static R sum4_u(R a, R b, R c, R d) { return dw_sum4_u(a, b, c, d); }
    __device__ __forceinline__ static R add_u(R a, R b) { return dw_add_u(a, b); }
    __device__ __forceinline__ static R mul_u(R a, R b) { return dw_mul_u(a, b); }
    __device__ __forceinline__ static R neg(R a) { return dw_neg(a); }
    __device__ __forceinline__ static R rcp(R a) { return dw_rcp(a); }
    // Kahan-compensated float partial sums of hi*hi + 2 hi*lo (relative accuracy ~1e-7 per
    // column sum, ample for a convergence test; block and grid stages run in FP64)
    typedef float Acc;
    __device__ __forceinline__ static void acc_dot(Acc& s, Acc& c, R a, R b) {
        float x = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.hi)));
        float y = __fsub_rn(x, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ static double acc_get(Acc s, Acc c) { return (double)s - (double)c; }
    __device__ __forceinline__ static float to_f(R x) { return __fadd_rn(x.hi, x.lo); }
    __device__ __forceinline__ static R from_f(float x) { return dw{x, 0.0f}; }
};

// FP32 arithmetic with every stored field value rounded to BF16 (8-bit significand, round to nearest
// even) and kept in an FP32 word: the values a BF16 store of the coarse levels would hold, used to
// measure how BF16 coarse-level storage affects convergence. Scratch (the Thomas stacks) is not
// rounded. It shares the FP32 workspaces and Thomas factors (id 1).
struct PolF32B : PolF32 {
    __device__ __forceinline__ static float rnd(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
    __device__ __forceinline__ static void st(S* p, size_t i, R x) { p[i] = rnd(x); }
};

}  // namespace tpmg

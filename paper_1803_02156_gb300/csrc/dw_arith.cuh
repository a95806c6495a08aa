// Double-word ("float-float") arithmetic of the complex-double steps on the
// fp32 pipe: every double carried as an unevaluated sum hi + lo of two floats
// (Dekker 1971), products through Dekker's TwoProduct via FMA, sums through
// Knuth's TwoSum, a row sum's errors collected in a second float (Ogita, Rump
// and Oishi 2005, Dot2).  Shared by the gathered and the footprint-staged
// double-word steps, so both round identically.
#pragma once

#include <cuda_runtime.h>

namespace cfd {
namespace {

// s + e = a + b exactly, s = fl(a + b) (Knuth's TwoSum; no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// (s, e) += (ah + al) (bh + bl): the product's high part enters s through
// TwoSum, its rounding error, the cross terms and the sum's error enter e.
__device__ __forceinline__ void dw_mac(float &s, float &e, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float pe = __fmaf_rn(ah, bh, -p);
    pe = __fmaf_rn(ah, bl, pe);
    pe = __fmaf_rn(al, bh, pe);
    float t, err;
    two_sum(s, p, t, err);
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, pe));
}

// x + g v for double-words x = (xh, xl), g = (gh, gl), v = (vh, vl), renormalised.
__device__ __forceinline__ void dw_axpy(float &xh, float &xl, float gh, float gl, float vh, float vl) {
    const float p = __fmul_rn(gh, vh);
    float pe = __fmaf_rn(gh, vh, -p);
    pe = __fmaf_rn(gh, vl, pe);
    pe = __fmaf_rn(gl, vh, pe);
    float t, err;
    two_sum(xh, p, t, err);
    const float lo = __fadd_rn(xl, __fadd_rn(pe, err));
    xh = __fadd_rn(t, lo);
    xl = __fsub_rn(lo, __fsub_rn(xh, t));
}

__device__ __forceinline__ float4 ld_nc4(const float4 *p) { return __ldg(p); }

// The same operations on two lanes at once with Blackwell's packed fp32x2
// instructions (FADD2, FMUL2, FFMA2: one issue slot for two round-to-nearest
// operations, each lane rounded exactly as the scalar instruction would).
// The step is issue bound, and the real and imaginary parts of a complex
// element run the same operation sequence, so pairing them halves the
// floating-point instructions; every lane's arithmetic is the scalar
// recipe's (dw_mac, two_sum, dw_axpy) bit for bit.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 swap2(float2 a) { return make_float2(a.y, a.x); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e) {
    s = __fadd2_rn(a, b);
    const float2 bv = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bv)))), __fadd2_rn(b, neg2(bv)));
}

// (s, e) += (hh + hl) (vh + vl) lanewise; nhh = -hh, nhl = -hl.  The product
// error is carried negated (ne = p - hh vh, exact, then minus the cross
// terms), which rounds to the negation of the scalar recipe's pe.
__device__ __forceinline__ void dw_mac2(float2 &s, float2 &e, float2 hh, float2 nhh, float2 nhl, float2 vh,
                                        float2 vl) {
    const float2 p = __fmul2_rn(hh, vh);
    float2 ne = __ffma2_rn(nhh, vh, p);
    ne = __ffma2_rn(nhh, vl, ne);
    ne = __ffma2_rn(nhl, vh, ne);
    float2 t, err;
    two_sum2(s, p, t, err);
    s = t;
    e = __fadd2_rn(e, __fadd2_rn(err, neg2(ne)));
}

// x + g v lanewise for double-words (xh, xl), g = (gh, gl) with ngh = -gh,
// ngl = -gl, v = (vh, vl); renormalised as dw_axpy.
__device__ __forceinline__ void dw_axpy2(float2 &xh, float2 &xl, float2 gh, float2 ngh, float2 ngl, float2 vh,
                                         float2 vl) {
    const float2 p = __fmul2_rn(gh, vh);
    float2 ne = __ffma2_rn(ngh, vh, p);
    ne = __ffma2_rn(ngh, vl, ne);
    ne = __ffma2_rn(ngl, vh, ne);
    float2 t, err;
    two_sum2(xh, p, t, err);
    const float2 lo = __fadd2_rn(xl, __fadd2_rn(err, neg2(ne)));
    xh = __fadd2_rn(t, lo);
    xl = __fadd2_rn(lo, neg2(__fadd2_rn(xh, neg2(t))));
}

// (s, e) <- (s + e, its rounding error) lanewise (Dekker's Fast2Sum, exact
// when |s| >= |e|): keeps the collected error term of a long sum at the
// size of one rounding of s, so its own roundings stay at 2^-48 of s.
__device__ __forceinline__ void renorm2(float2 &s, float2 &e) {
    const float2 t = __fadd2_rn(s, e);
    e = __fadd2_rn(e, neg2(__fadd2_rn(t, neg2(s))));
    s = t;
}

}  // namespace
}  // namespace cfd

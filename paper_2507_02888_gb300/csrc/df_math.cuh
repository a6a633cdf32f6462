// Double-float arithmetic for the tiered FP64 form: a value is the
// unevaluated sum hi + lo of two floats (48 significant bits), so FP64-grade
// results come from GB300's FP32 pipe, ~70x wider than its FP64 pipe.
// Products use the exact FMA residual of hi * hi plus the cross terms, sums
// Knuth's two-sum; every result is renormalised by a fast two-sum (Dekker
// 1971, the standard double-float arithmetic).  Each operation has a
// relative error of a few 2^-48.
#pragma once
#include <cuda_runtime.h>

#include "erfc_df_coeffs.h"

namespace ewald {

struct DF {
    float h, l;
};
struct CDF {
    DF x, y;
};

__device__ __forceinline__ DF df_from(double v) {
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.h + (double)a.l; }

// exact a + b of two floats (Knuth)
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bp = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.h, b.h), bp = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bp)), __fsub_rn(b.h, bp));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// a * b + c, the product's residual and c's low part folded before one
// renormalisation (the Horner step)
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const DF s = df_two_sum(p, c.h);
    const float t = __fadd_rn(s.l, __fadd_rn(e, c.l));
    const float h = __fadd_rn(s.h, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s.h))};
}

// a * b + sg * c * d (sg = +-1): the two leading products exactly (FMA
// residuals), their sum by two-sum, the cross terms into the residual
__device__ __forceinline__ DF df_dot2(DF a, DF b, DF c, DF d, float sg) {
    const float p1 = __fmul_rn(a.h, b.h), e1 = __fmaf_rn(a.h, b.h, -p1);
    const float cs = sg * c.h;
    const float p2 = __fmul_rn(cs, d.h), e2 = __fmaf_rn(cs, d.h, -p2);
    const float s = __fadd_rn(p1, p2), bp = __fsub_rn(s, p1);
    float t = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bp)), __fsub_rn(p2, bp));
    t = __fadd_rn(t, __fadd_rn(e1, e2));
    t = __fmaf_rn(a.h, b.l, t);
    t = __fmaf_rn(a.l, b.h, t);
    t = __fmaf_rn(cs, d.l, t);
    t = __fmaf_rn(sg * c.l, d.h, t);
    const float h = __fadd_rn(s, t);
    return {h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ CDF cdf_mul(const CDF &a, const CDF &b) {
    return {df_dot2(a.x, b.x, a.y, b.y, -1.0f), df_dot2(a.x, b.y, a.y, b.x, 1.0f)};
}

// An integer below 2^31 in magnitude, exactly: its top bits (exact in a
// float) plus its low byte.
__device__ __forceinline__ DF df_from_int(int v) {
    return df_two_sum(__fmul_rn(__int2float_rn(v >> 8), 256.0f), __int2float_rn(v & 255));
}

// A 64-bit fixed-point difference d (2^64 = one lattice period) as a
// double-float in units of 2^-32 of the period: d / 2^32, exact to 48 bits.
__device__ __forceinline__ DF df_from_fixed(long long d) {
    const DF hi = df_from_int((int)(d >> 32));
    const unsigned lo = (unsigned)d;
    const DF l = df_two_sum(__fmul_rn(__uint2float_rn(lo >> 8), 0x1p-24f), __fmul_rn(__uint2float_rn(lo & 255u), 0x1p-32f));
    return df_add(hi, l);
}

// 1 / sqrt(a): the hardware estimate, then two Newton steps in double-float
// (each squares the relative error: 2^-22 -> 2^-44 -> below 2^-48)
__device__ __forceinline__ DF df_rsqrt(DF a) {
    float y0;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(a.h));
    DF y = {y0, 0.0f};
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const DF t = df_mul(a, df_mul(y, y));  // a y^2, close to 1
        const DF e = df_add(DF{1.0f, 0.0f}, DF{-t.h, -t.l});
        y = df_fma(DF{0.5f * y.h, 0.5f * y.l}, e, y);  // y + (y / 2)(1 - a y^2)
    }
    return y;
}

// erfc(x) for 0 <= x < 4: the piece of width 1/8 holding x, Horner in
// s = x - c_m on its Taylor coefficients (erfc_df_coeffs.h)
__device__ __forceinline__ DF df_erfc(DF x) {
    const int m = min(max((int)(x.h * kErfcDfWidthInv), 0), kErfcDfPieces - 1);
    const DF s = df_add(x, DF{-((float)m + 0.5f) / kErfcDfWidthInv, 0.0f});
    const float2 *a = kErfcDf[m];
    float2 c = __ldg(a + kErfcDfDeg);
    DF p = {c.x, c.y};
#pragma unroll
    for (int k = kErfcDfDeg - 1; k >= 0; --k) {
        c = __ldg(a + k);
        p = df_fma(p, s, DF{c.x, c.y});
    }
    return p;
}

}  // namespace ewald

// Double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2 (about 48
// significant bits, the FP32 exponent range).  The operations are built from error-free
// transformations:
//   two_sum       Knuth's TwoSum (TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact rounding error;
//   fast_two_sum  Dekker's Fast2Sum (1971) for |a| >= |b| (or a = 0);
//   two_prod      Dekker's TwoProduct, written with one fused multiply-add: e = fma(a, b, -fl(a b)).
// Additions use the "sloppy" double-float sum (hi parts by TwoSum, lo parts added in FP32, one
// renormalisation), whose error is a few units of 2^-48 of the larger operand.  The intrinsics with an
// explicit rounding mode (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from contracting or
// reassociating the error terms.
//
// On GB300 the FP64 pipe issues about 2 thread-operations per SM cycle against 128 for FP32, so a
// double-float operation (3-15 FP32 instructions) is several times cheaper than one FP64 instruction.
#pragma once

#include <cuda_runtime.h>

struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo) {
    df r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
__device__ __forceinline__ df df_of(float x) { return df_make(x, 0.0f); }

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_neg(df a) { return df_make(-a.hi, -a.lo); }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a * b: hi product and its exact error, plus the cross terms a.hi b.lo + a.lo b.hi
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a * b with b a plain FP32 value
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}
// c - a * b with one renormalisation: the product's hi part enters TwoSum with c.hi, its error term
// and c.lo are added in FP32
__device__ __forceinline__ df df_fms(df c, df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df s = two_sum(c.hi, -p);
    s.lo = __fadd_rn(s.lo, __fsub_rn(c.lo, e));
    return fast_two_sum(s.hi, s.lo);
}
// c + a * b
__device__ __forceinline__ df df_fma(df c, df a, df b) { return df_fms(c, df_neg(a), b); }
__device__ __forceinline__ df df_sqr(df a) { return df_mul(a, a); }

// 1 / d for d.hi > 0 (normal): the hardware FP32 reciprocal approximation r0 (rcp.approx.ftz.f32,
// within 1 ulp) refined by one Newton-Raphson step r = r0 + r0 (1 - d r0), with 1 - d r0 formed from
// the exact product d.hi r0 (TwoProduct; 1 - fl(d.hi r0) is exact by Sterbenz's lemma) minus d.lo r0.
// The step squares the relative error: about 2^-45.
__device__ __forceinline__ df df_rcp(df d) {
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d.hi));
    const float p = __fmul_rn(d.hi, r0);
    const float pe = __fmaf_rn(d.hi, r0, -p);
    float e = __fsub_rn(__fsub_rn(1.0f, p), pe);
    e = __fmaf_rn(-d.lo, r0, e);
    return fast_two_sum(r0, __fmul_rn(r0, e));
}

// FP64 -> double-float, on the integer pipe: with x = M 2^(E - 1075) (M the 53-bit significand),
// hi = round(M / 2^29) 2^(E - 1046) is assembled from its bit fields (a carry of the rounding moves
// into the exponent field) and the remainder R = M - round(M / 2^29) 2^29 (|R| <= 2^28) gives
// lo = (R 2^-29) 2^(E - 1046), rounded to FP32.  Outside 2^-103 <= |x| < 2^126 (and for 0) hi is the
// FP32 rounding of x and lo = 0.
__device__ __forceinline__ df df_from_double(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ffull);
    if (E < 920 || E > 1149) return df_make(__double2float_rn(x), 0.0f);
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned q = (unsigned)((M + (1ull << 28)) >> 29);                  // 2^23 <= q <= 2^24
    const int R = (int)((long long)M - ((long long)q << 29));                 // |R| <= 2^28
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __int_as_float((int)((((unsigned)(E - 896)) << 23) + (q - (1u << 23))) | (int)sign);
    const float scale = __int_as_float((E - 919) << 23);                      // 2^(E - 1046)
    float lo = __fmul_rn(__fmul_rn((float)R, 1.862645149230957e-09f), scale);  // R 2^-29 2^(E - 1046)
    if (sign) lo = -lo;
    return df_make(hi, lo);
}

// double-float -> FP64 (exact: both parts convert exactly, their sum has at most 49 significant bits)
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// hi is positive, finite and at least 2^-lg_min, at most 2^lg_max (on the bit pattern)
__device__ __forceinline__ bool df_in_range(df a, int lg_min, int lg_max) {
    const int bits = __float_as_int(a.hi);
    const int e = (bits >> 23) & 0xff;
    return bits > 0 && e >= 127 - lg_min && e <= 127 + lg_max;
}

// Natural logarithm of m 2^e (m > 0 in double-float) on the FP32 pipe: m is brought into
// [1/sqrt 2, sqrt 2) by one halving, s = (m - 1) / (m + 1) and ln m = 2 atanh s = 2 s sum_k s^2k / (2k + 1),
// the series summed by Horner's rule through s^22 (|s| < 0.172: the first omitted term is below 2^-58
// of the sum), plus e ln 2.  About 2^-44 relative error in ln m.
__device__ __forceinline__ df df_log_scaled(df m, int e) {
    if (m.hi > 1.41421354f) {
        m.hi *= 0.5f;
        m.lo *= 0.5f;
        ++e;
    }
    const df s = df_mul(df_sub(m, df_of(1.0f)), df_rcp(df_add(m, df_of(1.0f))));
    const df s2 = df_mul(s, s);
    df acc = df_rcp(df_of(23.0f));
#pragma unroll
    for (int k = 21; k >= 1; k -= 2) acc = df_fma(df_rcp(df_of((float)k)), s2, acc);
    const df lnm = df_mul(df_make(2.0f * s.hi, 2.0f * s.lo), acc);
    const df ln2 = df_from_double(0.6931471805599453);
    return df_add(lnm, df_mulf(ln2, __int2float_rn(e)));
}

// Product accumulator for log-determinants in double-float: the mantissa is renormalised into [1, 2)
// after every factor (exact scaling by a power of two) and the binary exponent kept as an integer, so
// many pivots are multiplied with one logarithm at the end.
struct DFLogAcc {
    df mant;
    int expo;
    __device__ __forceinline__ void init() {
        mant = df_of(1.0f);
        expo = 0;
    }
    __device__ __forceinline__ void mul(df x) {
        mant = df_mul(mant, x);
        const int e = ((__float_as_int(mant.hi) >> 23) & 0xff) - 127;
        const float sc = __int_as_float((127 - e) << 23);
        mant.hi = __fmul_rn(mant.hi, sc);
        mant.lo = __fmul_rn(mant.lo, sc);
        expo += e;
    }
    // multiplies by x > 0 given in FP64: x = m 2^e split on its bit fields (m in [1, 2) exact in FP64,
    // rounded to double-float), so pivots of any FP64 magnitude enter exactly up to the rounding of m
    __device__ __forceinline__ void mul_fp64(double x) {
        const long long b = __double_as_longlong(x);
        const int e = (int)((b >> 52) & 0x7ff) - 1023;
        mul(df_from_double(__longlong_as_double((b & 0xFFFFFFFFFFFFFll) | (1023ll << 52))));
        expo += e;
    }
    // product over the 32 lanes of a warp (all lanes call); the total is valid in lane 0
    __device__ __forceinline__ void warp_product() {
        for (int o = 16; o > 0; o >>= 1) {
            df m2;
            m2.hi = __shfl_down_sync(0xffffffffu, mant.hi, o);
            m2.lo = __shfl_down_sync(0xffffffffu, mant.lo, o);
            const int e2 = __shfl_down_sync(0xffffffffu, expo, o);
            mul(m2);
            expo += e2;
        }
    }
    __device__ __forceinline__ double log_value() const {
        return log(df_to_double(mant)) + (double)expo * 0.6931471805599453;
    }
    // the logarithm in double-float on the FP32 pipe (df_log_scaled)
    __device__ __forceinline__ df log_df() const { return df_log_scaled(mant, expo); }
};

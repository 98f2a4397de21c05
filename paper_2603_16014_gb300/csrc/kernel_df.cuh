// Kernel values and kernel factors in double-float arithmetic (df64.cuh), for the kernels that need more
// than FP32 without spending FP64 instructions: the posterior of FP32-transform digital nets and the
// eta-gradient contractions of FP64-mode fits.
//
// A kernel value is returned with a fixed power-of-two scale s (K s), so that digital nets keep their
// exact integer form: eta s^-1 is formed once per dimension and eta K = (eta s^-1)(K s) costs one
// double-float product.
//   DSI order 2 (Eq. 2.6): s = 2^33; 2^33 K(X / 2^32) = 3 2^32 - 2 b X - 5 2^(32 - b), b = clz(X) + 1
//     (3 2^32 at X = 0), an integer below 2^34 in magnitude: exact.
//   SI of smoothness alpha = 1..4 (Eq. 2.5): s = 1; K(u) = c0 - c1 P_alpha(w), w = u (1 - u), u = X / 2^32
//     (order 2: pi^4/45 - (2 pi^4/3) w^2): u and 1 - u are exact, w and the rest carry about 2^-47
//     relative error.
#pragma once

#include "df64.cuh"
#include "mtgp.h"

// v exactly as a float for |v| < 2^22: the bias 2^23 + 2^22 puts v into the mantissa field
__device__ __forceinline__ float small_int_float(int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; }

__device__ __forceinline__ df dsi2_scaled_df(uint32_t X) {
    const int b = __clz(X) + 1;
    const long long t5 = X ? (5LL << (b <= 32 ? 32 - b : 0)) : 0LL;
    const long long I = (3LL << 32) - 2LL * (long long)b * (long long)X - t5;
    // I = 2^20 Ih + Il with |Ih| < 2^14 and 0 <= Il < 2^20: both floats exact, TwoSum exact
    const int ih = (int)(I >> 20), il = (int)(I & 0xFFFFFLL);
    return two_sum(small_int_float(ih) * 1048576.0f, small_int_float(il));
}

// constants of the SI kernel of smoothness alpha (Eq. 2.5, the Bernoulli polynomial B_{2 alpha}(u) in
// w = u (1 - u)) as double-float pairs: K = c0 - c1 P_alpha(w) with P_1 = w, P_2 = w^2,
// P_3 = w^2 (1/2 + w), P_4 = w^2 (2/3 + w (4/3 + w))
struct Si2Consts {
    df c0, c1, two_thirds, four_thirds;
    int alpha;
};
__device__ __forceinline__ Si2Consts si2_consts(int alpha = 2) {
    Si2Consts c;
    c.alpha = alpha;
    const double c0 = alpha == 1 ? 3.2898681336964529 : alpha == 3 ? 2.0346861239688983
                    : alpha == 4 ? 2.0081547123958887 : 2.1646464674222763;
    const double c1 = alpha == 1 ? 19.739208802178717 : alpha == 3 ? 85.456817206693728
                    : alpha == 4 ? 60.244641371876660 : 64.939394022668291;
    c.c0 = df_from_double(c0);
    c.c1 = df_from_double(c1);
    c.two_thirds = df_from_double(2.0 / 3.0);
    c.four_thirds = df_from_double(4.0 / 3.0);
    return c;
}

__device__ __forceinline__ df si2_df(uint32_t X, const Si2Consts& c) {
    // u = X 2^-32 from the two 16-bit halves (both exact floats), joined by TwoSum: exact
    const df u = two_sum(small_int_float((int)(X >> 16)) * 0x1p-16f, small_int_float((int)(X & 0xFFFFu)) * 0x1p-32f);
    const df w = df_mul(u, df_sub(df_of(1.0f), u));
    df pw;
    if (c.alpha == 1) {
        pw = w;
    } else {
        pw = df_sqr(w);
        if (c.alpha == 3) pw = df_mul(pw, df_add(df_of(0.5f), w));
        else if (c.alpha == 4) pw = df_mul(pw, df_add(c.two_thirds, df_mul(w, df_add(c.four_thirds, w))));
    }
    return df_fms(c.c0, c.c1, pw);
}

// K s for a design kind (MTGP_DNET: the DSI order-2 value, scale 2^33; otherwise the SI value of the
// smoothness held by c)
__device__ __forceinline__ df kval_scaled_df(int kind, uint32_t X, const Si2Consts& c) {
    return kind == MTGP_DNET ? dsi2_scaled_df(X) : si2_df(X, c);
}
__device__ __forceinline__ double kval_scale_inv(int kind) { return kind == MTGP_DNET ? 0x1p-33 : 1.0; }

// 1 + t for a double-float t
__device__ __forceinline__ df df_one_plus(df t) {
    df s = two_sum(1.0f, t.hi);
    s.lo = __fadd_rn(s.lo, t.lo);
    return fast_two_sum(s.hi, s.lo);
}

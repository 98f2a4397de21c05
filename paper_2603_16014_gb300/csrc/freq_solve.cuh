// Per-frequency FP64 work of the equal-size path (Corollary "equal sizes"):
//   Lambda(f) = R o M(f) + sigma2 I  (T x T, Hermitian),  L D L^H factorisation,
//   log det, quad = rhat^H Lambda^-1 rhat, and for the gradient
//   G = Lambda^-1 - alpha alpha^H  (alpha = Lambda^-1 rhat) with its contractions:
//     dL/dsigma2 += tr G,  Gamma_tu += Re(G[u][t] mu_tu),  adjoint weights W_c(f).
#pragma once

#include <type_traits>

#include "mtgp_internal.cuh"

template <bool CPLX>
using Vt = typename std::conditional<CPLX, cx<double>, double>::type;

__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ cx<double> vmul(cx<double> a, cx<double> b) { return a * b; }
__device__ __forceinline__ double vscale(double a, double s) { return a * s; }
__device__ __forceinline__ cx<double> vscale(cx<double> a, double s) { return mk(a.re * s, a.im * s); }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ cx<double> vadd(cx<double> a, cx<double> b) { return a + b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ cx<double> vsub(cx<double> a, cx<double> b) { return a - b; }

// float <-> double on the integer pipe (every conversion instruction occupies the FP64 pipe like an
// FMA).  Normal numbers and zero convert exactly / round to nearest; FP32 subnormals flush to zero
// and doubles beyond the FP32 range become +-inf (values the spectra and weights never take).
__device__ __forceinline__ double f2d(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    unsigned long long mag = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
    mag = (e == 0u) ? 0ull : mag;
    mag = (e == 0xffu) ? ((0x7ffull << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)) : mag;
    return __longlong_as_double((long long)(sign | mag));
}
__device__ __forceinline__ float d2f(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned long long a = b & 0x7fffffffffffffffull;
    const unsigned ex = (unsigned)(a >> 52);
    // rebias the exponent (1023 -> 127) and round the mantissa at bit 29 (carry may bump the exponent)
    unsigned f = (unsigned)(((a - (896ull << 52)) + (1ull << 28)) >> 29);
    f = (ex <= 896u) ? 0u : f;
    f = (ex >= 1151u) ? 0x7f800000u : f;
    f = (ex == 0x7ffu && (a & 0xfffffffffffffull)) ? 0x7fc00000u : f;
    return __uint_as_float(sign | f);
}
template <typename S>
__device__ __forceinline__ double to_d(S x) { return (double)x; }
template <>
__device__ __forceinline__ double to_d<float>(float x) { return f2d(x); }
template <typename S>
__device__ __forceinline__ S from_d(double x) { return (S)x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return d2f(x); }

template <typename S, bool CPLX>
__device__ __forceinline__ Vt<CPLX> load_elem(const void* p, long long i) {
    if constexpr (CPLX) {
        cx<S> v = reinterpret_cast<const cx<S>*>(p)[i];
        return mk(to_d<S>(v.re), to_d<S>(v.im));
    } else {
        return to_d<S>(reinterpret_cast<const S*>(p)[i]);
    }
}
template <typename S, bool CPLX>
__device__ __forceinline__ void store_elem(void* p, long long i, Vt<CPLX> v) {
    if constexpr (CPLX) {
        reinterpret_cast<cx<S>*>(p)[i] = mk(from_d<S>(v.re), from_d<S>(v.im));
    } else {
        reinterpret_cast<S*>(p)[i] = from_d<S>(v);
    }
}
template <bool CPLX>
__device__ __forceinline__ Vt<CPLX> ld(const double* p, long long i) {
    if constexpr (CPLX) return mk(p[2 * i], p[2 * i + 1]);
    else return p[i];
}
template <bool CPLX>
__device__ __forceinline__ void st(double* p, long long i, Vt<CPLX> v) {
    if constexpr (CPLX) {
        p[2 * i] = v.re;
        p[2 * i + 1] = v.im;
    } else {
        p[i] = v;
    }
}

// 1 / x in FP64: the hardware reciprocal approximation r (rcp.approx.ftz.f64, about 20 correct bits)
// refined by one step of the third-order Householder iteration for 1/x, the geometric series
// 1/x = r / (1 - e) = r (1 + e + e^2 + ...) with e = 1 - x r truncated after e^2, which leaves a
// relative error of about e^3 (below FP64 rounding); exact division outside binary exponents
// [-1000, 1000], tested on the bit pattern so the common path issues no FP64 compare.
__device__ __forceinline__ double fast_rcp(double x) {
    const unsigned ex = (unsigned)(__double_as_longlong(x) >> 52) & 0x7ffu;
    if (ex < 23u || ex > 2023u) return 1.0 / x;
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    // with e = 1 - x r:  1/x = r (1 + e + e^2 + ...); r (1 + e + e^2) leaves a relative error e^3
    const double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

// x > 0 and finite, tested on the bit pattern (sign clear, not zero, exponent not all ones)
__device__ __forceinline__ bool pos_finite(double x) {
    long long b = __double_as_longlong(x);
    return b > 0 && (b >> 52) < 0x7ff;
}

// Product accumulator for log-determinants: keeps mantissa and binary exponent apart so many
// pivots can be multiplied with one log at the end (the exponent is read from the bit pattern).
struct LogAcc {
    double mant;
    long long expo;
    __device__ __forceinline__ void init() {
        mant = 1.0;
        expo = 0;
    }
    __device__ __forceinline__ void mul(double x) {
        mant *= x;
        long long bits = __double_as_longlong(mant);
        int e = (int)((bits >> 52) & 0x7ff) - 1023;
        // renormalise the mantissa into [1, 2)
        bits = (bits & ~(0x7ffLL << 52)) | (1023LL << 52);
        mant = __longlong_as_double(bits);
        expo += e;
    }
    __device__ __forceinline__ double log_value() const { return log(mant) + (double)expo * 0.6931471805599453; }
    // product over the 32 lanes of a warp (all lanes call); the total is valid in lane 0
    __device__ __forceinline__ void warp_product() {
        for (int o = 16; o > 0; o >>= 1) {
            double m2 = __shfl_down_sync(0xffffffffu, mant, o);
            long long e2 = __shfl_down_sync(0xffffffffu, expo, o);
            mul(m2);
            expo += e2;
        }
    }
};

// Solve one frequency.  mu[t][u] (t <= u) are the first-column transforms M(f); rh[t] = rhat_t(f).
// Multiplies the pivots into lacc (log det), adds quad to acc[1]; with grad adds tr G to acc[2] and
// Gamma (upper triangle, row-major) to acc[3..]; writes the adjoint weights to w[t][u] (t < u, and
// w[0][0] = sum_t R_tt G_tt for the shared diagonal column) and alpha to al.
//   factor:  right-looking L D L^H, S_ij <- S_ij - L_ik conj(S_jk) for i >= j > k
//   inverse: Z[k][j] = -sum_{i>k} conj(L_ik) Z[i][j] (j > k),  Z[k][k] = 1/D_k - sum_{i>k} conj(L_ik) Z[i][k]
template <int T, bool CPLX>
__device__ __forceinline__ void solve_freq(Vt<CPLX> (&mu)[T][T], const Vt<CPLX> (&rh)[T], const double* sR, double sig,
                                           bool clamp, bool grad, LogAcc& lacc, double* acc, Vt<CPLX> (&w)[T][T],
                                           Vt<CPLX> (&al)[T], bool want_alpha, int& bad,
                                           const double* sigv = nullptr) {
    // sigv (optional): per-task noise (sorted order); its gradient traces go to acc[3 + T(T+1)/2 + t]
    using V = Vt<CPLX>;
    double mu0 = creal(mu[0][0]);
    double ind0 = 1.0;
    if (clamp && mu0 < 0.0) {
        mu0 = 0.0;
        ind0 = 0.0;
    }
    // lower triangle of Lambda(f): S[i][j] = Lambda[i][j] = R_ji conj(mu_ji) for i > j
    V S[T][T];
    double D[T], iD[T];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        D[i] = fma(sR[i * T + i], mu0, sigv ? sigv[i] : sig);
#pragma unroll
        for (int j = 0; j < i; ++j) S[i][j] = vscale(cconj(mu[j][i]), sR[j * T + i]);
    }
    V L[T][T];
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (!pos_finite(D[k])) {
            bad = 1;
            D[k] = 1.0;
        }
        iD[k] = fast_rcp(D[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) L[i][k] = vscale(S[i][k], iD[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) {
            D[i] -= creal(vmul(L[i][k], cconj(S[i][k])));
#pragma unroll
            for (int j = k + 1; j < i; ++j) S[i][j] = vsub(S[i][j], vmul(L[i][k], cconj(S[j][k])));
        }
    }
#pragma unroll
    for (int k = 0; k < T; ++k) lacc.mul(D[k]);
    V u[T];
#pragma unroll
    for (int k = 0; k < T; ++k) {
        V r = rh[k];
#pragma unroll
        for (int j = 0; j < k; ++j) r = vsub(r, vmul(L[k][j], u[j]));
        u[k] = r;
        acc[1] = fma(cabs2(r), iD[k], acc[1]);
    }
    if (!grad && !want_alpha) return;
#pragma unroll
    for (int k = T - 1; k >= 0; --k) {
        V a = vscale(u[k], iD[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) a = vsub(a, vmul(cconj(L[i][k]), al[i]));
        al[k] = a;
    }
    if (!grad) return;
    // lower triangle of Z = Lambda^-1:  Zl[j][k] = Z[j][k] (j >= k)
    V Zl[T][T];
#pragma unroll
    for (int k = T - 1; k >= 0; --k) {
#pragma unroll
        for (int j = T - 1; j > k; --j) {
            // Z[j][k] = conj(Z[k][j]) = -sum_{i>k} L_ik Z[j][i]
            V z = czero<V>();
#pragma unroll
            for (int i = k + 1; i < T; ++i) {
                V zji = (j >= i) ? Zl[j][i] : cconj(Zl[i][j]);
                z = vsub(z, vmul(L[i][k], zji));
            }
            Zl[j][k] = z;
        }
        double zkk = iD[k];
#pragma unroll
        for (int i = k + 1; i < T; ++i) zkk -= creal(vmul(cconj(L[i][k]), Zl[i][k]));
        Zl[k][k] = cfromreal<V>(zkk);
    }
    double wdiag = 0.0;
    int q = 3;
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int uu = t; uu < T; ++uu) {
            // G[uu][t] = Z[uu][t] - alpha_uu conj(alpha_t)   (uu >= t)
            if (uu == t) {
                double gd = creal(Zl[t][t]) - cabs2(al[t]);
                acc[2] += gd;
                if (sigv) acc[3 + T * (T + 1) / 2 + t] += gd;
                acc[q] = fma(gd, mu0, acc[q]);
                wdiag = fma(sR[t * T + t], gd, wdiag);
            } else {
                V g = vsub(Zl[uu][t], vmul(al[uu], cconj(al[t])));
                acc[q] += creal(vmul(g, mu[t][uu]));
                w[t][uu] = vscale(g, 2.0 * sR[t * T + uu]);
            }
            ++q;
        }
    }
    w[0][0] = cfromreal<V>(wdiag * ind0);
}

// ------------------------------------------------------------------- double-float solve (real data)

#include "df64.cuh"

// Working range of the double-float solve: pivots in [2^-kDfPivMin, 2^kDfPivMax], the quadratic form
// below 2^100, |alpha_k| and the diagonal of Lambda^-1 below 2^50 keep every product and sum of the
// recurrences inside the FP32 exponent range with their low parts normal.
constexpr int kDfPivMin = 50, kDfPivMax = 62;

// The recurrences of solve_freq for real data (digital nets) in double-float arithmetic, for
// FP32-transform mode, where the spectra mu arrive as FP32 values.  rh: transformed residuals,
// sR: R (T x T), sig: sigma2, all double-float.  Returns false, with no accumulator touched, when a
// pivot or an intermediate leaves the working range; the caller then solves the frequency with the
// FP64 recurrences.  A non-positive pivot sets `bad` (reported as not positive definite) and
// continues with D = 1, as the FP64 solve does.  acc[1] += quad, acc[2] += tr G, acc[3..] += Gamma;
// w receives the adjoint weights rounded to FP32.
template <int T>
__device__ __forceinline__ bool solve_freq_df(const float (&mu)[T][T], const df (&rh)[T], const df* sR, df sig,
                                              bool clamp, bool grad, DFLogAcc& lacc, df* acc, float (&w)[T][T],
                                              int& bad) {
    float mu0 = mu[0][0];
    float ind0 = 1.0f;
    if (clamp && mu0 < 0.0f) {
        mu0 = 0.0f;
        ind0 = 0.0f;
    }
    df S[T][T], D[T], iD[T], L[T][T];
#pragma unroll
    for (int i = 0; i < T; ++i) {
        D[i] = df_add(df_mulf(sR[i * T + i], mu0), sig);
#pragma unroll
        for (int j = 0; j < i; ++j) S[i][j] = df_mulf(sR[j * T + i], mu[j][i]);
    }
    int badk = 0;
#pragma unroll
    for (int k = 0; k < T; ++k) {
        if (!(D[k].hi > 0.0f) || !isfinite(D[k].hi)) {
            badk = 1;
            D[k] = df_of(1.0f);
        } else if (!df_in_range(D[k], kDfPivMin, kDfPivMax)) {
            return false;
        }
        iD[k] = df_rcp(D[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) L[i][k] = df_mul(S[i][k], iD[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) {
            D[i] = df_fms(D[i], L[i][k], S[i][k]);
#pragma unroll
            for (int j = k + 1; j < i; ++j) S[i][j] = df_fms(S[i][j], L[i][k], S[j][k]);
        }
    }
    df u[T];
    df quad = df_of(0.0f);
#pragma unroll
    for (int k = 0; k < T; ++k) {
        df r = rh[k];
#pragma unroll
        for (int j = 0; j < k; ++j) r = df_fms(r, L[k][j], u[j]);
        u[k] = r;
        quad = df_fma(quad, df_sqr(r), iD[k]);
    }
    if (!isfinite(quad.hi) || quad.hi > 0x1p100f) return false;
    if (!grad) {
#pragma unroll
        for (int k = 0; k < T; ++k) lacc.mul(D[k]);
        acc[1] = df_add(acc[1], quad);
        bad |= badk;
        return true;
    }
    df al[T];
    float big = 0.0f;
#pragma unroll
    for (int k = T - 1; k >= 0; --k) {
        df a = df_mul(u[k], iD[k]);
#pragma unroll
        for (int i = k + 1; i < T; ++i) a = df_fms(a, L[i][k], al[i]);
        al[k] = a;
        big = fmaxf(big, fabsf(a.hi));
    }
    // lower triangle of Z = Lambda^-1
    df Zl[T][T];
#pragma unroll
    for (int k = T - 1; k >= 0; --k) {
#pragma unroll
        for (int j = T - 1; j > k; --j) {
            df z = df_of(0.0f);
#pragma unroll
            for (int i = k + 1; i < T; ++i) z = df_fms(z, L[i][k], (j >= i) ? Zl[j][i] : Zl[i][j]);
            Zl[j][k] = z;
        }
        df zkk = iD[k];
#pragma unroll
        for (int i = k + 1; i < T; ++i) zkk = df_fms(zkk, L[i][k], Zl[i][k]);
        Zl[k][k] = zkk;
        big = fmaxf(big, zkk.hi);
    }
    // |alpha_k|^2 and Z_kk bound every entry of G = Z - alpha alpha^T (Cauchy-Schwarz on Z)
    if (!isfinite(big) || big > 0x1p50f) return false;
#pragma unroll
    for (int k = 0; k < T; ++k) lacc.mul(D[k]);
    acc[1] = df_add(acc[1], quad);
    bad |= badk;
    df wdiag = df_of(0.0f);
    int q = 3;
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int uu = t; uu < T; ++uu) {
            if (uu == t) {
                const df gd = df_fms(Zl[t][t], al[t], al[t]);
                acc[2] = df_add(acc[2], gd);
                acc[q] = df_add(acc[q], df_mulf(gd, mu0));
                wdiag = df_fma(wdiag, sR[t * T + t], gd);
            } else {
                const df g = df_fms(Zl[uu][t], al[uu], al[t]);
                acc[q] = df_add(acc[q], df_mulf(g, mu[t][uu]));
                // 2 R_tu g in double-float: its high part is the product rounded to FP32
                const df r2 = df_make(2.0f * sR[t * T + uu].hi, 2.0f * sR[t * T + uu].lo);
                w[t][uu] = df_mul(r2, g).hi;
            }
            ++q;
        }
    }
    w[0][0] = wdiag.hi * ind0;
    return true;
}

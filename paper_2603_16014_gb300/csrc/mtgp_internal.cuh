// Internal declarations shared by the CUDA translation units of the fast-MTGP library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mtgp.h"

#define MTGP_TMAX MTGP_MAX_TASKS
#define MTGP_MAX_COLS (MTGP_TMAX * (MTGP_TMAX + 1) / 2)

// status bits written by kernels (atomicOr); mtgp_sync maps the lowest set bit to an error code
#define ST_NOT_PD 1
#define ST_NUMERIC 2
#define ST_TIMEOUT 4

// ------------------------------------------------------------------------------- complex

template <typename S>
struct cx {
    S re, im;
};

template <typename S>
__host__ __device__ __forceinline__ cx<S> mk(S a, S b) { cx<S> r; r.re = a; r.im = b; return r; }
template <typename S>
__host__ __device__ __forceinline__ cx<S> operator+(cx<S> a, cx<S> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename S>
__host__ __device__ __forceinline__ cx<S> operator-(cx<S> a, cx<S> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename S>
__host__ __device__ __forceinline__ cx<S> operator*(cx<S> a, cx<S> b) {
    return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename S>
__host__ __device__ __forceinline__ cx<S> operator*(S a, cx<S> b) { return mk(a * b.re, a * b.im); }
template <typename S>
__host__ __device__ __forceinline__ cx<S> conj(cx<S> a) { return mk(a.re, -a.im); }
template <typename S>
__host__ __device__ __forceinline__ S norm2(cx<S> a) { return a.re * a.re + a.im * a.im; }

// Scalar-or-complex value used by the solvers: real problems (digital nets) use V = double,
// lattices use V = cx<double>.
__host__ __device__ __forceinline__ double cconj(double a) { return a; }
__host__ __device__ __forceinline__ cx<double> cconj(cx<double> a) { return conj(a); }
__host__ __device__ __forceinline__ double creal(double a) { return a; }
__host__ __device__ __forceinline__ double creal(cx<double> a) { return a.re; }
__host__ __device__ __forceinline__ double cabs2(double a) { return a * a; }
__host__ __device__ __forceinline__ double cabs2(cx<double> a) { return norm2(a); }
template <typename V> __host__ __device__ __forceinline__ V czero();
template <> __host__ __device__ __forceinline__ double czero<double>() { return 0.0; }
template <> __host__ __device__ __forceinline__ cx<double> czero<cx<double>>() { return mk(0.0, 0.0); }
template <typename V> __host__ __device__ __forceinline__ V cfromreal(double a);
template <> __host__ __device__ __forceinline__ double cfromreal<double>(double a) { return a; }
template <> __host__ __device__ __forceinline__ cx<double> cfromreal<cx<double>>(double a) { return mk(a, 0.0); }

// --------------------------------------------------------------------- fixed-point kernels

#define MTGP_2POW_M32 2.3283064365386962890625e-10  // 2^-32 exactly
#define MTGP_PI4_45 2.1646464674222763    // pi^4 / 45
#define MTGP_2PI4_3 64.939394022668291    // 2 pi^4 / 3

// Univariate SI kernel of Eq. 2.5 with alpha = 2: (2 pi)^4 / 4! * (1/30 - u^2 (1 - u)^2)
// = pi^4/45 - (2 pi^4 / 3) (u (1 - u))^2, u = X / 2^32 = (x - x') mod 1.  The kernel is
// symmetric under u -> 1 - u, so u is folded to [0, 1/2] in integer arithmetic first.
template <typename S>
__device__ __forceinline__ S si2_kernel(uint32_t X) {
    uint32_t Y = (X > 0x80000000u) ? (0u - X) : X;
    S u = (S)Y * (S)MTGP_2POW_M32;
    S w = u * ((S)1 - u);
    return (S)MTGP_PI4_45 - (S)MTGP_2PI4_3 * (w * w);
}

template <typename S>
__device__ __forceinline__ S pow2_neg(int b);  // 2^-b for 0 <= b <= 96
template <>
__device__ __forceinline__ float pow2_neg<float>(int b) { return __int_as_float((127 - b) << 23); }
template <>
__device__ __forceinline__ double pow2_neg<double>(int b) {
    return __longlong_as_double((long long)(1023 - b) << 52);
}

// Univariate DSI kernel of Eq. 2.6, order-2 term: -1 - beta(x) x + 5/2 (1 - 2^-beta(x)),
// beta(x) = -floor(log2 x) = clz(X) + 1 for x = X / 2^32 > 0, and 3/2 at x = 0.
template <typename S>
__device__ __forceinline__ S dsi2_kernel(uint32_t X) {
    if (X == 0u) return (S)1.5;
    int b = __clz(X) + 1;
    S x = (S)X * (S)MTGP_2POW_M32;
    return (S)1.5 - (S)b * x - (S)2.5 * pow2_neg<S>(b);
}

// FP32 without conversion instructions (they issue through the MIO queue): x = X 2^-32 is assembled from
// X shifted to its leading one (the exponent field from clz, the mantissa rounded to nearest with ties
// away from zero), beta = clz(X) + 1 as the float 2^23 + beta - 2^23 (exact), 2^-beta from its exponent.
template <>
__device__ __forceinline__ float dsi2_kernel<float>(uint32_t X) {
    const int lz = __clz(X);
    const uint32_t m = X << lz;                                   // leading one at bit 31
    const float x = __uint_as_float((uint32_t)(125 - lz) * 8388608u + (m >> 8) + ((m >> 7) & 1u));
    const float bf = __int_as_float(0x4B000000 | (lz + 1)) - 8388608.0f;
    const float pw = __int_as_float((126 - lz) << 23);            // 2^-(lz + 1)
    const float k = __fmaf_rn(-2.5f, pw, __fmaf_rn(-bf, x, 1.5f));
    return X == 0u ? 1.5f : k;
}

// FP64 forms assembled on the integer pipe.  |v| 2^-s as a double from integer fields: exact for
// v < 2^53, truncated to 53 significant bits above; the callers' scalings never underflow.
__device__ __forceinline__ double u64_times_pow2(unsigned long long v, int s, bool negative) {
    if (v == 0ull) return 0.0;
    const int lz = __clzll((long long)v);
    const unsigned long long m = v << lz;
    unsigned long long bits = ((unsigned long long)(1086 - lz - s) << 52) + ((m >> 11) & 0xFFFFFFFFFFFFFull);
    if (negative) bits |= 0x8000000000000000ull;
    return __longlong_as_double((long long)bits);
}

// SI kernel: u (1 - u) 2^64 = Y (2^32 - Y) is an exact 64-bit integer, leaving two FP64 operations.
template <>
__device__ __forceinline__ double si2_kernel<double>(uint32_t X) {
    const uint32_t Y = (X > 0x80000000u) ? (0u - X) : X;
    const double w = u64_times_pow2((unsigned long long)Y * (0x100000000ull - Y), 64, false);
    return fma(-MTGP_2PI4_3, w * w, MTGP_PI4_45);
}

// DSI kernel: 2^33 K(X / 2^32) = 3 2^32 - 2 b X - 5 2^(32-b) is an exact integer (|.| < 2^39), so K is
// exact and costs no FP64 operation.
template <>
__device__ __forceinline__ double dsi2_kernel<double>(uint32_t X) {
    long long I = 3LL << 32;
    if (X != 0u) {
        const int b = __clz(X) + 1;
        I -= 2LL * b * (long long)X + (5LL << (32 - b));
    }
    return u64_times_pow2((unsigned long long)(I < 0 ? -I : I), 33, I < 0);
}

// SI kernel of smoothness alpha = 1, 3, 4 (Eq. 2.5): the Bernoulli polynomial B_{2 alpha}(u) written
// in w = u (1 - u):  B2 = 1/6 - w,  B6 = -w^3 - w^2 / 2 + 1/42,  B8 = w^4 + 4/3 w^3 + 2/3 w^2 - 1/30.
template <typename S>
__device__ __forceinline__ S si_kernel_alpha(uint32_t X, int alpha) {
    const uint32_t Y = (X > 0x80000000u) ? (0u - X) : X;
    S w;
    if constexpr (sizeof(S) == 8) {
        w = u64_times_pow2((unsigned long long)Y * (0x100000000ull - Y), 64, false);
    } else {
        const S u = (S)Y * (S)MTGP_2POW_M32;
        w = u * ((S)1 - u);
    }
    if (alpha == 1) return (S)3.2898681336964529 - (S)19.739208802178717 * w;          // 2 pi^2 (1/6 - w)
    if (alpha == 3) return (S)2.0346861239688983 - (S)85.456817206693728 * (w * w * ((S)0.5 + w));
    // alpha = 4: -(2 pi^8 / 315) B8
    return (S)2.0081547123958887 - (S)60.244641371876660 * (w * w * ((S)2 / (S)3 + w * ((S)4 / (S)3 + w)));
}

template <typename S>
__device__ __forceinline__ S kernel1d(int kind, uint32_t X, int alpha = 2) {
    if (kind == MTGP_LATTICE) return alpha == 2 ? si2_kernel<S>(X) : si_kernel_alpha<S>(X, alpha);
    return dsi2_kernel<S>(X);
}

// Binary digits x_1..x_21 of x = X / 2^32 spread three bits apart: bit 3 (21 - a) holds x_a, so the
// word times 2^-60 is sum_{a <= 21} x_a 8^{1-a} (the standard Morton bit-interleave masks).
__device__ __forceinline__ unsigned long long spread3_top21(uint32_t X) {
    unsigned long long v = (unsigned long long)(X >> 11);
    v = (v | (v << 32)) & 0x001F00000000FFFFull;
    v = (v | (v << 16)) & 0x001F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// The four orders of the adaptive-smoothness DSI kernel (Eq. 2.6) at x = X / 2^32, with
// beta = clz(X) + 1, t_nu = 2^(-nu beta) and beta(0) = t_nu(0) = 0:
//   K1 = 1/6 - t1/2   (the order-one Walsh kernel: the printed form is read with mean zero)
//   K2 = 3/2 - beta x - 5/2 t1
//   K3 = 25/18 + beta x^2 - 5 x + 5 t1 x - 43/18 t2
//   K4 = 407/294 - 2/3 beta x^3 + 5 x^2 - 5 t1 x^2 - 43/9 x + 43/9 t2 x - 701/294 t3 + beta (D/48 - 1/42),
// D = sum_{a >= 1} (1 - 2 x_a) 8^(1-a) = 8/7 - 2 sum_a x_a 8^(1-a); digits past the 21st move D by
// less than 2^-61 and are dropped.
template <typename S>
__device__ __forceinline__ void dsi_orders(uint32_t X, S k[4]) {
    if (X == 0u) {
        k[0] = (S)(1.0 / 6.0);
        k[1] = (S)1.5;
        k[2] = (S)(25.0 / 18.0);
        k[3] = (S)(407.0 / 294.0);
        return;
    }
    const int b = __clz(X) + 1;
    const S bs = (S)b;
    const S x = (S)X * (S)MTGP_2POW_M32;
    const S t1 = pow2_neg<S>(b), t2 = pow2_neg<S>(2 * b), t3 = pow2_neg<S>(3 * b);
    const S x2 = x * x;
    k[0] = (S)(1.0 / 6.0) - (S)0.5 * t1;
    k[1] = (S)1.5 - bs * x - (S)2.5 * t1;
    k[2] = (S)(25.0 / 18.0) + bs * x2 - (S)5 * x + (S)5 * t1 * x - (S)(43.0 / 18.0) * t2;
    const S D = (S)(8.0 / 7.0) - (S)2 * ((S)spread3_top21(X) * pow2_neg<S>(60));
    k[3] = (S)(407.0 / 294.0) - (S)(2.0 / 3.0) * bs * x2 * x + (S)5 * x2 * ((S)1 - t1)
         - (S)(43.0 / 9.0) * x * ((S)1 - t2) - (S)(701.0 / 294.0) * t3 + bs * (D * (S)(1.0 / 48.0) - (S)(1.0 / 42.0));
}

// Univariate kernel of a handle: the DSI mixture sum_a b_a K_a when weights b are given (digital
// nets), else the single kernel of kernel1d.
template <typename S>
__device__ __forceinline__ S kernel1d_b(int kind, uint32_t X, int alpha, const S* b) {
    if (b == nullptr) return kernel1d<S>(kind, X, alpha);
    S k[4];
    dsi_orders<S>(X, k);
    return b[0] * k[0] + b[1] * k[1] + b[2] * k[2] + b[3] * k[3];
}

// Point z_i (unshifted) in coordinate j.  Lattice (Def. 2.1): v(i) g mod 1 = bitrev32(i) * g
// mod 2^32.  Digital net (Def. 2.2): XOR of generating-matrix columns g_p for the set bits of i.
__device__ __forceinline__ uint32_t point_word(int kind, uint32_t i, int j, const uint32_t* gen,
                                               int gen_cols) {
    if (kind == MTGP_LATTICE) return __brev(i) * gen[j];
    const uint32_t* g = gen + (size_t)j * gen_cols;
    uint32_t z = 0;
    while (i) {
        int p = __ffs(i) - 1;
        z ^= g[p];
        i &= i - 1;
    }
    return z;
}

// The combination x_{t,i} - x_{u,0} (lattice, mod 1) or x_{t,i} XOR x_{u,0} (digital net) that a
// first column of block (t, u) evaluates: z_i (+/-) Delta_t (-/XOR) Delta_u.
__device__ __forceinline__ uint32_t pair_word(int kind, uint32_t z, uint32_t dt, uint32_t du) {
    return kind == MTGP_LATTICE ? (z + dt - du) : (z ^ dt ^ du);
}

// ------------------------------------------------------------------------------- columns

// One first column of the block Gram matrix K~_{t,u} (sorted tasks, n_t >= n_u); for equal sizes
// all diagonal blocks share column 0.
struct ColDesc {
    long long off;  // element offset in the column buffers
    int n;          // length n_t
    int t, u;       // sorted task pair (t <= u)
    // complex (lattice) columns are real, so two of equal length share one complex transform: the
    // lead (role 1) in the real part, its partner (role 2) in the imaginary part of the lead's array
    // (src); role 0 is a column transformed alone
    long long src;
    int role;
};

struct Handle;

// ------------------------------------------------------------------------------- launchers

struct ThetaPtrs {
    const double* eta;
    const double* W;
    int s;
    const double* v;
    const double* sigma2;
    int nsig;  // noise values: 1 (shared sigma2) or T (per task, caller order); 0 reads as 1
    const double* bmix;  // DSI mixture weights b (4), or nullptr for the order-2 kernel alone
};

// noise variance of sorted task t
__device__ __forceinline__ double noise_of(const ThetaPtrs& th, const int* order, int t) {
    return th.nsig > 1 ? th.sigma2[order[t]] : th.sigma2[0];
}

// k_columns.cu
void launch_colgen(const Handle* h, const double* eta, void* out, cudaStream_t st);
void launch_points(const Handle* h, uint32_t* x, cudaStream_t st);
void launch_y_load(const Handle* h, const double* y, cudaStream_t st);
// paired columns: after the forward transform, Z = F(a + i b) -> F(a) = (Z + conj(Z(-f))) / 2 and
// F(b) = (Z - conj(Z(-f))) / (2i) into the lead's and the partner's arrays; before the adjoint
// transform, the lead's weights w_a + i w_b
void launch_pair_split(const Handle* h, void* spec, cudaStream_t st);
// posterior variance, unequal sizes: per (class block, query) sums of kappa^H Lambda~^-1 kappa over the
// transformed rows of B queries (N doubles / complex values per query), from the tree solver's factor
void launch_var_tree(const Handle* h, double* rows, int B, double* part, cudaStream_t st);
void launch_pair_pack(const Handle* h, void* wgt, cudaStream_t st);
void launch_eta_grad(const Handle* h, const double* eta, const void* omega, double* partials,
                     int nblk_max, cudaStream_t st);
int eta_grad_blocks(const Handle* h);

// k_transform.cu
// forward (DIT, bit-reversed input -> natural output) or adjoint (DIF, natural -> bit-reversed)
// transform of `narr` arrays of length 2^m at element offsets `offs` (device array).
void launch_transform(const Handle* h, void* base, bool fp32, bool complex_data, int m,
                      const long long* offs_dev, int narr, bool dif, cudaStream_t st);
void launch_twiddles(Handle* h, cudaStream_t st);

// k_solve.cu
int solve_equal_blocks(const Handle* h);
// gcv = 1: the GCV loss instead of the MLE loss; partial columns 2 and 3 then hold ||Lambda^-1 rhat||^2
// and trace(Lambda^-1).  gcv = 2 (equal sizes): the GCV gradient pass, reading [A, B] from gcv_ab,
// with the MLE gradient's partial layout and adjoint weights.
void launch_solve_equal(const Handle* h, ThetaPtrs th, bool grad, double* partials, cudaStream_t st,
                        int gcv = 0, const double* gcv_ab = nullptr);
void launch_solve_tree(const Handle* h, ThetaPtrs th, bool grad, double* partials, cudaStream_t st,
                       bool gcv = false);
int solve_tree_blocks(const Handle* h);
void launch_finalize(const Handle* h, ThetaPtrs th, bool grad, const double* partials, int nsolve,
                     const double* eta_partials, int neta, double* out, double* tau, double* g_eta,
                     double* g_W, double* g_v, double* g_s2, cudaStream_t st, int gcv = 0);

// k_fused_rt.cu: yhat rounded to double-float pairs (hi, lo) for the double-float solve
void launch_yhat_df(const double* yhat, float* yhat_df, long long n, cudaStream_t st);
// k_fused_rt.cu: theta-independent design words of the register-tile kernels, per handle:
// z_j(l) for the 32 lane offsets (d x 32), z_j(32 k) for k < n / 32 (d x n/32), shift XORs per column (C x d)
long long rt_words_len(const Handle* h);
void launch_rt_words(const Handle* h, cudaStream_t st);

// k_fused.cu (equal sizes)
bool fused_supported(const Handle* h);
long long fused_partials_len(const Handle* h);
void launch_fused(const Handle* h, ThetaPtrs th, bool grad, bool store_alpha, double* out, double* tau,
                  double* g_eta, double* g_W, double* g_v, double* g_s2, cudaStream_t st);
// split of n = 2^m between kernels A/C (2^a) and B (2^(m-a)); a_pref < 0 picks the default
bool fused_plan(int m, int ncols, int d, bool fp32, bool cplx, int a_pref, int* a_out, int* lgL_out);
// kernel family of a fit's fused evaluation: the generic shared-memory kernels (any split, complex
// spectra, FP64 transforms), or the register-tile kernels for FP32 real spectra with d <= 16 and both
// tile sizes in 2^5 .. 2^9 (k_fused_rt.cu), whose kernel B solves in FP64 (FUSED_RT) or in
// double-float (FUSED_RT_DF)
enum { FUSED_GENERIC = 0, FUSED_RT = 1, FUSED_RT_DF = 2 };
int fused_variant(bool fp32, bool cplx, bool solve_df, int d, int m, int a, bool store_alpha);
bool fused_rt_ok(bool cplx, bool fp32, int d, int m, int a);
int fused_rt_threads(int phase, int C, int m, int a);
size_t fused_rt_smem(int phase, int T, int C, int m, int a);
void fused_rt_phase(int phase, bool dfs, int T, int dmax, const void* single, const void* fits, const int2* items,
                    int nitems, int grid, int threads, size_t smem, cudaStream_t st);
int fused_rt_resident_blocks(int phase, bool dfs, int T, int dmax, int threads, size_t smem);
// device descriptor of one fit (fused_desc_size() bytes, written to desc) with split a and the given
// partial-sum buffer (2^a (NQ + 1) + 2^(m-a) d doubles) and counters (2 unsigned)
size_t fused_desc_size();
void fused_make_desc(const Handle* h, ThetaPtrs th, double* out, double* tau, double* g_eta, double* g_W,
                     double* g_v, double* g_s2, bool grad, int a, double* partials, unsigned* counters, void* desc);
// one phase (0 = A, 1 = B, 2 = C) of one class: `single` (host descriptor) launches one fit with a grid of
// its blocks, otherwise a persistent grid walks `nitems` (fit, block) items over the device descriptors
void fused_phase(int phase, int variant, bool fp32, bool cplx, int T, int dmax, const void* single, const void* fits,
                 const int2* items, int nitems, int grid, int threads, size_t smem, cudaStream_t st);
size_t fused_smem(int phase, int variant, int T, int C, int m, int a, bool fp32, bool cplx);
int fused_threads(int phase, int variant, int a, int d, int C, int m);
int fused_resident_blocks(int phase, int variant, bool fp32, bool cplx, int T, int dmax, int threads, size_t smem);

// k_mlp.cu: input width, output width and largest batch of a network
void mlp_shape(const mtgp_mlp_t* m, int* in_width, int* out_width, int* max_batch);

// records the message returned by mtgp_last_error_string for the calling thread (mtgp_api.cu)
void mtgp_set_error(const char* msg);

// kernel timing (mtgp_api.cu): no-ops unless profiling is enabled on the handle
void mtgp_prof_begin(const Handle* h, const char* name, cudaStream_t st);
void mtgp_prof_end(const Handle* h, cudaStream_t st);

// k_posterior.cu
// k_posterior_df.cu: posterior of equal-size FP32-transform digital nets in double-float arithmetic
// (order-2 DSI kernel, d <= 16, n = 2^10 .. 2^18); xqw: query words, design: sorted design words, beta64:
// K~^-1 r (FP64, sorted layout)
bool posterior_df_ok(const Handle* h);
void posterior_df_release(const Handle* h);
int posterior_df_run(const Handle* h, ThetaPtrs th, int nq, const uint32_t* xqw, const int* task, const uint32_t* design,
                     const double* beta64, double* mean, double* var, cudaStream_t st);
int posterior_run(Handle* h, ThetaPtrs th, int nq, const double* xq, const int* task, double* mean,
                  double* var, cudaStream_t st);

// ------------------------------------------------------------------------------- handle

struct Handle {
    int kind, d, T, prec;
    bool fp32;           // transform precision
    bool solve_df;       // FP32 transforms: per-frequency solve in double-float (else FP64)
    bool cplx;           // lattice spectra are complex
    bool equal;          // all n_t equal
    int gen_cols;
    int m_user[MTGP_TMAX];
    int order[MTGP_TMAX];    // sorted position -> caller task
    int rank[MTGP_TMAX];     // caller task -> sorted position
    int m[MTGP_TMAX];        // sorted
    long long n[MTGP_TMAX];  // sorted
    long long N;
    long long yoff[MTGP_TMAX];  // element offset of sorted task t in yhat / per-task vectors
    int mmax;

    int ncols;
    ColDesc cols[MTGP_MAX_COLS];
    int col_of[MTGP_TMAX][MTGP_TMAX];  // sorted (t, u) with t <= u -> column
    long long col_elems;               // total elements over columns

    // device buffers
    uint32_t* gen;       // lattice: d words; dnet: d * gen_cols
    uint32_t* shift;     // sorted T x d
    ColDesc* cols_dev;
    int ngroups;
    int group_m[MTGP_TMAX];
    int group_first[MTGP_TMAX];
    int group_count[MTGP_TMAX];
    // the arrays the general path transforms (leads and lone columns), per group, and the pairs
    long long* lead_offs_dev;
    int group_lfirst[MTGP_TMAX];
    int group_lcount[MTGP_TMAX];
    int npairs;
    long long* pairs_dev;  // (lead offset, partner offset, length) per pair
    long long* yoffs_dev;  // per sorted task offset (for y transforms)

    void* twid;          // twiddle table e^{-2 pi i k / 2^mmax}, k < 2^{mmax-1}, double2 and float2
    void* twid32;
    double* yhat;        // FP64 (complex for lattice), sorted tasks, length N
    float* yhat_df;      // FP32-transform equal-size digital nets: yhat as double-float pairs (hi, lo), or null
    uint32_t* rt_words;  // the same handles: design words of the register-tile kernels (rt_words_len), or null
    void* spec;          // column spectra (E = fp32 ? float : double, complex for lattice)
    void* wgt;           // adjoint weights, same layout as spec
    double* S;           // tree solver scratch (pair layout, FP64 (complex))
    double* Z;           // tree solver selected inverse
    double* r;           // residual / forward-solve vector (N, FP64 (complex))
    double* alpha;       // Lambda^-1 rhat (N, FP64 (complex))
    double* tau;         // sorted optimal means (T)
    double* partials;    // per-block partial sums
    long long partials_len;
    int* status;
    double* out_tmp;     // NLL outputs of calls that only need the solve (posterior)
    double* gcv_h;       // GCV, unequal sizes: class-0 columns of Lambda^-1 (T + 1 rows, on first use)
    double* pi_buf;      // cubature, unequal sizes: Pi = E K~^-1 E^T from the tree solver (T x T, on first use)
    unsigned* counters;  // last-block election counters of the fused kernels (reset by the last block)
    struct Prof* prof;   // kernel timing log (host side)
    long long ws_bytes;
    bool y_set;
    int smooth;          // SI kernel smoothness alpha of Eq. 2.5 (lattices; 2 unless set)
    bool noise_pt;       // one noise variance per task (general path only)
    bool dsi_mix;        // digital nets: DSI mixture weights b set (general path only)
    double* bmix;        // device: b (4 doubles) then dL/db of the last gradient call (4 doubles)
    double* hio;         // device staging of the host-buffer entry point: packed theta, then outputs
    // the host-buffer entry point replays one CUDA graph (staging, kernels) per (device addresses of
    // the page-locked theta and out, s, configuration); a call that changes which kernels run bumps cfg_gen
    unsigned cfg_gen;
    cudaStream_t cap_stream;
    cudaGraphExec_t hio_exec;
    const void* hio_key_th;
    void* hio_key_out;
    int hio_key_s;
    unsigned hio_key_gen;
    bool hio_nograph;    // capture failed once: the direct launches are used from then on
};

// columns of the per-block partial sums of the general solvers: [log det, quad, trace G, Gamma (T(T+1)/2)]
// and, with per-task noise, the T per-task traces of G
inline int solve_nq(const Handle* h) { return 3 + h->T * (h->T + 1) / 2 + (h->noise_pt ? h->T : 0); }

__device__ __forceinline__ void set_status(int* st, int bit) { atomicOr(st, bit); }

struct mtgp_s {
    Handle h;
};

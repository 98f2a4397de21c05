// Posterior mean and variance (Eq. 3.2) of equal-size digital-net fits in FP32-transform mode, in
// double-float arithmetic (df64.cuh) on the FP32 pipe.
//
//   mean_t(x) = tau_t + sum_u R_tu sum_i Q(x, x_ui) beta_u[i]
//   var_t(x)  = R_tt Q(x, x) - sum_f kappa(f)^T Lambda(f)^-1 kappa(f),  kappa_u = R_tu H q_u(x) / sqrt(n)
//
// with q_u(x)[i] = Q(x, x_ui), H the Walsh-Hadamard transform of length n = 2^m and Lambda(f) = R o mu(f) +
// noise per frequency (Theorem "fast MTGP computations", Corollary "equal sizes").  Every kernel value is
// exact: 2^33 K(x) of the order-2 DSI kernel (Eq. 2.6) is an integer below 2^34 in magnitude, whose
// double-float form is exact; the factors 1 + eta_j K, their product, the transform and the quadratic
// forms run in double-float (about 2^-46 relative per operation), so the cancellation in the mean
// (sum_i |Q beta| reaches 10^5 |mean| on smooth data with small noise) costs no accuracy that matters.
//
// Kernels:
//   k_pd_factor   Lambda(f) = L D L^T per frequency from the FP32 spectra: 1/D and L as double-float
//                 pairs, frequency f = h 2^a + lo stored at lo 2^(m-a) + h so that a block of one low
//                 index reads its factors contiguously;
//   k_pd_rows     one block per (point chunk of 2^a, query), one warp per task: the row values
//                 R_tu Q(x, x_ui) of the chunk, their contribution to the mean, and Walsh stages 0..a-1
//                 in registers and lane shuffles -> rows;
//   k_pd_quad     one block per (low index lo, query), one warp per task: stages a..m-1 of the rows'
//                 elements h 2^a + lo, then per frequency w = L^-1 kappa and sum_k w_k^2 / D_k;
//   k_pd_finish   one warp per query: the mean and the variance from the block sums (fixed order);
//   k_pd_mean     mean-only calls: one thread per query against a slice of the design points.
#include <cstring>

#include "mtgp_internal.cuh"
#include "kernel_df.cuh"

namespace {

constexpr int kPdMeanThreads = 256;
constexpr int kPdTile = 128;  // design points per shared-memory tile of the mean-only kernel

struct PdParams {
    int d, T, m, a;
    long long n;
    int order[MTGP_TMAX], rank[MTGP_TMAX];
    int colidx[MTGP_TMAX][MTGP_TMAX];
    long long coloff[MTGP_MAX_COLS];
};

// Q(x, x') = prod_j (1 + eta_j K(X_j)) from the XORed words X_j = x_j XOR x'_j, with es_j = eta_j 2^-33 (the
// scale of dsi2_scaled_df)
template <int DMAX>
__device__ __forceinline__ df q_df_words(const uint32_t (&X)[DMAX], const df* es, int d) {
    df q = df_of(1.0f);
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
        if (j < d) q = df_mul(q, df_one_plus(df_mul(es[j], dsi2_scaled_df(X[j]))));
    return q;
}

// task covariance R = W W^T + diag(v) of sorted tasks, as double-float (shared, T x T)
__device__ void load_R_df(df* sR, const PdParams& p, const ThetaPtrs& th) {
    for (int e = threadIdx.x; e < p.T * p.T; e += blockDim.x) {
        const int t = e / p.T, u = e % p.T;
        const int tc = p.order[t], uc = p.order[u];
        double r = 0.0;
        for (int k = 0; k < th.s; ++k) r += th.W[tc * th.s + k] * th.W[uc * th.s + k];
        if (t == u) r += th.v[tc];
        sR[e] = df_from_double(r);
    }
}

// eta_j 2^-33 as double-float (shared)
__device__ void load_eta_scaled(df* es, const PdParams& p, const ThetaPtrs& th) {
    if (threadIdx.x < p.d) es[threadIdx.x] = df_from_double(th.eta[threadIdx.x] * 0x1p-33);
}

__device__ __forceinline__ float2 f2(df v) { return make_float2(v.hi, v.lo); }
__device__ __forceinline__ df fd(float2 v) { return df_make(v.x, v.y); }

__device__ __forceinline__ df shfl_xor_df(df v, int m) {
    return df_make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
__device__ __forceinline__ df shfl_down_df(df v, int m) {
    return df_make(__shfl_down_sync(0xffffffffu, v.hi, m), __shfl_down_sync(0xffffffffu, v.lo, m));
}

// Walsh-Hadamard stages over a warp's register tile (lane l holds elements l + 32 e): the butterflies over
// the register index, then over the lane index (the lane with the bit clear keeps x + y, its partner y - x)
template <int LOGE>
__device__ __forceinline__ void wht_tile_df(df (&x)[1 << LOGE], int lane) {
#pragma unroll
    for (int b = 0; b < LOGE; ++b) {
#pragma unroll
        for (int e = 0; e < (1 << LOGE); ++e) {
            if (!(e & (1 << b))) {
                const df u = x[e], v = x[e | (1 << b)];
                x[e] = df_add(u, v);
                x[e | (1 << b)] = df_sub(u, v);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const bool upper = (lane >> b) & 1;
#pragma unroll
        for (int e = 0; e < (1 << LOGE); ++e) {
            const df y = shfl_xor_df(x[e], 1 << b);
            x[e] = upper ? df_sub(y, x[e]) : df_add(x[e], y);
        }
    }
}

// sum of a double-float over the warp (valid in lane 0)
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_down_df(v, o));
    return v;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------------- factor

// Lambda(f) = L D L^T for every frequency (real symmetric: Walsh spectra of real columns): diagonal
// blocks share column 0 (clamped at zero: its FP32 spectrum may round below), block (t, u) of the lower
// triangle is R_ut mu_tu(f).  Stores 1/D_k at k n + idx and L_ik at (T + i (i - 1) / 2 + k) n + idx,
// idx = lo 2^(m - a) + h for f = h 2^a + lo.
template <int T>
__global__ void __launch_bounds__(256) k_pd_factor(const float* __restrict__ spec, PdParams p, ThetaPtrs th,
                                                   float2* __restrict__ fac) {
    __shared__ df sR[T * T];
    __shared__ df s_noise[T];
    load_R_df(sR, p, th);
    if (threadIdx.x < T) s_noise[threadIdx.x] = df_from_double(noise_of(th, p.order, threadIdx.x));
    __syncthreads();
    const long long n = p.n;
    const int lgH = p.m - p.a;
    const long long lomask = (1LL << p.a) - 1;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n; f += (long long)gridDim.x * blockDim.x) {
        float mu[T][T];
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int u = t; u < T; ++u) mu[t][u] = spec[p.coloff[p.colidx[t][u]] + f];
        const float mu0 = mu[0][0] < 0.0f ? 0.0f : mu[0][0];
        const long long idx = ((f & lomask) << lgH) + (f >> p.a);
        df D[T], invD[T], L[T][T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            df dk = df_add(df_mulf(sR[k * T + k], mu0), s_noise[k]);
#pragma unroll
            for (int j = 0; j < k; ++j) dk = df_fms(dk, df_mul(L[k][j], L[k][j]), D[j]);
            D[k] = dk;
            invD[k] = df_rcp(dk);
            fac[(long long)k * n + idx] = f2(invD[k]);
#pragma unroll
            for (int i = k + 1; i < T; ++i) {
                df a = df_mulf(sR[k * T + i], mu[k][i]);
#pragma unroll
                for (int j = 0; j < k; ++j) a = df_fms(a, df_mul(L[i][j], L[k][j]), D[j]);
                L[i][k] = df_mul(a, invD[k]);
                fac[(long long)(T + i * (i - 1) / 2 + k) * n + idx] = f2(L[i][k]);
            }
        }
    }
}

// ---------------------------------------------------------------------------------- rows and mean

// Block (chunk c, query b), warp u = sorted task u, lane l holds the chunk's elements i = c 2^a + l + 32 e:
// v = R_{t_b u} Q(x_b, x_ui) with x_ui = z(i) XOR Delta_u, z(i) = z(l) XOR z(c 2^a + 32 e) from the design
// word table; the mean contribution sum_i v beta_u[i]; stages 0..a-1 of the row -> rows[(b T + u) n + i].
// mpart[b gridDim.x + c] = the block's mean contribution (tasks added in order).
template <int DMAX, int LOGE>
__global__ void __launch_bounds__(256) k_pd_rows(const uint32_t* __restrict__ xqw, const int* __restrict__ task, int q0,
                                                 PdParams p, ThetaPtrs th, const uint32_t* __restrict__ rtw,
                                                 const uint32_t* __restrict__ shift, const float2* __restrict__ beta,
                                                 float2* __restrict__ rows, float2* __restrict__ mpart) {
    constexpr int E = 1 << LOGE;
    __shared__ df sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ df s_es[MTGP_MAX_DIM];
    __shared__ df s_m[MTGP_TMAX];
    __shared__ uint32_t s_zh[DMAX][E];
    load_R_df(sR, p, th);
    load_eta_scaled(s_es, p, th);
    const int c = blockIdx.x, b = blockIdx.y, q = q0 + b;
    const int lane = threadIdx.x & 31, u = threadIdx.x >> 5;
    const int d = p.d;
    const long long n = p.n, n32 = n >> 5;
    const long long base = (long long)c << p.a;
    for (int e = threadIdx.x; e < d * E; e += blockDim.x) {
        const int j = e / E, k = e - j * E;
        s_zh[j][k] = rtw[32 * d + (long long)j * n32 + (base >> 5) + k];
    }
    uint32_t wl[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) wl[j] = j < d ? xqw[(long long)q * d + j] ^ shift[u * d + j] ^ rtw[j * 32 + lane] : 0u;
    const int tq = p.rank[task[q]];
    __syncthreads();
    const df r = sR[tq * p.T + u];
    const float2* bu = beta + (long long)u * n + base;
    df x[E];
    df macc = df_of(0.0f);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        uint32_t X[DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) X[j] = j < d ? wl[j] ^ s_zh[j][e] : 0u;
        const df v = df_mul(r, q_df_words<DMAX>(X, s_es, d));
        x[e] = v;
        macc = df_fma(macc, v, fd(bu[lane + 32 * e]));
    }
    wht_tile_df<LOGE>(x, lane);
    float2* out = rows + ((long long)b * p.T + u) * n + base;
#pragma unroll
    for (int e = 0; e < E; ++e) out[lane + 32 * e] = f2(x[e]);
    macc = warp_sum_df(macc);
    if (lane == 0) s_m[u] = macc;
    __syncthreads();
    if (threadIdx.x == 0) {
        df s = s_m[0];
        for (int uu = 1; uu < p.T; ++uu) s = df_add(s, s_m[uu]);
        mpart[(long long)b * gridDim.x + c] = f2(s);
    }
}

// ---------------------------------------------------------------------------------- quadratic forms

// Block (low index lo, query b), warp u = task u: the row elements h 2^a + lo (h = l + 32 e) through stages
// a..m-1 give kappa_u 2^(m/2) at f = h 2^a + lo; then per frequency w = L^-1 kappa and sum_k w_k^2 / D_k.
// vpart[b gridDim.x + lo] = the block's sum (warps added in order), scaled by 2^m.
template <int T, int LOGE>
__global__ void __launch_bounds__(256) k_pd_quad(const float2* __restrict__ rows, const float2* __restrict__ fac, PdParams p,
                                                 float2* __restrict__ vpart) {
    constexpr int E = 1 << LOGE;
    constexpr int H = 32 * E;
    __shared__ df s_k[T][H];
    __shared__ df s_red[T];
    const int lo = blockIdx.x, b = blockIdx.y;
    const int lane = threadIdx.x & 31, u = threadIdx.x >> 5;
    const long long n = p.n;
    const float2* in = rows + ((long long)b * T + u) * n + lo;
    df x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = fd(in[(long long)(lane + 32 * e) << p.a]);
    wht_tile_df<LOGE>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) s_k[u][lane + 32 * e] = x[e];
    __syncthreads();
    df acc = df_of(0.0f);
    const float2* fb = fac + ((long long)lo << (p.m - p.a));
    for (int hh = threadIdx.x; hh < H; hh += blockDim.x) {
        df w[T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            df r = s_k[k][hh];
#pragma unroll
            for (int j = 0; j < k; ++j) r = df_fms(r, fd(fb[(long long)(T + k * (k - 1) / 2 + j) * n + hh]), w[j]);
            w[k] = r;
            acc = df_fma(acc, df_mul(r, r), fd(fb[(long long)k * n + hh]));
        }
    }
    acc = warp_sum_df(acc);
    if (lane == 0) s_red[u] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        df s = s_red[0];
        for (int uu = 1; uu < T; ++uu) s = df_add(s, s_red[uu]);
        vpart[(long long)b * gridDim.x + lo] = f2(s);
    }
}

// ---------------------------------------------------------------------------------- totals

// One warp per query of the batch: mean = tau_t + sum of the chunk contributions, var = R_tt Q(x, x) -
// 2^-m sum of the low-index sums (lanes over the rows, then a shuffle tree: a fixed order).  Q(x, x) =
// prod_j (1 + 3/2 eta_j) in FP64 (K(0) = 3/2).
__global__ void k_pd_finish(const float2* __restrict__ mpart, int nchunk, const float2* __restrict__ vpart, int nlo,
                            const int* __restrict__ task, int q0, int B, PdParams p, ThetaPtrs th,
                            const double* __restrict__ tau_sorted, double* __restrict__ mean, double* __restrict__ var) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B) return;
    df sm = df_of(0.0f), sv = df_of(0.0f);
    for (int k = lane; k < nchunk; k += 32) sm = df_add(sm, fd(mpart[(long long)b * nchunk + k]));
    if (var)
        for (int k = lane; k < nlo; k += 32) sv = df_add(sv, fd(vpart[(long long)b * nlo + k]));
    sm = warp_sum_df(sm);
    sv = warp_sum_df(sv);
    if (lane == 0) {
        const int q = q0 + b;
        const int tq = p.rank[task[q]];
        mean[q] = tau_sorted[tq] + df_to_double(sm);
        if (var) {
            const int tc = p.order[tq];
            double rtt = th.v[tc];
            for (int k = 0; k < th.s; ++k) rtt += th.W[tc * th.s + k] * th.W[tc * th.s + k];
            double prior = rtt;
            for (int j = 0; j < p.d; ++j) prior *= 1.0 + 1.5 * th.eta[j];
            var[q] = prior - ldexp(df_to_double(sv), -p.m);
        }
    }
}

// ---------------------------------------------------------------------------------- mean only

// One thread per query against slice k = blockIdx.y of the design points (slice k: task k / spt, points
// (k mod spt) chunk ..): design words (with the task shift) and beta staged through shared tiles;
// part[k nq + q] = R_{t_q u} sum_i Q(x_q, x_ui) beta_u[i].
template <int DMAX>
__global__ void __launch_bounds__(kPdMeanThreads) k_pd_mean(const uint32_t* __restrict__ xqw, const int* __restrict__ task,
                                                            int nq, const uint32_t* __restrict__ dw,
                                                            const float2* __restrict__ beta, PdParams p, ThetaPtrs th,
                                                            long long chunk, int spt, double* __restrict__ part) {
    __shared__ df sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ df s_es[MTGP_MAX_DIM];
    __shared__ uint32_t s_x[kPdTile * DMAX];
    __shared__ df s_b[kPdTile];
    load_R_df(sR, p, th);
    load_eta_scaled(s_es, p, th);
    const int k = blockIdx.y, u = k / spt;
    const long long i_begin = (long long)(k - u * spt) * chunk;
    const long long i_end = i_begin + chunk < p.n ? i_begin + chunk : p.n;
    const int d = p.d;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = q < nq;
    uint32_t w[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) w[j] = (act && j < d) ? xqw[(long long)q * d + j] : 0u;
    const int tq = act ? p.rank[task[q]] : 0;
    df acc = df_of(0.0f);
    for (long long i0 = i_begin; i0 < i_end; i0 += kPdTile) {
        const int cnt = (int)((i_end - i0) < kPdTile ? (i_end - i0) : kPdTile);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * d; e += blockDim.x) s_x[e] = dw[((long long)u * p.n + i0) * d + e];
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) s_b[e] = fd(beta[(long long)u * p.n + i0 + e]);
        __syncthreads();
        if (act) {
            for (int i = 0; i < cnt; ++i) {
                uint32_t X[DMAX];
#pragma unroll
                for (int j = 0; j < DMAX; ++j) X[j] = j < d ? w[j] ^ s_x[i * d + j] : 0u;
                acc = df_fma(acc, q_df_words<DMAX>(X, s_es, d), s_b[i]);
            }
        }
    }
    if (act) part[(long long)k * nq + q] = df_to_double(df_mul(sR[tq * p.T + u], acc));
}

// mean[q] = tau_t + sum_k part[k][q] (slices added in order)
__global__ void k_pd_mean_sum(const double* __restrict__ part, int nslices, const int* __restrict__ task, int nq,
                              PdParams p, const double* __restrict__ tau_sorted, double* __restrict__ mean) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double m = 0.0;
    for (int k = 0; k < nslices; ++k) m += part[(long long)k * nq + q];
    mean[q] = tau_sorted[p.rank[task[q]]] + m;
}

// beta (FP64) -> double-float pairs
__global__ void k_pd_beta(const double* __restrict__ beta, float2* __restrict__ out, long long N) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        out[i] = f2(df_from_double(beta[i]));
}

}  // namespace

// ---------------------------------------------------------------------------------- host

#include <map>
#include <mutex>

namespace {

struct PdScratch {
    float2* beta = nullptr;
    long long beta_cap = 0;
    float2* fac = nullptr;
    long long fac_cap = 0;
    float2* rows = nullptr;
    long long rows_cap = 0;
    float2* mpart = nullptr;
    long long mpart_cap = 0;
    float2* vpart = nullptr;
    long long vpart_cap = 0;
    double* part = nullptr;
    long long part_cap = 0;
};
std::map<const Handle*, PdScratch> g_pd;
std::mutex g_pd_mu;

template <typename P>
bool grow(P*& ptr, long long& cap, long long need) {
    if (need <= cap) return true;
    cudaFree(ptr);
    ptr = nullptr;
    cap = 0;
    if (cudaMalloc(&ptr, sizeof(P) * (size_t)need) != cudaSuccess) return false;
    cap = need;
    return true;
}

// low part of the two-pass transform: chunks of 2^a points for the rows, 2^(m-a) frequencies per block of
// the quadratic forms, both register tiles of 2^5 .. 2^9 elements (-1: outside that range)
int pd_split(int m) {
    int a = m - 8;
    if (a < 5) a = 5;
    if (a > 9) a = 9;
    return (m - a >= 5 && m - a <= 9) ? a : -1;
}

PdParams pd_params(const Handle* h, int a) {
    PdParams p;
    std::memset(&p, 0, sizeof(p));
    p.d = h->d;
    p.T = h->T;
    p.m = h->m[0];
    p.a = a;
    p.n = h->n[0];
    for (int t = 0; t < MTGP_TMAX; ++t) {
        p.order[t] = t < h->T ? h->order[t] : 0;
        p.rank[t] = t < h->T ? h->rank[t] : 0;
        for (int u = 0; u < MTGP_TMAX; ++u) p.colidx[t][u] = (t < h->T && u < h->T && t <= u) ? h->col_of[t][u] : 0;
    }
    for (int c = 0; c < MTGP_MAX_COLS; ++c) p.coloff[c] = c < h->ncols ? h->cols[c].off : 0;
    return p;
}

int blocks_for(long long work) {
    long long b = (work + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

template <int T>
void launch_factor(const Handle* h, const PdParams& p, ThetaPtrs th, float2* fac, cudaStream_t st) {
    k_pd_factor<T><<<blocks_for(p.n), 256, 0, st>>>(static_cast<const float*>(h->spec), p, th, fac);
}
template <int T, int LOGE>
void launch_quad_t(const float2* rows, const float2* fac, const PdParams& p, int B, float2* vpart, cudaStream_t st) {
    k_pd_quad<T, LOGE><<<dim3(1u << p.a, (unsigned)B), 32 * T, 0, st>>>(rows, fac, p, vpart);
}
template <int T>
void launch_quad_e(const float2* rows, const float2* fac, const PdParams& p, int B, float2* vpart, cudaStream_t st) {
    switch (p.m - p.a - 5) {
        case 0: launch_quad_t<T, 0>(rows, fac, p, B, vpart, st); break;
        case 1: launch_quad_t<T, 1>(rows, fac, p, B, vpart, st); break;
        case 2: launch_quad_t<T, 2>(rows, fac, p, B, vpart, st); break;
        case 3: launch_quad_t<T, 3>(rows, fac, p, B, vpart, st); break;
        default: launch_quad_t<T, 4>(rows, fac, p, B, vpart, st); break;
    }
}
template <int DMAX, int LOGE>
void launch_rows_t(const uint32_t* xqw, const int* task, int q0, int B, const PdParams& p, ThetaPtrs th, const Handle* h,
                   const float2* beta, float2* rows, float2* mpart, cudaStream_t st) {
    k_pd_rows<DMAX, LOGE><<<dim3((unsigned)(p.n >> p.a), (unsigned)B), 32 * p.T, 0, st>>>(xqw, task, q0, p, th, h->rt_words,
                                                                                       h->shift, beta, rows, mpart);
}
template <int DMAX>
void launch_rows_e(const uint32_t* xqw, const int* task, int q0, int B, const PdParams& p, ThetaPtrs th, const Handle* h,
                   const float2* beta, float2* rows, float2* mpart, cudaStream_t st) {
    switch (p.a - 5) {
        case 0: launch_rows_t<DMAX, 0>(xqw, task, q0, B, p, th, h, beta, rows, mpart, st); break;
        case 1: launch_rows_t<DMAX, 1>(xqw, task, q0, B, p, th, h, beta, rows, mpart, st); break;
        case 2: launch_rows_t<DMAX, 2>(xqw, task, q0, B, p, th, h, beta, rows, mpart, st); break;
        case 3: launch_rows_t<DMAX, 3>(xqw, task, q0, B, p, th, h, beta, rows, mpart, st); break;
        default: launch_rows_t<DMAX, 4>(xqw, task, q0, B, p, th, h, beta, rows, mpart, st); break;
    }
}

}  // namespace

bool posterior_df_ok(const Handle* h) {
    return h->equal && h->fp32 && !h->cplx && h->kind == MTGP_DNET && !h->dsi_mix && h->d <= 16 &&
           h->rt_words != nullptr && pd_split(h->m[0]) >= 0;
}

void posterior_df_release(const Handle* h) {
    std::lock_guard<std::mutex> lk(g_pd_mu);
    auto it = g_pd.find(h);
    if (it == g_pd.end()) return;
    PdScratch& s = it->second;
    cudaFree(s.beta);
    cudaFree(s.fac);
    cudaFree(s.rows);
    cudaFree(s.mpart);
    cudaFree(s.vpart);
    cudaFree(s.part);
    g_pd.erase(it);
}

int posterior_df_run(const Handle* h, ThetaPtrs th, int nq, const uint32_t* xqw, const int* task, const uint32_t* design,
                     const double* beta64, double* mean, double* var, cudaStream_t st) {
    PdScratch* s;
    {
        std::lock_guard<std::mutex> lk(g_pd_mu);
        s = &g_pd[h];
    }
    const int a = pd_split(h->m[0]);
    const PdParams p = pd_params(h, a);
    const int T = h->T, d = h->d;
    const long long n = p.n, N = (long long)T * n;
    if (!grow(s->beta, s->beta_cap, N)) return MTGP_ERR_CUDA;
    k_pd_beta<<<blocks_for(N), 256, 0, st>>>(beta64, s->beta, N);
    if (!var) {
        // mean only: slices of the design points so that query blocks x slices fill the GPU several times
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long long qblocks = (nq + kPdMeanThreads - 1) / kPdMeanThreads;
        long long want = (16LL * nsm / T + qblocks - 1) / qblocks;
        const long long cap = (32LL << 20) / ((long long)nq * T);
        if (want > cap) want = cap;
        if (want < 1) want = 1;
        long long chunk = (n + want - 1) / want;
        chunk = (chunk + kPdTile - 1) / kPdTile * kPdTile;
        const int spt = (int)((n + chunk - 1) / chunk), ns = T * spt;
        if (!grow(s->part, s->part_cap, (long long)ns * nq)) return MTGP_ERR_CUDA;
        mtgp_prof_begin(h, "post_mean", st);
        const dim3 grid((unsigned)qblocks, (unsigned)ns);
        if (d <= 8) k_pd_mean<8><<<grid, kPdMeanThreads, 0, st>>>(xqw, task, nq, design, s->beta, p, th, chunk, spt, s->part);
        else k_pd_mean<16><<<grid, kPdMeanThreads, 0, st>>>(xqw, task, nq, design, s->beta, p, th, chunk, spt, s->part);
        k_pd_mean_sum<<<(unsigned)qblocks, kPdMeanThreads, 0, st>>>(s->part, ns, task, nq, p, h->tau, mean);
        mtgp_prof_end(h, st);
        return MTGP_OK;
    }
    // mean and variance: the factors once, then batches of queries whose rows (8 bytes per value) stay within
    // 512 MB
    if (!grow(s->fac, s->fac_cap, (long long)(T + T * (T - 1) / 2) * n)) return MTGP_ERR_CUDA;
    int B = (int)((64LL << 20) / N);
    if (B < 1) B = 1;
    if (B > 1024) B = 1024;
    if (B > nq) B = nq;
    const int nchunk = (int)(n >> a), nlo = 1 << a;
    if (!grow(s->rows, s->rows_cap, (long long)B * N) || !grow(s->mpart, s->mpart_cap, (long long)B * nchunk) ||
        !grow(s->vpart, s->vpart_cap, (long long)B * nlo))
        return MTGP_ERR_CUDA;
    mtgp_prof_begin(h, "var_factor", st);
    switch (T) {
        case 1: launch_factor<1>(h, p, th, s->fac, st); break;
        case 2: launch_factor<2>(h, p, th, s->fac, st); break;
        case 3: launch_factor<3>(h, p, th, s->fac, st); break;
        case 4: launch_factor<4>(h, p, th, s->fac, st); break;
        case 5: launch_factor<5>(h, p, th, s->fac, st); break;
        case 6: launch_factor<6>(h, p, th, s->fac, st); break;
        case 7: launch_factor<7>(h, p, th, s->fac, st); break;
        default: launch_factor<8>(h, p, th, s->fac, st); break;
    }
    mtgp_prof_end(h, st);
    for (int q0 = 0; q0 < nq; q0 += B) {
        const int Bb = (nq - q0) < B ? (nq - q0) : B;
        mtgp_prof_begin(h, "var_rows", st);
        if (d <= 8) launch_rows_e<8>(xqw, task, q0, Bb, p, th, h, s->beta, s->rows, s->mpart, st);
        else launch_rows_e<16>(xqw, task, q0, Bb, p, th, h, s->beta, s->rows, s->mpart, st);
        mtgp_prof_end(h, st);
        mtgp_prof_begin(h, "var_quad", st);
        switch (T) {
            case 1: launch_quad_e<1>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 2: launch_quad_e<2>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 3: launch_quad_e<3>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 4: launch_quad_e<4>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 5: launch_quad_e<5>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 6: launch_quad_e<6>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            case 7: launch_quad_e<7>(s->rows, s->fac, p, Bb, s->vpart, st); break;
            default: launch_quad_e<8>(s->rows, s->fac, p, Bb, s->vpart, st); break;
        }
        k_pd_finish<<<(unsigned)((Bb + 7) / 8), 256, 0, st>>>(s->mpart, nchunk, s->vpart, nlo, task, q0, Bb, p, th, h->tau,
                                                              mean, var);
        mtgp_prof_end(h, st);
    }
    return MTGP_OK;
}

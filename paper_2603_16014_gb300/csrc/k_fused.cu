// Equal-size fast path: NLL (+ gradient) in three kernels, everything between them L2-resident.
//
//   A  first kernel columns c_p (p < C) generated on the fly for a contiguous chunk of 2^a indices,
//      forward butterfly stages 0..a-1 in shared memory                        -> spec
//   B  stages a..m-1 for a tile of low indices, then per frequency f the FP64 solve of
//      Lambda(f) = R o M(f) + sigma2 I (freq_solve.cuh); with the gradient, the adjoint weights
//      W_c(f) replace the spectra in shared memory and the transposed (DIF) stages m-1..a run on
//      them                                                                     -> wgt
//   C  DIF stages a-1..0 on a contiguous chunk, then dL/deta_j = Re sum_i omega_c[i] dc_c[i]/deta_j
//      with the kernel values regenerated from the index.
// Block partial sums are reduced by the last block of B (NLL only) or C, in a fixed order, so the
// results do not depend on block scheduling.  Columns: c = 0 is the diagonal block's column (shared
// by all tasks for equal sizes), then one per task pair t < u.
#include <cstring>

#include "freq_solve.cuh"

namespace {

template <typename S, bool CPLX>
struct El;
template <typename S>
struct El<S, false> { using T = S; };
template <typename S>
struct El<S, true> { using T = cx<S>; };

template <typename S>
__device__ __forceinline__ S el_re(S x) { return x; }
template <typename S>
__device__ __forceinline__ S el_re(cx<S> x) { return x.re; }
template <typename S>
__device__ __forceinline__ S bmul(S x, cx<S>) { return x; }
template <typename S>
__device__ __forceinline__ cx<S> bmul(cx<S> x, cx<S> w) { return x * w; }

struct FusedParams {
    int kind, d, T, C, gen_cols, m, a, lgL, grad, clamp, store_alpha, mtw, s;
    long long n, N;
    int colt[MTGP_MAX_COLS], colu[MTGP_MAX_COLS];
    int colidx[MTGP_TMAX][MTGP_TMAX];
    int order[MTGP_TMAX], rank[MTGP_TMAX];
};

// butterfly stages [s_first .. s_last] (DIT ascending, DIF descending) over groups of 2^lgH values
// spaced L apart in shared memory, for `ncol` columns stored back to back (colstride elements).
template <typename S, bool CPLX, bool DIF>
__device__ __forceinline__ void smem_stages(typename El<S, CPLX>::T* buf, int ncol, int colstride, int lgH, int lgL,
                                            int s0, long long lo0, const cx<S>* tw, int mtw) {
    using E = typename El<S, CPLX>::T;
    const int L = 1 << lgL;
    const int lgnb = lgH + lgL - 1;
    const int nb = 1 << lgnb;
    for (int st = 0; st < lgH; ++st) {
        const int s = DIF ? (s0 + lgH - 1 - st) : (s0 + st);
        const int ls = s - s0;
        for (int e = threadIdx.x; e < nb * ncol; e += blockDim.x) {
            const int c = e >> lgnb;
            const int b = e & (nb - 1);
            const int lo = b & (L - 1);
            const int hb = b >> lgL;
            const int hlo = hb & ((1 << ls) - 1);
            const int h1 = ((hb >> ls) << (ls + 1)) | hlo;
            const int h2 = h1 + (1 << ls);
            E* col = buf + (long long)c * colstride;
            E x1 = col[(h1 << lgL) + lo];
            E x2 = col[(h2 << lgL) + lo];
            cx<S> w;
            if (CPLX) w = tw[(lo0 + lo + ((long long)hlo << s0)) << (mtw - 1 - s)];
            if (!DIF) {
                E t = bmul(x2, w);
                col[(h1 << lgL) + lo] = x1 + t;
                col[(h2 << lgL) + lo] = x1 - t;
            } else {
                col[(h1 << lgL) + lo] = x1 + x2;
                col[(h2 << lgL) + lo] = bmul(x1 - x2, w);
            }
        }
        __syncthreads();
    }
}

__device__ void load_R_f(double* sR, const FusedParams& p, const ThetaPtrs& th) {
    for (int e = threadIdx.x; e < p.T * p.T; e += blockDim.x) {
        int t = e / p.T, u = e % p.T;
        int tc = p.order[t], uc = p.order[u];
        double r = 0.0;
        for (int k = 0; k < th.s; ++k) r += th.W[tc * th.s + k] * th.W[uc * th.s + k];
        if (t == u) r += th.v[tc];
        sR[e] = r;
    }
}

// deterministic block reduction of one value (all threads call; result valid in thread 0)
__device__ __forceinline__ double block_sum(double v, double* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += scratch[w];
    return r;
}

template <typename S>
__device__ __forceinline__ S block_sum_s(S v, S* scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    S r = (S)0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += scratch[w];
    return r;
}

// sum of column q of a (nrows x ncols) partial array, fixed order, all threads call
__device__ double sum_partials(const double* part, int nrows, int ncols, int q, double* scratch) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nrows; b += blockDim.x) v += part[(long long)b * ncols + q];
    return block_sum(v, scratch);
}

// totals of the ncols columns of an (nrows x ncols) partial array into out[q]: warp w sums columns
// q = w, w + nwarps, ...; lane l adds rows l, l + 32, ... (fixed order), then a shuffle tree.
__device__ void reduce_columns(const double* part, int nrows, int ncols, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < ncols; q += nw) {
        double v = 0.0;
        for (int b = lane; b < nrows; b += 32) v += part[(long long)b * ncols + q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) out[q] = v;
    }
    __syncthreads();
}

// last-block election: true in exactly one block, after all blocks have written their partials
__device__ bool last_block(unsigned* counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

struct OutPtrs {
    double* out;
    double* tau;
    double* g_eta;
    double* g_W;
    double* g_v;
    double* g_s2;
};

__device__ __forceinline__ int gq(int t, int u, int T) { return t * T - t * (t - 1) / 2 + (u - t); }

// final outputs from the totals (thread 0)
__device__ void write_outputs(const double* tot, const double* etot, const FusedParams& p, const ThetaPtrs& th,
                              const double* tau_sorted, OutPtrs o) {
    const double LOG2PI = 1.8378770664093453;
    o.out[0] = 0.5 * (tot[0] + tot[1] + (double)p.N * LOG2PI);
    o.out[1] = tot[1];
    o.out[2] = tot[0];
    if (o.tau)
        for (int t = 0; t < p.T; ++t) o.tau[p.order[t]] = tau_sorted[t];
    if (!p.grad) return;
    const int T = p.T;
    o.g_s2[0] = 0.5 * tot[2];
    for (int j = 0; j < p.d; ++j) o.g_eta[j] = 0.5 * etot[j];
    for (int tc = 0; tc < T; ++tc) {
        int t = p.rank[tc];
        for (int k = 0; k < th.s; ++k) {
            double g = 0.0;
            for (int uc = 0; uc < T; ++uc) {
                int u = p.rank[uc];
                double G = (t <= u) ? tot[3 + gq(t, u, T)] : tot[3 + gq(u, t, T)];
                g += G * th.W[uc * th.s + k];
            }
            o.g_W[tc * th.s + k] = g;
        }
        o.g_v[tc] = 0.5 * tot[3 + gq(t, t, T)];
    }
}

// ---------------------------------------------------------------------------------- kernel A

// design-point words of the chunk [base, base + 2^a): z(base + lo) = z(base) (+) z(lo) (lattice: +,
// digital net: XOR; both follow from the linearity in the index bits used in Sec. 3.3)
template <int DMAX>
__device__ __forceinline__ void chunk_point(int kind, int d, uint32_t lo, const uint32_t* s_zhi, const uint32_t* s_gen,
                                            int gen_cols, uint32_t (&z)[DMAX]) {
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            uint32_t zl = point_word(kind, lo, j, s_gen, gen_cols);
            z[j] = (kind == MTGP_LATTICE) ? s_zhi[j] + zl : (s_zhi[j] ^ zl);
        }
    }
}

__device__ __forceinline__ void load_design_smem(const FusedParams& p, const uint32_t* gen, const uint32_t* shift,
                                                 const double* eta, long long base, uint32_t* s_gen, uint32_t* s_sh,
                                                 uint32_t* s_zhi) {
    const int d = p.d;
    const int ng = (p.kind == MTGP_LATTICE) ? d : d * p.gen_cols;
    for (int e = threadIdx.x; e < ng; e += blockDim.x) s_gen[e] = gen[e];
    for (int e = threadIdx.x; e < p.T * d; e += blockDim.x) s_sh[e] = shift[e];
    __syncthreads();
    if (threadIdx.x < d) s_zhi[threadIdx.x] = point_word(p.kind, (uint32_t)base, threadIdx.x, s_gen, p.gen_cols);
}

template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512)
k_fused_a(void* spec, FusedParams p, const uint32_t* __restrict__ gen, const uint32_t* __restrict__ shift,
          const double* __restrict__ eta, const cx<S>* __restrict__ tw) {
    using E = typename El<S, CPLX>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ uint32_t s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_sh[MTGP_TMAX * MTGP_MAX_DIM];
    __shared__ uint32_t s_gen[MTGP_MAX_DIM * 32];
    const int HA = 1 << p.a;
    const long long base = (long long)blockIdx.x << p.a;
    const int d = p.d;
    if (threadIdx.x < d) s_eta[threadIdx.x] = (S)eta[threadIdx.x];
    load_design_smem(p, gen, shift, eta, base, s_gen, s_sh, s_zhi);
    __syncthreads();
    for (int lo = threadIdx.x; lo < HA; lo += blockDim.x) {
        uint32_t z[DMAX];
        chunk_point<DMAX>(p.kind, d, (uint32_t)lo, s_zhi, s_gen, p.gen_cols, z);
        for (int c = 0; c < p.C; ++c) {
            const int t = p.colt[c], u = p.colu[c];
            S q = (S)1;
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                if (j < d) {
                    uint32_t X = pair_word(p.kind, z[j], s_sh[t * d + j], s_sh[u * d + j]);
                    q *= (S)1 + s_eta[j] * kernel1d<S>(p.kind, X);
                }
            }
            if constexpr (CPLX) buf[c * HA + lo] = mk(q, (S)0);
            else buf[c * HA + lo] = q;
        }
    }
    __syncthreads();
    smem_stages<S, CPLX, false>(buf, p.C, HA, p.a, 0, 0, 0, tw, p.mtw);
    E* out = reinterpret_cast<E*>(spec);
    for (int e = threadIdx.x; e < HA * p.C; e += blockDim.x) {
        const int c = e >> p.a;
        const int lo = e & (HA - 1);
        out[(long long)c * p.n + base + lo] = buf[e];
    }
}

// ---------------------------------------------------------------------------------- kernel B

constexpr int kBThreads = 256;

template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kBThreads, 2)
k_fused_b(void* spec, void* wgt, const double* __restrict__ yhat, double* alpha_out, const double* tau_sorted,
          FusedParams p, ThetaPtrs th, const cx<S>* __restrict__ tw, double* partials, unsigned* counter, OutPtrs o,
          int* status) {
    using E = typename El<S, CPLX>::T;
    using V = Vt<CPLX>;
    constexpr int NQ = 3 + T * (T + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ double sR[T * T];
    __shared__ double s_sig;
    __shared__ double s_scr[32];
    __shared__ double s_tot[NQ];
    load_R_f(sR, p, th);
    if (threadIdx.x == 0) s_sig = th.sigma2[0];
    const int lgH = p.m - p.a;
    const int HB = 1 << lgH;
    const int L = 1 << p.lgL;
    const int tile = HB * L;
    const int lgT = lgH + p.lgL;
    const long long lo0 = (long long)blockIdx.x << p.lgL;
    // observations of this thread's first frequency, requested before the transform stages so the
    // (L2-flushed) loads overlap them
    V rh0[T];
    {
        const int r = threadIdx.x;
        const long long f = ((long long)(r >> p.lgL) << p.a) + lo0 + (r & (L - 1));
#pragma unroll
        for (int t = 0; t < T; ++t) rh0[t] = (r < tile && f != 0) ? ld<CPLX>(yhat, (long long)t * p.n + f) : czero<V>();
    }
    const E* in = reinterpret_cast<const E*>(spec);
    for (int e = threadIdx.x; e < tile * p.C; e += blockDim.x) {
        const int c = e >> lgT;
        const int r = e & (tile - 1);
        const int h = r >> p.lgL, l = r & (L - 1);
        buf[e] = in[(long long)c * p.n + ((long long)h << p.a) + lo0 + l];
    }
    __syncthreads();
    smem_stages<S, CPLX, false>(buf, p.C, tile, lgH, p.lgL, p.a, lo0, tw, p.mtw);
    const double sig = s_sig;
    double acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    LogAcc lacc;
    lacc.init();
    int bad = 0;
    for (int r = threadIdx.x; r < tile; r += blockDim.x) {
        const int h = r >> p.lgL, l = r & (L - 1);
        const long long f = ((long long)h << p.a) + lo0 + l;
        V mu[T][T], w[T][T], al[T], rh[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
#pragma unroll
            for (int u = t; u < T; ++u) {
                E x = buf[p.colidx[t][u] * tile + r];
                if constexpr (CPLX) mu[t][u] = mk(to_d<S>(x.re), to_d<S>(x.im));
                else mu[t][u] = to_d<S>(x);
            }
            rh[t] = (r == (int)threadIdx.x) ? rh0[t] : ((f == 0) ? czero<V>() : ld<CPLX>(yhat, (long long)t * p.n + f));
        }
        solve_freq<T, CPLX>(mu, rh, sR, sig, p.clamp != 0, p.grad != 0, lacc, acc, w, al, p.store_alpha != 0, bad);
        if (p.store_alpha) {
#pragma unroll
            for (int t = 0; t < T; ++t) st<CPLX>(alpha_out, (long long)t * p.n + f, al[t]);
        }
        if (p.grad) {
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int u = t; u < T; ++u) {
                    if (u != t || t == 0) {
                        V x = w[t][u];
                        E e;
                        if constexpr (CPLX) e = mk(from_d<S>(x.re), from_d<S>(x.im));
                        else e = from_d<S>(x);
                        buf[p.colidx[t][u] * tile + r] = e;
                    }
                }
        }
    }
    // one logarithm per warp: multiply the lanes' mantissa/exponent products first
    lacc.warp_product();
    acc[0] = ((threadIdx.x & 31) == 0) ? lacc.log_value() : 0.0;
    if (bad) set_status(status, ST_NOT_PD);
    __syncthreads();
    if (p.store_alpha && !p.grad) {
        // the posterior's variance pass reads the fully transformed spectra
        E* so = reinterpret_cast<E*>(spec);
        for (int e = threadIdx.x; e < tile * p.C; e += blockDim.x) {
            const int c = e / tile;
            const int r = e - c * tile;
            const int h = r >> p.lgL, l = r & (L - 1);
            so[(long long)c * p.n + ((long long)h << p.a) + lo0 + l] = buf[e];
        }
    }
    if (p.grad) {
        smem_stages<S, CPLX, true>(buf, p.C, tile, lgH, p.lgL, p.a, lo0, tw, p.mtw);
        E* wo = reinterpret_cast<E*>(wgt);
        for (int e = threadIdx.x; e < tile * p.C; e += blockDim.x) {
            const int c = e / tile;
            const int r = e - c * tile;
            const int h = r >> p.lgL, l = r & (L - 1);
            wo[(long long)c * p.n + ((long long)h << p.a) + lo0 + l] = buf[e];
        }
    }
    // block partials: transpose through shared memory, then one warp per column
    __syncthreads();
    double* s_acc = reinterpret_cast<double*>(smem_raw);
#pragma unroll
    for (int q = 0; q < NQ; ++q) s_acc[q * blockDim.x + threadIdx.x] = acc[q];
    __syncthreads();
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int q = warp; q < NQ; q += nw) {
            double v = 0.0;
            for (int b = lane; b < (int)blockDim.x; b += 32) v += s_acc[q * blockDim.x + b];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) partials[(long long)blockIdx.x * NQ + q] = v;
        }
    }
    if (p.grad) return;  // kernel C finishes
    if (!last_block(counter)) return;
    reduce_columns(partials, gridDim.x, NQ, s_tot);
    if (threadIdx.x == 0) {
        write_outputs(s_tot, nullptr, p, th, tau_sorted, o);
        *counter = 0u;
    }
}

// ---------------------------------------------------------------------------------- kernel C

template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512)
k_fused_c(const void* wgt, FusedParams p, const uint32_t* __restrict__ gen, const uint32_t* __restrict__ shift,
          const double* __restrict__ eta, const cx<S>* __restrict__ tw, const double* partials_b, int nb,
          double* partials_c, unsigned* counter, ThetaPtrs th, const double* tau_sorted, OutPtrs o) {
    using E = typename El<S, CPLX>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ uint32_t s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_sh[MTGP_TMAX * MTGP_MAX_DIM];
    __shared__ uint32_t s_gen[MTGP_MAX_DIM * 32];
    __shared__ double s_scr[32];
    __shared__ double s_tot[3 + MTGP_MAX_COLS];
    __shared__ double s_etot[MTGP_MAX_DIM];
    const int HA = 1 << p.a;
    const long long base = (long long)blockIdx.x << p.a;
    const int d = p.d;
    if (threadIdx.x < d) s_eta[threadIdx.x] = (S)eta[threadIdx.x];
    load_design_smem(p, gen, shift, eta, base, s_gen, s_sh, s_zhi);
    const E* in = reinterpret_cast<const E*>(wgt);
    for (int e = threadIdx.x; e < HA * p.C; e += blockDim.x) {
        const int c = e >> p.a;
        const int lo = e & (HA - 1);
        buf[e] = in[(long long)c * p.n + base + lo];
    }
    __syncthreads();
    smem_stages<S, CPLX, true>(buf, p.C, HA, p.a, 0, 0, 0, tw, p.mtw);
    // per-thread sums in the transform precision; one conversion per block after the block sum
    S part[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) part[j] = (S)0;
    for (int lo = threadIdx.x; lo < HA; lo += blockDim.x) {
        uint32_t z[DMAX];
        chunk_point<DMAX>(p.kind, d, (uint32_t)lo, s_zhi, s_gen, p.gen_cols, z);
        for (int c = 0; c < p.C; ++c) {
            const S w = el_re(buf[c * HA + lo]);
            const int t = p.colt[c], u = p.colu[c];
            S kv[DMAX], pre[DMAX];
            S pr = (S)1;
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                if (j < d) {
                    uint32_t X = pair_word(p.kind, z[j], s_sh[t * d + j], s_sh[u * d + j]);
                    kv[j] = kernel1d<S>(p.kind, X);
                    pre[j] = pr;
                    pr *= (S)1 + s_eta[j] * kv[j];
                }
            }
            S suf = w;
#pragma unroll
            for (int j = DMAX - 1; j >= 0; --j) {
                if (j < d) {
                    part[j] += kv[j] * pre[j] * suf;
                    suf *= (S)1 + s_eta[j] * kv[j];
                }
            }
        }
    }
    __shared__ S s_scr_s[32];
    for (int j = 0; j < d; ++j) {
        S v = block_sum_s<S>(j < DMAX ? part[j] : (S)0, s_scr_s);
        if (threadIdx.x == 0) partials_c[(long long)blockIdx.x * d + j] = (double)v;
    }
    if (!last_block(counter)) return;
    const int NQ = 3 + p.T * (p.T + 1) / 2;
    reduce_columns(partials_b, nb, NQ, s_tot);
    reduce_columns(partials_c, gridDim.x, d, s_etot);
    if (threadIdx.x == 0) {
        write_outputs(s_tot, s_etot, p, th, tau_sorted, o);
        *counter = 0u;
    }
}

}  // namespace

// ---------------------------------------------------------------------------------- host side

namespace {

size_t elem_size(const Handle* h) { return (h->fp32 ? 4 : 8) * (h->cplx ? 2 : 1); }

// split n = 2^m into a low part 2^a (kernels A, C) and a high part 2^(m-a) (kernel B)
bool plan(const Handle* h, int* a_out, int* lgL_out) {
    const int m = h->m[0];
    if (!h->equal || m < 4) return false;
    const size_t es = elem_size(h);
    const size_t cap = 96 * 1024;
    const int C = h->ncols;
    // kernel B tiles hold 2^(m-a) frequencies (one per thread at 2^8); kernels A and C hold 2^a values
    int a = m - 8;
    if (a < m / 2) a = m / 2;
    while (a > 1 && (size_t)C * ((size_t)1 << a) * es > cap) --a;
    if (a < 1 || a > m - 1) return false;
    if ((size_t)C * ((size_t)1 << (m - a)) * es > cap) return false;
    *a_out = a;
    *lgL_out = 0;
    return true;
}

FusedParams make_params(const Handle* h, ThetaPtrs th, bool grad, bool store_alpha, int a, int lgL) {
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    p.kind = h->kind;
    p.d = h->d;
    p.T = h->T;
    p.C = h->ncols;
    p.gen_cols = h->gen_cols;
    p.m = h->m[0];
    p.a = a;
    p.lgL = lgL;
    p.grad = grad ? 1 : 0;
    p.clamp = h->fp32 ? 1 : 0;
    p.store_alpha = store_alpha ? 1 : 0;
    p.mtw = h->mmax;
    p.s = th.s;
    p.n = h->n[0];
    p.N = h->N;
    for (int c = 0; c < h->ncols; ++c) {
        p.colt[c] = h->cols[c].t;
        p.colu[c] = h->cols[c].u;
    }
    for (int t = 0; t < MTGP_TMAX; ++t) {
        p.order[t] = t < h->T ? h->order[t] : 0;
        p.rank[t] = t < h->T ? h->rank[t] : 0;
        for (int u = 0; u < MTGP_TMAX; ++u) p.colidx[t][u] = (t < h->T && u < h->T && t <= u) ? h->col_of[t][u] : 0;
    }
    return p;
}

template <typename F>
void set_smem(F* fn, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int T, bool CPLX, typename S>
void launch_b(const Handle* h, FusedParams p, ThetaPtrs th, OutPtrs o, cudaStream_t st) {
    size_t smem = elem_size(h) * p.C * ((size_t)1 << (p.m - p.a + p.lgL));
    const size_t red = (size_t)(3 + T * (T + 1) / 2) * kBThreads * sizeof(double);
    if (red > smem) smem = red;
    set_smem(k_fused_b<T, CPLX, S>, smem);
    const int grid = 1 << (p.a - p.lgL);
    const void* twp = h->fp32 ? h->twid32 : h->twid;
    mtgp_prof_begin(h, "fused_b", st);
    k_fused_b<T, CPLX, S><<<grid, kBThreads, smem, st>>>(h->spec, h->wgt, h->yhat, h->alpha, h->tau, p, th,
                                                   reinterpret_cast<const cx<S>*>(twp), h->partials, h->counters, o,
                                                   h->status);
    mtgp_prof_end(h, st);
}

template <bool CPLX, typename S>
void dispatch_b(const Handle* h, FusedParams p, ThetaPtrs th, OutPtrs o, cudaStream_t st) {
    switch (h->T) {
        case 1: launch_b<1, CPLX, S>(h, p, th, o, st); break;
        case 2: launch_b<2, CPLX, S>(h, p, th, o, st); break;
        case 3: launch_b<3, CPLX, S>(h, p, th, o, st); break;
        case 4: launch_b<4, CPLX, S>(h, p, th, o, st); break;
        case 5: launch_b<5, CPLX, S>(h, p, th, o, st); break;
        case 6: launch_b<6, CPLX, S>(h, p, th, o, st); break;
        case 7: launch_b<7, CPLX, S>(h, p, th, o, st); break;
        default: launch_b<8, CPLX, S>(h, p, th, o, st); break;
    }
}

template <bool CPLX, typename S>
void run_fused(const Handle* h, FusedParams p, ThetaPtrs th, OutPtrs o, cudaStream_t st) {
    using E = typename El<S, CPLX>::T;
    const void* twp = h->fp32 ? h->twid32 : h->twid;
    const cx<S>* tw = reinterpret_cast<const cx<S>*>(twp);
    const size_t smem_a = sizeof(E) * p.C * ((size_t)1 << p.a);
    const int grid_a = 1 << (p.m - p.a);
    const int thr_a = (1 << p.a) < 512 ? ((1 << p.a) < 64 ? 64 : (1 << p.a)) : 512;
    mtgp_prof_begin(h, "fused_a", st);
    if (h->d <= 4) {
        set_smem(k_fused_a<S, CPLX, 4>, smem_a);
        k_fused_a<S, CPLX, 4><<<grid_a, thr_a, smem_a, st>>>(h->spec, p, h->gen, h->shift, th.eta, tw);
    } else if (h->d <= 8) {
        set_smem(k_fused_a<S, CPLX, 8>, smem_a);
        k_fused_a<S, CPLX, 8><<<grid_a, thr_a, smem_a, st>>>(h->spec, p, h->gen, h->shift, th.eta, tw);
    } else if (h->d <= 16) {
        set_smem(k_fused_a<S, CPLX, 16>, smem_a);
        k_fused_a<S, CPLX, 16><<<grid_a, thr_a, smem_a, st>>>(h->spec, p, h->gen, h->shift, th.eta, tw);
    } else {
        set_smem(k_fused_a<S, CPLX, 32>, smem_a);
        k_fused_a<S, CPLX, 32><<<grid_a, thr_a, smem_a, st>>>(h->spec, p, h->gen, h->shift, th.eta, tw);
    }
    mtgp_prof_end(h, st);
    dispatch_b<CPLX, S>(h, p, th, o, st);
    if (!p.grad) return;
    const int nb = 1 << (p.a - p.lgL);
    const int NQ = 3 + h->T * (h->T + 1) / 2;
    double* part_c = h->partials + (long long)nb * NQ;
    mtgp_prof_begin(h, "fused_c", st);
    if (h->d <= 4) {
        set_smem(k_fused_c<S, CPLX, 4>, smem_a);
        k_fused_c<S, CPLX, 4><<<grid_a, thr_a, smem_a, st>>>(h->wgt, p, h->gen, h->shift, th.eta, tw, h->partials, nb, part_c, h->counters + 1, th, h->tau, o);
    } else if (h->d <= 8) {
        set_smem(k_fused_c<S, CPLX, 8>, smem_a);
        k_fused_c<S, CPLX, 8><<<grid_a, thr_a, smem_a, st>>>(h->wgt, p, h->gen, h->shift, th.eta, tw, h->partials, nb, part_c, h->counters + 1, th, h->tau, o);
    } else if (h->d <= 16) {
        set_smem(k_fused_c<S, CPLX, 16>, smem_a);
        k_fused_c<S, CPLX, 16><<<grid_a, thr_a, smem_a, st>>>(h->wgt, p, h->gen, h->shift, th.eta, tw, h->partials, nb, part_c, h->counters + 1, th, h->tau, o);
    } else {
        set_smem(k_fused_c<S, CPLX, 32>, smem_a);
        k_fused_c<S, CPLX, 32><<<grid_a, thr_a, smem_a, st>>>(h->wgt, p, h->gen, h->shift, th.eta, tw, h->partials, nb, part_c, h->counters + 1, th, h->tau, o);
    }
    mtgp_prof_end(h, st);
}

}  // namespace

bool fused_supported(const Handle* h) {
    int a, lgL;
    return plan(h, &a, &lgL);
}

long long fused_partials_len(const Handle* h) {
    int a, lgL;
    if (!plan(h, &a, &lgL)) return 0;
    const int NQ = 3 + h->T * (h->T + 1) / 2;
    return ((long long)1 << (a - lgL)) * NQ + ((long long)1 << (h->m[0] - a)) * h->d;
}

void launch_fused(const Handle* h, ThetaPtrs th, bool grad, bool store_alpha, double* out, double* tau, double* g_eta,
                  double* g_W, double* g_v, double* g_s2, cudaStream_t st) {
    int a = 0, lgL = 0;
    plan(h, &a, &lgL);
    FusedParams p = make_params(h, th, grad, store_alpha, a, lgL);
    OutPtrs o{out, tau, g_eta, g_W, g_v, g_s2};
    if (h->fp32) {
        if (h->cplx) run_fused<true, float>(h, p, th, o, st);
        else run_fused<false, float>(h, p, th, o, st);
    } else {
        if (h->cplx) run_fused<true, double>(h, p, th, o, st);
        else run_fused<false, double>(h, p, th, o, st);
    }
}

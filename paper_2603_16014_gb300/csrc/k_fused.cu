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
#include "fused_common.cuh"
#include "kernel_df.cuh"

namespace {

template <typename S, bool CPLX, int DMAX>
__device__ __forceinline__ void fused_a_body(const FitDesc& f, int blk) {
    using E = typename El<S, CPLX>::T;
    const FusedParams& p = f.p;
    void* spec = f.spec;
    const uint32_t* gen = f.gen;
    const uint32_t* shift = f.shift;
    const double* eta = f.th.eta;
    const cx<S>* tw = reinterpret_cast<const cx<S>*>(f.tw);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ uint32_t s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_sh[MTGP_TMAX * MTGP_MAX_DIM];
    __shared__ uint32_t s_gen[MTGP_MAX_DIM * 32];
    const int HA = 1 << p.a;
    const long long base = (long long)blk << p.a;
    const int d = p.d;
    __shared__ uint32_t s_z[kZTab];
    const bool ztab = HA * d <= kZTab;
    load_design_smem(p, gen, shift, eta, base, s_gen, s_sh, s_zhi);
    __syncthreads();
    if (ztab) chunk_table(p.kind, d, p.a, s_zhi, s_gen, p.gen_cols, s_z);  // chunk points, once per (coordinate, element)
    pdl_wait();  // parameters and the spectra buffer belong to earlier work in the stream
    pdl_trigger();
    if (blk == 0) check_theta_block(f.th, d, p.T, f.status);
    if (threadIdx.x < d) s_eta[threadIdx.x] = (S)eta[threadIdx.x];
    __syncthreads();
    if (ztab) {
        // one work item per (column, element)
        for (int e = threadIdx.x; e < HA * p.C; e += blockDim.x) {
            const int c = e >> p.a, lo = e & (HA - 1);
            const int t = p.colt[c], u = p.colu[c];
            S q = (S)1;
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                if (j < d) {
                    uint32_t X = pair_word(p.kind, s_z[(j << p.a) + lo], s_sh[t * d + j], s_sh[u * d + j]);
                    q *= (S)1 + s_eta[j] * kernel1d<S>(p.kind, X, p.alpha);
                }
            }
            if constexpr (CPLX) buf[e] = mk(q, (S)0);
            else buf[e] = q;
        }
    } else {
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
                        q *= (S)1 + s_eta[j] * kernel1d<S>(p.kind, X, p.alpha);
                    }
                }
                if constexpr (CPLX) buf[c * HA + lo] = mk(q, (S)0);
                else buf[c * HA + lo] = q;
            }
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
__device__ __forceinline__ void fused_b_body(const FitDesc& f, int blk) {
    using E = typename El<S, CPLX>::T;
    const FusedParams& p = f.p;
    const ThetaPtrs& th = f.th;
    void* spec = f.spec;
    void* wgt = f.wgt;
    const double* yhat = f.yhat;
    double* alpha_out = f.alpha;
    const double* tau_sorted = f.tau;
    const cx<S>* tw = reinterpret_cast<const cx<S>*>(f.tw);
    double* partials = f.partials;
    unsigned* counter = f.counters;
    int* status = f.status;
    using V = Vt<CPLX>;
    constexpr int NQ = 3 + T * (T + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ double sR[T * T];
    __shared__ double s_sig;
    __shared__ double s_tot[NQ];
    load_R_f(sR, p, th);
    if (threadIdx.x == 0) s_sig = th.sigma2[0];
    const int lgH = p.m - p.a;
    const int HB = 1 << lgH;
    const int L = 1 << p.lgL;
    const int tile = HB * L;
    const int lgT = lgH + p.lgL;
    const long long lo0 = (long long)blk << p.lgL;
    // observations of this thread's first frequency, requested before the transform stages so the
    // (L2-flushed) loads overlap them
    V rh0[T];
    {
        const int r = threadIdx.x;
        const long long f = ((long long)(r >> p.lgL) << p.a) + lo0 + (r & (L - 1));
#pragma unroll
        for (int t = 0; t < T; ++t) rh0[t] = (r < tile && f != 0) ? ld<CPLX>(yhat, (long long)t * p.n + f) : czero<V>();
    }
    pdl_wait();  // the spectra come from kernel A
    pdl_trigger();
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
            if (lane == 0) partials[(long long)blk * NQ + q] = v;
        }
    }
    if (p.grad) return;  // kernel C finishes
    if (!last_block(counter, f.nb)) return;
    reduce_columns(partials, f.nb, NQ, s_tot);
    write_outputs(s_tot, nullptr, p, th, tau_sorted, f.o);
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------------- kernel C

// eta contraction of one item over dimensions 0 .. nd-1 of X in double-float: pd_j += K_j s pre_j suf_j,
// pre_j = pre0 prod_{k < j} (1 + eta_k K_k), suf_j = suf0 prod_{j < k < nd} (1 + eta_k K_k) (suf0 carries the
// adjoint weight); es_j = eta_j / s.  Returns pre0 times the product of the nd factors.
template <int NH>
__device__ __forceinline__ df contract_df_pass(const uint32_t* X, int nd, const df* es, int kind, const Si2Consts& sc,
                                               df pre0, df suf0, df* pd) {
    df fv[NH], kp[NH];
    df pr = pre0;
#pragma unroll
    for (int j = 0; j < NH; ++j) {
        if (j < nd) {
            const df ks = kval_scaled_df(kind, X[j], sc);
            fv[j] = df_one_plus(df_mul(es[j], ks));
            kp[j] = df_mul(ks, pr);
            pr = df_mul(pr, fv[j]);
        }
    }
    df suf = suf0;
#pragma unroll
    for (int j = NH - 1; j >= 0; --j) {
        if (j < nd) {
            pd[j] = df_fma(pd[j], kp[j], suf);
            suf = df_mul(suf, fv[j]);
        }
    }
    return pr;
}

template <typename S, bool CPLX, int DMAX>
__device__ __forceinline__ void fused_c_body(const FitDesc& f, int blk) {
    using E = typename El<S, CPLX>::T;
    const FusedParams& p = f.p;
    const ThetaPtrs& th = f.th;
    const void* wgt = f.wgt;
    const uint32_t* gen = f.gen;
    const uint32_t* shift = f.shift;
    const double* eta = f.th.eta;
    const cx<S>* tw = reinterpret_cast<const cx<S>*>(f.tw);
    const int nb = f.nb;
    const double* partials_b = f.partials;
    double* partials_c = f.partials + (long long)f.nb * (3 + p.T * (p.T + 1) / 2);
    unsigned* counter = f.counters + 1;
    const double* tau_sorted = f.tau;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ uint32_t s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_sh[MTGP_TMAX * MTGP_MAX_DIM];
    __shared__ uint32_t s_gen[MTGP_MAX_DIM * 32];
    __shared__ double s_tot[3 + MTGP_MAX_COLS];
    __shared__ double s_etot[MTGP_MAX_DIM];
    __shared__ uint32_t s_z[kZTab];
    const int HA = 1 << p.a;
    const long long base = (long long)blk << p.a;
    const int d = p.d;
    if (threadIdx.x < d) s_eta[threadIdx.x] = (S)eta[threadIdx.x];
    load_design_smem(p, gen, shift, eta, base, s_gen, s_sh, s_zhi);
    const bool ztab = HA * d <= kZTab;
    if (ztab) {
        __syncthreads();
        chunk_table(p.kind, d, p.a, s_zhi, s_gen, p.gen_cols, s_z);
    }
    pdl_wait();  // the adjoint weights and kernel B's partial sums
    pdl_trigger();
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
    // dL/deta_j += w K_j prod_{k<j} (1 + eta_k K_k) prod_{k>j} (1 + eta_k K_k) per (column, element)
    auto item = [&](const uint32_t* zc, int zstride, int c, S w) {
        const int t = p.colt[c], u = p.colu[c];
        S kv[DMAX], pre[DMAX];
        S pr = (S)1;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < d) {
                uint32_t X = pair_word(p.kind, zc[j * zstride], s_sh[t * d + j], s_sh[u * d + j]);
                kv[j] = kernel1d<S>(p.kind, X, p.alpha);
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
    };
    // FP64 fits (d <= 16): the contraction in double-float on the FP32 pipe (kernel_df.cuh), K_j s exact for
    // digital nets and to ~2^-47 for lattices, sums rescaled by 1/s at the end; it feeds only the eta
    // gradient (FP64 tolerance 1e-7 of its largest entry against ~2^-46 per term)
    bool done = false;
    if constexpr (std::is_same<S, double>::value && DMAX <= 16) {
        __shared__ df s_es[DMAX];
        const double sinv = kval_scale_inv(p.kind);
        if (threadIdx.x < d) s_es[threadIdx.x] = df_from_double(eta[threadIdx.x] * sinv);
        __syncthreads();
        const Si2Consts sc = si2_consts(p.alpha);
        df pd[DMAX];
#pragma unroll
        for (int j = 0; j < DMAX; ++j) pd[j] = df_of(0.0f);
        auto item_df = [&](const uint32_t* zc, int zstride, int c, double w) {
            const int t = p.colt[c], u = p.colu[c];
            uint32_t X[DMAX];
#pragma unroll
            for (int j = 0; j < DMAX; ++j)
                X[j] = j < d ? pair_word(p.kind, zc[j * zstride], s_sh[t * d + j], s_sh[u * d + j]) : 0u;
            const df wd = df_from_double(w);
            if constexpr (DMAX <= 8) {
                contract_df_pass<DMAX>(X, d, s_es, p.kind, sc, df_of(1.0f), wd, pd);
            } else {
                // two passes of 8 dimensions: the upper factors' product rides in the lower pass's suffix,
                // the lower factors' product in the upper pass's prefix (upper factors formed twice)
                df up = df_of(1.0f);
#pragma unroll
                for (int j = 8; j < DMAX; ++j)
                    if (j < d) up = df_mul(up, df_one_plus(df_mul(s_es[j], kval_scaled_df(p.kind, X[j], sc))));
                const df lowp = contract_df_pass<8>(X, d < 8 ? d : 8, s_es, p.kind, sc, df_of(1.0f), df_mul(wd, up), pd);
                contract_df_pass<8>(X + 8, d - 8, s_es + 8, p.kind, sc, lowp, wd, pd + 8);
            }
        };
        if (ztab) {
            for (int e = threadIdx.x; e < HA * p.C; e += blockDim.x) {
                const int c = e >> p.a, lo = e & (HA - 1);
                item_df(s_z + lo, HA, c, (double)el_re(buf[e]));
            }
        } else {
            for (int lo = threadIdx.x; lo < HA; lo += blockDim.x) {
                uint32_t z[DMAX];
                chunk_point<DMAX>(p.kind, d, (uint32_t)lo, s_zhi, s_gen, p.gen_cols, z);
                for (int c = 0; c < p.C; ++c) item_df(z, 1, c, (double)el_re(buf[c * HA + lo]));
            }
        }
#pragma unroll
        for (int j = 0; j < DMAX; ++j) part[j] = (S)(df_to_double(pd[j]) * sinv);
        done = true;
    }
    if (!done && ztab) {
        for (int e = threadIdx.x; e < HA * p.C; e += blockDim.x) {
            const int c = e >> p.a, lo = e & (HA - 1);
            item(s_z + lo, HA, c, el_re(buf[e]));
        }
    } else if (!done) {
        for (int lo = threadIdx.x; lo < HA; lo += blockDim.x) {
            uint32_t z[DMAX];
            chunk_point<DMAX>(p.kind, d, (uint32_t)lo, s_zhi, s_gen, p.gen_cols, z);
            for (int c = 0; c < p.C; ++c) item(z, 1, c, el_re(buf[c * HA + lo]));
        }
    }
    // the d block sums together: a shuffle tree per warp, one shared row per warp, warps added in
    // order by thread j (the same order as one block sum per coordinate, one barrier instead of 2d)
    __shared__ S s_red[16][DMAX];
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < d) {
                S v = part[j];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) s_red[warp][j] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x < d) {
            S v = (S)0;
            for (int w = 0; w < nw; ++w) v += s_red[w][threadIdx.x];
            partials_c[(long long)blk * d + threadIdx.x] = (double)v;
        }
    }
    if (!last_block(counter, f.na)) return;
    const int NQ = 3 + p.T * (p.T + 1) / 2;
    reduce_columns2(partials_b, nb, NQ, s_tot, partials_c, f.na, d, s_etot);
    write_outputs(s_tot, s_etot, p, th, tau_sorted, f.o);
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------------- kernels

template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512) k_fused_a(FitDesc f) { fused_a_body<S, CPLX, DMAX>(f, blockIdx.x); }

template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kBThreads, 2) k_fused_b(FitDesc f) { fused_b_body<T, CPLX, S>(f, blockIdx.x); }

template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512) k_fused_c(FitDesc f) { fused_c_body<S, CPLX, DMAX>(f, blockIdx.x); }

// Batched fits: a persistent grid walks a table of (fit, block) items, largest fits first.
template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512) k_batch_a(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        fused_a_body<S, CPLX, DMAX>(fits[w.x], w.y);
        __syncthreads();
    }
}

template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kBThreads, 2) k_batch_b(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        fused_b_body<T, CPLX, S>(fits[w.x], w.y);
        __syncthreads();
    }
}

template <typename S, bool CPLX, int DMAX>
__global__ void __launch_bounds__(512) k_batch_c(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        fused_c_body<S, CPLX, DMAX>(fits[w.x], w.y);
        __syncthreads();
    }
}

}  // namespace

// ---------------------------------------------------------------------------------- host side

bool fused_plan_cap(int m, int ncols, int d, bool fp32, bool cplx, int a_pref, size_t cap, int* a_out, int* lgL_out);

// split n = 2^m into a low part 2^a (kernels A, C) and a high part 2^(m-a) (kernel B); a_pref >= 0
// asks for a specific split (the autotuner), -1 for the default (B tiles of 2^8 frequencies)
// Tiles are kept within 96 KB of shared memory where a split allows it (two blocks per SM), else within
// 200 KB (one block per SM; e.g. FP64 lattice spectra of 8 tasks).
bool fused_plan(int m, int ncols, int d, bool fp32, bool cplx, int a_pref, int* a_out, int* lgL_out) {
    if (fused_plan_cap(m, ncols, d, fp32, cplx, a_pref, 96 * 1024, a_out, lgL_out)) return true;
    return fused_plan_cap(m, ncols, d, fp32, cplx, a_pref, 200 * 1024, a_out, lgL_out);
}

bool fused_plan_cap(int m, int ncols, int d, bool fp32, bool cplx, int a_pref, size_t cap, int* a_out, int* lgL_out) {
    if (m < 4) return false;
    const size_t es = elem_size_of(fp32, cplx);
    int a;
    if (a_pref >= 0) {
        a = a_pref;
    } else if (fused_rt_ok(cplx, fp32, d, m, m - 8 < 5 ? 5 : (m - 8 > 9 ? 9 : m - 8))) {
        // FP32 real spectra: both halves in the register-tile kernels' range (B tiles of 2^8
        // frequencies where possible)
        a = m - 8 < 5 ? 5 : (m - 8 > 9 ? 9 : m - 8);
    } else {
        a = m - 8;
        if (a < m / 2) a = m / 2;
        while (a > 1 && (size_t)ncols * ((size_t)1 << a) * es > cap) --a;
    }
    if (fused_rt_ok(cplx, fp32, d, m, a)) {
        *a_out = a;
        *lgL_out = 0;
        return true;
    }
    if (a < 1 || a > m - 1) return false;
    if ((size_t)ncols * ((size_t)1 << a) * es > cap) return false;
    if ((size_t)ncols * ((size_t)1 << (m - a)) * es > cap) return false;
    *a_out = a;
    *lgL_out = 0;
    return true;
}

namespace {

bool plan(const Handle* h, int* a_out, int* lgL_out) {
    if (!h->equal) return false;
    return fused_plan(h->m[0], h->ncols, h->d, h->fp32, h->cplx, -1, a_out, lgL_out);
}

FusedParams make_params(const Handle* h, ThetaPtrs th, bool grad, bool store_alpha, int a, int lgL) {
    FusedParams p;
    std::memset(&p, 0, sizeof(p));
    p.kind = h->kind;
    p.alpha = h->smooth;
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

FitDesc make_desc(const Handle* h, ThetaPtrs th, OutPtrs o, bool grad, bool store_alpha, int a, int lgL) {
    FitDesc f;
    std::memset(&f, 0, sizeof(f));
    f.p = make_params(h, th, grad, store_alpha, a, lgL);
    f.th = th;
    f.o = o;
    f.gen = h->gen;
    f.shift = h->shift;
    f.tw = h->fp32 ? h->twid32 : h->twid;
    f.spec = h->spec;
    f.wgt = h->wgt;
    f.yhat = h->yhat;
    f.yhat_df = reinterpret_cast<const float2*>(h->yhat_df);
    f.rtw = h->rt_words;
    f.alpha = h->alpha;
    f.tau = h->tau;
    f.partials = h->partials;
    f.counters = h->counters;
    f.status = h->status;
    f.na = 1 << (f.p.m - a);
    f.nb = 1 << (a - lgL);
    return f;
}

// ---- shared dispatch: one phase of one class, single fit (fits == nullptr) or a batch item table

size_t smem_ac(int C, int a, size_t es) { return es * C * ((size_t)1 << a); }
size_t smem_b(int T, int C, int lgH, size_t es) {
    size_t s = es * C * ((size_t)1 << lgH);
    const size_t red = (size_t)(3 + T * (T + 1) / 2) * kBThreads * sizeof(double);
    return s > red ? s : red;
}
// A and C threads: with the chunk-point table the (column, element) items are spread over twice the
// chunk length, otherwise one thread per element; between 64 and 512
int threads_ac(int a, int d) {
    const int t = ((1 << a) * d <= kZTab) ? (2 << a) : (1 << a);
    return t < 512 ? (t < 64 ? 64 : t) : 512;
}

template <typename S, bool CPLX, int DMAX>
void phase_ac(bool is_c, const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid,
              int threads, size_t smem, cudaStream_t st) {
    if (!is_c) {
        if (single) {
            set_smem(k_fused_a<S, CPLX, DMAX>, smem);
            launch_pdl(k_fused_a<S, CPLX, DMAX>, grid, threads, smem, st, *single);
        } else {
            set_smem(k_batch_a<S, CPLX, DMAX>, smem);
            k_batch_a<S, CPLX, DMAX><<<grid, threads, smem, st>>>(fits, items, nitems);
        }
    } else {
        if (single) {
            set_smem(k_fused_c<S, CPLX, DMAX>, smem);
            launch_pdl(k_fused_c<S, CPLX, DMAX>, grid, threads, smem, st, *single);
        } else {
            set_smem(k_batch_c<S, CPLX, DMAX>, smem);
            k_batch_c<S, CPLX, DMAX><<<grid, threads, smem, st>>>(fits, items, nitems);
        }
    }
}

template <typename S, bool CPLX>
void phase_ac_d(int dmax, bool is_c, const FitDesc* single, const FitDesc* fits, const int2* items, int nitems,
                int grid, int threads, size_t smem, cudaStream_t st) {
    if (dmax <= 4) phase_ac<S, CPLX, 4>(is_c, single, fits, items, nitems, grid, threads, smem, st);
    else if (dmax <= 8) phase_ac<S, CPLX, 8>(is_c, single, fits, items, nitems, grid, threads, smem, st);
    else if (dmax <= 16) phase_ac<S, CPLX, 16>(is_c, single, fits, items, nitems, grid, threads, smem, st);
    else phase_ac<S, CPLX, 32>(is_c, single, fits, items, nitems, grid, threads, smem, st);
}

template <int T, bool CPLX, typename S>
void phase_b_t(const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid, size_t smem,
               cudaStream_t st) {
    if (single) {
        set_smem(k_fused_b<T, CPLX, S>, smem);
        launch_pdl(k_fused_b<T, CPLX, S>, grid, kBThreads, smem, st, *single);
    } else {
        set_smem(k_batch_b<T, CPLX, S>, smem);
        k_batch_b<T, CPLX, S><<<grid, kBThreads, smem, st>>>(fits, items, nitems);
    }
}

template <bool CPLX, typename S>
void phase_b(int T, const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid, size_t smem,
             cudaStream_t st) {
    switch (T) {
        case 1: phase_b_t<1, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 2: phase_b_t<2, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 3: phase_b_t<3, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 4: phase_b_t<4, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 5: phase_b_t<5, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 6: phase_b_t<6, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        case 7: phase_b_t<7, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
        default: phase_b_t<8, CPLX, S>(single, fits, items, nitems, grid, smem, st); break;
    }
}

}  // namespace

int fused_variant(bool fp32, bool cplx, bool solve_df, int d, int m, int a, bool store_alpha) {
    if (store_alpha || !fused_rt_ok(cplx, fp32, d, m, a)) return FUSED_GENERIC;
    return (fp32 && solve_df) ? FUSED_RT_DF : FUSED_RT;
}

// one phase (0 = A, 1 = B, 2 = C) for one class; single != nullptr launches one fit with a grid of
// its own blocks, otherwise a persistent grid over `nitems` batch items
void fused_phase(int phase, int variant, bool fp32, bool cplx, int T, int dmax, const void* single_v,
                 const void* fits_v, const int2* items, int nitems, int grid, int threads_acq, size_t smem,
                 cudaStream_t st) {
    if (variant != FUSED_GENERIC) {
        fused_rt_phase(phase, variant == FUSED_RT_DF, T, dmax, single_v, fits_v, items, nitems, grid, threads_acq, smem,
                       st);
        return;
    }
    const FitDesc* single = static_cast<const FitDesc*>(single_v);
    const FitDesc* fits = static_cast<const FitDesc*>(fits_v);
    if (phase == 1) {
        if (fp32) {
            if (cplx) phase_b<true, float>(T, single, fits, items, nitems, grid, smem, st);
            else phase_b<false, float>(T, single, fits, items, nitems, grid, smem, st);
        } else {
            if (cplx) phase_b<true, double>(T, single, fits, items, nitems, grid, smem, st);
            else phase_b<false, double>(T, single, fits, items, nitems, grid, smem, st);
        }
        return;
    }
    const bool is_c = phase == 2;
    if (fp32) {
        if (cplx) phase_ac_d<float, true>(dmax, is_c, single, fits, items, nitems, grid, threads_acq, smem, st);
        else phase_ac_d<float, false>(dmax, is_c, single, fits, items, nitems, grid, threads_acq, smem, st);
    } else {
        if (cplx) phase_ac_d<double, true>(dmax, is_c, single, fits, items, nitems, grid, threads_acq, smem, st);
        else phase_ac_d<double, false>(dmax, is_c, single, fits, items, nitems, grid, threads_acq, smem, st);
    }
}

size_t fused_desc_size() { return sizeof(FitDesc); }

void fused_make_desc(const Handle* h, ThetaPtrs th, double* out, double* tau, double* g_eta, double* g_W, double* g_v,
                     double* g_s2, bool grad, int a, double* partials, unsigned* counters, void* desc) {
    OutPtrs o{out, tau, g_eta, g_W, g_v, g_s2};
    FitDesc f = make_desc(h, th, o, grad, false, a, 0);
    f.partials = partials;
    f.counters = counters;
    std::memcpy(desc, &f, sizeof(FitDesc));
}

int fused_threads(int phase, int variant, int a, int d, int C, int m) {
    if (variant != FUSED_GENERIC) return fused_rt_threads(phase, C, m, a);
    return phase == 1 ? kBThreads : threads_ac(a, d);
}

namespace {
template <typename F>
int occ(F* fn, int threads, size_t smem) {
    set_smem(fn, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    cudaGetLastError();  // a failed query must not surface as a later launch error
    return nb;
}
template <typename S, bool CPLX>
int occ_ac(bool is_c, int dmax, int threads, size_t smem) {
    if (!is_c) {
        if (dmax <= 4) return occ(k_batch_a<S, CPLX, 4>, threads, smem);
        if (dmax <= 8) return occ(k_batch_a<S, CPLX, 8>, threads, smem);
        if (dmax <= 16) return occ(k_batch_a<S, CPLX, 16>, threads, smem);
        return occ(k_batch_a<S, CPLX, 32>, threads, smem);
    }
    if (dmax <= 4) return occ(k_batch_c<S, CPLX, 4>, threads, smem);
    if (dmax <= 8) return occ(k_batch_c<S, CPLX, 8>, threads, smem);
    if (dmax <= 16) return occ(k_batch_c<S, CPLX, 16>, threads, smem);
    return occ(k_batch_c<S, CPLX, 32>, threads, smem);
}
template <bool CPLX, typename S>
int occ_b(int T, size_t smem) {
    switch (T) {
        case 1: return occ(k_batch_b<1, CPLX, S>, kBThreads, smem);
        case 2: return occ(k_batch_b<2, CPLX, S>, kBThreads, smem);
        case 3: return occ(k_batch_b<3, CPLX, S>, kBThreads, smem);
        case 4: return occ(k_batch_b<4, CPLX, S>, kBThreads, smem);
        case 5: return occ(k_batch_b<5, CPLX, S>, kBThreads, smem);
        case 6: return occ(k_batch_b<6, CPLX, S>, kBThreads, smem);
        case 7: return occ(k_batch_b<7, CPLX, S>, kBThreads, smem);
        default: return occ(k_batch_b<8, CPLX, S>, kBThreads, smem);
    }
}
}  // namespace

int fused_resident_blocks(int phase, int variant, bool fp32, bool cplx, int T, int dmax, int threads, size_t smem) {
    if (variant != FUSED_GENERIC) return fused_rt_resident_blocks(phase, variant == FUSED_RT_DF, T, dmax, threads, smem);
    if (phase == 1) {
        if (fp32) return cplx ? occ_b<true, float>(T, smem) : occ_b<false, float>(T, smem);
        return cplx ? occ_b<true, double>(T, smem) : occ_b<false, double>(T, smem);
    }
    const bool is_c = phase == 2;
    if (fp32) return cplx ? occ_ac<float, true>(is_c, dmax, threads, smem) : occ_ac<float, false>(is_c, dmax, threads, smem);
    return cplx ? occ_ac<double, true>(is_c, dmax, threads, smem) : occ_ac<double, false>(is_c, dmax, threads, smem);
}
size_t fused_smem(int phase, int variant, int T, int C, int m, int a, bool fp32, bool cplx) {
    if (variant != FUSED_GENERIC) return fused_rt_smem(phase, T, C, m, a);
    const size_t es = elem_size_of(fp32, cplx);
    return phase == 1 ? smem_b(T, C, m - a, es) : smem_ac(C, a, es);
}
int fused_threads_ac(int a, int d) { return threads_ac(a, d); }

bool fused_supported(const Handle* h) {
    if (h->noise_pt) return false;  // the fused solve takes one shared noise variance
    if (h->dsi_mix) return false;   // the fused column passes evaluate the order-2 DSI kernel only
    int a, lgL;
    return plan(h, &a, &lgL);
}

// B blocks' rows hold NQ sums (generic kernels) or NQ + 1 slots (register-tile kernels: the pivot product
// as mantissa and exponent), then C blocks' d sums, then NQ totals of B's rows (register-tile kernel C)
long long fused_partials_len(const Handle* h) {
    int a, lgL;
    if (!plan(h, &a, &lgL)) return 0;
    const int NQ = 3 + h->T * (h->T + 1) / 2;
    return ((long long)1 << (a - lgL)) * (NQ + 1) + ((long long)1 << (h->m[0] - a)) * h->d + NQ;
}

void launch_fused(const Handle* h, ThetaPtrs th, bool grad, bool store_alpha, double* out, double* tau, double* g_eta,
                  double* g_W, double* g_v, double* g_s2, cudaStream_t st) {
    int a = 0, lgL = 0;
    plan(h, &a, &lgL);
    OutPtrs o{out, tau, g_eta, g_W, g_v, g_s2};
    const FitDesc f = make_desc(h, th, o, grad, store_alpha, a, lgL);
    const int C = h->ncols, m = f.p.m;
    const int var = fused_variant(h->fp32, h->cplx, h->solve_df, h->d, m, a, store_alpha);
    for (int ph = 0; ph < (grad ? 3 : 2); ++ph) {
        static const char* names[3] = {"fused_a", "fused_b", "fused_c"};
        mtgp_prof_begin(h, names[ph], st);
        fused_phase(ph, var, h->fp32, h->cplx, h->T, h->d, &f, nullptr, nullptr, 0, ph == 1 ? f.nb : f.na,
                    fused_threads(ph, var, a, h->d, C, m), fused_smem(ph, var, h->T, C, m, a, h->fp32, h->cplx), st);
        mtgp_prof_end(h, st);
    }
}

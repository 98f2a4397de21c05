// Equal-size fast path for real spectra (digital nets, Walsh-Hadamard transforms): the three fused
// kernels of k_fused.cu with every transform held in registers.
//
// A tile of 2^k elements of one first column (k = a for kernels A and C, k = m - a for kernel B) is
// owned by one warp: lane l holds the E = 2^(k-5) elements l + 32 e.  The unnormalised Walsh-Hadamard
// transform is the tensor product of 2 x 2 butterflies over the index bits, which commute, so a tile's
// stages run as butterflies over the register index e (bits 5 .. k-1) and then over the lane index with
// warp shuffles (bits 0..4): no shared-memory passes and no barriers inside a transform.  The adjoint
// (DIF) transform of real Walsh data is the same operation (H^T = H).
//
//   A  columns c_p of the chunk [base, base + 2^a) from the design words (z(base + l + 32 e) =
//      z(l) XOR z(base + 32 e), both constructions are linear in the index bits), stages 0..a-1 -> spec
//   B  stages a..m-1 of the tile f = h 2^a + lo0, a shared-memory transpose to one thread per
//      frequency, the per-frequency solve (Corollary "equal sizes"), weights back through shared memory,
//      adjoint stages m-1..a                                                  -> wgt
//   C  adjoint stages a-1..0, then dL/deta_j = sum_i omega_c[i] dc_c[i]/deta_j with the kernel values
//      regenerated from the design words; the last block reduces every block's partial sums.
// The kernels serve FP32-transform mode (float spectra) with d <= 16 and tiles of 2^5 .. 2^9 elements.
// Kernel B solves in double-float arithmetic (df64.cuh) unless the handle asks for FP64: the spectra are
// FP32 values, so the solve keeps about 48 bits on the FP32 pipe instead of FP64 on the much narrower
// FP64 pipe; a frequency whose pivots leave the double-float range is solved again in FP64.
#include "fused_common.cuh"

namespace {

// ------------------------------------------------------------------ register-tile Walsh-Hadamard

// butterflies over the register index: (x[e], x[e + 2^b]) -> (x[e] + x[e + 2^b], x[e] - x[e + 2^b])
template <typename S, int LOGE>
__device__ __forceinline__ void wht_regs(S (&x)[1 << LOGE]) {
#pragma unroll
    for (int b = 0; b < LOGE; ++b) {
#pragma unroll
        for (int e = 0; e < (1 << LOGE); ++e) {
            if (!(e & (1 << b))) {
                const S u = x[e], v = x[e | (1 << b)];
                x[e] = u + v;
                x[e | (1 << b)] = u - v;
            }
        }
    }
}

// butterflies over the lane index: the lane with bit b clear keeps x + y, its partner y - x
// (= x_lower - x_upper), one fused multiply-add with the sign +-1 (exact as an addition)
template <typename S, int LOGE>
__device__ __forceinline__ void wht_lanes(S (&x)[1 << LOGE], int lane) {
#pragma unroll
    for (int b = 0; b < 5; ++b) {
        const S sg = ((lane >> b) & 1) ? S(-1) : S(1);
#pragma unroll
        for (int e = 0; e < (1 << LOGE); ++e) {
            const S y = __shfl_xor_sync(0xffffffffu, x[e], 1 << b);
            x[e] = __fmaf_rn(sg, x[e], y);
        }
    }
}

template <typename S, int LOGE>
__device__ __forceinline__ void wht_tile(S (&x)[1 << LOGE], int lane) {
    wht_regs<S, LOGE>(x);
    wht_lanes<S, LOGE>(x, lane);
}

// Design words of a chunk, in shared memory: zl[j][l] = z_j(l) for the 32 lane offsets, zh[j][e] =
// z_j(base + 32 e), dl[c][j] = Delta_t XOR Delta_u of column c = (t, u).
constexpr int kRtMaxE = 16;
constexpr int kRtACWarps = 16;  // kernels A and C: 512 threads per block
struct RtDesign {
    uint32_t zl[MTGP_MAX_DIM][32];
    uint32_t zh[MTGP_MAX_DIM][kRtMaxE];
    uint32_t dl[MTGP_MAX_COLS][MTGP_MAX_DIM];
    uint32_t gen[MTGP_MAX_DIM * 32];
};

// fills RtDesign for the chunk starting at `base` with 2^loge words per lane (all threads call; ends
// with a barrier); reads only handle constants, so it runs before the grid dependency wait.  With the
// handle's word table the chunk's words are one round of loads; without it (the no-allocation entry
// point) they are assembled from the generating matrices.
__device__ __forceinline__ void rt_design(const FitDesc& f, long long base, int loge, RtDesign& s) {
    const FusedParams& p = f.p;
    const int d = p.d, E = 1 << loge;
    if (f.rtw) {
        const long long n32 = p.n >> 5;
        const uint32_t* zl = f.rtw;
        const uint32_t* z32 = f.rtw + 32 * d;
        const uint32_t* dl = z32 + (long long)d * n32;
        for (int e = threadIdx.x; e < 32 * d; e += blockDim.x) s.zl[e >> 5][e & 31] = zl[e];
        for (int e = threadIdx.x; e < E * d; e += blockDim.x) {
            const int j = e >> loge, k = e & (E - 1);
            s.zh[j][k] = z32[(long long)j * n32 + (base >> 5) + k];
        }
        for (int e = threadIdx.x; e < p.C * d; e += blockDim.x) s.dl[e / d][e % d] = dl[e];
        __syncthreads();
        return;
    }
    for (int e = threadIdx.x; e < d * p.gen_cols; e += blockDim.x) s.gen[e] = f.gen[e];
    for (int e = threadIdx.x; e < p.C * d; e += blockDim.x) {
        const int c = e / d, j = e - c * d;
        s.dl[c][j] = f.shift[p.colt[c] * d + j] ^ f.shift[p.colu[c] * d + j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * d; e += blockDim.x) {
        const int j = e >> 5, l = e & 31;
        s.zl[j][l] = point_word(MTGP_DNET, (uint32_t)l, j, s.gen, p.gen_cols);
    }
    for (int e = threadIdx.x; e < E * d; e += blockDim.x) {
        const int j = e >> loge, k = e & (E - 1);
        s.zh[j][k] = point_word(MTGP_DNET, (uint32_t)(base + 32 * k), j, s.gen, p.gen_cols);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------- kernel A

// The chunk's column entries prod_j (1 + eta_j K_j), one (column, element) item per thread, each formed in
// double-float (every factor from the exact product eta_j K_j) and rounded to FP32 once: that halves the
// FP32 spectra's error against the d roundings of a plain FP32 product (the NLL error of FP32-transform
// mode follows it).  Items go to the shared tile (column-major, 2^a per column).
// the factor 1 + eta_j K_j of one item in double-float (from the exact product eta_j K_j)
__device__ __forceinline__ df rt_factor(const RtDesign& s, const float* s_eta, int j, int lane, int e, int c) {
    const float k = dsi2_kernel<float>(s.zl[j][lane] ^ s.zh[j][e] ^ s.dl[c][j]);
    const float ej = s_eta[j];
    const float pk = __fmul_rn(ej, k);
    df f = two_sum(1.0f, pk);
    f.lo = __fadd_rn(f.lo, __fmaf_rn(ej, k, -pk));
    return f;
}

// prod_j (1 + eta_j K_j) of one (column, element) item: the d factors are independent, so they are
// formed first and multiplied in a balanced tree (depth log2 DMAX instead of a chain of d products)
template <int DMAX>
__device__ __forceinline__ float rt_item(const RtDesign& s, const float* s_eta, int d, int a, int it) {
    const int c = it >> a, lo = it & ((1 << a) - 1), lane = lo & 31, e = lo >> 5;
    df f[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) f[j] = j < d ? rt_factor(s, s_eta, j, lane, e, c) : df_of(1.0f);
#pragma unroll
    for (int w = 1; w < DMAX; w <<= 1)
#pragma unroll
        for (int j = 0; j + w < DMAX; j += 2 * w) f[j] = df_mul(f[j], f[j + w]);
    return f[0].hi;
}

// The chunk's column entries prod_j (1 + eta_j K_j), (column, element) items spread over the block, each
// formed in double-float and rounded to FP32 once: that halves the FP32 spectra's error against the d
// roundings of a plain FP32 product (the NLL error of FP32-transform mode follows it).  Two items per
// iteration give each thread two independent chains.  Items go to the shared tile (column-major, 2^a
// per column).
template <int DMAX>
__device__ __forceinline__ void rt_a_generate(const RtDesign& s, const float* s_eta, int d, int C, int a, float* tile) {
    const int n_items = C << a, stride = blockDim.x;
    int it = threadIdx.x;
    for (; it + stride < n_items; it += 2 * stride) {
        const float v0 = rt_item<DMAX>(s, s_eta, d, a, it);
        const float v1 = rt_item<DMAX>(s, s_eta, d, a, it + stride);
        tile[it] = v0;
        tile[it + stride] = v1;
    }
    if (it < n_items) tile[it] = rt_item<DMAX>(s, s_eta, d, a, it);
}

// forward stages 0..a-1 of one column: shared tile -> registers -> global (contiguous)
template <int LOGE>
__device__ __forceinline__ void rt_a_transform(const float* tile, float* out, int lane) {
    constexpr int E = 1 << LOGE;
    float x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = tile[lane + 32 * e];
    wht_tile<float, LOGE>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) out[lane + 32 * e] = x[e];
}

template <int DMAX>
__device__ __forceinline__ void rt_a_body(const FitDesc& f, int blk) {
    const FusedParams& p = f.p;
    __shared__ RtDesign s;
    __shared__ float s_eta[MTGP_MAX_DIM];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tile = reinterpret_cast<float*>(smem_raw);  // C x 2^a
    const int loge = p.a - 5;
    const long long base = (long long)blk << p.a;
    rt_design(f, base, loge, s);
    pdl_wait();  // parameters and the spectra buffer belong to earlier work in the stream
    pdl_trigger();
    if (blk == 0) check_theta_block(f.th, p.d, p.T, f.status);
    if (threadIdx.x < p.d) s_eta[threadIdx.x] = d2f(f.th.eta[threadIdx.x]);
    __syncthreads();
    rt_a_generate<DMAX>(s, s_eta, p.d, p.C, p.a, tile);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* spec = reinterpret_cast<float*>(f.spec);
    for (int c = warp; c < p.C; c += nw) {
        const float* tc = tile + (c << p.a);
        float* out = spec + (long long)c * p.n + base;
        switch (loge) {
            case 0: rt_a_transform<0>(tc, out, lane); break;
            case 1: rt_a_transform<1>(tc, out, lane); break;
            case 2: rt_a_transform<2>(tc, out, lane); break;
            case 3: rt_a_transform<3>(tc, out, lane); break;
            default: rt_a_transform<4>(tc, out, lane); break;
        }
    }
}

// ---------------------------------------------------------------------------------- kernel B

constexpr int kRtBThreads = 256;

// forward (or adjoint) stages of one column of the tile: global (stride 2^a) <-> shared (contiguous)
template <typename S, int LOGE>
__device__ __forceinline__ void rt_b_fwd(const S* in, int a, S* tile, int lane) {
    constexpr int E = 1 << LOGE;
    S x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = in[(long long)(lane + 32 * e) << a];
    wht_tile<S, LOGE>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) tile[lane + 32 * e] = x[e];
}
template <typename S, int LOGE>
__device__ __forceinline__ void rt_b_adj(const S* tile, int a, S* out, int lane) {
    constexpr int E = 1 << LOGE;
    S x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = tile[lane + 32 * e];
    wht_tile<S, LOGE>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) out[(long long)(lane + 32 * e) << a] = x[e];
}
__device__ __forceinline__ void rt_b_pass(bool adj, int loge, const float* gin, float* gout, int a, float* tile,
                                          int lane) {
    if (!adj) {
        switch (loge) {
            case 0: rt_b_fwd<float, 0>(gin, a, tile, lane); break;
            case 1: rt_b_fwd<float, 1>(gin, a, tile, lane); break;
            case 2: rt_b_fwd<float, 2>(gin, a, tile, lane); break;
            case 3: rt_b_fwd<float, 3>(gin, a, tile, lane); break;
            default: rt_b_fwd<float, 4>(gin, a, tile, lane); break;
        }
    } else {
        switch (loge) {
            case 0: rt_b_adj<float, 0>(tile, a, gout, lane); break;
            case 1: rt_b_adj<float, 1>(tile, a, gout, lane); break;
            case 2: rt_b_adj<float, 2>(tile, a, gout, lane); break;
            case 3: rt_b_adj<float, 3>(tile, a, gout, lane); break;
            default: rt_b_adj<float, 4>(tile, a, gout, lane); break;
        }
    }
}

// Partial sums of the register-tile kernels travel between blocks as double-float pairs stored in the
// 8-byte slots of the partial-sum buffer, so no block spends warp-wide FP64 instructions on them (on
// GB300 one warp-wide FP64 instruction occupies an SM's FP64 unit for about 17 cycles).
__device__ __forceinline__ void put_df(double* slot, df v) { *reinterpret_cast<float2*>(slot) = make_float2(v.hi, v.lo); }
__device__ __forceinline__ df get_df(const double* slot) {
    const float2 x = *reinterpret_cast<const float2*>(slot);
    return df_make(x.x, x.y);
}

// Column sums of a (rows x ncols) double-float block in shared memory, one warp per column, a fixed
// order: lane l adds rows l, l + 32, ..., then a shuffle tree; lane 0 stores the total into out[q].
__device__ __forceinline__ void block_sums_df(const df* s_v, int rows, int ncols, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < ncols; q += nw) {
        df v = df_of(0.0f);
        for (int r = lane; r < rows; r += 32) v = df_add(v, s_v[q * rows + r]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            df w;
            w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
            w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
            v = df_add(v, w);
        }
        if (lane == 0) put_df(out + q, v);
    }
}

// Total of one column of the register-tile kernels' partial sums, by one warp (fixed order, 8 loads in
// flight per lane; the total is valid in lane 0).  Kernel B's rows hold NQ + 1 slots: the block's pivot
// product as a double-float mantissa (slot 0) and binary exponent (slot 1), then the NQ - 1 sums; column 0
// is the log-determinant (one logarithm for the whole evaluation), columns 1 .. NQ - 1 the sums, columns
// NQ .. NQ + d - 1 kernel C's d sums (rows of d).
__device__ double rt_column_total(const double* pb, int nb, int NQ, const double* pc, int na, int d, int col) {
    const int lane = threadIdx.x & 31;
    const int NQR = NQ + 1;
    if (col == 0) {
        // the rows' mantissas and exponents loaded 8 at a time before they are multiplied in (the same
        // order as one row after another): one memory round trip per 8 rows instead of one per row
        DFLogAcc acc;
        acc.init();
        for (int b0 = lane; b0 < nb; b0 += 256) {
            df mk[8];
            int ek[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int bb = b0 + 32 * k;
                mk[k] = bb < nb ? get_df(pb + (long long)bb * NQR) : df_of(1.0f);
                ek[k] = bb < nb ? __float_as_int(get_df(pb + (long long)bb * NQR + 1).hi) : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc.mul(mk[k]);
                acc.expo += ek[k];
            }
        }
        acc.warp_product();
        return df_to_double(acc.log_df());
    }
    const bool inb = col < NQ;
    const double* part = inb ? pb + col + 1 : pc + (col - NQ);
    const int nrows = inb ? nb : na, stride = inb ? NQR : d;
    df v = df_of(0.0f);
    for (int b0 = lane; b0 < nrows; b0 += 256) {
        df t[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int bb = b0 + 32 * k;
            t[k] = bb < nrows ? get_df(part + (long long)bb * stride) : df_of(0.0f);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) v = df_add(v, t[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return df_to_double(v);
}

// Final totals (the last block, one warp per column): tot[0 .. NQ - 1] from kernel B's rows, or copied from
// btot when earlier blocks already formed them; etot the d eta totals of kernel C's rows (if pc is given).
__device__ void rt_final_totals(const double* pb, int nb, int NQ, const double* pc, int na, int d, double* tot,
                                double* etot, const double* btot = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ncol = NQ + (pc ? d : 0);
    if (btot && (int)threadIdx.x < NQ) tot[threadIdx.x] = btot[threadIdx.x];
    for (int col = (btot ? NQ : 0) + warp; col < ncol; col += nw) {
        const double v = rt_column_total(pb, nb, NQ, pc, na, d, col);
        if (lane == 0) {
            if (col < NQ) tot[col] = v;
            else etot[col - NQ] = v;
        }
    }
    __syncthreads();
}

// observation of sorted task t at frequency fr as double-float (fr = 0: the residual vanishes, tau at
// its optimum), from the double-float copy when the handle keeps one
__device__ __forceinline__ df rhat_df(const FitDesc& f, int t, long long fr) {
    if (fr == 0) return df_of(0.0f);
    const long long i = (long long)t * f.p.n + fr;
    if (f.yhat_df) {
        const float2 x = f.yhat_df[i];
        return df_make(x.x, x.y);
    }
    return df_from_double(f.yhat[i]);
}

// One frequency by the FP64 recurrences (the double-float solve's fallback), out of line so that the
// double-float kernels carry one copy: spectra from the tile column r, contributions added to fbacc
// (FP64, the caller's), weights written back to the tile; returns the frequency's pivot product.
struct FbOut {
    double mant;
    int expo;
    int bad;
};
template <int T>
__device__ __noinline__ FbOut rt_b_fp64_fallback(const float* s_sp, float* s_wt, int HB, int r, const int* colidx,
                                                 const double* yh, long long n, long long fr, const double* sR,
                                                 double sig, bool clamp, bool grad, double* fbacc) {
    double mu[T][T], w[T][T], al[T], rh[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
#pragma unroll
        for (int u = t; u < T; ++u) mu[t][u] = f2d(s_sp[colidx[t * MTGP_TMAX + u] * HB + r]);
        rh[t] = fr == 0 ? 0.0 : yh[(long long)t * n + fr];
    }
    LogAcc lacc;
    lacc.init();
    int b = 0;
    solve_freq<T, false>(mu, rh, sR, sig, clamp, grad, lacc, fbacc, w, al, false, b);
    if (grad) {
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int u = t; u < T; ++u)
                if (u != t || t == 0) s_wt[colidx[t * MTGP_TMAX + u] * HB + r] = d2f(w[t][u]);
    }
    FbOut o;
    o.mant = lacc.mant;
    o.expo = (int)lacc.expo;
    o.bad = b;
    return o;
}

// DFS: the double-float solve, else the FP64 solve of freq_solve.cuh (float spectra in both cases)
template <int T, bool DFS>
__device__ __forceinline__ void rt_b_body(const FitDesc& f, int blk) {
    using S = float;
    const FusedParams& p = f.p;
    const ThetaPtrs& th = f.th;
    constexpr int NQ = 3 + T * (T + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S* s_sp = reinterpret_cast<S*>(smem_raw);  // C x HB: spectra, then adjoint weights
    __shared__ double sR[T * T];
    __shared__ df sRdf[T * T];
    __shared__ double s_sig;
    __shared__ double s_tot[NQ];
    __shared__ df s_lm[32];
    __shared__ int s_le[32];
    __shared__ int s_cidx[MTGP_TMAX * MTGP_TMAX];
    load_R_f(sR, p, th);
    if (threadIdx.x == 0) s_sig = th.sigma2[0];
    for (int e = threadIdx.x; e < MTGP_TMAX * MTGP_TMAX; e += blockDim.x) s_cidx[e] = p.colidx[e / MTGP_TMAX][e % MTGP_TMAX];
    const int lgH = p.m - p.a, HB = 1 << lgH, loge = lgH - 5;
    const long long lo0 = blk;  // one low index per block (lgL = 0)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // observations of this thread's first frequency, requested before the transform stages so the loads
    // (from DRAM after an L2 flush) overlap them; they do not depend on earlier kernels
    df rh0[T];
    if constexpr (DFS) {
        const long long fr0 = ((long long)threadIdx.x << p.a) + lo0;
#pragma unroll
        for (int t = 0; t < T; ++t) rh0[t] = (int)threadIdx.x < HB ? rhat_df(f, t, fr0) : df_of(0.0f);
    }
    pdl_wait();  // the spectra come from kernel A
    pdl_trigger();
    const S* spec = reinterpret_cast<const S*>(f.spec);
    for (int c = warp; c < p.C; c += nw)
        rt_b_pass(false, loge, spec + (long long)c * p.n + lo0, nullptr, p.a, s_sp + c * HB, lane);
    if (DFS && threadIdx.x < T * T) sRdf[threadIdx.x] = df_from_double(sR[threadIdx.x]);
    __syncthreads();
    const bool clamp = p.clamp != 0, grad = p.grad != 0;
    int bad = 0;
    // per-thread sums: double-float (DFS) or FP64; entry 0 (log det) is kept by the product accumulators
    df accd[DFS ? NQ : 1];
    double acc[NQ];  // DFS: contributions of frequencies solved by the FP64 fallback
#pragma unroll
    for (int q = 0; q < (DFS ? NQ : 1); ++q) accd[q] = df_of(0.0f);
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    DFLogAcc lacc_df;
    lacc_df.init();
    LogAcc lacc;
    lacc.init();
    bool any_fb = !DFS;  // FP64 sums to fold into the double-float ones
    const double sig = s_sig;
    const df sigdf = df_from_double(sig);
    for (int r = threadIdx.x; r < HB; r += blockDim.x) {
        const long long fr = ((long long)r << p.a) + lo0;
        if constexpr (DFS) {
            float mu[T][T], w[T][T];
            df rh[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int u = t; u < T; ++u) mu[t][u] = s_sp[s_cidx[t * MTGP_TMAX + u] * HB + r];
                rh[t] = r == (int)threadIdx.x ? rh0[t] : rhat_df(f, t, fr);
            }
            if (solve_freq_df<T>(mu, rh, sRdf, sigdf, clamp, grad, lacc_df, accd, w, bad)) {
                if (grad) {
#pragma unroll
                    for (int t = 0; t < T; ++t)
#pragma unroll
                        for (int u = t; u < T; ++u)
                            if (u != t || t == 0) s_sp[s_cidx[t * MTGP_TMAX + u] * HB + r] = w[t][u];
                }
            } else {
                const FbOut o = rt_b_fp64_fallback<T>(s_sp, s_sp, HB, r, s_cidx, f.yhat, p.n, fr, sR, sig, clamp, grad,
                                                      acc);
                lacc_df.mul_fp64(o.mant);
                lacc_df.expo += o.expo;
                bad |= o.bad;
                any_fb = true;
            }
        } else {
            double mu[T][T], w[T][T], al[T], rh[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int u = t; u < T; ++u) mu[t][u] = f2d(s_sp[s_cidx[t * MTGP_TMAX + u] * HB + r]);
                rh[t] = fr == 0 ? 0.0 : f.yhat[(long long)t * p.n + fr];
            }
            solve_freq<T, false>(mu, rh, sR, sig, clamp, grad, lacc, acc, w, al, false, bad);
            if (grad) {
#pragma unroll
                for (int t = 0; t < T; ++t)
#pragma unroll
                    for (int u = t; u < T; ++u)
                        if (u != t || t == 0) s_sp[s_cidx[t * MTGP_TMAX + u] * HB + r] = d2f(w[t][u]);
            }
        }
    }
    if (bad) set_status(f.status, ST_NOT_PD);
    // log-determinant: the FP64 pivot products (if any) join the double-float one, a double-float product
    // over each warp, then one logarithm per block (thread 0)
    if constexpr (!DFS) {
        lacc_df.mul_fp64(lacc.mant);
        lacc_df.expo += (int)lacc.expo;
    }
    lacc_df.warp_product();
    if (lane == 0) {
        s_lm[warp] = lacc_df.mant;
        s_le[warp] = lacc_df.expo;
    }
    __syncthreads();  // weights complete in shared memory
    if (grad) {
        S* wgt = reinterpret_cast<S*>(f.wgt);
        for (int c = warp; c < p.C; c += nw)
            rt_b_pass(true, loge, nullptr, wgt + (long long)c * p.n + lo0, p.a, s_sp + c * HB, lane);
        __syncthreads();  // the tile area is reused for the partial sums
    }
    // block partial sums as double-float pairs: the pivot product as mantissa and exponent (slots 0, 1),
    // then the other sums through shared memory, one warp per entry (slots 2..)
    double* partials = f.partials + (long long)blk * (NQ + 1);
    const int nt = blockDim.x;
    df* s_v = reinterpret_cast<df*>(smem_raw);
    if (any_fb) {
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            const df fb = df_from_double(acc[q]);
            s_v[(q - 1) * nt + threadIdx.x] = DFS ? df_add(accd[DFS ? q : 0], fb) : fb;
        }
    } else {
#pragma unroll
        for (int q = 1; q < NQ; ++q) s_v[(q - 1) * nt + threadIdx.x] = accd[DFS ? q : 0];
    }
    __syncthreads();
    block_sums_df(s_v, nt, NQ - 1, partials + 2);
    if (threadIdx.x == 0) {
        DFLogAcc tot;
        tot.init();
        for (int w = 0; w < nw; ++w) {
            tot.mul(s_lm[w]);
            tot.expo += s_le[w];
        }
        put_df(partials, tot.mant);
        put_df(partials + 1, df_make(__int_as_float(tot.expo), 0.0f));
    }
    if (grad) return;  // kernel C finishes
    if (!last_block(f.counters, f.nb)) return;
    rt_final_totals(f.partials, f.nb, NQ, nullptr, 0, 0, s_tot, nullptr);
    write_outputs(s_tot, nullptr, p, th, f.tau, f.o);
    if (threadIdx.x == 0) *f.counters = 0u;
}

// ---------------------------------------------------------------------------------- kernel C

// adjoint stages a-1..0 of one column: global (contiguous) -> registers -> shared tile
template <int LOGE>
__device__ __forceinline__ void rt_c_transform(const float* in, float* tile, int lane) {
    constexpr int E = 1 << LOGE;
    float x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = in[lane + 32 * e];
    wht_tile<float, LOGE>(x, lane);
#pragma unroll
    for (int e = 0; e < E; ++e) tile[lane + 32 * e] = x[e];
}

// the eta contractions of the chunk, one (column, element) item per thread:
//   dL/deta_j += w K_j prod_{k != j} (1 + eta_k K_k)
// with prefix / suffix products (no division by 1 + eta K, which may vanish).  The forward pass keeps
// only the factors and K_j times the prefix product, so an item holds 2 d values.
template <int DMAX>
__device__ __forceinline__ void rt_c_item(const RtDesign& s, const float* s_eta, int d, int a, int it, const float* tile,
                                          float (&part)[DMAX]) {
    const int c = it >> a, lo = it & ((1 << a) - 1), lane = lo & 31, e = lo >> 5;
    float fv[DMAX], kp[DMAX];
    float pr = 1.0f;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            const float k = dsi2_kernel<float>(s.zl[j][lane] ^ s.zh[j][e] ^ s.dl[c][j]);
            fv[j] = fmaf(s_eta[j], k, 1.0f);
            kp[j] = k * pr;
            pr *= fv[j];
        }
    }
    float suf = tile[it];
#pragma unroll
    for (int j = DMAX - 1; j >= 0; --j) {
        if (j < d) {
            part[j] = fmaf(kp[j], suf, part[j]);
            suf *= fv[j];
        }
    }
}

// the eta contractions of the chunk, (column, element) items spread over the block, two per iteration
// (PAIR and d <= 8; otherwise one, within the register budget):
//   dL/deta_j += w K_j prod_{k != j} (1 + eta_k K_k)
// with prefix / suffix products (no division by 1 + eta K, which may vanish)
template <int DMAX, bool PAIR>
__device__ __forceinline__ void rt_c_contract(const RtDesign& s, const float* s_eta, int d, int C, int a,
                                              const float* tile, float (&part)[DMAX]) {
    const int n_items = C << a, stride = blockDim.x;
    int it = threadIdx.x;
    if constexpr (PAIR && DMAX <= 8) {
        // both items add into the same sums in item order, so the result equals one item at a time; only
        // their kernel values and products overlap
        for (; it + stride < n_items; it += 2 * stride) {
            rt_c_item<DMAX>(s, s_eta, d, a, it, tile, part);
            rt_c_item<DMAX>(s, s_eta, d, a, it + stride, tile, part);
        }
    }
    for (; it < n_items; it += stride) rt_c_item<DMAX>(s, s_eta, d, a, it, tile, part);
}

// PAIR: two contraction items per loop iteration (the single-fit kernel; the batch kernel, which keeps more
// state live across its item loop, takes one at a time within the register budget); the sums are the same
template <int DMAX, bool PAIR>
__device__ __forceinline__ void rt_c_body(const FitDesc& f, int blk) {
    using S = float;
    const FusedParams& p = f.p;
    __shared__ RtDesign s;
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ S s_red[kRtACWarps][DMAX];
    __shared__ double s_tot[3 + MTGP_MAX_COLS];
    __shared__ double s_etot[MTGP_MAX_DIM];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* tile = reinterpret_cast<float*>(smem_raw);  // C x 2^a adjoint weights
    const int loge = p.a - 5, d = p.d;
    const long long base = (long long)blk << p.a;
    __shared__ double s_W[MTGP_TMAX * MTGP_TMAX];
    if (threadIdx.x < d) s_eta[threadIdx.x] = d2f(f.th.eta[threadIdx.x]);
    // W for the final outputs, staged now so the last block does not wait for it
    for (int e = threadIdx.x; e < p.T * f.th.s; e += blockDim.x) s_W[e] = f.th.W[e];
    rt_design(f, base, loge, s);
    pdl_wait();  // the adjoint weights and kernel B's partial sums
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int NQ = 3 + p.T * (p.T + 1) / 2;
    double* partials_c = f.partials + (long long)f.nb * (NQ + 1);  // after B's NQ + 1 slots per block
    double* btot = partials_c + (long long)f.na * d;
    // kernel B's column totals, column q by block q mod na, on the last warp (idle while the first warps
    // transform the columns): the last block then reduces only kernel C's rows
    if (warp == nw - 1)
        for (int col = blk; col < NQ; col += f.na) {
            const double v = rt_column_total(f.partials, f.nb, NQ, nullptr, 0, 0, col);
            if (lane == 0) btot[col] = v;
        }
    const S* wgt = reinterpret_cast<const S*>(f.wgt);
    for (int c = warp; c < p.C; c += nw) {
        const float* in = wgt + (long long)c * p.n + base;
        float* tc = tile + (c << p.a);
        switch (loge) {
            case 0: rt_c_transform<0>(in, tc, lane); break;
            case 1: rt_c_transform<1>(in, tc, lane); break;
            case 2: rt_c_transform<2>(in, tc, lane); break;
            case 3: rt_c_transform<3>(in, tc, lane); break;
            default: rt_c_transform<4>(in, tc, lane); break;
        }
    }
    __syncthreads();
    S part[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) part[j] = S(0);
    rt_c_contract<DMAX, PAIR>(s, s_eta, d, p.C, p.a, tile, part);
    // the d block sums: a shuffle tree per warp, one shared row per warp, warps added in order
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
        S v = S(0);
        for (int w = 0; w < nw; ++w) v += s_red[w][threadIdx.x];
        put_df(partials_c + (long long)blk * d + threadIdx.x, df_of(v));
    }
    if (!last_block(f.counters + 1, f.na)) return;
    rt_final_totals(f.partials, f.nb, NQ, partials_c, f.na, d, s_tot, s_etot, btot);
    write_outputs(s_tot, s_etot, p, f.th, f.tau, f.o, s_W);
    if (threadIdx.x == 0) f.counters[1] = 0u;
}

// ---------------------------------------------------------------------------------- kernels

template <int DMAX>
__global__ void __launch_bounds__(512, 2) k_rt_a(FitDesc f) { rt_a_body<DMAX>(f, blockIdx.x); }
template <int T, bool DFS>
__global__ void __launch_bounds__(kRtBThreads, (T <= 4 ? 2 : 1)) k_rt_b(FitDesc f) { rt_b_body<T, DFS>(f, blockIdx.x); }
template <int DMAX>
__global__ void __launch_bounds__(512, 2) k_rt_c(FitDesc f) { rt_c_body<DMAX, true>(f, blockIdx.x); }

template <int DMAX>
__global__ void __launch_bounds__(512, 2) k_rt_batch_a(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        rt_a_body<DMAX>(fits[w.x], w.y);
        __syncthreads();
    }
}
template <int T, bool DFS>
__global__ void __launch_bounds__(kRtBThreads, (T <= 4 ? 2 : 1)) k_rt_batch_b(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        rt_b_body<T, DFS>(fits[w.x], w.y);
        __syncthreads();
    }
}
template <int DMAX>
__global__ void __launch_bounds__(512, 2) k_rt_batch_c(const FitDesc* fits, const int2* items, int nitems) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        rt_c_body<DMAX, false>(fits[w.x], w.y);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------- host dispatch

template <typename F>
int occupancy(F* fn, int threads, size_t smem) {
    set_smem(fn, smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) nb = 1;
    cudaGetLastError();  // a failed query must not surface as a later launch error
    return nb;
}

template <int DMAX>
int rt_ac(bool is_c, const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid, int threads,
          size_t smem, cudaStream_t st, bool query) {
    if (!is_c) {
        if (query) return occupancy(k_rt_batch_a<DMAX>, threads, smem);
        if (single) {
            set_smem(k_rt_a<DMAX>, smem);
            launch_pdl(k_rt_a<DMAX>, grid, threads, smem, st, *single);
        } else {
            set_smem(k_rt_batch_a<DMAX>, smem);
            k_rt_batch_a<DMAX><<<grid, threads, smem, st>>>(fits, items, nitems);
        }
    } else {
        if (query) return occupancy(k_rt_batch_c<DMAX>, threads, smem);
        if (single) {
            set_smem(k_rt_c<DMAX>, smem);
            launch_pdl(k_rt_c<DMAX>, grid, threads, smem, st, *single);
        } else {
            set_smem(k_rt_batch_c<DMAX>, smem);
            k_rt_batch_c<DMAX><<<grid, threads, smem, st>>>(fits, items, nitems);
        }
    }
    return 0;
}

template <int T, bool DFS>
int rt_b_t(const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid, size_t smem,
           cudaStream_t st, bool query) {
    if (query) return occupancy(k_rt_batch_b<T, DFS>, kRtBThreads, smem);
    if (single) {
        set_smem(k_rt_b<T, DFS>, smem);
        launch_pdl(k_rt_b<T, DFS>, grid, kRtBThreads, smem, st, *single);
    } else {
        set_smem(k_rt_batch_b<T, DFS>, smem);
        k_rt_batch_b<T, DFS><<<grid, kRtBThreads, smem, st>>>(fits, items, nitems);
    }
    return 0;
}

template <bool DFS>
int rt_b(int T, const FitDesc* single, const FitDesc* fits, const int2* items, int nitems, int grid, size_t smem,
         cudaStream_t st, bool query) {
    switch (T) {
        case 1: return rt_b_t<1, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 2: return rt_b_t<2, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 3: return rt_b_t<3, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 4: return rt_b_t<4, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 5: return rt_b_t<5, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 6: return rt_b_t<6, DFS>(single, fits, items, nitems, grid, smem, st, query);
        case 7: return rt_b_t<7, DFS>(single, fits, items, nitems, grid, smem, st, query);
        default: return rt_b_t<8, DFS>(single, fits, items, nitems, grid, smem, st, query);
    }
}

int rt_dispatch(int phase, bool dfs, int T, int dmax, const FitDesc* single, const FitDesc* fits, const int2* items,
                int nitems, int grid, int threads, size_t smem, cudaStream_t st, bool query) {
    if (phase == 1)
        return dfs ? rt_b<true>(T, single, fits, items, nitems, grid, smem, st, query)
                   : rt_b<false>(T, single, fits, items, nitems, grid, smem, st, query);
    const bool is_c = phase == 2;
    if (dmax <= 4) return rt_ac<4>(is_c, single, fits, items, nitems, grid, threads, smem, st, query);
    if (dmax <= 8) return rt_ac<8>(is_c, single, fits, items, nitems, grid, threads, smem, st, query);
    return rt_ac<16>(is_c, single, fits, items, nitems, grid, threads, smem, st, query);
}

}  // namespace

// FP32 real spectra, d <= 16, both tile sizes in 2^5 .. 2^9 (kernel B's tile: at most 29 x 512 floats)
bool fused_rt_ok(bool cplx, bool fp32, int d, int m, int a) {
    return !cplx && fp32 && d <= 16 && a >= 5 && a <= 9 && m - a >= 5 && m - a <= 9;
}

int fused_rt_threads(int phase, int C, int m, int a) {
    (void)C;
    (void)m;
    (void)a;
    return phase == 1 ? kRtBThreads : 32 * kRtACWarps;
}

// dynamic shared memory: kernels A and C hold the chunk's C x 2^a tile, kernel B the C x 2^(m-a) tile or
// its partial sums
size_t fused_rt_smem(int phase, int T, int C, int m, int a) {
    if (phase != 1) return sizeof(float) * (size_t)C * ((size_t)1 << a);
    const size_t tile = sizeof(float) * (size_t)C * ((size_t)1 << (m - a));
    const size_t red = (size_t)(2 + T * (T + 1) / 2) * kRtBThreads * 8;  // NQ - 1 entries of 8 bytes per thread
    return tile > red ? tile : red;
}

void fused_rt_phase(int phase, bool dfs, int T, int dmax, const void* single, const void* fits, const int2* items,
                    int nitems, int grid, int threads, size_t smem, cudaStream_t st) {
    rt_dispatch(phase, dfs, T, dmax, static_cast<const FitDesc*>(single), static_cast<const FitDesc*>(fits), items, nitems,
                grid, threads, smem, st, false);
}

int fused_rt_resident_blocks(int phase, bool dfs, int T, int dmax, int threads, size_t smem) {
    return rt_dispatch(phase, dfs, T, dmax, nullptr, nullptr, nullptr, 0, 0, threads, smem, nullptr, true);
}

namespace {
__global__ void k_yhat_df(const double* __restrict__ yhat, float2* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const df v = df_from_double(yhat[i]);
        out[i] = make_float2(v.hi, v.lo);
    }
}
}  // namespace

void launch_yhat_df(const double* yhat, float* yhat_df, long long n, cudaStream_t st) {
    const long long blocks = (n + 255) / 256;
    k_yhat_df<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(yhat, reinterpret_cast<float2*>(yhat_df), n);
}

namespace {
// z_j(l), l < 32; z_j(32 k), k < n / 32; Delta_t XOR Delta_u per column (digital nets, equal sizes)
__global__ void k_rt_words(uint32_t* __restrict__ out, int d, int C, long long n32, const uint32_t* __restrict__ gen,
                           int gen_cols, const uint32_t* __restrict__ shift, const int2* __restrict__ cols) {
    const long long tot = 32LL * d + (long long)d * n32 + (long long)C * d;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        uint32_t w;
        if (e < 32LL * d) {
            w = point_word(MTGP_DNET, (uint32_t)(e & 31), (int)(e >> 5), gen, gen_cols);
        } else if (e < 32LL * d + (long long)d * n32) {
            const long long r = e - 32LL * d;
            const int j = (int)(r / n32);
            w = point_word(MTGP_DNET, (uint32_t)((r - j * n32) << 5), j, gen, gen_cols);
        } else {
            const long long r = e - 32LL * d - (long long)d * n32;
            const int c = (int)(r / d), j = (int)(r - (long long)c * d);
            w = shift[cols[c].x * d + j] ^ shift[cols[c].y * d + j];
        }
        out[e] = w;
    }
}
}  // namespace

long long rt_words_len(const Handle* h) {
    if (!h->equal || !h->fp32 || h->cplx || h->d > 16 || h->m[0] < 10) return 0;
    return 32LL * h->d + (long long)h->d * (h->n[0] >> 5) + (long long)h->ncols * h->d;
}

void launch_rt_words(const Handle* h, cudaStream_t st) {
    int2 cols[MTGP_MAX_COLS];
    for (int c = 0; c < h->ncols; ++c) cols[c] = make_int2(h->cols[c].t, h->cols[c].u);
    int2* dcols = nullptr;
    if (cudaMalloc(&dcols, sizeof(int2) * h->ncols) != cudaSuccess) return;
    cudaMemcpy(dcols, cols, sizeof(int2) * h->ncols, cudaMemcpyHostToDevice);
    const long long tot = rt_words_len(h);
    k_rt_words<<<(unsigned)((tot + 255) / 256 < 1024 ? (tot + 255) / 256 : 1024), 256, 0, st>>>(
        h->rt_words, h->d, h->ncols, h->n[0] >> 5, h->gen, h->gen_cols, h->shift, dcols);
    cudaStreamSynchronize(st);
    cudaFree(dcols);
}

// Design points, first kernel columns, observation loading and the eta-gradient pass.
//
// First column of block (t, u) (sorted tasks, n_t >= n_u), Theorem "fast MTGP computations" item 3:
//   c_{tu}[i] = Q(x_{t,i}, x_{u,0}) = prod_j (1 + eta_j K(z_{i,j} (+) Delta_{t,j} (-) Delta_{u,j})),  i < n_t,
// in radical-inverse order, generated on the fly from the index i (Def. 2.1 / 2.2, Eq. 2.4-2.6).
// The task covariance R and the noise enter later, per frequency, so the columns depend on eta only.
#include "mtgp_internal.cuh"
#include "kernel_df.cuh"

namespace {

constexpr int kThreads = 256;

struct ColParams {
    ColDesc cols[MTGP_MAX_COLS];
    long long tile0[MTGP_MAX_COLS + 1];  // first 256-element tile of each column (prefix sums)
    int alpha;           // SI smoothness
    const double* bmix;  // DSI mixture weights (4), or nullptr
};

// Points of a tile of 256 consecutive indices t0 + lo (t0 a multiple of 256): the index bits of t0
// and lo are disjoint, and both constructions are linear in them (lattice: bitrev(t0 | lo) g =
// bitrev(t0) g + bitrev(lo) g mod 2^32; digital net: XOR of the generator columns of the set bits),
// so z(t0 + lo) = z(t0) (+) z(lo).  Each thread keeps z(lo) of its own lo in shared memory; z(t0) is
// formed once per tile by d threads.
__device__ __forceinline__ uint32_t combine_word(int kind, uint32_t zhi, uint32_t zlo) {
    return kind == MTGP_LATTICE ? zhi + zlo : (zhi ^ zlo);
}

template <typename S, bool CPLX>
__global__ void __launch_bounds__(kThreads)
k_colgen(void* out, ColParams cp, int kind, int d, const uint32_t* __restrict__ gen, int gen_cols,
         const uint32_t* __restrict__ shift, const double* __restrict__ eta) {
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ S s_b[4];
    __shared__ uint32_t s_dt[MTGP_MAX_DIM], s_du[MTGP_MAX_DIM], s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_zlo[MTGP_MAX_DIM * kThreads];
    const ColDesc c = cp.cols[blockIdx.y];
    const int tid = threadIdx.x;
    if (tid < d) {
        s_eta[tid] = (S)eta[tid];
        s_dt[tid] = shift[c.t * d + tid];
        s_du[tid] = shift[c.u * d + tid];
    }
    if (cp.bmix && tid < 4) s_b[tid] = (S)cp.bmix[tid];
    const S* bw = cp.bmix ? s_b : nullptr;
    for (int j = 0; j < d; ++j) s_zlo[j * kThreads + tid] = point_word(kind, (uint32_t)tid, j, gen, gen_cols);
    for (long long t0 = (long long)blockIdx.x * kThreads; t0 < c.n; t0 += (long long)gridDim.x * kThreads) {
        __syncthreads();  // the previous tile's reads of s_zhi are done
        if (tid < d) s_zhi[tid] = point_word(kind, (uint32_t)t0, tid, gen, gen_cols);
        __syncthreads();
        const long long i = t0 + tid;
        if (i < c.n) {
            S q = (S)1;
            for (int j = 0; j < d; ++j) {
                const uint32_t z = combine_word(kind, s_zhi[j], s_zlo[j * kThreads + tid]);
                const uint32_t X = pair_word(kind, z, s_dt[j], s_du[j]);
                q *= (S)1 + s_eta[j] * kernel1d_b<S>(kind, X, cp.alpha, bw);
            }
            if (CPLX) {
                // a pair's lead writes the real part, its partner the imaginary part of the lead's element
                S* o = reinterpret_cast<S*>(out);
                if (c.role == 0) reinterpret_cast<cx<S>*>(out)[c.off + i] = mk(q, (S)0);
                else if (c.role == 1) o[2 * (c.off + i)] = q;
                else o[2 * (c.src + i) + 1] = q;
            } else {
                reinterpret_cast<S*>(out)[c.off + i] = q;
            }
        }
    }
}

__global__ void k_points(uint32_t* __restrict__ x, int kind, int d, const uint32_t* __restrict__ gen, int gen_cols,
                         const uint32_t* __restrict__ shift_sorted, int sorted_t, long long n, long long out_off) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * d;
         e += (long long)gridDim.x * blockDim.x) {
        long long i = e / d;
        int j = (int)(e - i * d);
        uint32_t z = point_word(kind, (uint32_t)i, j, gen, gen_cols);
        uint32_t dt = shift_sorted[sorted_t * d + j];
        x[(out_off + i) * d + j] = (kind == MTGP_LATTICE) ? z + dt : z ^ dt;
    }
}

__global__ void k_y_load(double* __restrict__ yhat, const double* __restrict__ y, long long n, long long in_off,
                         long long out_off, int cplx) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = y[in_off + i];
        if (cplx) {
            yhat[2 * (out_off + i)] = v;
            yhat[2 * (out_off + i) + 1] = 0.0;
        } else {
            yhat[out_off + i] = v;
        }
    }
}

__global__ void k_scale(double* __restrict__ a, long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] *= s;
}

// dL/deta_j = Re sum_c sum_i omega_c[i] dc_c[i]/deta_j, omega = DIF(adjoint weights); the derivative
// of the product is K_j prod_{l != j} (1 + eta_l K_l), formed with prefix and suffix products
// (no division: a factor 1 + eta K may vanish).  With DSI mixture weights (MIX) the same pass also
// forms dL/db_a = Re sum omega dc/db_a, dc/db_a = sum_j eta_j K_a(x_j) prod_{l != j} (1 + eta_l K_l),
// written after the d eta entries of each block's partials.
template <typename S, bool CPLX, bool MIX>
__global__ void __launch_bounds__(kThreads)
k_eta_grad(const void* omega, ColParams cp, int ncols, int kind, int d, const uint32_t* __restrict__ gen,
           int gen_cols, const uint32_t* __restrict__ shift, const double* __restrict__ eta,
           double* __restrict__ partials) {
    constexpr int NB = MIX ? 4 : 0;
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ S s_b[4];
    __shared__ double s_red[kThreads / 32][MTGP_MAX_DIM + 4];
    __shared__ uint32_t s_dt[MTGP_MAX_DIM], s_du[MTGP_MAX_DIM], s_zhi[MTGP_MAX_DIM];
    __shared__ uint32_t s_zlo[MTGP_MAX_DIM * kThreads];
    const int tid = threadIdx.x;
    if (tid < d) s_eta[tid] = (S)eta[tid];
    if (MIX && tid < 4) s_b[tid] = (S)cp.bmix[tid];
    for (int j = 0; j < d; ++j) s_zlo[j * kThreads + tid] = point_word(kind, (uint32_t)tid, j, gen, gen_cols);
    const S* bw = MIX ? s_b : nullptr;
    // per-thread sums in the transform precision (FP32 additions keep the FP64 pipe free; a thread
    // adds a few hundred terms), FP64 from the warp sums on
    S acc[MTGP_MAX_DIM + NB];
    for (int j = 0; j < d + NB; ++j) acc[j] = (S)0;
    // 256-element tiles of the columns, tile g of all columns (column c owns tiles tile0[c] ..)
    const long long ntiles = cp.tile0[ncols];
    for (long long g = blockIdx.x; g < ntiles; g += gridDim.x) {
        int c = 0;
        while (c + 1 < ncols && g >= cp.tile0[c + 1]) ++c;
        const ColDesc cd = cp.cols[c];
        const long long t0 = (g - cp.tile0[c]) * kThreads;
        __syncthreads();  // the previous tile's reads of the shared words are done
        if (tid < d) {
            s_zhi[tid] = point_word(kind, (uint32_t)t0, tid, gen, gen_cols);
            s_dt[tid] = shift[cd.t * d + tid];
            s_du[tid] = shift[cd.u * d + tid];
        }
        __syncthreads();
        const long long i = t0 + tid;
        if (i >= cd.n) continue;
        S w;
        if (CPLX) {
            // a partner's transformed weights are the imaginary part of its lead's array
            const cx<S> o = reinterpret_cast<const cx<S>*>(omega)[(cd.role == 2 ? cd.src : cd.off) + i];
            w = cd.role == 2 ? o.im : o.re;
        } else {
            w = reinterpret_cast<const S*>(omega)[cd.off + i];
        }
        S kv[MTGP_MAX_DIM];
        S pre[MTGP_MAX_DIM];
        S fac[MTGP_MAX_DIM];
        uint32_t xw[MIX ? MTGP_MAX_DIM : 1];
        S p = (S)1;
        for (int j = 0; j < d; ++j) {
            const uint32_t z = combine_word(kind, s_zhi[j], s_zlo[j * kThreads + tid]);
            const uint32_t X = pair_word(kind, z, s_dt[j], s_du[j]);
            if (MIX) xw[j] = X;
            kv[j] = kernel1d_b<S>(kind, X, cp.alpha, bw);
            fac[j] = fma(s_eta[j], kv[j], (S)1);
            pre[j] = p;
            p *= fac[j];
        }
        // the adjoint weight rides in the suffix product: suf = w prod_{l > j} (1 + eta_l K_l)
        S suf = w;
        for (int j = d - 1; j >= 0; --j) {
            const S ps = pre[j] * suf;
            acc[j] = fma(kv[j], ps, acc[j]);
            if (MIX) {
                S ko[4];
                dsi_orders<S>(xw[j], ko);
                const S f = s_eta[j] * ps;
                for (int a = 0; a < 4; ++a) acc[d + a] = fma(f, ko[a], acc[d + a]);
            }
            suf *= fac[j];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < d + NB; ++j) {
        double v = (double)acc[j];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[warp][j] = v;
    }
    __syncthreads();
    if (threadIdx.x < d + NB) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_red[w][threadIdx.x];
        partials[(long long)blockIdx.x * (d + NB) + threadIdx.x] = v;
    }
}

// The same contraction for FP64 fits in double-float arithmetic (no mixture, d <= DMAX):
// K_j s exact (digital nets) or to ~2^-47 (lattices), the factors, prefix products and the per-thread sums
// as double-float pairs on the FP32 pipe, the block sums in FP64.  Only the eta gradient depends on it;
// its terms carry ~2^-46 relative error against the FP64 gradient tolerance of 1e-7.
template <bool CPLX, int DMAX>
__global__ void __launch_bounds__(kThreads)
k_eta_grad_df(const void* omega, ColParams cp, int ncols, int kind, int d, const uint32_t* __restrict__ gen,
              int gen_cols, const uint32_t* __restrict__ shift, const double* __restrict__ eta,
              double* __restrict__ partials) {
    __shared__ df s_es[DMAX];
    __shared__ double s_red[kThreads / 32][DMAX];
    __shared__ uint32_t s_dt[DMAX], s_du[DMAX], s_zhi[DMAX];
    __shared__ uint32_t s_zlo[DMAX * kThreads];
    const int tid = threadIdx.x;
    const double sinv = kval_scale_inv(kind);
    if (tid < d) s_es[tid] = df_from_double(eta[tid] * sinv);
    for (int j = 0; j < d; ++j) s_zlo[j * kThreads + tid] = point_word(kind, (uint32_t)tid, j, gen, gen_cols);
    const Si2Consts sc = si2_consts(cp.alpha);
    df acc[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) acc[j] = df_of(0.0f);
    const long long ntiles = cp.tile0[ncols];
    for (long long g = blockIdx.x; g < ntiles; g += gridDim.x) {
        int c = 0;
        while (c + 1 < ncols && g >= cp.tile0[c + 1]) ++c;
        const ColDesc cd = cp.cols[c];
        const long long t0 = (g - cp.tile0[c]) * kThreads;
        __syncthreads();  // the previous tile's reads of the shared words are done
        if (tid < d) {
            s_zhi[tid] = point_word(kind, (uint32_t)t0, tid, gen, gen_cols);
            s_dt[tid] = shift[cd.t * d + tid];
            s_du[tid] = shift[cd.u * d + tid];
        }
        __syncthreads();
        const long long i = t0 + tid;
        if (i >= cd.n) continue;
        double w;
        if (CPLX) {
            const cx<double> o = reinterpret_cast<const cx<double>*>(omega)[(cd.role == 2 ? cd.src : cd.off) + i];
            w = cd.role == 2 ? o.im : o.re;
        } else {
            w = reinterpret_cast<const double*>(omega)[cd.off + i];
        }
        df fv[DMAX], kp[DMAX];
        df pr = df_of(1.0f);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < d) {
                const uint32_t z = combine_word(kind, s_zhi[j], s_zlo[j * kThreads + tid]);
                const df ks = kval_scaled_df(kind, pair_word(kind, z, s_dt[j], s_du[j]), sc);
                fv[j] = df_one_plus(df_mul(s_es[j], ks));
                kp[j] = df_mul(ks, pr);
                pr = df_mul(pr, fv[j]);
            }
        }
        // the adjoint weight rides in the suffix product: suf = w prod_{l > j} (1 + eta_l K_l)
        df suf = df_from_double(w);
#pragma unroll
        for (int j = DMAX - 1; j >= 0; --j) {
            if (j < d) {
                acc[j] = df_fma(acc[j], kp[j], suf);
                suf = df_mul(suf, fv[j]);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        if (j < d) {
            double v = df_to_double(acc[j]) * sinv;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) s_red[warp][j] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < d) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_red[w][threadIdx.x];
        partials[(long long)blockIdx.x * d + threadIdx.x] = v;
    }
}

// F(a), F(b) from Z = F(a + i b) for real a, b (Hermitian spectra): F(a)[f] = (Z[f] + conj Z[-f]) / 2,
// F(b)[f] = -i (Z[f] - conj Z[-f]) / 2, -f = (n - f) mod n.  One thread takes f and -f together, so
// the lead's array is overwritten in place.
template <typename S>
__global__ void k_pair_split(cx<S>* __restrict__ spec, const long long* __restrict__ pairs, int npairs) {
    const int pr = blockIdx.y;
    if (pr >= npairs) return;
    const long long offa = pairs[3 * pr], offb = pairs[3 * pr + 1], n = pairs[3 * pr + 2];
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f <= n / 2;
         f += (long long)gridDim.x * blockDim.x) {
        const long long g = (n - f) & (n - 1);
        const cx<S> zf = spec[offa + f], zg = spec[offa + g];
        const S h = (S)0.5;
        spec[offa + f] = mk(h * (zf.re + zg.re), h * (zf.im - zg.im));
        spec[offb + f] = mk(h * (zf.im + zg.im), h * (zg.re - zf.re));
        if (g != f) {
            spec[offa + g] = mk(h * (zg.re + zf.re), h * (zg.im - zf.im));
            spec[offb + g] = mk(h * (zg.im + zf.im), h * (zf.re - zg.re));
        }
    }
}

// the lead's weights become w_a + i w_b (the adjoint transform is linear; both transformed weight
// arrays are real up to rounding, the eta adjoint reads the real part for a and the imaginary for b)
template <typename S>
__global__ void k_pair_pack(cx<S>* __restrict__ wgt, const long long* __restrict__ pairs, int npairs) {
    const int pr = blockIdx.y;
    if (pr >= npairs) return;
    const long long offa = pairs[3 * pr], offb = pairs[3 * pr + 1], n = pairs[3 * pr + 2];
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n; f += (long long)gridDim.x * blockDim.x) {
        const cx<S> wa = wgt[offa + f], wb = wgt[offb + f];
        wgt[offa + f] = mk(wa.re - wb.im, wa.im + wb.re);
    }
}

ColParams make_params(const Handle* h) {
    ColParams cp;
    for (int c = 0; c < h->ncols; ++c) cp.cols[c] = h->cols[c];
    cp.alpha = h->smooth;
    cp.bmix = h->dsi_mix ? h->bmix : nullptr;
    cp.tile0[0] = 0;
    for (int c = 0; c < h->ncols; ++c) cp.tile0[c + 1] = cp.tile0[c] + (h->cols[c].n + kThreads - 1) / kThreads;
    return cp;
}

}  // namespace

void launch_colgen(const Handle* h, const double* eta, void* out, cudaStream_t st) {
    long long maxn = 0;
    for (int c = 0; c < h->ncols; ++c) maxn = maxn > h->cols[c].n ? maxn : h->cols[c].n;
    long long bx = (maxn + kThreads - 1) / kThreads;
    if (bx > 4096) bx = 4096;
    dim3 grid((unsigned)bx, (unsigned)h->ncols);
    ColParams cp = make_params(h);
    if (h->fp32) {
        if (h->cplx) k_colgen<float, true><<<grid, kThreads, 0, st>>>(out, cp, h->kind, h->d, h->gen, h->gen_cols, h->shift, eta);
        else k_colgen<float, false><<<grid, kThreads, 0, st>>>(out, cp, h->kind, h->d, h->gen, h->gen_cols, h->shift, eta);
    } else {
        if (h->cplx) k_colgen<double, true><<<grid, kThreads, 0, st>>>(out, cp, h->kind, h->d, h->gen, h->gen_cols, h->shift, eta);
        else k_colgen<double, false><<<grid, kThreads, 0, st>>>(out, cp, h->kind, h->d, h->gen, h->gen_cols, h->shift, eta);
    }
}

void launch_points(const Handle* h, uint32_t* x, cudaStream_t st) {
    long long off = 0;
    for (int tc = 0; tc < h->T; ++tc) {
        int t = h->rank[tc];
        long long n = h->n[t];
        long long work = n * h->d;
        int blocks = (int)((work + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_points<<<blocks, 256, 0, st>>>(x, h->kind, h->d, h->gen, h->gen_cols, h->shift, t, n, off);
        off += n;
    }
}

void launch_y_load(const Handle* h, const double* y, cudaStream_t st) {
    long long in_off = 0;
    for (int tc = 0; tc < h->T; ++tc) {
        int t = h->rank[tc];
        long long n = h->n[t];
        int blocks = (int)((n + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_y_load<<<blocks, 256, 0, st>>>(h->yhat, y, n, in_off, h->yoff[t], h->cplx ? 1 : 0);
        in_off += n;
    }
    // yhat_t = V_{m_t}^dagger y_t, FP64, one launch per distinct length
    for (int t = 0; t < h->T;) {
        int t2 = t;
        while (t2 < h->T && h->m[t2] == h->m[t]) ++t2;
        launch_transform(h, h->yhat, false, h->cplx, h->m[t], h->yoffs_dev + t, t2 - t, false, st);
        t = t2;
    }
    for (int t = 0; t < h->T; ++t) {
        long long n = h->n[t];
        long long len = h->cplx ? 2 * n : n;
        int blocks = (int)((len + 255) / 256);
        if (blocks > 4096) blocks = 4096;
        k_scale<<<blocks, 256, 0, st>>>(h->yhat + (h->cplx ? 2 : 1) * h->yoff[t], len, 1.0 / sqrt((double)n));
    }
}

int eta_grad_blocks(const Handle* h) {
    long long b = (h->col_elems + kThreads - 1) / kThreads;
    if (b > 1216) b = 1216;
    return (int)b;
}

// FP64 fits whose eta contraction runs in double-float: the SI kernels of smoothness 1..4 and the order-2
// DSI kernel (no mixture), d <= 16
static bool eta_grad_df_ok(const Handle* h) {
    return !h->fp32 && !h->dsi_mix && h->d <= 16;
}

void launch_eta_grad(const Handle* h, const double* eta, const void* omega, double* partials, int nblk,
                     cudaStream_t st) {
    ColParams cp = make_params(h);
#define MTGP_ETA_GRAD(S, C, M) \
    k_eta_grad<S, C, M><<<nblk, kThreads, 0, st>>>(omega, cp, h->ncols, h->kind, h->d, h->gen, h->gen_cols, \
                                                   h->shift, eta, partials)
    if (h->dsi_mix) {
        if (h->fp32) MTGP_ETA_GRAD(float, false, true);
        else MTGP_ETA_GRAD(double, false, true);
    } else if (h->fp32) {
        if (h->cplx) MTGP_ETA_GRAD(float, true, false);
        else MTGP_ETA_GRAD(float, false, false);
    } else if (eta_grad_df_ok(h)) {
#define MTGP_ETA_GRAD_DF(C, DM) \
    k_eta_grad_df<C, DM><<<nblk, kThreads, 0, st>>>(omega, cp, h->ncols, h->kind, h->d, h->gen, h->gen_cols, h->shift, \
                                                    eta, partials)
        if (h->d <= 8) {
            if (h->cplx) MTGP_ETA_GRAD_DF(true, 8);
            else MTGP_ETA_GRAD_DF(false, 8);
        } else {
            if (h->cplx) MTGP_ETA_GRAD_DF(true, 16);
            else MTGP_ETA_GRAD_DF(false, 16);
        }
#undef MTGP_ETA_GRAD_DF
    } else {
        if (h->cplx) MTGP_ETA_GRAD(double, true, false);
        else MTGP_ETA_GRAD(double, false, false);
    }
#undef MTGP_ETA_GRAD
}

static dim3 pair_grid(const Handle* h) {
    long long maxn = 0;
    for (int c = 0; c < h->ncols; ++c) maxn = maxn > h->cols[c].n ? maxn : h->cols[c].n;
    long long bx = (maxn + kThreads - 1) / kThreads;
    if (bx > 2048) bx = 2048;
    return dim3((unsigned)bx, (unsigned)h->npairs);
}

void launch_pair_split(const Handle* h, void* spec, cudaStream_t st) {
    if (h->npairs == 0) return;
    if (h->fp32) k_pair_split<float><<<pair_grid(h), kThreads, 0, st>>>(reinterpret_cast<cx<float>*>(spec), h->pairs_dev, h->npairs);
    else k_pair_split<double><<<pair_grid(h), kThreads, 0, st>>>(reinterpret_cast<cx<double>*>(spec), h->pairs_dev, h->npairs);
}

void launch_pair_pack(const Handle* h, void* wgt, cudaStream_t st) {
    if (h->npairs == 0) return;
    if (h->fp32) k_pair_pack<float><<<pair_grid(h), kThreads, 0, st>>>(reinterpret_cast<cx<float>*>(wgt), h->pairs_dev, h->npairs);
    else k_pair_pack<double><<<pair_grid(h), kThreads, 0, st>>>(reinterpret_cast<cx<double>*>(wgt), h->pairs_dev, h->npairs);
}

// Design points, first kernel columns, observation loading and the eta-gradient pass.
//
// First column of block (t, u) (sorted tasks, n_t >= n_u), Theorem "fast MTGP computations" item 3:
//   c_{tu}[i] = Q(x_{t,i}, x_{u,0}) = prod_j (1 + eta_j K(z_{i,j} (+) Delta_{t,j} (-) Delta_{u,j})),  i < n_t,
// in radical-inverse order, generated on the fly from the index i (Def. 2.1 / 2.2, Eq. 2.4-2.6).
// The task covariance R and the noise enter later, per frequency, so the columns depend on eta only.
#include "mtgp_internal.cuh"

namespace {

constexpr int kThreads = 256;

struct ColParams {
    ColDesc cols[MTGP_MAX_COLS];
    int alpha;           // SI smoothness
    const double* bmix;  // DSI mixture weights (4), or nullptr
};

template <typename S, bool CPLX>
__global__ void __launch_bounds__(kThreads)
k_colgen(void* out, ColParams cp, int kind, int d, const uint32_t* __restrict__ gen, int gen_cols,
         const uint32_t* __restrict__ shift, const double* __restrict__ eta) {
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ S s_b[4];
    __shared__ uint32_t s_dt[MTGP_MAX_DIM], s_du[MTGP_MAX_DIM];
    const ColDesc c = cp.cols[blockIdx.y];
    if (threadIdx.x < d) {
        s_eta[threadIdx.x] = (S)eta[threadIdx.x];
        s_dt[threadIdx.x] = shift[c.t * d + threadIdx.x];
        s_du[threadIdx.x] = shift[c.u * d + threadIdx.x];
    }
    if (cp.bmix && threadIdx.x < 4) s_b[threadIdx.x] = (S)cp.bmix[threadIdx.x];
    const S* bw = cp.bmix ? s_b : nullptr;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < c.n;
         i += (long long)gridDim.x * blockDim.x) {
        S q = (S)1;
        for (int j = 0; j < d; ++j) {
            uint32_t z = point_word(kind, (uint32_t)i, j, gen, gen_cols);
            uint32_t X = pair_word(kind, z, s_dt[j], s_du[j]);
            q *= (S)1 + s_eta[j] * kernel1d_b<S>(kind, X, cp.alpha, bw);
        }
        if (CPLX) {
            reinterpret_cast<cx<S>*>(out)[c.off + i] = mk(q, (S)0);
        } else {
            reinterpret_cast<S*>(out)[c.off + i] = q;
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
           double* __restrict__ partials, long long total) {
    constexpr int NB = MIX ? 4 : 0;
    __shared__ S s_eta[MTGP_MAX_DIM];
    __shared__ S s_b[4];
    __shared__ double s_red[kThreads / 32][MTGP_MAX_DIM + 4];
    if (threadIdx.x < d) s_eta[threadIdx.x] = (S)eta[threadIdx.x];
    if (MIX && threadIdx.x < 4) s_b[threadIdx.x] = (S)cp.bmix[threadIdx.x];
    __syncthreads();
    const S* bw = MIX ? s_b : nullptr;
    double acc[MTGP_MAX_DIM + NB];
    for (int j = 0; j < d + NB; ++j) acc[j] = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // locate the column
        int c = 0;
        while (c + 1 < ncols && e >= cp.cols[c + 1].off) ++c;
        const ColDesc cd = cp.cols[c];
        long long i = e - cd.off;
        S w;
        if (CPLX) w = reinterpret_cast<const cx<S>*>(omega)[e].re;
        else w = reinterpret_cast<const S*>(omega)[e];
        S kv[MTGP_MAX_DIM];
        S pre[MTGP_MAX_DIM];
        uint32_t xw[MIX ? MTGP_MAX_DIM : 1];
        S p = (S)1;
        for (int j = 0; j < d; ++j) {
            uint32_t z = point_word(kind, (uint32_t)i, j, gen, gen_cols);
            uint32_t X = pair_word(kind, z, shift[cd.t * d + j], shift[cd.u * d + j]);
            if (MIX) xw[j] = X;
            kv[j] = kernel1d_b<S>(kind, X, cp.alpha, bw);
            pre[j] = p;
            p *= (S)1 + s_eta[j] * kv[j];
        }
        S suf = (S)1;
        for (int j = d - 1; j >= 0; --j) {
            acc[j] += (double)(w * kv[j] * pre[j] * suf);
            if (MIX) {
                S ko[4];
                dsi_orders<S>(xw[j], ko);
                const S f = w * s_eta[j] * (pre[j] * suf);
                for (int a = 0; a < 4; ++a) acc[d + a] += (double)(f * ko[a]);
            }
            suf *= (S)1 + s_eta[j] * kv[j];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < d + NB; ++j) {
        double v = acc[j];
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

ColParams make_params(const Handle* h) {
    ColParams cp;
    for (int c = 0; c < h->ncols; ++c) cp.cols[c] = h->cols[c];
    cp.alpha = h->smooth;
    cp.bmix = h->dsi_mix ? h->bmix : nullptr;
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

void launch_eta_grad(const Handle* h, const double* eta, const void* omega, double* partials, int nblk,
                     cudaStream_t st) {
    ColParams cp = make_params(h);
#define MTGP_ETA_GRAD(S, C, M) \
    k_eta_grad<S, C, M><<<nblk, kThreads, 0, st>>>(omega, cp, h->ncols, h->kind, h->d, h->gen, h->gen_cols, \
                                                   h->shift, eta, partials, h->col_elems)
    if (h->dsi_mix) {
        if (h->fp32) MTGP_ETA_GRAD(float, false, true);
        else MTGP_ETA_GRAD(double, false, true);
    } else if (h->fp32) {
        if (h->cplx) MTGP_ETA_GRAD(float, true, false);
        else MTGP_ETA_GRAD(float, false, false);
    } else {
        if (h->cplx) MTGP_ETA_GRAD(double, true, false);
        else MTGP_ETA_GRAD(double, false, false);
    }
#undef MTGP_ETA_GRAD
}

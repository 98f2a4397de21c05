// Posterior mean and variance of f(t, x) (Eq. 3.2) with the optimal mean tau plugged in.
//
//   mean_t(x) = tau_t + sum_u R_{tu} sum_i Q(x, x_{u,i}) beta_u[i],   beta = K~^-1 r = V Lambda^-1 rhat,
//   var_t(x)  = R_tt Q(x, x) - kappa^H Lambda^-1 kappa,             kappa_u = R_{tu} V_{m_u}^dagger q_u(x),
// with q_u(x)[i] = Q(x, x_{u,i}).  alpha = Lambda^-1 rhat comes from the solve; beta_t = V_{m_t} alpha_t
// is the inverse transform (V = conj o DIF o conj / sqrt(n) for lattices, FWHT / sqrt(n) for nets).
#include <type_traits>

#include "mtgp_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 256;

__global__ void k_query_words(const double* __restrict__ xq, long long total, uint32_t* __restrict__ out,
                              int* status) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double x = xq[e];
        uint32_t w;
        if (!(x == x)) {
            set_status(status, ST_NUMERIC);
            w = 0;
        } else if (x >= 1.0) {
            w = 0xFFFFFFFFu;  // points equal to 1 map to the largest value below 1
        } else if (x <= 0.0) {
            w = 0u;
        } else {
            w = (uint32_t)floor(x * 4294967296.0);
        }
        out[e] = w;
    }
}

// sorted design points, N x d words
__global__ void k_design_words(uint32_t* __restrict__ out, int kind, int d, const uint32_t* __restrict__ gen,
                               int gen_cols, const uint32_t* __restrict__ shift, int t, long long n, long long off) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * d;
         e += (long long)gridDim.x * blockDim.x) {
        long long i = e / d;
        int j = (int)(e - i * d);
        uint32_t z = point_word(kind, (uint32_t)i, j, gen, gen_cols);
        uint32_t dt = shift[t * d + j];
        out[(off + i) * d + j] = (kind == MTGP_LATTICE) ? z + dt : z ^ dt;
    }
}

// beta buffer <- alpha (conjugated for lattices, so the DIF transform yields conj(V alpha) * sqrt(n))
__global__ void k_beta_prep(const double* __restrict__ alpha, double* __restrict__ beta, long long N, int cplx) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (cplx) {
            beta[2 * i] = alpha[2 * i];
            beta[2 * i + 1] = -alpha[2 * i + 1];
        } else {
            beta[i] = alpha[i];
        }
    }
}

// beta_real[i] = Re(beta_buf[i]) / sqrt(n_t)
__global__ void k_beta_finish(const double* __restrict__ beta, double* __restrict__ breal, long long n, long long off,
                              int cplx, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = cplx ? beta[2 * (off + i)] : beta[off + i];
        breal[off + i] = v * scale;
    }
}

struct PostParams {
    int kind, d, T, alpha;
    const double* bmix;  // DSI mixture weights (4), or nullptr
    long long n[MTGP_TMAX];
    long long yoff[MTGP_TMAX];
    int order[MTGP_TMAX];
    int rank[MTGP_TMAX];
};

template <typename S>
__device__ __forceinline__ S qkernel(int kind, const uint32_t* xa, const uint32_t* xb, const S* eta, int d, int alpha,
                                     const S* bmix) {
    S q = (S)1;
    for (int j = 0; j < d; ++j) {
        uint32_t X = (kind == MTGP_LATTICE) ? (xa[j] - xb[j]) : (xa[j] ^ xb[j]);
        q *= (S)1 + eta[j] * kernel1d_b<S>(kind, X, alpha, bmix);
    }
    return q;
}

// shared copy of the mixture weights (nullptr when the handle has none)
__device__ __forceinline__ const double* load_bmix(double* s_bm, const PostParams& p) {
    if (p.bmix && threadIdx.x < 4) s_bm[threadIdx.x] = p.bmix[threadIdx.x];
    return p.bmix ? s_bm : nullptr;
}

__device__ void load_R_post(double* sR, const PostParams& p, const ThetaPtrs& th) {
    for (int e = threadIdx.x; e < p.T * p.T; e += blockDim.x) {
        int t = e / p.T, u = e % p.T;
        int tc = p.order[t], uc = p.order[u];
        double r = 0.0;
        for (int k = 0; k < th.s; ++k) r += th.W[tc * th.s + k] * th.W[uc * th.s + k];
        if (t == u) r += th.v[tc];
        sR[e] = r;
    }
}

// Posterior mean, split over queries (blockIdx.x, one thread per query) and over slices of the design
// points (blockIdx.y): slice k is chunk c of sorted task u, with k = first[u] + c.  Design points
// and beta stream through shared-memory tiles; part[k][q] = R_{t_q u} sum_{i in slice} Q(x_q, x_ui) beta_u[i].
struct MeanSlices {
    long long chunk;             // points per slice (multiple of kTile)
    int first[MTGP_TMAX + 1];    // first slice of each sorted task; first[T] = number of slices
};

__global__ void __launch_bounds__(kThreads)
k_post_mean_part(const uint32_t* __restrict__ xqw, const int* __restrict__ task, int nq, const uint32_t* __restrict__ dw,
                 const double* __restrict__ beta, PostParams p, MeanSlices sl, ThetaPtrs th, double* __restrict__ part) {
    __shared__ double sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ double s_eta[MTGP_MAX_DIM];
    __shared__ uint32_t s_x[kTile * MTGP_MAX_DIM];
    __shared__ double s_b[kTile];
    __shared__ double s_bm[4];
    load_R_post(sR, p, th);
    if (threadIdx.x < p.d) s_eta[threadIdx.x] = th.eta[threadIdx.x];
    const double* bm = load_bmix(s_bm, p);
    const int k = blockIdx.y;
    int u = 0;
    while (u + 1 < p.T && sl.first[u + 1] <= k) ++u;
    const long long i_begin = (long long)(k - sl.first[u]) * sl.chunk;
    const long long i_end = (i_begin + sl.chunk) < p.n[u] ? (i_begin + sl.chunk) : p.n[u];
    const int d = p.d;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = q < nq;
    uint32_t xq[MTGP_MAX_DIM];
    int tq = 0;
    if (act) {
        for (int j = 0; j < d; ++j) xq[j] = xqw[(long long)q * d + j];
        tq = p.rank[task[q]];
    }
    __syncthreads();
    double acc = 0.0;
    for (long long i0 = i_begin; i0 < i_end; i0 += kTile) {
        const int cnt = (int)((i_end - i0) < kTile ? (i_end - i0) : kTile);
        __syncthreads();
        for (int e = threadIdx.x; e < cnt * d; e += blockDim.x) s_x[e] = dw[(p.yoff[u] + i0) * d + e];
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) s_b[e] = beta[p.yoff[u] + i0 + e];
        __syncthreads();
        if (act) {
            for (int i = 0; i < cnt; ++i) acc += qkernel<double>(p.kind, xq, s_x + i * d, s_eta, d, p.alpha, bm) * s_b[i];
        }
    }
    if (act) part[(long long)k * nq + q] = sR[tq * p.T + u] * acc;
}

// mean[q] = tau_{t_q} + sum_k part[k][q] (slices added in order)
__global__ void k_post_mean_sum(const double* __restrict__ part, int nslices, const int* __restrict__ task, int nq,
                                PostParams p, const double* __restrict__ tau_sorted, double* __restrict__ mean) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double m = 0.0;
    for (int k = 0; k < nslices; ++k) m += part[(long long)k * nq + q];
    mean[q] = tau_sorted[p.rank[task[q]]] + m;
}

// rows of the variance batch: qrow[(b * T + u) * n + i] = R_{t_b u} Q(x_b, x_{u,i})  (equal sizes)
template <bool CPLX>
__global__ void k_var_rows(const uint32_t* __restrict__ xqw, const int* __restrict__ task, int q0, int B,
                           const uint32_t* __restrict__ dw, PostParams p, ThetaPtrs th, double* __restrict__ rows) {
    __shared__ double sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ double s_eta[MTGP_MAX_DIM];
    __shared__ double s_bm[4];
    load_R_post(sR, p, th);
    if (threadIdx.x < p.d) s_eta[threadIdx.x] = th.eta[threadIdx.x];
    const double* bm = load_bmix(s_bm, p);
    __syncthreads();
    const long long n = p.n[0];
    const long long total = (long long)B * p.T * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long i = e % n;
        long long bu = e / n;
        int u = (int)(bu % p.T);
        int b = (int)(bu / p.T);
        int q = q0 + b;
        int tq = p.rank[task[q]];
        double v = sR[tq * p.T + u] * qkernel<double>(p.kind, xqw + (long long)q * p.d, dw + (p.yoff[u] + i) * p.d, s_eta, p.d, p.alpha, bm);
        if (CPLX) {
            rows[2 * e] = v;
            rows[2 * e + 1] = 0.0;
        } else {
            rows[e] = v;
        }
    }
}

template <bool CPLX>
using Vt = typename std::conditional<CPLX, cx<double>, double>::type;

__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ cx<double> vmul(cx<double> a, cx<double> b) { return a * b; }
__device__ __forceinline__ double vscale(double a, double s) { return a * s; }
__device__ __forceinline__ cx<double> vscale(cx<double> a, double s) { return mk(a.re * s, a.im * s); }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ cx<double> vsub(cx<double> a, cx<double> b) { return a - b; }

template <typename S, bool CPLX>
__device__ __forceinline__ Vt<CPLX> load_spec(const void* ptr, long long i) {
    if constexpr (CPLX) {
        cx<S> v = reinterpret_cast<const cx<S>*>(ptr)[i];
        return mk((double)v.re, (double)v.im);
    } else {
        return (double)reinterpret_cast<const S*>(ptr)[i];
    }
}

struct VarParams {
    int T, clamp;
    long long n;
    int colidx[MTGP_TMAX][MTGP_TMAX];
    long long coloff[MTGP_MAX_COLS];
};

// once per posterior call: Lambda(f) = L D L^H per frequency; stores 1/D_k (T x n doubles) then the
// strict lower L_ik (T(T-1)/2 x n, complex for lattices), each entry index-major so threads coalesce
template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kThreads)
k_var_factor(const void* spec, PostParams pp, VarParams p, ThetaPtrs th, double* __restrict__ fac) {
    using V = Vt<CPLX>;
    __shared__ double sR[T * T];
    __shared__ double s_sigv[T];
    load_R_post(sR, pp, th);
    if (threadIdx.x < T) s_sigv[threadIdx.x] = noise_of(th, pp.order, threadIdx.x);
    __syncthreads();
    const long long n = p.n;
    V* facL = reinterpret_cast<V*>(fac + (long long)T * n);
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n; f += (long long)gridDim.x * blockDim.x) {
        V mu[T][T];
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int u = t; u < T; ++u) mu[t][u] = load_spec<S, CPLX>(spec, p.coloff[p.colidx[t][u]] + f);
        double mu0 = creal(mu[0][0]);
        if (p.clamp && mu0 < 0.0) mu0 = 0.0;
        V lam[T][T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
            lam[i][i] = cfromreal<V>(sR[i * T + i] * mu0 + s_sigv[i]);
#pragma unroll
            for (int j = 0; j < i; ++j) lam[i][j] = vscale(cconj(mu[j][i]), sR[j * T + i]);
        }
        double D[T];
        V L[T][T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            double dk = creal(lam[k][k]);
#pragma unroll
            for (int j = 0; j < k; ++j) dk -= cabs2(L[k][j]) * D[j];
            D[k] = dk;
            fac[(long long)k * n + f] = 1.0 / dk;
#pragma unroll
            for (int i = k + 1; i < T; ++i) {
                V a = lam[i][k];
#pragma unroll
                for (int j = 0; j < k; ++j) a = vsub(a, vscale(vmul(L[i][j], cconj(L[k][j])), D[j]));
                L[i][k] = vscale(a, 1.0 / dk);
                facL[(long long)(i * (i - 1) / 2 + k) * n + f] = L[i][k];
            }
        }
    }
}

// one CTA per query: sum_f kappa(f)^H Lambda(f)^-1 kappa(f) with kappa(f) = transformed rows / sqrt(n),
// through the stored factors: w = L^-1 kappa, sum_k |w_k|^2 / D_k
template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kThreads)
k_var_quad(const double* __restrict__ rows, const double* __restrict__ fac, const int* __restrict__ task, int q0,
           const uint32_t* __restrict__ xqw, PostParams pp, VarParams p, ThetaPtrs th, double* __restrict__ var) {
    using V = Vt<CPLX>;
    __shared__ double sR[T * T];
    __shared__ double s_eta[MTGP_MAX_DIM];
    __shared__ double s_red[kThreads / 32];
    __shared__ double s_bm[4];
    load_R_post(sR, pp, th);
    if (threadIdx.x < pp.d) s_eta[threadIdx.x] = th.eta[threadIdx.x];
    const double* bm = load_bmix(s_bm, pp);
    __syncthreads();
    const int b = blockIdx.x;
    const long long n = p.n;
    const double inv_n = 1.0 / (double)n;
    const V* facL = reinterpret_cast<const V*>(fac + (long long)T * n);
    double acc = 0.0;
    for (long long f = threadIdx.x; f < n; f += blockDim.x) {
        V w[T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            long long e = ((long long)b * T + k) * n + f;
            V r;
            if constexpr (CPLX) r = mk(rows[2 * e], rows[2 * e + 1]);
            else r = rows[e];
#pragma unroll
            for (int j = 0; j < k; ++j) r = vsub(r, vmul(facL[(long long)(k * (k - 1) / 2 + j) * n + f], w[j]));
            w[k] = r;
            acc += cabs2(r) * fac[(long long)k * n + f];
        }
    }
    acc *= inv_n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w2 = 0; w2 < kThreads / 32; ++w2) s += s_red[w2];
        int q = q0 + b;
        int tq = pp.rank[task[q]];
        const uint32_t* x = xqw + (long long)q * pp.d;
        double prior = sR[tq * T + tq] * qkernel<double>(pp.kind, x, x, s_eta, pp.d, pp.alpha, bm);
        var[q] = prior - s;
    }
}

template <int T, bool CPLX, typename S>
void run_var(bool factor, int B, const double* rows, const void* spec, double* fac, const int* task, int q0,
             const uint32_t* xqw, PostParams pp, VarParams vp, ThetaPtrs th, double* var, cudaStream_t st) {
    if (factor) {
        long long blocks = (vp.n + kThreads - 1) / kThreads;
        k_var_factor<T, CPLX, S><<<(int)(blocks < 4096 ? blocks : 4096), kThreads, 0, st>>>(spec, pp, vp, th, fac);
    } else {
        k_var_quad<T, CPLX, S><<<B, kThreads, 0, st>>>(rows, fac, task, q0, xqw, pp, vp, th, var);
    }
}

// rows of the variance batch, unequal sizes: rows[b * N + yoff[u] + i] = R_{t_b u} Q(x_b, x_{u,i}) / sqrt(n_u)
// (the 1 / sqrt(n_u) of V^dagger folded in), tasks in the sorted observation layout
template <bool CPLX>
__global__ void k_var_rows_all(const uint32_t* __restrict__ xqw, const int* __restrict__ task, int q0, int B,
                               const uint32_t* __restrict__ dw, PostParams p, ThetaPtrs th, long long N,
                               double* __restrict__ rows) {
    __shared__ double sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ double s_eta[MTGP_MAX_DIM];
    __shared__ double s_bm[4];
    load_R_post(sR, p, th);
    if (threadIdx.x < p.d) s_eta[threadIdx.x] = th.eta[threadIdx.x];
    const double* bm = load_bmix(s_bm, p);
    __syncthreads();
    if (threadIdx.x < p.T * p.T) sR[threadIdx.x] *= 1.0 / sqrt((double)p.n[threadIdx.x % p.T]);
    __syncthreads();
    const long long total = (long long)B * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long idx = e % N;
        const int b = (int)(e / N);
        int u = 0;
        while (u + 1 < p.T && idx >= p.yoff[u + 1]) ++u;
        const int q = q0 + b;
        const int tq = p.rank[task[q]];
        const double v = sR[tq * p.T + u] * qkernel<double>(p.kind, xqw + (long long)q * p.d, dw + idx * p.d, s_eta,
                                                             p.d, p.alpha, bm);
        if (CPLX) {
            rows[2 * e] = v;
            rows[2 * e + 1] = 0.0;
        } else {
            rows[e] = v;
        }
    }
}

// var[q0 + b] = R_{tt} Q(x_b, x_b) - sum of the per-class-block quadratic forms (in block order)
__global__ void k_var_tree_sum(const double* __restrict__ part, int nblk, int B, int q0, const int* __restrict__ task,
                               const uint32_t* __restrict__ xqw, PostParams p, ThetaPtrs th, double* __restrict__ var) {
    __shared__ double sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ double s_eta[MTGP_MAX_DIM];
    __shared__ double s_bm[4];
    load_R_post(sR, p, th);
    if (threadIdx.x < p.d) s_eta[threadIdx.x] = th.eta[threadIdx.x];
    const double* bm = load_bmix(s_bm, p);
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[(long long)b * nblk + k];
    const int q = q0 + b;
    const int tq = p.rank[task[q]];
    const uint32_t* x = xqw + (long long)q * p.d;
    var[q] = sR[tq * p.T + tq] * qkernel<double>(p.kind, x, x, s_eta, p.d, p.alpha, bm) - s;
}

// factor = true: per-frequency factors into fac; false: the quadratic forms of B queries
template <bool CPLX, typename S>
void dispatch_var(bool factor, int T, int B, const double* rows, const void* spec, double* fac, const int* task,
                  int q0, const uint32_t* xqw, PostParams pp, VarParams vp, ThetaPtrs th, double* var,
                  cudaStream_t st) {
    switch (T) {
        case 1: run_var<1, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 2: run_var<2, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 3: run_var<3, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 4: run_var<4, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 5: run_var<5, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 6: run_var<6, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        case 7: run_var<7, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
        default: run_var<8, CPLX, S>(factor, B, rows, spec, fac, task, q0, xqw, pp, vp, th, var, st); break;
    }
}

int grid_for(long long work) {
    long long b = (work + 255) / 256;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

// Scratch needed by posterior_run beyond the handle's fixed workspace is carved from `h->S`-sized
// buffers allocated on first use (see mtgp_api.cu: post_* fields are not part of Handle to keep
// the header small; they live in a static map keyed by handle).
#include <map>
#include <mutex>

namespace {
struct PostScratch {
    uint32_t* design = nullptr;  // N x d words (sorted)
    double* beta_c = nullptr;    // N (complex for lattice)
    double* beta = nullptr;      // N real
    uint32_t* xq = nullptr;      // nq x d words
    long long xq_cap = 0;
    double* rows = nullptr;      // variance batch rows
    long long rows_cap = 0;
    long long* offs = nullptr;   // row offsets of the variance batch (multiples of n)
    int offs_cap = 0;
    int offs_kind = -1;          // 0: equal sizes (i n), 1: unequal sizes (b N + yoff[u], u-major)
    int offs_B = 0;
    double* fac = nullptr;       // per-frequency L D L^H factors of Lambda (variance)
    long long fac_cap = 0;
    double* part = nullptr;      // mean partial sums, slices x nq
    long long part_cap = 0;
    double* vpart = nullptr;     // variance, unequal sizes: per (query, class block) sums
    long long vpart_cap = 0;
};
std::map<const Handle*, PostScratch> g_post;
std::mutex g_post_mu;
}  // namespace

void posterior_release(const Handle* h) {
    posterior_df_release(h);
    std::lock_guard<std::mutex> lk(g_post_mu);
    auto it = g_post.find(h);
    if (it == g_post.end()) return;
    cudaFree(it->second.design);
    cudaFree(it->second.beta_c);
    cudaFree(it->second.beta);
    cudaFree(it->second.xq);
    cudaFree(it->second.rows);
    cudaFree(it->second.offs);
    cudaFree(it->second.fac);
    cudaFree(it->second.part);
    cudaFree(it->second.vpart);
    g_post.erase(it);
}

int posterior_run(Handle* h, ThetaPtrs th, int nq, const double* xq, const int* task, double* mean, double* var,
                  cudaStream_t st) {
    PostScratch* ps;
    {
        std::lock_guard<std::mutex> lk(g_post_mu);
        ps = &g_post[h];
    }
    const int d = h->d;
    const long long N = h->N;
    const int es = h->cplx ? 2 : 1;
    if (!ps->design) {
        if (cudaMalloc(&ps->design, (size_t)N * d * sizeof(uint32_t)) != cudaSuccess) return MTGP_ERR_CUDA;
        if (cudaMalloc(&ps->beta_c, (size_t)N * es * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
        if (cudaMalloc(&ps->beta, (size_t)N * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
        for (int t = 0; t < h->T; ++t)
            k_design_words<<<grid_for(h->n[t] * d), 256, 0, st>>>(ps->design, h->kind, d, h->gen, h->gen_cols, h->shift, t,
                                                                h->n[t], h->yoff[t]);
    }
    if ((long long)nq * d > ps->xq_cap) {
        cudaFree(ps->xq);
        ps->xq_cap = (long long)nq * d;
        if (cudaMalloc(&ps->xq, (size_t)ps->xq_cap * sizeof(uint32_t)) != cudaSuccess) return MTGP_ERR_CUDA;
    }
    k_query_words<<<grid_for((long long)nq * d), 256, 0, st>>>(xq, (long long)nq * d, ps->xq, h->status);
    // beta = V alpha
    k_beta_prep<<<grid_for(N), 256, 0, st>>>(h->alpha, ps->beta_c, N, h->cplx ? 1 : 0);
    for (int t = 0; t < h->T;) {
        int t2 = t;
        while (t2 < h->T && h->m[t2] == h->m[t]) ++t2;
        launch_transform(h, ps->beta_c, false, h->cplx, h->m[t], h->yoffs_dev + t, t2 - t, true, st);
        t = t2;
    }
    for (int t = 0; t < h->T; ++t)
        k_beta_finish<<<grid_for(h->n[t]), 256, 0, st>>>(ps->beta_c, ps->beta, h->n[t], h->yoff[t], h->cplx ? 1 : 0,
                                                       1.0 / sqrt((double)h->n[t]));
    if (posterior_df_ok(h)) return posterior_df_run(h, th, nq, ps->xq, task, ps->design, ps->beta, mean, var, st);
    PostParams pp;
    pp.kind = h->kind;
    pp.alpha = h->smooth;
    pp.bmix = h->dsi_mix ? h->bmix : nullptr;
    pp.d = d;
    pp.T = h->T;
    for (int t = 0; t < MTGP_TMAX; ++t) {
        pp.n[t] = t < h->T ? h->n[t] : 0;
        pp.yoff[t] = t < h->T ? h->yoff[t] : 0;
        pp.order[t] = t < h->T ? h->order[t] : 0;
        pp.rank[t] = t < h->T ? h->rank[t] : 0;
    }
    // tau (sorted) lives in h->tau (filled by the solver for unequal sizes, by mtgp_set_y for equal)
    // slices of the design points so that query blocks x slices fill the GPU several times over,
    // with the partial sums capped at 32 M doubles
    {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const long long qblocks = (nq + kThreads - 1) / kThreads;
        long long want = (16LL * nsm + qblocks - 1) / qblocks;
        const long long cap = (32LL << 20) / nq;
        if (want > cap) want = cap;
        if (want < 1) want = 1;
        long long chunk = (N + want - 1) / want;
        chunk = (chunk + kTile - 1) / kTile * kTile;
        MeanSlices sl;
        sl.chunk = chunk;
        int ns = 0;
        for (int t = 0; t < MTGP_TMAX + 1; ++t) {
            sl.first[t] = ns;
            if (t < h->T) ns += (int)((h->n[t] + chunk - 1) / chunk);
        }
        if ((long long)ns * nq > ps->part_cap) {
            cudaFree(ps->part);
            ps->part_cap = (long long)ns * nq;
            if (cudaMalloc(&ps->part, (size_t)ps->part_cap * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
        }
        mtgp_prof_begin(h, "post_mean", st);
        dim3 grid((unsigned)qblocks, (unsigned)ns);
        k_post_mean_part<<<grid, kThreads, 0, st>>>(ps->xq, task, nq, ps->design, ps->beta, pp, sl, th, ps->part);
        k_post_mean_sum<<<(unsigned)qblocks, kThreads, 0, st>>>(ps->part, ns, task, nq, pp, h->tau, mean);
        mtgp_prof_end(h, st);
    }
    if (!var) return MTGP_OK;
    if (!h->equal) {
        // unequal sizes: rows of a batch of queries, their transforms per task, then the quadratic
        // forms through the tree solver's factor class by class
        const long long per_q = N * es;
        int B = (int)((64LL << 20) / per_q);
        if (B < 1) B = 1;
        if (B > 1024) B = 1024;
        if (B > nq) B = nq;
        if ((long long)B * per_q > ps->rows_cap) {
            cudaFree(ps->rows);
            ps->rows_cap = (long long)B * per_q;
            if (cudaMalloc(&ps->rows, (size_t)ps->rows_cap * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
        }
        const int T = h->T;
        if (B * T > ps->offs_cap || ps->offs_kind != 1 || ps->offs_B != B) {
            // offsets of query b's task-u row: b N + yoff[u], grouped by task (u-major)
            cudaFree(ps->offs);
            ps->offs_cap = B * T;
            if (cudaMalloc(&ps->offs, (size_t)ps->offs_cap * sizeof(long long)) != cudaSuccess) return MTGP_ERR_CUDA;
            long long* tmp = new long long[ps->offs_cap];
            for (int u = 0; u < T; ++u)
                for (int b = 0; b < B; ++b) tmp[u * B + b] = (long long)b * N + h->yoff[u];
            cudaMemcpyAsync(ps->offs, tmp, (size_t)ps->offs_cap * sizeof(long long), cudaMemcpyHostToDevice, st);
            cudaStreamSynchronize(st);
            delete[] tmp;
            ps->offs_kind = 1;
            ps->offs_B = B;
        }
        const int nblk = solve_tree_blocks(h);
        if ((long long)B * nblk > ps->vpart_cap) {
            cudaFree(ps->vpart);
            ps->vpart_cap = (long long)B * nblk;
            if (cudaMalloc(&ps->vpart, (size_t)ps->vpart_cap * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
        }
        for (int q0 = 0; q0 < nq; q0 += B) {
            const int Bb = (nq - q0) < B ? (nq - q0) : B;
            mtgp_prof_begin(h, "var_rows", st);
            if (h->cplx) k_var_rows_all<true><<<grid_for((long long)Bb * N), 256, 0, st>>>(ps->xq, task, q0, Bb, ps->design, pp, th, N, ps->rows);
            else k_var_rows_all<false><<<grid_for((long long)Bb * N), 256, 0, st>>>(ps->xq, task, q0, Bb, ps->design, pp, th, N, ps->rows);
            mtgp_prof_end(h, st);
            mtgp_prof_begin(h, "var_xform", st);
            for (int u = 0; u < T; ++u)
                launch_transform(h, ps->rows, false, h->cplx, h->m[u], ps->offs + (long long)u * B, Bb, false, st);
            mtgp_prof_end(h, st);
            mtgp_prof_begin(h, "var_quad", st);
            launch_var_tree(h, ps->rows, Bb, ps->vpart, st);
            k_var_tree_sum<<<(Bb + 127) / 128, 128, 0, st>>>(ps->vpart, nblk, Bb, q0, task, ps->xq, pp, th, var);
            mtgp_prof_end(h, st);
        }
        return MTGP_OK;
    }
    const long long n = h->n[0];
    // batch so the rows stay within ~512 MB
    long long per_q = (long long)h->T * n * es;
    int B = (int)((64LL << 20) / per_q);
    if (B < 1) B = 1;
    if (B > 1024) B = 1024;
    if (B > nq) B = nq;
    if ((long long)B * per_q > ps->rows_cap) {
        cudaFree(ps->rows);
        ps->rows_cap = (long long)B * per_q;
        if (cudaMalloc(&ps->rows, (size_t)ps->rows_cap * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
    }
    // offsets of the B*T rows for the batched transform
    if (B * h->T > ps->offs_cap || ps->offs_kind != 0) {
        cudaFree(ps->offs);
        ps->offs_kind = 0;
        ps->offs_cap = B * h->T;
        if (cudaMalloc(&ps->offs, (size_t)ps->offs_cap * sizeof(long long)) != cudaSuccess) return MTGP_ERR_CUDA;
        long long* tmp = new long long[ps->offs_cap];
        for (int i = 0; i < ps->offs_cap; ++i) tmp[i] = (long long)i * n;
        cudaMemcpyAsync(ps->offs, tmp, (size_t)ps->offs_cap * sizeof(long long), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
        delete[] tmp;
    }
    long long* offs_dev = ps->offs;
    VarParams vp;
    vp.T = h->T;
    vp.clamp = h->fp32 ? 1 : 0;
    vp.n = n;
    for (int t = 0; t < MTGP_TMAX; ++t)
        for (int u = 0; u < MTGP_TMAX; ++u) vp.colidx[t][u] = (t < h->T && u < h->T && t <= u) ? h->col_of[t][u] : 0;
    for (int c = 0; c < MTGP_MAX_COLS; ++c) vp.coloff[c] = c < h->ncols ? h->cols[c].off : 0;
    const long long fac_need = (long long)h->T * n + (long long)h->T * (h->T - 1) / 2 * n * es;
    if (fac_need > ps->fac_cap) {
        cudaFree(ps->fac);
        ps->fac_cap = fac_need;
        if (cudaMalloc(&ps->fac, (size_t)fac_need * sizeof(double)) != cudaSuccess) return MTGP_ERR_CUDA;
    }
    auto var_step = [&](bool factor, int Bb, int q0) {
        if (h->fp32) {
            if (h->cplx) dispatch_var<true, float>(factor, h->T, Bb, ps->rows, h->spec, ps->fac, task, q0, ps->xq, pp, vp, th, var, st);
            else dispatch_var<false, float>(factor, h->T, Bb, ps->rows, h->spec, ps->fac, task, q0, ps->xq, pp, vp, th, var, st);
        } else {
            if (h->cplx) dispatch_var<true, double>(factor, h->T, Bb, ps->rows, h->spec, ps->fac, task, q0, ps->xq, pp, vp, th, var, st);
            else dispatch_var<false, double>(factor, h->T, Bb, ps->rows, h->spec, ps->fac, task, q0, ps->xq, pp, vp, th, var, st);
        }
    };
    mtgp_prof_begin(h, "var_factor", st);
    var_step(true, 0, 0);
    mtgp_prof_end(h, st);
    for (int q0 = 0; q0 < nq; q0 += B) {
        int Bb = (nq - q0) < B ? (nq - q0) : B;
        long long work = (long long)Bb * h->T * n;
        mtgp_prof_begin(h, "var_rows", st);
        if (h->cplx) k_var_rows<true><<<grid_for(work), 256, 0, st>>>(ps->xq, task, q0, Bb, ps->design, pp, th, ps->rows);
        else k_var_rows<false><<<grid_for(work), 256, 0, st>>>(ps->xq, task, q0, Bb, ps->design, pp, th, ps->rows);
        mtgp_prof_end(h, st);
        mtgp_prof_begin(h, "var_xform", st);
        launch_transform(h, ps->rows, false, h->cplx, h->m[0], offs_dev, Bb * h->T, false, st);
        mtgp_prof_end(h, st);
        mtgp_prof_begin(h, "var_quad", st);
        var_step(false, Bb, q0);
        mtgp_prof_end(h, st);
    }
    return MTGP_OK;
}

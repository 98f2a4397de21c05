// C ABI entry points: argument validation, workspace layout and the launch sequence of each call.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mtgp_internal.cuh"

void posterior_release(const Handle* h);

struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
struct Prof {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    ProfRec cur{};
};

static cudaEvent_t prof_event(Prof* p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void mtgp_prof_begin(const Handle* h, const char* name, cudaStream_t st) {
    Prof* p = h->prof;
    if (!p || !p->on) return;
    p->cur.name = name;
    p->cur.a = prof_event(p);
    p->cur.b = prof_event(p);
    cudaEventRecord(p->cur.a, st);
}

void mtgp_prof_end(const Handle* h, cudaStream_t st) {
    Prof* p = h->prof;
    if (!p || !p->on) return;
    cudaEventRecord(p->cur.b, st);
    p->recs.push_back(p->cur);
}

namespace {

thread_local std::string g_err;

int fail(int code, const char* msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return MTGP_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

__global__ void k_tau_equal(const double* yhat, double* tau, int T, long long n, int cplx) {
    int t = threadIdx.x;
    if (t < T) tau[t] = yhat[(cplx ? 2 : 1) * (long long)t * n] / sqrt((double)n);
}

__global__ void k_check_theta(ThetaPtrs th, int d, int T, int* status) {
    int bad = 0;
    for (int j = threadIdx.x; j < d; j += blockDim.x)
        if (!isfinite(th.eta[j]) || th.eta[j] < 0.0) bad = 1;
    for (int e = threadIdx.x; e < T * th.s; e += blockDim.x)
        if (!isfinite(th.W[e])) bad = 1;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        if (!isfinite(th.v[t]) || th.v[t] < 0.0) bad = 1;
    for (int t = threadIdx.x; t < (th.nsig > 1 ? th.nsig : 1); t += blockDim.x)
        if (!isfinite(th.sigma2[t]) || th.sigma2[t] < 0.0) bad = 1;
    if (th.bmix && threadIdx.x < 4)
        if (!isfinite(th.bmix[threadIdx.x]) || th.bmix[threadIdx.x] < 0.0) bad = 1;
    if (bad) atomicOr(status, ST_NUMERIC);
}

__global__ void k_check_y(const double* y, long long N, int* status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(y[i])) {
            atomicOr(status, ST_NUMERIC);
            return;
        }
}

// Multitask Bayesian cubature (Sec. 3.5, multitask cubature theorem, gamma = 1 for the product kernels
// of Eq. 2.4): mu = tau + R E K~^-1 (y - E^T tau) with (E K~^-1 r)_t = sqrt(n_t) alpha_t(0), and
// Sigma = R - R Pi R, Pi = E K~^-1 E^T = n Lambda(0)^-1 (equal sizes) or from the tree solver.
struct CubParams {
    int T, s, equal, cplx, fp32, clamp;
    long long n[MTGP_TMAX], yoff[MTGP_TMAX];
    int order[MTGP_TMAX], rank[MTGP_TMAX];
    int colidx[MTGP_TMAX][MTGP_TMAX];
    long long coloff[MTGP_MAX_COLS];
};

__global__ void k_cubature(CubParams p, ThetaPtrs th, const void* spec, const double* alpha, const double* tau_sorted,
                           const double* pi_sorted, double* mu, double* Sigma, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int T = p.T;
    double R[MTGP_TMAX][MTGP_TMAX], Pi[MTGP_TMAX][MTGP_TMAX];  // caller order
    for (int t = 0; t < T; ++t)
        for (int u = 0; u < T; ++u) {
            double r = 0.0;
            for (int k = 0; k < th.s; ++k) r += th.W[t * th.s + k] * th.W[u * th.s + k];
            R[t][u] = r + (t == u ? th.v[t] : 0.0);
        }
    if (p.equal) {
        // Lambda(0) in sorted order from the transformed first columns at frequency 0
        double L[MTGP_TMAX][MTGP_TMAX];
        for (int t = 0; t < T; ++t)
            for (int u = t; u < T; ++u) {
                const double sig = noise_of(th, p.order, t);
                const long long e = p.coloff[p.colidx[t][u]];
                double mu0;
                if (p.fp32) mu0 = p.cplx ? (double)((const float*)spec)[2 * e] : (double)((const float*)spec)[e];
                else mu0 = p.cplx ? ((const double*)spec)[2 * e] : ((const double*)spec)[e];
                if (t == u && p.clamp && mu0 < 0.0) mu0 = 0.0;
                const double v = R[p.order[t]][p.order[u]] * mu0 + (t == u ? sig : 0.0);
                L[t][u] = L[u][t] = v;
            }
        // Pi = n Lambda(0)^-1 by Cholesky
        for (int k = 0; k < T; ++k) {
            double dk = L[k][k];
            for (int j = 0; j < k; ++j) dk -= L[k][j] * L[k][j];
            if (!(dk > 0.0)) {
                set_status(status, ST_NOT_PD);
                dk = 1.0;
            }
            dk = sqrt(dk);
            L[k][k] = dk;
            for (int i = k + 1; i < T; ++i) {
                double a = L[i][k];
                for (int j = 0; j < k; ++j) a -= L[i][j] * L[k][j];
                L[i][k] = a / dk;
            }
        }
        for (int c = 0; c < T; ++c) {
            double x[MTGP_TMAX];
            for (int k = 0; k < T; ++k) {
                double a = (k == c) ? 1.0 : 0.0;
                for (int j = 0; j < k; ++j) a -= L[k][j] * x[j];
                x[k] = a / L[k][k];
            }
            for (int k = T - 1; k >= 0; --k) {
                double a = x[k];
                for (int i = k + 1; i < T; ++i) a -= L[i][k] * x[i];
                x[k] = a / L[k][k];
            }
            for (int k = 0; k < T; ++k) Pi[p.order[k]][p.order[c]] = (double)p.n[0] * x[k];
        }
    } else {
        for (int t = 0; t < T; ++t)
            for (int u = 0; u < T; ++u) Pi[p.order[t]][p.order[u]] = pi_sorted[t * T + u];
    }
    for (int t = 0; t < T; ++t) {
        double m = tau_sorted[p.rank[t]];
        for (int u = 0; u < T; ++u) {
            const int su = p.rank[u];
            const double a0 = p.cplx ? alpha[2 * p.yoff[su]] : alpha[p.yoff[su]];
            m += R[t][u] * sqrt((double)p.n[su]) * a0;
        }
        mu[t] = m;
        for (int u = 0; u < T; ++u) {
            double rpr = 0.0;
            for (int a = 0; a < T; ++a)
                for (int b = 0; b < T; ++b) rpr += R[t][a] * Pi[a][b] * R[b][u];
            Sigma[t * T + u] = R[t][u] - rpr;
        }
    }
}

template <typename T>
cudaError_t dalloc(Handle* h, T** p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc((void**)p, bytes);
    if (e == cudaSuccess) h->ws_bytes += (long long)bytes;
    return e;
}

void free_all(Handle* h) {
    void* ptrs[] = {h->gen, h->shift, h->cols_dev, h->yoffs_dev, h->twid, h->twid32, h->yhat, h->yhat_df, h->rt_words,
                    h->spec,
                    h->wgt, h->S, h->Z, h->r, h->alpha, h->tau, h->partials, h->status, h->out_tmp, h->counters,
                    h->gcv_h, h->pi_buf, h->bmix, h->hio, h->lead_offs_dev, h->pairs_dev};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->hio_exec) cudaGraphExecDestroy(h->hio_exec);
    h->hio_exec = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    if (h->prof) {
        for (auto& r : h->prof->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (auto e : h->prof->pool) cudaEventDestroy(e);
        delete h->prof;
        h->prof = nullptr;
    }
}

int validate_theta(const Handle* h, const double* eta, const double* W, int s, const double* v, const double* sigma2) {
    if (!eta || !W || !v || !sigma2) return fail(MTGP_ERR_INVALID_ARG, "theta pointer is NULL");
    if (s < 1 || s > h->T) return fail(MTGP_ERR_INVALID_ARG, "s must satisfy 1 <= s <= T");
    return MTGP_OK;
}

// First-column spectra of the general path: columns, forward transforms (paired columns of a
// lattice share one complex transform), split of the pairs.
static void forward_columns(Handle* h, const double* eta, cudaStream_t st) {
    mtgp_prof_begin(h, "colgen", st);
    launch_colgen(h, eta, h->spec, st);
    mtgp_prof_end(h, st);
    mtgp_prof_begin(h, "xform_dit", st);
    for (int g = 0; g < h->ngroups; ++g)
        launch_transform(h, h->spec, h->fp32, h->cplx, h->group_m[g], h->lead_offs_dev + h->group_lfirst[g],
                         h->group_lcount[g], false, st);
    launch_pair_split(h, h->spec, st);
    mtgp_prof_end(h, st);
}

// Adjoint transforms of the gradient weights (paired columns packed as w_a + i w_b first).
static void adjoint_columns(Handle* h, cudaStream_t st) {
    mtgp_prof_begin(h, "xform_dif", st);
    launch_pair_pack(h, h->wgt, st);
    for (int g = 0; g < h->ngroups; ++g)
        launch_transform(h, h->wgt, h->fp32, h->cplx, h->group_m[g], h->lead_offs_dev + h->group_lfirst[g],
                         h->group_lcount[g], true, st);
    mtgp_prof_end(h, st);
}

// NLL (and gradient) at theta; leaves alpha = Lambda^-1 rhat in h->alpha and tau in h->tau.
int run_nll(Handle* h, ThetaPtrs th, bool grad, double* out, double* tau, double* g_eta, double* g_W, double* g_v,
            double* g_s2, cudaStream_t st, bool store_alpha = false) {
    if (h->equal && fused_supported(h)) {
        // kernel A's block 0 checks the parameters
        launch_fused(h, th, grad, store_alpha, out, tau, g_eta, g_W, g_v, g_s2, st);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        return MTGP_OK;
    }
    k_check_theta<<<1, 64, 0, st>>>(th, h->d, h->T, h->status);
    forward_columns(h, th.eta, st);
    int nsolve;
    if (h->equal) {
        mtgp_prof_begin(h, "solve_equal", st);
        launch_solve_equal(h, th, grad, h->partials, st);
        mtgp_prof_end(h, st);
        nsolve = solve_equal_blocks(h);
    } else {
        mtgp_prof_begin(h, "solve_tree", st);
        launch_solve_tree(h, th, grad, h->partials, st);
        mtgp_prof_end(h, st);
        nsolve = solve_tree_blocks(h);
    }
    const int NQ = solve_nq(h);
    double* eta_part = h->partials + (long long)nsolve * NQ;
    int neta = 0;
    if (grad) {
        adjoint_columns(h, st);
        neta = eta_grad_blocks(h);
        mtgp_prof_begin(h, "eta_grad", st);
        launch_eta_grad(h, th.eta, h->wgt, eta_part, neta, st);
        mtgp_prof_end(h, st);
    }
    mtgp_prof_begin(h, "finalize", st);
    launch_finalize(h, th, grad, h->partials, nsolve, eta_part, neta, out, tau, g_eta, g_W, g_v, g_s2, st);
    mtgp_prof_end(h, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    return MTGP_OK;
}

}  // namespace

void mtgp_set_error(const char* msg) { g_err = msg; }

extern "C" {

const char* mtgp_last_error_string(void) { return g_err.c_str(); }

long long mtgp_workspace_bytes(const mtgp_t* hh) { return hh ? hh->h.ws_bytes : 0; }

int mtgp_create(mtgp_t** out, int kind, int d, int T, const int* m, const uint32_t* gen, int gen_cols,
                const uint32_t* shift, int precision) {
    if (!out) return fail(MTGP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (kind != MTGP_LATTICE && kind != MTGP_DNET) return fail(MTGP_ERR_INVALID_ARG, "kind must be MTGP_LATTICE or MTGP_DNET");
    if (d < 1 || d > MTGP_MAX_DIM) return fail(MTGP_ERR_INVALID_ARG, "d out of range [1, MTGP_MAX_DIM]");
    if (T < 1 || T > MTGP_MAX_TASKS) return fail(MTGP_ERR_INVALID_ARG, "T out of range [1, MTGP_MAX_TASKS]");
    if (!m || !gen || !shift) return fail(MTGP_ERR_INVALID_ARG, "m, gen and shift must be host arrays");
    const bool noise_pt = (precision & MTGP_NOISE_PER_TASK) != 0;
    const bool solve_fp64 = (precision & MTGP_SOLVE_FP64) != 0;
    precision &= ~(MTGP_NOISE_PER_TASK | MTGP_SOLVE_FP64);
    if (precision != MTGP_FP64 && precision != MTGP_FP32_TRANSFORM)
        return fail(MTGP_ERR_INVALID_ARG,
                    "precision must be MTGP_FP64 or MTGP_FP32_TRANSFORM (optionally | MTGP_NOISE_PER_TASK | MTGP_SOLVE_FP64)");
    int mmax = 0;
    for (int t = 0; t < T; ++t) {
        if (m[t] < 0 || m[t] > MTGP_MAX_M) return fail(MTGP_ERR_INVALID_ARG, "m[t] out of range [0, MTGP_MAX_M]");
        mmax = m[t] > mmax ? m[t] : mmax;
    }
    if (kind == MTGP_DNET && (gen_cols < mmax || gen_cols > 32))
        return fail(MTGP_ERR_INVALID_ARG, "gen_cols must satisfy max m <= gen_cols <= 32");
    mtgp_s* hs = new (std::nothrow) mtgp_s();
    if (!hs) return fail(MTGP_ERR_CUDA, "host allocation failed");
    Handle* h = &hs->h;
    std::memset(h, 0, sizeof(Handle));
    h->smooth = 2;
    h->noise_pt = noise_pt;
    h->kind = kind;
    h->d = d;
    h->T = T;
    h->prec = precision;
    h->fp32 = precision == MTGP_FP32_TRANSFORM;
    h->solve_df = h->fp32 && !solve_fp64;
    h->cplx = kind == MTGP_LATTICE;
    h->gen_cols = kind == MTGP_DNET ? gen_cols : 1;
    h->mmax = mmax;
    // sort tasks by decreasing size, ties by caller index (stable)
    std::vector<int> ord(T);
    for (int t = 0; t < T; ++t) ord[t] = t;
    for (int i = 1; i < T; ++i)
        for (int j = i; j > 0 && m[ord[j]] > m[ord[j - 1]]; --j) std::swap(ord[j], ord[j - 1]);
    h->equal = true;
    long long off = 0;
    for (int t = 0; t < T; ++t) {
        h->m_user[t] = m[t];
        h->order[t] = ord[t];
        h->rank[ord[t]] = t;
        h->m[t] = m[ord[t]];
        h->n[t] = 1LL << h->m[t];
        h->yoff[t] = off;
        off += h->n[t];
        if (h->m[t] != h->m[0]) h->equal = false;
    }
    h->N = off;
    // first columns: equal sizes share the diagonal column; otherwise one column per pair t <= u
    int c = 0;
    long long coff = 0;
    if (h->equal) {
        h->cols[c] = ColDesc{coff, (int)h->n[0], 0, 0};
        for (int t = 0; t < T; ++t) h->col_of[t][t] = 0;
        coff += h->n[0];
        ++c;
        for (int t = 0; t < T; ++t)
            for (int u = t + 1; u < T; ++u) {
                h->cols[c] = ColDesc{coff, (int)h->n[0], t, u};
                h->col_of[t][u] = c;
                coff += h->n[0];
                ++c;
            }
    } else {
        for (int t = 0; t < T; ++t)
            for (int u = t; u < T; ++u) {
                h->cols[c] = ColDesc{coff, (int)h->n[t], t, u};
                h->col_of[t][u] = c;
                coff += h->n[t];
                ++c;
            }
    }
    h->ncols = c;
    h->col_elems = coff;
    // group columns by length for batched transforms (columns are ordered by t, so lengths are runs)
    h->ngroups = 0;
    for (int i = 0; i < h->ncols;) {
        int j = i;
        while (j < h->ncols && h->cols[j].n == h->cols[i].n) ++j;
        int g = h->ngroups++;
        h->group_first[g] = i;
        h->group_count[g] = j - i;
        int mm = 0;
        while ((1LL << mm) < h->cols[i].n) ++mm;
        h->group_m[g] = mm;
        i = j;
    }
    // lattices: pair the columns of each group (two real columns per complex transform)
    std::vector<long long> lead_offs, pair_tab;
    h->npairs = 0;
    for (int g = 0; g < h->ngroups; ++g) {
        h->group_lfirst[g] = (int)lead_offs.size();
        const int c0 = h->group_first[g], cnt = h->group_count[g];
        for (int k = 0; k < cnt; ++k) {
            ColDesc& cd = h->cols[c0 + k];
            cd.src = cd.off;
            cd.role = 0;
        }
        for (int k = 0; k < cnt; k += 2) {
            ColDesc& a = h->cols[c0 + k];
            lead_offs.push_back(a.off);
            if (h->cplx && k + 1 < cnt) {
                ColDesc& b = h->cols[c0 + k + 1];
                a.role = 1;
                b.role = 2;
                b.src = a.off;
                pair_tab.push_back(a.off);
                pair_tab.push_back(b.off);
                pair_tab.push_back(a.n);
                ++h->npairs;
            } else if (k + 1 < cnt) {
                lead_offs.push_back(h->cols[c0 + k + 1].off);  // real data: every column alone
            }
        }
        h->group_lcount[g] = (int)lead_offs.size() - h->group_lfirst[g];
    }
    const size_t es = (h->fp32 ? 4 : 8) * (h->cplx ? 2 : 1);
    const size_t vs = h->cplx ? 2 : 1;  // doubles per FP64 value
    cudaError_t e;
#define AL(ptr, cnt)                                              \
    e = dalloc(h, &(ptr), (cnt));                                 \
    if (e != cudaSuccess) {                                       \
        free_all(h);                                              \
        delete hs;                                                \
        return cuda_fail(e, "cudaMalloc workspace");              \
    }
    AL(h->gen, (size_t)d * h->gen_cols);
    AL(h->shift, (size_t)T * d);
    AL(h->cols_dev, (size_t)h->ncols);
    AL(h->lead_offs_dev, lead_offs.size());
    AL(h->pairs_dev, pair_tab.size());
    AL(h->yoffs_dev, (size_t)T);
    {
        size_t half = mmax >= 1 ? ((size_t)1 << (mmax - 1)) : 1;
        double* tw64 = nullptr;
        float* tw32 = nullptr;
        AL(tw64, half * 2);
        AL(tw32, half * 2);
        h->twid = tw64;
        h->twid32 = tw32;
    }
    AL(h->yhat, (size_t)h->N * vs);
    {
        unsigned char* sp = nullptr;
        unsigned char* wg = nullptr;
        AL(sp, (size_t)h->col_elems * es);
        AL(wg, (size_t)h->col_elems * es);
        h->spec = sp;
        h->wgt = wg;
    }
    if (!h->equal) {
        AL(h->S, (size_t)h->col_elems * vs);
        AL(h->Z, (size_t)h->col_elems * vs);
    }
    AL(h->r, (size_t)h->N * vs);
    AL(h->alpha, (size_t)h->N * vs);
    if (h->equal && h->fp32 && !h->cplx) AL(h->yhat_df, (size_t)h->N * 2);
    if (rt_words_len(h) > 0) AL(h->rt_words, (size_t)rt_words_len(h));
    AL(h->tau, (size_t)MTGP_TMAX);
    {
        const int NQ = solve_nq(h);
        long long nsolve = h->equal ? solve_equal_blocks(h) : solve_tree_blocks(h);
        h->partials_len = nsolve * NQ + (long long)eta_grad_blocks(h) * (d + 4);
        long long fl = fused_partials_len(h);
        if (fl > h->partials_len) h->partials_len = fl;
        AL(h->partials, (size_t)h->partials_len);
    }
    AL(h->status, (size_t)1);
    AL(h->out_tmp, (size_t)4);
    AL(h->counters, (size_t)4);
    AL(h->bmix, (size_t)8);
    AL(h->hio, (size_t)(2 * (d + T * T + 2 * T) + 3 + T));
#undef AL
    h->prof = new Prof();
    // upload descriptors
    std::vector<uint32_t> shift_sorted((size_t)T * d);
    for (int t = 0; t < T; ++t)
        for (int j = 0; j < d; ++j) shift_sorted[(size_t)t * d + j] = shift[(size_t)h->order[t] * d + j];
    std::vector<long long> yoffs(T);
    for (int t = 0; t < T; ++t) yoffs[t] = h->yoff[t];
    bool okc = cudaMemcpy(h->gen, gen, (size_t)d * h->gen_cols * sizeof(uint32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(h->shift, shift_sorted.data(), shift_sorted.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(h->cols_dev, h->cols, (size_t)h->ncols * sizeof(ColDesc), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemcpy(h->lead_offs_dev, lead_offs.data(), lead_offs.size() * sizeof(long long),
                          cudaMemcpyHostToDevice) == cudaSuccess &&
               (pair_tab.empty() || cudaMemcpy(h->pairs_dev, pair_tab.data(), pair_tab.size() * sizeof(long long),
                                               cudaMemcpyHostToDevice) == cudaSuccess) &&
               cudaMemcpy(h->yoffs_dev, yoffs.data(), yoffs.size() * sizeof(long long), cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(h->status, 0, sizeof(int)) == cudaSuccess &&
               cudaMemset(h->counters, 0, 4 * sizeof(unsigned)) == cudaSuccess &&
               cudaMemset(h->bmix, 0, 8 * sizeof(double)) == cudaSuccess &&
               cudaMemset(h->tau, 0, MTGP_TMAX * sizeof(double)) == cudaSuccess;
    if (!okc) {
        free_all(h);
        delete hs;
        return fail(MTGP_ERR_CUDA, "uploading handle descriptors failed");
    }
    launch_twiddles(h, 0);
    if (h->rt_words) launch_rt_words(h, 0);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_all(h);
        delete hs;
        return cuda_fail(e, "twiddle table");
    }
    *out = hs;
    return MTGP_OK;
}

int mtgp_destroy(mtgp_t* hs) {
    if (!hs) return MTGP_OK;
    cudaDeviceSynchronize();
    posterior_release(&hs->h);
    free_all(&hs->h);
    delete hs;
    return MTGP_OK;
}

int mtgp_set_smoothness(mtgp_t* hs, int alpha) {
    if (!hs) return fail(MTGP_ERR_INVALID_ARG, "NULL handle");
    Handle* h = &hs->h;
    if (alpha < 1 || alpha > 4) return fail(MTGP_ERR_INVALID_ARG, "smoothness must be 1, 2, 3 or 4");
    ++h->cfg_gen;
    if (h->kind == MTGP_LATTICE) {
        h->smooth = alpha;
        return MTGP_OK;
    }
    // digital nets: the single order alpha of Eq. 2.6, i.e. mixture weights b = e_alpha
    if (alpha == 2) {
        h->dsi_mix = false;
        return MTGP_OK;
    }
    double b[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    b[alpha - 1] = 1.0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(h->bmix, b, sizeof(b), cudaMemcpyHostToDevice));
    h->dsi_mix = true;
    return MTGP_OK;
}

int mtgp_set_dsi_weights(mtgp_t* hs, const double* b, cudaStream_t st) {
    if (!hs) return fail(MTGP_ERR_INVALID_ARG, "NULL handle");
    Handle* h = &hs->h;
    if (h->kind != MTGP_DNET) return fail(MTGP_ERR_UNSUPPORTED, "mixture weights apply to digital nets (Eq. 2.6)");
    ++h->cfg_gen;
    if (!b) {
        h->dsi_mix = false;
        return MTGP_OK;
    }
    CK(cudaMemcpyAsync(h->bmix, b, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemsetAsync(h->bmix + 4, 0, 4 * sizeof(double), st));
    h->dsi_mix = true;
    return MTGP_OK;
}

int mtgp_dsi_weights_grad(mtgp_t* hs, double* g_b, cudaStream_t st) {
    if (!hs || !g_b) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    if (!h->dsi_mix) return fail(MTGP_ERR_INVALID_ARG, "no DSI mixture weights are set on this handle");
    CK(cudaMemcpyAsync(g_b, h->bmix + 4, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return MTGP_OK;
}

int mtgp_points(mtgp_t* hs, uint32_t* x, cudaStream_t st) {
    if (!hs || !x) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    launch_points(&hs->h, x, st);
    CK(cudaGetLastError());
    return MTGP_OK;
}

int mtgp_set_y(mtgp_t* hs, const double* y, cudaStream_t st) {
    if (!hs || !y) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    int blocks = (int)((h->N + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_check_y<<<blocks, 256, 0, st>>>(y, h->N, h->status);
    launch_y_load(h, y, st);
    if (h->equal) k_tau_equal<<<1, 32, 0, st>>>(h->yhat, h->tau, h->T, h->n[0], h->cplx ? 1 : 0);
    if (h->yhat_df) launch_yhat_df(h->yhat, h->yhat_df, h->N, st);
    CK(cudaGetLastError());
    h->y_set = true;
    return MTGP_OK;
}

int mtgp_nll(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
             double* out, double* tau, cudaStream_t st) {
    if (!hs || !out) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    return run_nll(h, th, false, out, tau, nullptr, nullptr, nullptr, nullptr, st);
}

int mtgp_nll_grad(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                  double* out, double* tau, double* g_eta, double* g_W, double* g_v, double* g_sigma2,
                  cudaStream_t st) {
    if (!hs || !out) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    if (!g_eta || !g_W || !g_v || !g_sigma2) return fail(MTGP_ERR_INVALID_ARG, "gradient outputs must not be NULL");
    Handle* h = &hs->h;
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    return run_nll(h, th, true, out, tau, g_eta, g_W, g_v, g_sigma2, st);
}

// theta from page-locked host memory into the handle's staging buffer (one small block; the fused
// kernels wait for it through their programmatic-launch wait)
__global__ void k_stage_in(const double* __restrict__ src, double* __restrict__ dst, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// device address of page-locked host memory, or nullptr if it has none (pageable memory)
static void* mapped_ptr(const void* host) {
    void* dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, const_cast<void*>(host), 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return dp;
}

// copy in, evaluate, copy out on stream st (the launches of the host-buffer entry point).  With
// page-locked buffers the kernels read theta through k_stage_in and write the results straight into
// the host buffer (no DMA copies); pageable buffers go through cudaMemcpyAsync.
static int enqueue_nll_grad_host(Handle* h, const double* theta, int s, double* out, const double* th_map,
                                 double* out_map, cudaStream_t st) {
    const int d = h->d, T = h->T, nsig = h->noise_pt ? T : 1;
    const size_t nth = (size_t)d + (size_t)T * s + T + nsig;
    const size_t nout = 3 + (size_t)T + nth;
    double* dth = h->hio;
    const bool zero_copy = th_map && out_map;
    double* dout = zero_copy ? out_map : h->hio + nth;
    if (zero_copy) {
        k_stage_in<<<1, 64, 0, st>>>(th_map, dth, (int)nth);
        CK(cudaGetLastError());
    } else {
        CK(cudaMemcpyAsync(dth, theta, nth * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    ThetaPtrs th{dth, dth + d, s, dth + d + (size_t)T * s, dth + d + (size_t)T * s + T, nsig,
                 h->dsi_mix ? h->bmix : nullptr};
    double* g = dout + 3 + T;
    int rc = run_nll(h, th, true, dout, dout + 3, g, g + d, g + d + (size_t)T * s, g + d + (size_t)T * s + T, st);
    if (rc) return rc;
    if (!zero_copy) CK(cudaMemcpyAsync(out, dout, nout * sizeof(double), cudaMemcpyDeviceToHost, st));
    return MTGP_OK;
}

static void drop_hio_graph(Handle* h) {
    if (h->hio_exec) cudaGraphExecDestroy(h->hio_exec);
    h->hio_exec = nullptr;
}

// capture the copy-in / kernels / copy-out sequence into h->hio_exec; false if the capture fails
static bool capture_hio_graph(Handle* h, const double* theta, int s, double* out, const double* th_map,
                              double* out_map) {
    drop_hio_graph(h);
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        h->cap_stream = nullptr;
        return false;
    }
    if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    const int rc = enqueue_nll_grad_host(h, theta, s, out, th_map, out_map, h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(h->cap_stream, &graph);
    bool ok = rc == MTGP_OK && ec == cudaSuccess && graph != nullptr;
    if (ok) ok = cudaGraphInstantiate(&h->hio_exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        h->hio_exec = nullptr;
        cudaGetLastError();  // the failed capture's error is not the caller's
    }
    return ok;
}

int mtgp_nll_grad_host(mtgp_t* hs, const double* theta, int s, double* out, cudaStream_t st) {
    if (!hs || !theta || !out) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    if (s < 1 || s > h->T) return fail(MTGP_ERR_INVALID_ARG, "s must satisfy 1 <= s <= T");
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    // looked up on every call: a buffer that is no longer page-locked must not reach a kernel
    const double* th_map = static_cast<const double*>(mapped_ptr(theta));
    double* out_map = static_cast<double*>(mapped_ptr(out));
    const bool profiling = h->prof && h->prof->on;
    if (th_map && out_map && !profiling && !h->hio_nograph) {
        const bool same = h->hio_exec && h->hio_key_th == th_map && h->hio_key_out == out_map &&
                          h->hio_key_s == s && h->hio_key_gen == h->cfg_gen;
        if (!same) {
            h->hio_key_th = th_map;
            h->hio_key_out = out_map;
            h->hio_key_s = s;
            h->hio_key_gen = h->cfg_gen;
            if (!capture_hio_graph(h, theta, s, out, th_map, out_map)) h->hio_nograph = true;  // direct from now on
        }
        if (h->hio_exec) {
            CK(cudaGraphLaunch(h->hio_exec, st));
            return MTGP_OK;
        }
    }
    return enqueue_nll_grad_host(h, theta, s, out, th_map, out_map, st);
}

// GCV loss at the GCV mean: generic path (column generation, transforms, per-frequency or tree
// solve in GCV mode, finalize)
static int run_gcv(Handle* h, ThetaPtrs th, double* out, double* tau, cudaStream_t st) {
    if (!h->equal && !h->gcv_h) {
        long long P0 = 0;
        for (int t = 0; t < h->T; ++t) P0 += h->n[t] / h->n[h->T - 1];
        const size_t bytes = sizeof(double) * (size_t)(h->T + 1) * (size_t)P0 * (h->cplx ? 2 : 1);
        CK(cudaMalloc(&h->gcv_h, bytes));
        h->ws_bytes += (long long)bytes;
    }
    k_check_theta<<<1, 64, 0, st>>>(th, h->d, h->T, h->status);
    forward_columns(h, th.eta, st);
    int nsolve;
    if (h->equal) {
        mtgp_prof_begin(h, "solve_equal_gcv", st);
        launch_solve_equal(h, th, false, h->partials, st, 1);
        mtgp_prof_end(h, st);
        nsolve = solve_equal_blocks(h);
    } else {
        mtgp_prof_begin(h, "solve_tree_gcv", st);
        launch_solve_tree(h, th, false, h->partials, st, true);
        mtgp_prof_end(h, st);
        nsolve = solve_tree_blocks(h);
    }
    mtgp_prof_begin(h, "finalize", st);
    launch_finalize(h, th, false, h->partials, nsolve, nullptr, 0, out, tau, nullptr, nullptr, nullptr, nullptr, st, 1);
    mtgp_prof_end(h, st);
    CK(cudaGetLastError());
    return MTGP_OK;
}

int mtgp_cubature(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                  double* mu, double* Sigma, cudaStream_t st) {
    if (!hs || !mu || !Sigma) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    if (!h->equal && !h->pi_buf) {
        CK(cudaMalloc(&h->pi_buf, sizeof(double) * MTGP_TMAX * MTGP_TMAX));
        h->ws_bytes += (long long)sizeof(double) * MTGP_TMAX * MTGP_TMAX;
    }
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    // the MLE solve leaves alpha, tau (sorted), the transformed spectra (equal sizes) or Pi (nested)
    rc = run_nll(h, th, false, h->out_tmp, nullptr, nullptr, nullptr, nullptr, nullptr, st, true);
    if (rc) return rc;
    CubParams cp;
    std::memset(&cp, 0, sizeof(cp));
    cp.T = h->T;
    cp.s = s;
    cp.equal = h->equal ? 1 : 0;
    cp.cplx = h->cplx ? 1 : 0;
    cp.fp32 = h->fp32 ? 1 : 0;
    cp.clamp = h->fp32 ? 1 : 0;
    for (int t = 0; t < MTGP_TMAX; ++t) {
        cp.n[t] = t < h->T ? h->n[t] : 1;
        cp.yoff[t] = t < h->T ? h->yoff[t] : 0;
        cp.order[t] = t < h->T ? h->order[t] : 0;
        cp.rank[t] = t < h->T ? h->rank[t] : 0;
        for (int u = 0; u < MTGP_TMAX; ++u) cp.colidx[t][u] = (t < h->T && u < h->T && t <= u) ? h->col_of[t][u] : 0;
    }
    for (int c = 0; c < MTGP_MAX_COLS; ++c) cp.coloff[c] = c < h->ncols ? h->cols[c].off : 0;
    k_cubature<<<1, 32, 0, st>>>(cp, th, h->spec, h->alpha, h->tau, h->pi_buf, mu, Sigma, h->status);
    CK(cudaGetLastError());
    return MTGP_OK;
}

// GCV gradient, equal sizes: the value pass, then a second per-frequency pass with the totals, the
// adjoint transforms and the eta pass of the MLE gradient
static int run_gcv_grad(Handle* h, ThetaPtrs th, double* out, double* tau, double* g_eta, double* g_W, double* g_v,
                        double* g_s2, cudaStream_t st) {
    int rc = run_gcv(h, th, out, tau, st);
    if (rc) return rc;
    mtgp_prof_begin(h, "solve_equal_gcv_grad", st);
    launch_solve_equal(h, th, true, h->partials, st, 2, out + 1);
    mtgp_prof_end(h, st);
    const int nsolve = solve_equal_blocks(h);
    const int NQ = solve_nq(h);
    double* eta_part = h->partials + (long long)nsolve * NQ;
    adjoint_columns(h, st);
    const int neta = eta_grad_blocks(h);
    mtgp_prof_begin(h, "eta_grad", st);
    launch_eta_grad(h, th.eta, h->wgt, eta_part, neta, st);
    mtgp_prof_end(h, st);
    mtgp_prof_begin(h, "finalize", st);
    launch_finalize(h, th, true, h->partials, nsolve, eta_part, neta, out, nullptr, g_eta, g_W, g_v, g_s2, st, 2);
    mtgp_prof_end(h, st);
    CK(cudaGetLastError());
    return MTGP_OK;
}

int mtgp_gcv_grad(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                  double* out, double* tau, double* g_eta, double* g_W, double* g_v, double* g_sigma2,
                  cudaStream_t st) {
    if (!hs || !out || !g_eta || !g_W || !g_v || !g_sigma2) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    if (!h->equal) return fail(MTGP_ERR_UNSUPPORTED, "the GCV gradient needs equal task sizes");
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    return run_gcv_grad(h, th, out, tau, g_eta, g_W, g_v, g_sigma2, st);
}

int mtgp_gcv(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
             double* out, double* tau, cudaStream_t st) {
    if (!hs || !out) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Handle* h = &hs->h;
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    return run_gcv(h, th, out, tau, st);
}

int mtgp_posterior(mtgp_t* hs, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                   int nq, const double* xq, const int* task, double* mean, double* var, cudaStream_t st) {
    if (!hs || !xq || !task || !mean) return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    if (nq < 0) return fail(MTGP_ERR_INVALID_ARG, "nq < 0");
    Handle* h = &hs->h;
    int rc = validate_theta(h, eta, W, s, v, sigma2);
    if (rc) return rc;
    if (!h->y_set) return fail(MTGP_ERR_STATE, "mtgp_set_y must be called first");
    if (nq == 0) return MTGP_OK;
    ThetaPtrs th{eta, W, s, v, sigma2, h->noise_pt ? h->T : 1, h->dsi_mix ? h->bmix : nullptr};
    // the solve leaves alpha = Lambda^-1 rhat and tau in the workspace
    rc = run_nll(h, th, false, h->out_tmp, nullptr, nullptr, nullptr, nullptr, nullptr, st, true);
    if (rc) return rc;
    rc = posterior_run(h, th, nq, xq, task, mean, var, st);
    if (rc) return rc == MTGP_ERR_CUDA ? fail(rc, "posterior scratch allocation failed") : fail(rc, "posterior");
    CK(cudaGetLastError());
    return MTGP_OK;
}

int mtgp_profile(mtgp_t* hs, int enable) {
    if (!hs) return fail(MTGP_ERR_INVALID_ARG, "NULL handle");
    hs->h.prof->on = enable != 0;
    return MTGP_OK;
}

int mtgp_profile_read(mtgp_t* hs, int max_entries, char* names, double* total_ms, int* counts, int* n_out) {
    if (!hs || !n_out || (max_entries > 0 && (!names || !total_ms || !counts)))
        return fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    Prof* p = hs->h.prof;
    std::vector<std::string> nm;
    std::vector<double> tot;
    std::vector<int> cnt;
    for (auto& r : p->recs) {
        CK(cudaEventSynchronize(r.b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        size_t i = 0;
        while (i < nm.size() && nm[i] != r.name) ++i;
        if (i == nm.size()) {
            nm.push_back(r.name);
            tot.push_back(0.0);
            cnt.push_back(0);
        }
        tot[i] += ms;
        cnt[i] += 1;
        p->pool.push_back(r.a);
        p->pool.push_back(r.b);
    }
    p->recs.clear();
    int n = (int)nm.size();
    *n_out = n;
    for (int i = 0; i < n && i < max_entries; ++i) {
        std::snprintf(names + 32 * i, 32, "%s", nm[i].c_str());
        total_ms[i] = tot[i];
        counts[i] = cnt[i];
    }
    return MTGP_OK;
}

int mtgp_sync(mtgp_t* hs, cudaStream_t st) {
    if (!hs) return fail(MTGP_ERR_INVALID_ARG, "NULL handle");
    Handle* h = &hs->h;
    int s = 0;
    CK(cudaMemcpyAsync(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemsetAsync(h->status, 0, sizeof(int), st));
    CK(cudaStreamSynchronize(st));
    if (s & ST_NUMERIC) return fail(MTGP_ERR_NUMERIC, "non-finite value in an input or intermediate");
    if (s & ST_NOT_PD) return fail(MTGP_ERR_NOT_PD, "non-positive pivot: Lambda-tilde is not numerically HPD");
    if (s & ST_TIMEOUT) return fail(MTGP_ERR_TIMEOUT, "a bounded device wait gave up");
    return MTGP_OK;
}

}  // extern "C"

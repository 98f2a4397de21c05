// Batched fits: many independent equal-size fits advanced together.
//
// Each fit keeps its own workspace (an ordinary handle).  One NLL + gradient evaluation of the whole
// batch is three phases (kernels A, B, C of k_fused.cu); within a phase the fits are grouped into
// classes that share a kernel specialisation -- (design kind, T) for the per-frequency FP64 solve,
// (design kind, dimension bucket) for the generation / adjoint kernels -- and each class runs as one
// persistent launch over a table of (fit, block) items ordered largest fit first.  Classes of one
// phase run concurrently on side streams.  An optimiser step adds one Adam update on the packed
// parameters (log eta, W, log v, log sigma2); a run of steps can be captured in one CUDA graph.
// The split of each fit's transform between kernels A/C and B can be chosen by timing (autotune).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "mtgp_internal.cuh"

namespace {

constexpr int kSide = 16;

struct Cls {
    int phase;
    int variant;      // FUSED_GENERIC / FUSED_RT / FUSED_RT_DF
    bool fp32;        // transform precision of the class's fits
    bool cplx;
    int key;          // T (phase B) or dimension bucket (phases A, C)
    int2* items;      // device
    int nitems;
    int grid, threads;
    size_t smem;
};

int dbucket(int d) { return d <= 4 ? 4 : d <= 8 ? 8 : d <= 16 ? 16 : 32; }

__global__ void k_batch_theta_in(const double* nat, double* lg, double* nv, const int* pinfo, long long np, double* m1,
                                 double* m2) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        double x = nat[p];
        lg[p] = pinfo[2 * p + 1] ? log(x) : x;
        nv[p] = x;
        m1[p] = 0.0;
        m2[p] = 0.0;
    }
}

// Adam on the packed parameters; positive parameters live in log space (chain rule d/dlog x = x d/dx).
// The objective's value at the parameters this step used is recorded in trace (if given).
__global__ void k_batch_adam(double* lg, double* nv, const double* g, double* m1, double* m2, const int* pinfo,
                             long long np, const int* tstep, int step, double lr, const double* out, double* trace,
                             int nfits) {
    const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    const int t = *tstep + step + 1;
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        const bool islog = pinfo[2 * p + 1] != 0;
        double gg = g[p];
        if (islog) gg *= nv[p];
        const double a = b1 * m1[p] + (1.0 - b1) * gg;
        const double b = b2 * m2[p] + (1.0 - b2) * gg * gg;
        m1[p] = a;
        m2[p] = b;
        const double x = lg[p] - lr * (a / c1) / (sqrt(b / c2) + eps);
        lg[p] = x;
        nv[p] = islog ? exp(x) : x;
        if (trace && p < nfits) trace[(long long)step * nfits + p] = out[3 * p];
    }
}

__global__ void k_batch_tick(int* tstep, int k) { *tstep += k; }

}  // namespace

struct mtgp_batch_s {
    int nfits = 0, s = 1;
    std::vector<mtgp_t*> fits;
    std::vector<int> a;
    std::vector<long long> poff, yoff, partoff;
    long long np = 0;
    double *th_log = nullptr, *th_nat = nullptr, *g_nat = nullptr, *m1 = nullptr, *m2 = nullptr;
    double *out = nullptr, *tau = nullptr, *partials = nullptr;
    unsigned* counters = nullptr;
    int* pinfo = nullptr;
    int* tstep = nullptr;
    unsigned char* descs = nullptr;
    std::vector<unsigned char> descs_host;
    std::vector<Cls> cls[3];
    cudaStream_t side[kSide] = {};
    cudaEvent_t evfork = nullptr, evjoin[kSide] = {};
    cudaGraphExec_t gexec = nullptr;
    int gsteps = 0;
    double glr = 0.0;
    double* gtrace = nullptr;
    int nsm = 1;
    void* fdesc = nullptr;  // proposal descriptors (device), built on first use
    float* pfeat = nullptr;  // mtgp_propose: features (nfits x 258) and prediction (nfits x 37), on first use
    float* ppred = nullptr;
    double* jcur = nullptr;   // mtgp_propose with the exact-NLL judge: log parameters before the call,
    double* jcur_nat = nullptr;  // the same natural parameters (restored exactly by the last candidate),
    double* jpred = nullptr;  // log parameters of the prediction, best candidate NLL and index per fit, sigma2 marks
    double* jbest = nullptr;
    int* jk = nullptr;
    unsigned char* is_s2 = nullptr;
};

namespace {

int bfail(int code, const char* msg) {
    mtgp_set_error(msg);
    return code;
}

int launch_status(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return MTGP_OK;
    char msg[256];
    std::snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
    return bfail(MTGP_ERR_CUDA, msg);
}

void free_classes(mtgp_batch_s* b) {
    for (int ph = 0; ph < 3; ++ph) {
        for (auto& c : b->cls[ph]) cudaFree(c.items);
        b->cls[ph].clear();
    }
}

// (re)build descriptors, partial-sum buffers and class item tables for the current splits
int build_plan(mtgp_batch_s* b) {
    cudaDeviceSynchronize();  // earlier launches may still read the old tables
    free_classes(b);
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    const size_t dsz = fused_desc_size();
    b->partoff.assign(b->nfits + 1, 0);
    for (int f = 0; f < b->nfits; ++f) {
        const Handle& h = b->fits[f]->h;
        const int NQ = 3 + h.T * (h.T + 1) / 2;
        const int m = h.m[0], a = b->a[f];
        b->partoff[f + 1] = b->partoff[f] + ((long long)1 << a) * (NQ + 1) + ((long long)1 << (m - a)) * h.d + NQ;
    }
    cudaFree(b->partials);
    b->partials = nullptr;
    if (cudaMalloc(&b->partials, sizeof(double) * (size_t)std::max<long long>(b->partoff[b->nfits], 1)) != cudaSuccess)
        return bfail(MTGP_ERR_CUDA, "batch partials allocation failed");
    b->descs_host.assign(dsz * b->nfits, 0);
    for (int f = 0; f < b->nfits; ++f) {
        const Handle& h = b->fits[f]->h;
        const long long o = b->poff[f];
        const int d = h.d, T = h.T, s = b->s;
        ThetaPtrs th{b->th_nat + o, b->th_nat + o + d, s, b->th_nat + o + d + (long long)T * s,
                     b->th_nat + o + d + (long long)T * s + T};
        fused_make_desc(&h, th, b->out + 3 * f, b->tau + (long long)MTGP_TMAX * f, b->g_nat + o, b->g_nat + o + d,
                        b->g_nat + o + d + (long long)T * s, b->g_nat + o + d + (long long)T * s + T, true, b->a[f],
                        b->partials + b->partoff[f], b->counters + 2 * f, b->descs_host.data() + dsz * f);
    }
    if (!b->descs) {
        if (cudaMalloc(&b->descs, dsz * b->nfits) != cudaSuccess) return bfail(MTGP_ERR_CUDA, "batch descriptor allocation failed");
    }
    if (cudaMemcpy(b->descs, b->descs_host.data(), dsz * b->nfits, cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(MTGP_ERR_CUDA, "batch descriptor upload failed");
    // classes, fits largest first
    std::vector<int> order(b->nfits);
    for (int f = 0; f < b->nfits; ++f) order[f] = f;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const Handle &hx = b->fits[x]->h, &hy = b->fits[y]->h;
        return hx.n[0] * hx.T * hx.T > hy.n[0] * hy.T * hy.T;
    });
    for (int ph = 0; ph < 3; ++ph) {
        // class key: (kernel family, transform precision, complex spectra, T or dimension bucket)
        std::map<std::tuple<int, int, int, int>, std::vector<int2>> items;
        std::map<std::tuple<int, int, int, int>, std::pair<size_t, int>> res;  // smem, threads
        for (int f : order) {
            const Handle& h = b->fits[f]->h;
            const int m = h.m[0], a = b->a[f];
            const int var = fused_variant(h.fp32, h.cplx, h.solve_df, h.d, m, a, false);
            const int key = ph == 1 ? h.T : dbucket(h.d);
            auto k = std::make_tuple(var, h.fp32 ? 1 : 0, h.cplx ? 1 : 0, key);
            const int nblk = ph == 1 ? (1 << a) : (1 << (m - a));
            for (int j = 0; j < nblk; ++j) items[k].push_back(make_int2(f, j));
            const size_t sm = fused_smem(ph, var, h.T, h.ncols, m, a, h.fp32, h.cplx);
            const int th = fused_threads(ph, var, a, h.d, h.ncols, m);
            auto& r = res[k];
            r.first = std::max(r.first, sm);
            r.second = std::max(r.second, th);
        }
        for (auto& kv : items) {
            Cls c;
            c.phase = ph;
            c.variant = std::get<0>(kv.first);
            c.fp32 = std::get<1>(kv.first) != 0;
            c.cplx = std::get<2>(kv.first) != 0;
            c.key = std::get<3>(kv.first);
            c.nitems = (int)kv.second.size();
            c.smem = res[kv.first].first;
            c.threads = res[kv.first].second;
            const int T = ph == 1 ? c.key : 1;
            const int per_sm = fused_resident_blocks(ph, c.variant, c.fp32, c.cplx, T, c.key, c.threads, c.smem);
            c.grid = std::min(c.nitems, per_sm * b->nsm);
            if (cudaMalloc(&c.items, sizeof(int2) * c.nitems) != cudaSuccess)
                return bfail(MTGP_ERR_CUDA, "batch item table allocation failed");
            cudaMemcpy(c.items, kv.second.data(), sizeof(int2) * c.nitems, cudaMemcpyHostToDevice);
            b->cls[ph].push_back(c);
        }
    }
    return MTGP_OK;
}

// ---- learned proposal: per-fit spectral features, training targets and the map back to parameters ----

constexpr int kFeat = 8 * 32 + 2, kOut = 37, kDmaxProp = 12;

struct FeatDesc {
    const double* yhat;
    long long yoff[MTGP_TMAX];  // element offset of caller task t's transformed observations
    long long poff;             // offset of the fit's packed parameters
    int T, m, d, cplx;
};

// bin(f) = floor(4 q / m), q = 8 floor(log2 f) + the three bits after f's leading one (zero-filled)
__device__ __forceinline__ int freq_bin(unsigned long long f, int m) {
    const int L = 63 - __clzll((long long)f);
    const int frac3 = L >= 3 ? (int)((f >> (L - 3)) & 7ull) : (int)((f << (3 - L)) & 7ull);
    return (4 * (8 * L + frac3)) / m;
}

// one block per fit: per task, log of the mean |yhat(f)|^2 over each of 32 log-spaced frequency bins
// (f = 1..n-1; empty bins repeat the previous value), then log2 n and d.  A warp takes 32 consecutive
// frequencies; their bins form contiguous runs, summed by a segmented warp scan in a fixed order, and
// the run's last lane adds the run to the warp's own bin row, so the sums are deterministic.
__global__ void __launch_bounds__(256) k_batch_features(const FeatDesc* __restrict__ fds, float* __restrict__ feat) {
    __shared__ double s_sum[8][32], s_cnt[8][32];
    const FeatDesc& fd = fds[blockIdx.x];
    float* out = feat + (long long)blockIdx.x * kFeat;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n = 1ll << fd.m;
    for (int t = 0; t < MTGP_TMAX; ++t) {
        if (t >= fd.T) {
            if (threadIdx.x < 32) out[t * 32 + threadIdx.x] = 0.f;
            continue;
        }
        s_sum[warp][lane] = 0.0;
        s_cnt[warp][lane] = 0.0;
        __syncthreads();
        const double* y = fd.yhat + (fd.cplx ? 2 : 1) * fd.yoff[t];
        for (long long base = (long long)warp * 32; base < n; base += 256) {
            const long long f = base + lane;
            int bin = 32;  // past the last frequency: no bin
            double e = 0.0, c = 0.0;
            if (f < n) {
                bin = f == 0 ? 0 : freq_bin((unsigned long long)f, fd.m);
                if (f > 0) {
                    if (fd.cplx) {
                        const double re = y[2 * f], im = y[2 * f + 1];
                        e = re * re + im * im;
                    } else {
                        e = y[f] * y[f];
                    }
                    c = 1.0;
                }
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double ue = __shfl_up_sync(0xffffffffu, e, o);
                const double uc = __shfl_up_sync(0xffffffffu, c, o);
                const int ub = __shfl_up_sync(0xffffffffu, bin, o);
                if (lane >= o && ub == bin) {
                    e += ue;
                    c += uc;
                }
            }
            const int nb = __shfl_down_sync(0xffffffffu, bin, 1);
            if ((lane == 31 || nb != bin) && bin < 32) {
                s_sum[warp][bin] += e;
                s_cnt[warp][bin] += c;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float prev = 0.f;
            for (int k = 0; k < 32; ++k) {
                double sm = 0.0, cn = 0.0;
                for (int w = 0; w < 8; ++w) {
                    sm += s_sum[w][k];
                    cn += s_cnt[w][k];
                }
                if (k == 0 || cn > 0.0) prev = (float)log(sm / (cn > 1.0 ? cn : 1.0) + 1e-30);
                out[t * 32 + k] = prev;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[256] = (float)fd.m;
        out[257] = (float)fd.d;
    }
}

// one thread per fit: [log eta (12), canonical W (8 x 2), log v (8), log sigma2] and its mask; a fit
// whose parameters give a non-finite entry gets target 0 and mask 0 throughout
__global__ void k_batch_targets(const FeatDesc* __restrict__ fds, const double* __restrict__ nat, int nfits,
                                float* __restrict__ tgt, float* __restrict__ mask) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfits) return;
    const FeatDesc& fd = fds[f];
    const double* p = nat + fd.poff;
    float t[kOut], mk[kOut];
    const int d = fd.d, T = fd.T;
    for (int j = 0; j < kDmaxProp; ++j) {
        t[j] = j < d ? (float)log(p[j]) : 0.f;
        mk[j] = j < d ? 1.f : 0.f;
    }
    // W Q with Q the rotation taking row 0 to (r, 0), then column 1 negated if W[1][1] < 0
    const double* W = p + d;
    const double a = W[0], b = W[1], r = sqrt(a * a + b * b);
    const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
    const double w11 = T > 1 ? -W[2] * sn + W[3] * c : 0.0;
    const double sg = w11 < 0.0 ? -1.0 : 1.0;
    for (int u = 0; u < MTGP_TMAX; ++u) {
        float w0 = 0.f, w1 = 0.f, m = 0.f;
        if (u < T) {
            w0 = (float)(W[2 * u] * c + W[2 * u + 1] * sn);
            w1 = u == 0 ? 0.f : (float)(sg * (-W[2 * u] * sn + W[2 * u + 1] * c));
            m = 1.f;
        }
        t[kDmaxProp + 2 * u] = w0;
        t[kDmaxProp + 2 * u + 1] = w1;
        mk[kDmaxProp + 2 * u] = m;
        mk[kDmaxProp + 2 * u + 1] = m;
        t[kDmaxProp + 16 + u] = u < T ? (float)log(p[d + 2 * T + u]) : 0.f;
        mk[kDmaxProp + 16 + u] = m;
    }
    t[kOut - 1] = (float)log(p[d + 3 * T]);
    mk[kOut - 1] = 1.f;
    bool ok = true;
    for (int k = 0; k < kOut; ++k) ok = ok && isfinite(t[k]);
    float* to = tgt + (long long)f * kOut;
    float* mo = mask + (long long)f * kOut;
    for (int k = 0; k < kOut; ++k) {
        to[k] = ok ? t[k] : 0.f;
        mo[k] = ok ? mk[k] : 0.f;
    }
}

// one thread per fit: parameters from a prediction (exp of the log entries clamped to [-40, 20]);
// Adam moments of the fit cleared
__global__ void k_batch_propose(const FeatDesc* __restrict__ fds, const float* __restrict__ pred, int nfits,
                                double* __restrict__ lg, double* __restrict__ nv, double* __restrict__ m1,
                                double* __restrict__ m2) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfits) return;
    const FeatDesc& fd = fds[f];
    const float* q = pred + (long long)f * kOut;
    const int d = fd.d, T = fd.T;
    const long long o = fd.poff;
    auto put_log = [&](long long k, float z) {
        double x = (double)z;
        x = x < -40.0 ? -40.0 : (x > 20.0 ? 20.0 : x);
        lg[o + k] = x;
        nv[o + k] = exp(x);
    };
    for (int j = 0; j < d; ++j) put_log(j, q[j]);
    for (int k = 0; k < 2 * T; ++k) {
        lg[o + d + k] = (double)q[kDmaxProp + k];
        nv[o + d + k] = (double)q[kDmaxProp + k];
    }
    for (int u = 0; u < T; ++u) put_log(d + 2 * T + u, q[kDmaxProp + 16 + u]);
    put_log(d + 3 * T, q[kOut - 1]);
    for (long long k = 0; k < d + 3 * T + 1; ++k) {
        m1[o + k] = 0.0;
        m2[o + k] = 0.0;
    }
}

// Starting-point candidates judged by the exact NLL: candidate k blends the log parameters before the
// call (c) and of the prediction (p) as lam p + (1 - lam) c (W linearly), with log sigma2 raised by
// dls2 (guards against an under-predicted noise level, whose quadratic form grows like 1 / sigma2).
// The last candidate is the starting point the caller set: the judged start is never worse than it.
constexpr int kJudgeCand = 5;
__device__ __forceinline__ void judge_candidate(int k, double& lam, double& dls2) {
    const double L[kJudgeCand] = {1.0, 1.0, 0.5, 0.25, 0.0};
    const double S[kJudgeCand] = {0.0, 4.605170185988092, 0.0, 0.0, 0.0};  // ln 100
    lam = L[k];
    dls2 = S[k];
}

__global__ void k_judge_set(int k, const int* __restrict__ kfit, const int* __restrict__ pinfo,
                            const unsigned char* __restrict__ is_s2, long long np, const double* __restrict__ cur,
                            const double* __restrict__ cur_nat, const double* __restrict__ pred, double* __restrict__ lg,
                            double* __restrict__ nv, double* __restrict__ m1, double* __restrict__ m2) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np; q += (long long)gridDim.x * blockDim.x) {
        int kk = k;
        if (kfit) {
            kk = kfit[pinfo[2 * q]];
            if (kk < 0) kk = kJudgeCand - 1;  // no finite candidate: the caller's start
        }
        double lam, dls2;
        judge_candidate(kk, lam, dls2);
        if (kk == kJudgeCand - 1) {
            // the caller's own start, exactly
            lg[q] = cur[q];
            nv[q] = cur_nat[q];
        } else {
            double x = lam * pred[q] + (1.0 - lam) * cur[q];
            if (is_s2[q]) x += dls2;
            const bool islog = pinfo[2 * q + 1] != 0;
            lg[q] = x;
            nv[q] = islog ? exp(x) : x;
        }
        m1[q] = 0.0;
        m2[q] = 0.0;
    }
}

__global__ void k_judge_keep(int k, int first, int nfits, const double* __restrict__ out, double* __restrict__ best,
                             int* __restrict__ kbest) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfits) return;
    const double v = out[3 * f];
    if (first) {
        best[f] = INFINITY;
        kbest[f] = -1;
    }
    if (isfinite(v) && v < best[f]) {
        best[f] = v;
        kbest[f] = k;
    }
}

int ensure_fdesc(mtgp_batch_s* b) {
    if (b->fdesc) return MTGP_OK;
    if (b->s != 2) return bfail(MTGP_ERR_UNSUPPORTED, "the proposal is defined for s = 2");
    std::vector<FeatDesc> v(b->nfits);
    for (int f = 0; f < b->nfits; ++f) {
        const Handle& h = b->fits[f]->h;
        if (h.d > kDmaxProp) return bfail(MTGP_ERR_UNSUPPORTED, "the proposal is defined for d <= 12");
        FeatDesc& x = v[f];
        std::memset(&x, 0, sizeof(x));
        x.yhat = h.yhat;
        for (int t = 0; t < h.T; ++t) x.yoff[t] = h.yoff[h.rank[t]];
        x.poff = b->poff[f];
        x.T = h.T;
        x.m = h.m[0];
        x.d = h.d;
        x.cplx = h.cplx ? 1 : 0;
    }
    if (cudaMalloc(&b->fdesc, sizeof(FeatDesc) * v.size()) != cudaSuccess)
        return bfail(MTGP_ERR_CUDA, "proposal table allocation failed");
    cudaMemcpy(b->fdesc, v.data(), sizeof(FeatDesc) * v.size(), cudaMemcpyHostToDevice);
    return MTGP_OK;
}

// with MTGP_BATCH_CHECK set in the environment every class launch is checked (outside graph capture)
void check_launch(const Cls& c, int T) {
    static const bool on = std::getenv("MTGP_BATCH_CHECK") != nullptr;
    if (!on) return;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        std::fprintf(stderr, "batch launch failed: %s phase=%d variant=%d fp32=%d cplx=%d key=%d T=%d grid=%d threads=%d smem=%zu items=%d\n",
                     cudaGetErrorString(e), c.phase, c.variant, (int)c.fp32, (int)c.cplx, c.key, T, c.grid, c.threads, c.smem,
                     c.nitems);
}

// the three phases of one batched NLL + gradient evaluation on stream st (classes forked to side streams)
void launch_eval(mtgp_batch_s* b, cudaStream_t st) {
    for (int ph = 0; ph < 3; ++ph) {
        const auto& cl = b->cls[ph];
        if (cl.size() == 1) {
            const Cls& c = cl[0];
            const int T = ph == 1 ? c.key : 1;
            fused_phase(ph, c.variant, c.fp32, c.cplx, T, c.key, nullptr, b->descs, c.items, c.nitems, c.grid, c.threads, c.smem, st);
            check_launch(c, T);
            continue;
        }
        cudaEventRecord(b->evfork, st);
        for (size_t i = 0; i < cl.size(); ++i) {
            const Cls& c = cl[i];
            cudaStream_t ss = b->side[i % kSide];
            cudaStreamWaitEvent(ss, b->evfork, 0);
            const int T = ph == 1 ? c.key : 1;
            fused_phase(ph, c.variant, c.fp32, c.cplx, T, c.key, nullptr, b->descs, c.items, c.nitems, c.grid, c.threads, c.smem, ss);
            check_launch(c, T);
        }
        const int used = (int)std::min<size_t>(cl.size(), kSide);
        for (int i = 0; i < used; ++i) {
            cudaEventRecord(b->evjoin[i], b->side[i]);
            cudaStreamWaitEvent(st, b->evjoin[i], 0);
        }
    }
}

void launch_steps(mtgp_batch_s* b, int steps, double lr, double* trace, cudaStream_t st) {
    const int thr = 256;
    const int blocks = (int)std::min<long long>((b->np + thr - 1) / thr, 4096);
    for (int k = 0; k < steps; ++k) {
        launch_eval(b, st);
        k_batch_adam<<<blocks, thr, 0, st>>>(b->th_log, b->th_nat, b->g_nat, b->m1, b->m2, b->pinfo, b->np, b->tstep, k,
                                             lr, b->out, trace, b->nfits);
    }
    k_batch_tick<<<1, 1, 0, st>>>(b->tstep, steps);
}

}  // namespace

extern "C" {

int mtgp_batch_create(mtgp_batch_t** out, int nfits, const int* kind, const int* d, const int* T, const int* m,
                      const uint32_t* gen, const int* gen_cols, const uint32_t* shift, int s, const int* precision) {
    if (!out) return bfail(MTGP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nfits < 1 || !kind || !d || !T || !m || !gen || !gen_cols || !shift || !precision)
        return bfail(MTGP_ERR_INVALID_ARG, "nfits < 1 or NULL host array");
    if (s < 1) return bfail(MTGP_ERR_INVALID_ARG, "s must be >= 1");
    for (int f = 0; f < nfits; ++f) {
        if (precision[f] & MTGP_NOISE_PER_TASK)
            return bfail(MTGP_ERR_UNSUPPORTED, "batched fits take one noise variance per fit");
        const int pr = precision[f] & ~MTGP_SOLVE_FP64;
        if (pr != MTGP_FP64 && pr != MTGP_FP32_TRANSFORM)
            return bfail(MTGP_ERR_INVALID_ARG, "precision[f] must be MTGP_FP64 or MTGP_FP32_TRANSFORM (optionally | MTGP_SOLVE_FP64)");
        if (T[f] < s) return bfail(MTGP_ERR_INVALID_ARG, "every fit needs T >= s");
    }
    auto* b = new mtgp_batch_s();
    b->nfits = nfits;
    b->s = s;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    long long goff = 0, soff = 0, poff = 0, yoff = 0;
    b->poff.push_back(0);
    b->yoff.push_back(0);
    std::vector<int> pinfo;
    for (int f = 0; f < nfits; ++f) {
        std::vector<int> mm(T[f], m[f]);
        mtgp_t* hf = nullptr;
        int rc = mtgp_create(&hf, kind[f], d[f], T[f], mm.data(), gen + goff, gen_cols[f], shift + soff, precision[f]);
        if (rc) {
            mtgp_batch_destroy(b);
            return rc;
        }
        b->fits.push_back(hf);
        int a = 0, lgL = 0;
        if (!fused_plan(m[f], hf->h.ncols, hf->h.d, hf->h.fp32, hf->h.cplx, -1, &a, &lgL)) {
            mtgp_batch_destroy(b);
            return bfail(MTGP_ERR_UNSUPPORTED, "a fit's size is not handled by the fused kernels (m >= 4, tiles <= 96 KB)");
        }
        b->a.push_back(a);
        goff += kind[f] == MTGP_LATTICE ? d[f] : (long long)d[f] * gen_cols[f];
        soff += (long long)T[f] * d[f];
        const long long npf = d[f] + (long long)T[f] * s + T[f] + 1;
        for (long long q = 0; q < npf; ++q) {
            const bool is_w = q >= d[f] && q < d[f] + (long long)T[f] * s;
            pinfo.push_back(f);
            pinfo.push_back(is_w ? 0 : 1);
        }
        poff += npf;
        yoff += (long long)T[f] << m[f];
        b->poff.push_back(poff);
        b->yoff.push_back(yoff);
    }
    b->np = poff;
    bool ok = cudaMalloc(&b->th_log, sizeof(double) * poff) == cudaSuccess &&
              cudaMalloc(&b->th_nat, sizeof(double) * poff) == cudaSuccess &&
              cudaMalloc(&b->g_nat, sizeof(double) * poff) == cudaSuccess &&
              cudaMalloc(&b->m1, sizeof(double) * poff) == cudaSuccess &&
              cudaMalloc(&b->m2, sizeof(double) * poff) == cudaSuccess &&
              cudaMalloc(&b->out, sizeof(double) * 3 * nfits) == cudaSuccess &&
              cudaMalloc(&b->tau, sizeof(double) * MTGP_TMAX * nfits) == cudaSuccess &&
              cudaMalloc(&b->counters, sizeof(unsigned) * 2 * nfits) == cudaSuccess &&
              cudaMalloc(&b->pinfo, sizeof(int) * pinfo.size()) == cudaSuccess &&
              cudaMalloc(&b->tstep, sizeof(int)) == cudaSuccess;
    if (!ok) {
        mtgp_batch_destroy(b);
        return bfail(MTGP_ERR_CUDA, "batch allocation failed");
    }
    cudaMemcpy(b->pinfo, pinfo.data(), sizeof(int) * pinfo.size(), cudaMemcpyHostToDevice);
    cudaMemset(b->counters, 0, sizeof(unsigned) * 2 * nfits);
    cudaMemset(b->tstep, 0, sizeof(int));
    cudaMemset(b->th_nat, 0, sizeof(double) * poff);
    for (int i = 0; i < kSide; ++i) {
        cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&b->evjoin[i], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&b->evfork, cudaEventDisableTiming);
    int rc = build_plan(b);
    if (rc) {
        mtgp_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MTGP_OK;
}

int mtgp_batch_destroy(mtgp_batch_t* b) {
    if (!b) return MTGP_OK;
    cudaDeviceSynchronize();
    free_classes(b);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (auto* f : b->fits) mtgp_destroy(f);
    void* ptrs[] = {b->th_log, b->th_nat, b->g_nat, b->m1, b->m2, b->out, b->tau, b->partials, b->counters, b->pinfo,
                    b->tstep, b->descs, b->fdesc, b->pfeat, b->ppred, b->jcur, b->jcur_nat, b->jpred, b->jbest, b->jk,
                    b->is_s2};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < kSide; ++i) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->evjoin[i]) cudaEventDestroy(b->evjoin[i]);
    }
    if (b->evfork) cudaEventDestroy(b->evfork);
    delete b;
    return MTGP_OK;
}

int mtgp_batch_layout(const mtgp_batch_t* b, long long* param_offsets, long long* y_offsets) {
    if (!b || !param_offsets || !y_offsets) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    for (int f = 0; f <= b->nfits; ++f) {
        param_offsets[f] = b->poff[f];
        y_offsets[f] = b->yoff[f];
    }
    return MTGP_OK;
}

int mtgp_batch_set_y(mtgp_batch_t* b, const double* y, cudaStream_t st) {
    if (!b || !y) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    for (int f = 0; f < b->nfits; ++f) {
        int rc = mtgp_set_y(b->fits[f], y + b->yoff[f], st);
        if (rc) return rc;
    }
    return MTGP_OK;
}

int mtgp_batch_set_theta(mtgp_batch_t* b, const double* theta, cudaStream_t st) {
    if (!b || !theta) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    const int blocks = (int)std::min<long long>((b->np + 255) / 256, 4096);
    k_batch_theta_in<<<blocks, 256, 0, st>>>(theta, b->th_log, b->th_nat, b->pinfo, b->np, b->m1, b->m2);
    cudaMemsetAsync(b->tstep, 0, sizeof(int), st);
    return launch_status("mtgp_batch_set_theta");
}

int mtgp_batch_get_theta(mtgp_batch_t* b, double* theta, cudaStream_t st) {
    if (!b || !theta) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    cudaMemcpyAsync(theta, b->th_nat, sizeof(double) * b->np, cudaMemcpyDeviceToDevice, st);
    return MTGP_OK;
}

int mtgp_batch_nll_grad(mtgp_batch_t* b, double* nll, double* grad, cudaStream_t st) {
    if (!b) return bfail(MTGP_ERR_INVALID_ARG, "NULL handle");
    for (auto* f : b->fits)
        if (!f->h.y_set) return bfail(MTGP_ERR_STATE, "mtgp_batch_set_y must be called first");
    launch_eval(b, st);
    if (nll) {
        // out holds [NLL, quad, logdet] per fit
        cudaMemcpy2DAsync(nll, sizeof(double), b->out, 3 * sizeof(double), sizeof(double), b->nfits,
                          cudaMemcpyDeviceToDevice, st);
    }
    if (grad) cudaMemcpyAsync(grad, b->g_nat, sizeof(double) * b->np, cudaMemcpyDeviceToDevice, st);
    return launch_status("mtgp_batch_nll_grad");
}

int mtgp_batch_adam(mtgp_batch_t* b, int steps, double lr, int use_graph, double* trace, cudaStream_t st) {
    if (!b || steps < 1) return bfail(MTGP_ERR_INVALID_ARG, "NULL handle or steps < 1");
    for (auto* f : b->fits)
        if (!f->h.y_set) return bfail(MTGP_ERR_STATE, "mtgp_batch_set_y must be called first");
    if (!use_graph) {
        launch_steps(b, steps, lr, trace, st);
        return launch_status("mtgp_batch_adam");
    }
    if (!b->gexec || b->gsteps != steps || b->glr != lr || b->gtrace != trace) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t g;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return bfail(MTGP_ERR_CUDA, "cudaStreamBeginCapture failed (stream must be a non-default stream)");
        launch_steps(b, steps, lr, trace, st);
        if (cudaStreamEndCapture(st, &g) != cudaSuccess) return bfail(MTGP_ERR_CUDA, "graph capture failed");
        cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(MTGP_ERR_CUDA, "graph instantiation failed");
        b->gsteps = steps;
        b->glr = lr;
        b->gtrace = trace;
    }
    return cudaGraphLaunch(b->gexec, st) == cudaSuccess ? MTGP_OK : bfail(MTGP_ERR_CUDA, "graph launch failed");
}

int mtgp_batch_features(mtgp_batch_t* b, float* feat, cudaStream_t st) {
    if (!b || !feat) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    for (auto* f : b->fits)
        if (!f->h.y_set) return bfail(MTGP_ERR_STATE, "mtgp_batch_set_y must be called first");
    int rc = ensure_fdesc(b);
    if (rc) return rc;
    k_batch_features<<<b->nfits, 256, 0, st>>>(static_cast<const FeatDesc*>(b->fdesc), feat);
    return launch_status("mtgp_batch_features");
}

int mtgp_batch_targets(mtgp_batch_t* b, float* target, float* mask, cudaStream_t st) {
    if (!b || !target || !mask) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    int rc = ensure_fdesc(b);
    if (rc) return rc;
    k_batch_targets<<<(b->nfits + 127) / 128, 128, 0, st>>>(static_cast<const FeatDesc*>(b->fdesc), b->th_nat, b->nfits,
                                                            target, mask);
    return launch_status("mtgp_batch_targets");
}

int mtgp_batch_set_theta_proposal(mtgp_batch_t* b, const float* pred, cudaStream_t st) {
    if (!b || !pred) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    int rc = ensure_fdesc(b);
    if (rc) return rc;
    k_batch_propose<<<(b->nfits + 127) / 128, 128, 0, st>>>(static_cast<const FeatDesc*>(b->fdesc), pred, b->nfits,
                                                            b->th_log, b->th_nat, b->m1, b->m2);
    cudaMemsetAsync(b->tstep, 0, sizeof(int), st);
    return launch_status("mtgp_batch_set_theta_proposal");
}

int mtgp_batch_fit(mtgp_batch_t* b, const double* theta0, int steps, double lr, int use_graph, double* theta_out,
                   double* nll_out, double* trace, cudaStream_t st) {
    if (!b || steps < 1) return bfail(MTGP_ERR_INVALID_ARG, "NULL handle or steps < 1");
    if (!(lr > 0.0)) return bfail(MTGP_ERR_INVALID_ARG, "lr must be > 0");
    int rc;
    if (theta0) {
        rc = mtgp_batch_set_theta(b, theta0, st);
        if (rc) return rc;
    }
    rc = mtgp_batch_adam(b, steps, lr, use_graph, trace, st);
    if (rc) return rc;
    if (nll_out) {
        // the objective at the parameters the last step produced (one more batched evaluation)
        rc = mtgp_batch_nll_grad(b, nll_out, nullptr, st);
        if (rc) return rc;
    }
    if (theta_out) return mtgp_batch_get_theta(b, theta_out, st);
    return MTGP_OK;
}

int mtgp_propose(mtgp_batch_t* b, mtgp_mlp_t* net, float* pred, int judge, int* chosen, cudaStream_t st) {
    if (!b || !net) return bfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    if (judge < 0 || judge > 2) return bfail(MTGP_ERR_INVALID_ARG, "judge must be 0, 1 or 2");
    int in_w = 0, out_w = 0, max_b = 0;
    mlp_shape(net, &in_w, &out_w, &max_b);
    if (in_w != kFeat || out_w != kOut)
        return bfail(MTGP_ERR_INVALID_ARG, "the network must map 258 features to 37 outputs");
    for (auto* f : b->fits)
        if (!f->h.y_set) return bfail(MTGP_ERR_STATE, "mtgp_batch_set_y must be called first");
    int rc = ensure_fdesc(b);
    if (rc) return rc;
    if (!b->pfeat) {
        if (cudaMalloc(&b->pfeat, sizeof(float) * kFeat * (size_t)b->nfits) != cudaSuccess ||
            cudaMalloc(&b->ppred, sizeof(float) * kOut * (size_t)b->nfits) != cudaSuccess)
            return bfail(MTGP_ERR_CUDA, "proposal buffer allocation failed");
    }
    if (judge && !b->jcur) {
        std::vector<unsigned char> s2((size_t)b->np, 0);
        for (int f = 0; f < b->nfits; ++f) s2[(size_t)b->poff[f + 1] - 1] = 1;
        if (cudaMalloc(&b->jcur, sizeof(double) * b->np) != cudaSuccess ||
            cudaMalloc(&b->jcur_nat, sizeof(double) * b->np) != cudaSuccess ||
            cudaMalloc(&b->jpred, sizeof(double) * b->np) != cudaSuccess ||
            cudaMalloc(&b->jbest, sizeof(double) * b->nfits) != cudaSuccess ||
            cudaMalloc(&b->jk, sizeof(int) * b->nfits) != cudaSuccess ||
            cudaMalloc(&b->is_s2, (size_t)b->np) != cudaSuccess)
            return bfail(MTGP_ERR_CUDA, "proposal judge buffer allocation failed");
        cudaMemcpy(b->is_s2, s2.data(), (size_t)b->np, cudaMemcpyHostToDevice);
    }
    float* y = pred ? pred : b->ppred;
    if (judge) {
        cudaMemcpyAsync(b->jcur, b->th_log, sizeof(double) * b->np, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(b->jcur_nat, b->th_nat, sizeof(double) * b->np, cudaMemcpyDeviceToDevice, st);
    }
    k_batch_features<<<b->nfits, 256, 0, st>>>(static_cast<const FeatDesc*>(b->fdesc), b->pfeat);
    rc = launch_status("mtgp_propose (features)");
    if (rc) return rc;
    for (int r0 = 0; r0 < b->nfits; r0 += max_b) {
        const int rows = std::min(max_b, b->nfits - r0);
        rc = mtgp_mlp_forward(net, rows, b->pfeat + (size_t)r0 * kFeat, y + (size_t)r0 * kOut, st);
        if (rc) return rc;
    }
    rc = mtgp_batch_set_theta_proposal(b, y, st);
    if (rc || !judge) return rc;
    // the exact NLL judges the candidates; every fit keeps its best
    cudaMemcpyAsync(b->jpred, b->th_log, sizeof(double) * b->np, cudaMemcpyDeviceToDevice, st);
    const int blocks = (int)std::min<long long>((b->np + 255) / 256, 4096);
    // judge 1: all five candidates; judge 2: the quarter blend (p + 3 c) / 4 and c
    static const int kAll[kJudgeCand] = {0, 1, 2, 3, 4};
    static const int kBlend[2] = {3, 4};
    const int* cands = judge == 2 ? kBlend : kAll;
    const int ncand = judge == 2 ? 2 : kJudgeCand;
    for (int i = 0; i < ncand; ++i) {
        const int k = cands[i];
        k_judge_set<<<blocks, 256, 0, st>>>(k, nullptr, b->pinfo, b->is_s2, b->np, b->jcur, b->jcur_nat, b->jpred,
                                            b->th_log, b->th_nat, b->m1, b->m2);
        launch_eval(b, st);
        k_judge_keep<<<(b->nfits + 127) / 128, 128, 0, st>>>(k, i == 0, b->nfits, b->out, b->jbest, b->jk);
    }
    k_judge_set<<<blocks, 256, 0, st>>>(0, b->jk, b->pinfo, b->is_s2, b->np, b->jcur, b->jcur_nat, b->jpred,
                                        b->th_log, b->th_nat, b->m1, b->m2);
    cudaMemsetAsync(b->tstep, 0, sizeof(int), st);
    if (chosen) cudaMemcpyAsync(chosen, b->jk, sizeof(int) * b->nfits, cudaMemcpyDeviceToDevice, st);
    return launch_status("mtgp_propose (judge)");
}

int mtgp_batch_autotune(mtgp_batch_t* b, int reps, int* chosen, cudaStream_t st) {
    if (!b) return bfail(MTGP_ERR_INVALID_ARG, "NULL handle");
    for (auto* f : b->fits)
        if (!f->h.y_set) return bfail(MTGP_ERR_STATE, "mtgp_batch_set_y must be called first");
    if (reps < 1) reps = 3;
    const size_t dsz = fused_desc_size();
    std::vector<unsigned char> desc(dsz);
    std::map<std::tuple<int, int, int, int>, int> best;  // (kind, T, m, dbucket) -> split
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double* part = nullptr;
    unsigned* cnt = nullptr;
    long long partcap = 0;
    for (int f = 0; f < b->nfits; ++f) {
        const Handle& h = b->fits[f]->h;
        const int m = h.m[0];
        auto key = std::make_tuple(h.kind, h.T, m, dbucket(h.d));
        if (best.count(key)) continue;
        const long long o = b->poff[f];
        ThetaPtrs th{b->th_nat + o, b->th_nat + o + h.d, b->s, b->th_nat + o + h.d + (long long)h.T * b->s,
                     b->th_nat + o + h.d + (long long)h.T * b->s + h.T};
        float best_ms = 1e30f;
        int best_a = b->a[f];
        for (int a = 2; a <= m - 2; ++a) {
            int aa, lgL;
            if (!fused_plan(m, h.ncols, h.d, h.fp32, h.cplx, a, &aa, &lgL)) continue;
            const int NQ = 3 + h.T * (h.T + 1) / 2;
            const long long need = ((long long)1 << a) * (NQ + 1) + ((long long)1 << (m - a)) * h.d + NQ;
            if (need > partcap) {
                cudaFree(part);
                partcap = need;
                if (cudaMalloc(&part, sizeof(double) * partcap) != cudaSuccess) return bfail(MTGP_ERR_CUDA, "autotune scratch");
            }
            if (!cnt) {
                if (cudaMalloc(&cnt, 2 * sizeof(unsigned)) != cudaSuccess) return bfail(MTGP_ERR_CUDA, "autotune scratch");
                cudaMemset(cnt, 0, 2 * sizeof(unsigned));
            }
            fused_make_desc(&h, th, b->out + 3 * f, nullptr, b->g_nat + o, b->g_nat + o + h.d,
                            b->g_nat + o + h.d + (long long)h.T * b->s, b->g_nat + o + h.d + (long long)h.T * b->s + h.T,
                            true, a, part, cnt, desc.data());
            float tot = 0.f;
            for (int r = 0; r <= reps; ++r) {
                cudaEventRecord(e0, st);
                const int var = fused_variant(h.fp32, h.cplx, h.solve_df, h.d, m, a, false);
                for (int ph = 0; ph < 3; ++ph) {
                    const int grid = ph == 1 ? (1 << a) : (1 << (m - a));
                    fused_phase(ph, var, h.fp32, h.cplx, h.T, h.d, desc.data(), nullptr, nullptr, 0, grid,
                                fused_threads(ph, var, a, h.d, h.ncols, m),
                                fused_smem(ph, var, h.T, h.ncols, m, a, h.fp32, h.cplx), st);
                }
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (r > 0) tot += ms;  // first run warms up
            }
            if (tot < best_ms) {
                best_ms = tot;
                best_a = a;
            }
        }
        best[key] = best_a;
    }
    cudaFree(part);
    cudaFree(cnt);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int f = 0; f < b->nfits; ++f) {
        const Handle& h = b->fits[f]->h;
        b->a[f] = best[std::make_tuple(h.kind, h.T, h.m[0], dbucket(h.d))];
        if (chosen) chosen[f] = b->a[f];
    }
    return build_plan(b);
}

}  // extern "C"

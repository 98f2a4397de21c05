// Structures and helpers shared by the equal-size fused kernels: the generic path (k_fused.cu: any
// tile split, complex lattice spectra) and the register-tile path for real digital-net spectra
// (k_fused_rt.cu).  Everything lives in an anonymous namespace: each translation unit has its own copy.
#pragma once

#include <cstring>
#include <mutex>
#include <unordered_map>

#include "butterfly.cuh"
#include "freq_solve.cuh"

namespace {

template <typename S>
__device__ __forceinline__ S el_re(S x) { return x; }
template <typename S>
__device__ __forceinline__ S el_re(cx<S> x) { return x.re; }
struct FusedParams {
    int kind, d, T, C, gen_cols, m, a, lgL, grad, clamp, store_alpha, mtw, s, alpha;
    long long n, N;
    int colt[MTGP_MAX_COLS], colu[MTGP_MAX_COLS];
    int colidx[MTGP_TMAX][MTGP_TMAX];
    int order[MTGP_TMAX], rank[MTGP_TMAX];
};

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

// Column totals of one or two (nrows x ncols) partial arrays (fixed order): warp w sums columns
// w, w + nw, ... of the two arrays in turn; column q's lane l adds rows l, l + 32, ... (the loads of
// 8 rows are issued before their additions: one memory round trip per 8), then a shuffle tree.
__device__ void reduce_columns2(const double* part1, int nrows1, int ncols1, double* out1, const double* part2,
                                int nrows2, int ncols2, double* out2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int qq = warp; qq < ncols1 + ncols2; qq += nw) {
        const bool first = qq < ncols1;
        const double* part = first ? part1 : part2;
        const int nrows = first ? nrows1 : nrows2, ncols = first ? ncols1 : ncols2, q = first ? qq : qq - ncols1;
        double v = 0.0;
        for (int b0 = lane; b0 < nrows; b0 += 256) {
            double t[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int b = b0 + 32 * k;
                t[k] = b < nrows ? part[(long long)b * ncols + q] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) v += t[k];
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) (first ? out1 : out2)[q] = v;
    }
    __syncthreads();
}

__device__ void reduce_columns(const double* part, int nrows, int ncols, double* out) {
    reduce_columns2(part, nrows, ncols, out, nullptr, 0, 0, nullptr);
}

// last-block election: true in exactly one block, after all blocks have written their partials
__device__ bool last_block(unsigned* counter, unsigned nblocks) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == nblocks - 1);
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

// Everything one fit needs on the device: its parameters, theta / output pointers and buffers.
// Single-fit kernels take it by value; batched kernels read it from a device array.
struct FitDesc {
    FusedParams p;
    ThetaPtrs th;
    OutPtrs o;
    const uint32_t* gen;
    const uint32_t* shift;
    const void* tw;          // twiddles of the transform precision (lattices)
    void* spec;              // C x n spectra
    void* wgt;               // C x n adjoint weights
    const double* yhat;      // T x n observations, transformed
    const float2* yhat_df;   // the same as double-float pairs (FP32-transform digital nets), or null
    const uint32_t* rtw;     // design words of the register-tile kernels (rt_words_len layout), or null
    double* alpha;           // T x n Lambda^-1 rhat (posterior)
    const double* tau;       // T optimal means (sorted)
    double* partials;        // kernel B partials (nb x NQ), then kernel C partials (na x d)
    unsigned* counters;      // [0] B (NLL only), [1] C
    int* status;
    int na, nb;              // kernel A / C blocks, kernel B blocks
};

__device__ __forceinline__ int gq(int t, int u, int T) { return t * T - t * (t - 1) / 2 + (u - t); }

// Final outputs from the totals, written by all threads of the block (W and the sorted means are
// read into shared memory first, every output has its own thread).
// W_staged: W already in shared memory (caller staged it, with a barrier since), or null to load it here
__device__ void write_outputs(const double* tot, const double* etot, const FusedParams& p, const ThetaPtrs& th,
                              const double* tau_sorted, OutPtrs o, const double* W_staged = nullptr) {
    __shared__ double s_Wl[MTGP_TMAX * MTGP_TMAX];
    const double* s_W = W_staged ? W_staged : s_Wl;
    const int T = p.T, tid = threadIdx.x;
    const double LOG2PI = 1.8378770664093453;
    if (p.grad && !W_staged)
        for (int e = tid; e < T * th.s; e += blockDim.x) s_Wl[e] = th.W[e];
    if (tid == 0) {
        o.out[0] = 0.5 * (tot[0] + tot[1] + (double)p.N * LOG2PI);
        o.out[1] = tot[1];
        o.out[2] = tot[0];
    }
    if (o.tau && tid < T) o.tau[p.order[tid]] = tau_sorted[tid];
    if (!p.grad) return;
    __syncthreads();
    if (tid == 0) o.g_s2[0] = 0.5 * tot[2];
    if (tid < p.d) o.g_eta[tid] = 0.5 * etot[tid];
    for (int e = tid; e < T * th.s; e += blockDim.x) {
        const int tc = e / th.s, k = e - tc * th.s;
        const int t = p.rank[tc];
        double g = 0.0;
        for (int uc = 0; uc < T; ++uc) {
            const int u = p.rank[uc];
            const double G = (t <= u) ? tot[3 + gq(t, u, T)] : tot[3 + gq(u, t, T)];
            g += G * s_W[uc * th.s + k];
        }
        o.g_W[e] = g;
    }
    if (tid < T) o.g_v[tid] = 0.5 * tot[3 + gq(p.rank[tid], p.rank[tid], T)];
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

// chunk points as a table: s_z[j * 2^a + lo] = coordinate j of point base + lo (all threads call)
constexpr int kZTab = 2048;
__device__ __forceinline__ void chunk_table(int kind, int d, int a, const uint32_t* s_zhi, const uint32_t* s_gen,
                                            int gen_cols, uint32_t* s_z) {
    const int HA = 1 << a;
    for (int e = threadIdx.x; e < HA * d; e += blockDim.x) {
        const int j = e >> a, lo = e & (HA - 1);
        const uint32_t zl = point_word(kind, (uint32_t)lo, j, s_gen, gen_cols);
        s_z[e] = (kind == MTGP_LATTICE) ? s_zhi[j] + zl : (s_zhi[j] ^ zl);
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

// Programmatic dependent launch.  The wait returns once the grids this one depends on have finished
// and their writes are visible (at once when the launch did not allow early start); the trigger lets
// the next grid in the stream begin its independent prologue.  A, B and C each put the work that
// reads only handle constants (design words, task covariance, observations) before the wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// parameters that are non-finite or negative (eta, v, sigma2) flag ST_NUMERIC; run by block 0 of A
__device__ __forceinline__ void check_theta_block(const ThetaPtrs& th, int d, int T, int* status) {
    int bad = 0;
    for (int j = threadIdx.x; j < d; j += blockDim.x)
        if (!isfinite(th.eta[j]) || th.eta[j] < 0.0) bad = 1;
    for (int e = threadIdx.x; e < T * th.s; e += blockDim.x)
        if (!isfinite(th.W[e])) bad = 1;
    for (int t = threadIdx.x; t < T; t += blockDim.x)
        if (!isfinite(th.v[t]) || th.v[t] < 0.0) bad = 1;
    if (threadIdx.x == 0 && (!isfinite(th.sigma2[0]) || th.sigma2[0] < 0.0)) bad = 1;
    if (bad) set_status(status, ST_NUMERIC);
}

// ---------------------------------------------------------------------------------- host helpers

size_t elem_size_of(bool fp32, bool cplx) { return (fp32 ? 4 : 8) * (cplx ? 2 : 1); }

// Raise a kernel's dynamic shared-memory limit to `bytes` (the default limit counts static shared
// memory too, so any dynamic size may need it); remembered per kernel so each value is set once.
std::mutex g_smem_mu;
std::unordered_map<const void*, size_t> g_smem_set;

template <typename F>
void set_smem(F* fn, size_t bytes) {
    if (bytes == 0) return;
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t& cur = g_smem_set[reinterpret_cast<const void*>(fn)];
    if (bytes > cur) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        cur = bytes;
    }
}

// a single-fit launch that may start while the previous kernel in the stream finishes
template <typename... KArgs>
void launch_pdl(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t st, const FitDesc& f) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, f);
}

}  // namespace

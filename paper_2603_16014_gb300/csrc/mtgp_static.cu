// An NLL entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running where allocation is forbidden or unsafe (inside a
// region that must not synchronise the device, an allocator callback, a plugin host that owns the
// device heap, or a process that has already reserved all free memory for its own pool).  For them,
// mtgp_nll_equal_static evaluates the equal-size fast-MTGP NLL with every intermediate placed in one
// file-scope device array of fixed size, MTGP_STATIC_SCRATCH_BYTES, which the library image carries
// and every GPU that loads the library holds until the process exits.
//
// The host code here never passes the array's name to a kernel (in host code that name is only a
// host-side stand-in for the symbol): the first call on each device, with that device current, looks
// up the device address with cudaGetSymbolAddress and every later call on that device reuses it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "mtgp_internal.cuh"

#define MTGP_STATIC_SCRATCH_BYTES (8u << 20)
#define MTGP_STATIC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_static_scratch[MTGP_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
unsigned char* g_static_ptr[MTGP_STATIC_MAX_DEVICES] = {nullptr};

int static_fail(int code, const char* msg) {
    mtgp_set_error(msg);
    return code;
}

// device address of the scratch array on the current device (looked up once per device)
int scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(MTGP_ERR_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= MTGP_STATIC_MAX_DEVICES) return static_fail(MTGP_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return static_fail(MTGP_ERR_CUDA, msg);
        }
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return MTGP_OK;
}

struct StaticDesc {
    uint32_t gen[MTGP_MAX_DIM * 32];
    uint32_t shift[MTGP_TMAX * MTGP_MAX_DIM];
    long long yoffs[MTGP_TMAX];
    int ngen, nshift, T;
};

// writes the design description into the scratch array and clears what must start at zero
__global__ void k_static_setup(StaticDesc desc, uint32_t* gen, uint32_t* shift, long long* yoffs, unsigned* counters,
                               int* status) {
    for (int i = threadIdx.x; i < desc.ngen; i += blockDim.x) gen[i] = desc.gen[i];
    for (int i = threadIdx.x; i < desc.nshift; i += blockDim.x) shift[i] = desc.shift[i];
    if (threadIdx.x < desc.T) yoffs[threadIdx.x] = desc.yoffs[threadIdx.x];
    if (threadIdx.x < 4) counters[threadIdx.x] = 0u;
    if (status && threadIdx.x == 0) *status = 0;
}

// optimal means for equal sizes: tau_t = yhat_t(0) / sqrt(n) (sample means)
__global__ void k_static_tau(const double* yhat, double* tau_sorted, int T, long long n, int cplx) {
    int t = threadIdx.x;
    if (t < T) tau_sorted[t] = yhat[(cplx ? 2 : 1) * (long long)t * n] / sqrt((double)n);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int mtgp_nll_equal_static(int kind, int d, int T, int m, const uint32_t* gen, int gen_cols,
                                     const uint32_t* shift, int precision, const double* y, const double* eta,
                                     const double* W, int s, const double* v, const double* sigma2, double* out,
                                     double* tau, int* status, cudaStream_t stream) {
    // ---- host-side validation (no device work before it passes)
    if (kind != MTGP_LATTICE && kind != MTGP_DNET) return static_fail(MTGP_ERR_INVALID_ARG, "kind must be MTGP_LATTICE or MTGP_DNET");
    if (d < 1 || d > MTGP_MAX_DIM) return static_fail(MTGP_ERR_INVALID_ARG, "d out of range [1, MTGP_MAX_DIM]");
    if (T < 1 || T > MTGP_MAX_TASKS) return static_fail(MTGP_ERR_INVALID_ARG, "T out of range [1, MTGP_MAX_TASKS]");
    if (m < 4 || m > MTGP_MAX_M) return static_fail(MTGP_ERR_INVALID_ARG, "m must satisfy 4 <= m <= MTGP_MAX_M");
    if (precision != MTGP_FP64 && precision != MTGP_FP32_TRANSFORM)
        return static_fail(MTGP_ERR_INVALID_ARG, "precision must be MTGP_FP64 or MTGP_FP32_TRANSFORM");
    if (kind == MTGP_DNET && (gen_cols < m || gen_cols > 32))
        return static_fail(MTGP_ERR_INVALID_ARG, "gen_cols must satisfy m <= gen_cols <= 32");
    if (!gen || !shift || !y || !eta || !W || !v || !sigma2 || !out)
        return static_fail(MTGP_ERR_INVALID_ARG, "NULL argument");
    if (s < 1 || s > T) return static_fail(MTGP_ERR_INVALID_ARG, "s must satisfy 1 <= s <= T");

    // ---- a host-side handle whose device pointers all point into the scratch array
    Handle h;
    std::memset(&h, 0, sizeof(h));
    h.smooth = 2;
    h.kind = kind;
    h.d = d;
    h.T = T;
    h.prec = precision;
    h.fp32 = precision == MTGP_FP32_TRANSFORM;
    h.solve_df = h.fp32;
    h.cplx = kind == MTGP_LATTICE;
    h.equal = true;
    h.gen_cols = kind == MTGP_DNET ? gen_cols : 1;
    h.mmax = m;
    const long long n = 1LL << m;
    for (int t = 0; t < T; ++t) {
        h.m_user[t] = m;
        h.order[t] = t;
        h.rank[t] = t;
        h.m[t] = m;
        h.n[t] = n;
        h.yoff[t] = (long long)t * n;
    }
    h.N = n * T;
    int c = 0;
    h.cols[c++] = ColDesc{0, (int)n, 0, 0};
    for (int t = 0; t < T; ++t) h.col_of[t][t] = 0;
    for (int t = 0; t < T; ++t)
        for (int u = t + 1; u < T; ++u) {
            h.cols[c] = ColDesc{(long long)c * n, (int)n, t, u};
            h.col_of[t][u] = c;
            ++c;
        }
    h.ncols = c;
    h.col_elems = (long long)c * n;
    if (!fused_supported(&h)) return static_fail(MTGP_ERR_UNSUPPORTED, "this size is not handled by the fused kernels");

    const size_t es = (h.fp32 ? 4 : 8) * (h.cplx ? 2 : 1);
    const size_t vs = h.cplx ? 2 : 1;
    const size_t half = (size_t)1 << (m - 1);
    const int ngen = kind == MTGP_LATTICE ? d : d * gen_cols;
    size_t off = 0;
    const size_t o_gen = off;      off = align256(off + sizeof(uint32_t) * ngen);
    const size_t o_shift = off;    off = align256(off + sizeof(uint32_t) * T * d);
    const size_t o_yoffs = off;    off = align256(off + sizeof(long long) * T);
    const size_t o_tw64 = off;     off = align256(off + 2 * sizeof(double) * half);
    const size_t o_tw32 = off;     off = align256(off + 2 * sizeof(float) * half);
    const size_t o_yhat = off;     off = align256(off + sizeof(double) * vs * h.N);
    const size_t o_spec = off;     off = align256(off + es * h.col_elems);
    const size_t o_part = off;     off = align256(off + sizeof(double) * fused_partials_len(&h));
    const size_t o_tau = off;      off = align256(off + sizeof(double) * MTGP_TMAX);
    const size_t o_cnt = off;      off = align256(off + sizeof(unsigned) * 4);
    const size_t o_stat = off;     off = align256(off + sizeof(int));
    if (off > MTGP_STATIC_SCRATCH_BYTES) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "problem needs %zu bytes of scratch; the static scratch array holds %u bytes",
                      off, (unsigned)MTGP_STATIC_SCRATCH_BYTES);
        return static_fail(MTGP_ERR_INVALID_ARG, msg);
    }

    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    h.gen = reinterpret_cast<uint32_t*>(base + o_gen);
    h.shift = reinterpret_cast<uint32_t*>(base + o_shift);
    h.yoffs_dev = reinterpret_cast<long long*>(base + o_yoffs);
    h.twid = base + o_tw64;
    h.twid32 = base + o_tw32;
    h.yhat = reinterpret_cast<double*>(base + o_yhat);
    h.spec = base + o_spec;
    h.wgt = base + o_spec;  // unused by the NLL-only kernels
    h.partials = reinterpret_cast<double*>(base + o_part);
    h.tau = reinterpret_cast<double*>(base + o_tau);
    h.counters = reinterpret_cast<unsigned*>(base + o_cnt);
    h.status = status ? status : reinterpret_cast<int*>(base + o_stat);
    h.prof = nullptr;

    StaticDesc desc;
    std::memset(&desc, 0, sizeof(desc));
    std::memcpy(desc.gen, gen, sizeof(uint32_t) * ngen);
    std::memcpy(desc.shift, shift, sizeof(uint32_t) * T * d);
    for (int t = 0; t < T; ++t) desc.yoffs[t] = h.yoff[t];
    desc.ngen = ngen;
    desc.nshift = T * d;
    desc.T = T;
    k_static_setup<<<1, 256, 0, stream>>>(desc, h.gen, h.shift, h.yoffs_dev, h.counters, h.status);
    launch_twiddles(&h, stream);
    launch_y_load(&h, y, stream);
    k_static_tau<<<1, 32, 0, stream>>>(h.yhat, h.tau, T, n, h.cplx ? 1 : 0);
    ThetaPtrs th{eta, W, s, v, sigma2};
    launch_fused(&h, th, false, false, out, tau, nullptr, nullptr, nullptr, nullptr, stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        std::snprintf(msg, sizeof(msg), "kernel launch: %s", cudaGetErrorString(e));
        return static_fail(MTGP_ERR_CUDA, msg);
    }
    return MTGP_OK;
}

// Fast transforms V_m^dagger (Theorem "fast MTGP computations", closing sentence):
//   digital nets: unnormalised Walsh-Hadamard transform (FWHT);
//   lattices:     DFT of the bit-reversed vector, FFT(bitrev(a)).
// Both are the same radix-2 butterfly network.  Data arrive in radical-inverse order, which is
// already the bit-reversed order a decimation-in-time network wants, so the forward transform
// (DIT) runs with no permutation and writes natural frequency order.  Its transpose, the
// decimation-in-frequency network (DIF), maps natural order to bit-reversed order; it serves the
// adjoint (gradient) and the inverse transform V.
//
// A transform of length 2^m runs as one or two passes.  A pass covers butterfly stages
// [s0, s1): the elements whose indices differ only in bits s0..s1-1 form a group of 2^(s1-s0)
// values, staged in shared memory.  A CTA holds L groups with consecutive low indices so its
// global loads and stores are contiguous runs of L elements.
#include <cstdio>

#include "butterfly.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxTileBytes = 64 * 1024;

template <typename S, bool CPLX, bool DIF>
__global__ void __launch_bounds__(kThreads)
k_xform_pass(typename El<S, CPLX>::T* __restrict__ base, const long long* __restrict__ offs, int m,
             int s0, int s1, int lgL, const cx<S>* __restrict__ tw, int mtw) {
    using E = typename El<S, CPLX>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    E* buf = reinterpret_cast<E*>(smem_raw);
    const int lgH = s1 - s0;
    const int H = 1 << lgH;
    const int L = 1 << lgL;
    const int lotiles_lg = s0 - lgL;
    const long long tile = blockIdx.x;
    E* a = base + offs[blockIdx.y];
    const long long lo0 = (tile & ((1LL << lotiles_lg) - 1)) << lgL;
    const long long hibase = (tile >> lotiles_lg) << s1;
    for (int e = threadIdx.x; e < H * L; e += blockDim.x) {
        int h = e >> lgL, lo = e & (L - 1);
        buf[e] = a[hibase + ((long long)h << s0) + lo0 + lo];
    }
    __syncthreads();
    smem_stages<S, CPLX, DIF>(buf, 1, H * L, lgH, lgL, s0, lo0, tw, mtw);
    for (int e = threadIdx.x; e < H * L; e += blockDim.x) {
        int h = e >> lgL, lo = e & (L - 1);
        a[hibase + ((long long)h << s0) + lo0 + lo] = buf[e];
    }
}

template <typename S, bool CPLX, bool DIF>
void run_pass(void* base, const long long* offs, int narr, int m, int s0, int s1, const void* tw, int mtw,
              cudaStream_t st) {
    using E = typename El<S, CPLX>::T;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_xform_pass<S, CPLX, DIF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kMaxTileBytes);
        attr_set = true;
    }
    const int lgH = s1 - s0;
    int lgL = 0;
    while (lgL < s0 && ((size_t)sizeof(E) << (lgH + lgL + 1)) <= (size_t)kMaxTileBytes && lgL < 4) ++lgL;
    const size_t smem = sizeof(E) << (lgH + lgL);
    const long long tiles = 1LL << ((m - s1) + (s0 - lgL));
    dim3 grid((unsigned)tiles, (unsigned)narr);
    int threads = kThreads;
    if ((1 << (lgH + lgL - 1)) < threads) threads = (1 << (lgH + lgL - 1)) < 32 ? 32 : (1 << (lgH + lgL - 1));
    k_xform_pass<S, CPLX, DIF><<<grid, threads, smem, st>>>(reinterpret_cast<E*>(base), offs, m, s0, s1, lgL,
                                                             reinterpret_cast<const cx<S>*>(tw), mtw);
}

template <typename S, bool CPLX>
void run_transform(void* base, const long long* offs, int narr, int m, bool dif, const void* tw, int mtw,
                   cudaStream_t st) {
    if (m <= 0 || narr <= 0) return;
    const int maxlg = 12;
    if (m <= maxlg) {
        if (dif) run_pass<S, CPLX, true>(base, offs, narr, m, 0, m, tw, mtw, st);
        else run_pass<S, CPLX, false>(base, offs, narr, m, 0, m, tw, mtw, st);
        return;
    }
    const int a = m / 2;
    if (!dif) {
        run_pass<S, CPLX, false>(base, offs, narr, m, 0, a, tw, mtw, st);
        run_pass<S, CPLX, false>(base, offs, narr, m, a, m, tw, mtw, st);
    } else {
        run_pass<S, CPLX, true>(base, offs, narr, m, a, m, tw, mtw, st);
        run_pass<S, CPLX, true>(base, offs, narr, m, 0, a, tw, mtw, st);
    }
}

__global__ void k_twiddles(cx<double>* tw64, cx<float>* tw32, int mtw) {
    long long half = 1LL << (mtw - 1);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < half;
         k += (long long)gridDim.x * blockDim.x) {
        double s, c;
        // e^{-2 pi i k / 2^mtw} = cos(pi x) - i sin(pi x), x = k / 2^(mtw-1)
        sincospi((double)k / (double)half, &s, &c);
        tw64[k] = mk(c, -s);
        tw32[k] = mk((float)c, (float)-s);
    }
}

}  // namespace

void launch_transform(const Handle* h, void* base, bool fp32, bool complex_data, int m, const long long* offs_dev,
                      int narr, bool dif, cudaStream_t st) {
    if (fp32) {
        if (complex_data) run_transform<float, true>(base, offs_dev, narr, m, dif, h->twid32, h->mmax, st);
        else run_transform<float, false>(base, offs_dev, narr, m, dif, h->twid32, h->mmax, st);
    } else {
        if (complex_data) run_transform<double, true>(base, offs_dev, narr, m, dif, h->twid, h->mmax, st);
        else run_transform<double, false>(base, offs_dev, narr, m, dif, h->twid, h->mmax, st);
    }
}

void launch_twiddles(Handle* h, cudaStream_t st) {
    if (h->mmax < 1) return;
    long long half = 1LL << (h->mmax - 1);
    int blocks = (int)((half + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_twiddles<<<blocks, 256, 0, st>>>(reinterpret_cast<cx<double>*>(h->twid), reinterpret_cast<cx<float>*>(h->twid32),
                                       h->mmax);
}

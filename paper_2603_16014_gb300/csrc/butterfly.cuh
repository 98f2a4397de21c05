// Radix-2 butterfly networks on values staged in shared memory, shared by the fused kernels and the
// general transform.  Forward (DIT): x1 + w x2, x1 - w x2; transposed (DIF): x1 + x2, (x1 - x2) w, with
// w = e^{-2 pi i e / 2^(s+1)} taken from a table of 2^(mtw-1) entries (complex data only; the
// Walsh-Hadamard transform of real data has w = 1).
#pragma once

#include "mtgp_internal.cuh"

namespace {

template <typename S, bool CPLX>
struct El;
template <typename S>
struct El<S, false> { using T = S; };
template <typename S>
struct El<S, true> { using T = cx<S>; };

template <typename S>
__device__ __forceinline__ S bmul(S x, cx<S>) { return x; }
template <typename S>
__device__ __forceinline__ cx<S> bmul(cx<S> x, cx<S> w) { return x * w; }

// butterfly stages s0 .. s0+lgH-1 (DIT ascending, DIF descending) over groups of 2^lgH values spaced
// L apart in shared memory, for `ncol` columns stored back to back (colstride elements).  Two stages
// run per pass: a thread loads the 4 values two consecutive stages combine, applies both stages in
// registers (the same operations in the same order as two separate stages) and stores them back,
// halving shared-memory passes and barriers; an odd stage count leaves one single-stage pass.
template <typename S, bool CPLX, bool DIF>
__device__ __forceinline__ void smem_stage1(typename El<S, CPLX>::T* buf, int ncol, int colstride, int lgH, int lgL,
                                            int s0, long long lo0, const cx<S>* tw, int mtw, int s) {
    using E = typename El<S, CPLX>::T;
    const int L = 1 << lgL;
    const int lgnb = lgH + lgL - 1;
    const int nb = 1 << lgnb;
    const int ls = s - s0;
    for (int e = threadIdx.x; e < nb * ncol; e += blockDim.x) {
        const int c = e >> lgnb;
        const int b = e & (nb - 1);
        const int lo = b & (L - 1);
        const int hb = b >> lgL;
        const int hlo = hb & ((1 << ls) - 1);
        const int h1 = ((hb >> ls) << (ls + 1)) | hlo;
        const int h2 = h1 + (1 << ls);
        E* col = buf + (long long)c * colstride;
        E x1 = col[(h1 << lgL) + lo];
        E x2 = col[(h2 << lgL) + lo];
        cx<S> w;
        if (CPLX) w = tw[(lo0 + lo + ((long long)hlo << s0)) << (mtw - 1 - s)];
        if (!DIF) {
            E t = bmul(x2, w);
            col[(h1 << lgL) + lo] = x1 + t;
            col[(h2 << lgL) + lo] = x1 - t;
        } else {
            col[(h1 << lgL) + lo] = x1 + x2;
            col[(h2 << lgL) + lo] = bmul(x1 - x2, w);
        }
    }
}

// stages sl (relative ls) and sl + 1 in one pass
template <typename S, bool CPLX, bool DIF>
__device__ __forceinline__ void smem_stage2(typename El<S, CPLX>::T* buf, int ncol, int colstride, int lgH, int lgL,
                                            int s0, long long lo0, const cx<S>* tw, int mtw, int sl) {
    using E = typename El<S, CPLX>::T;
    const int L = 1 << lgL;
    const int lgng = lgH + lgL - 2;
    const int ng = 1 << lgng;
    const int ls = sl - s0;
    for (int e = threadIdx.x; e < ng * ncol; e += blockDim.x) {
        const int c = e >> lgng;
        const int g = e & (ng - 1);
        const int lo = g & (L - 1);
        const int hb = g >> lgL;
        const int hlo = hb & ((1 << ls) - 1);
        const int h0 = ((hb >> ls) << (ls + 2)) | hlo;
        E* col = buf + (long long)c * colstride;
        const int i0 = (h0 << lgL) + lo, step = 1 << (ls + lgL);
        E x0 = col[i0], x1 = col[i0 + step], x2 = col[i0 + 2 * step], x3 = col[i0 + 3 * step];
        cx<S> wa, wb, wc;
        if (CPLX) {
            const long long pos = lo0 + lo + ((long long)hlo << s0);
            const long long pos1 = lo0 + lo + ((long long)(hlo + (1 << ls)) << s0);
            wa = tw[pos << (mtw - 1 - sl)];        // stage sl, both pairs
            wb = tw[pos << (mtw - 2 - sl)];        // stage sl + 1, pair (x0, x2)
            wc = tw[pos1 << (mtw - 2 - sl)];       // stage sl + 1, pair (x1, x3)
        }
        if (!DIF) {
            E t = bmul(x1, wa);
            E y0 = x0 + t, y1 = x0 - t;
            t = bmul(x3, wa);
            E y2 = x2 + t, y3 = x2 - t;
            t = bmul(y2, wb);
            col[i0] = y0 + t;
            col[i0 + 2 * step] = y0 - t;
            t = bmul(y3, wc);
            col[i0 + step] = y1 + t;
            col[i0 + 3 * step] = y1 - t;
        } else {
            E y0 = x0 + x2, y2 = bmul(x0 - x2, wb);
            E y1 = x1 + x3, y3 = bmul(x1 - x3, wc);
            col[i0] = y0 + y1;
            col[i0 + step] = bmul(y0 - y1, wa);
            col[i0 + 2 * step] = y2 + y3;
            col[i0 + 3 * step] = bmul(y2 - y3, wa);
        }
    }
}

template <typename S, bool CPLX, bool DIF>
__device__ __forceinline__ void smem_stages(typename El<S, CPLX>::T* buf, int ncol, int colstride, int lgH, int lgL,
                                            int s0, long long lo0, const cx<S>* tw, int mtw) {
    if (!DIF) {
        int st = 0;
        for (; st + 1 < lgH; st += 2) {
            smem_stage2<S, CPLX, false>(buf, ncol, colstride, lgH, lgL, s0, lo0, tw, mtw, s0 + st);
            __syncthreads();
        }
        if (st < lgH) {
            smem_stage1<S, CPLX, false>(buf, ncol, colstride, lgH, lgL, s0, lo0, tw, mtw, s0 + st);
            __syncthreads();
        }
    } else {
        int st = lgH;  // stages still to run: s0 + st - 1 down to s0
        for (; st >= 2; st -= 2) {
            smem_stage2<S, CPLX, true>(buf, ncol, colstride, lgH, lgL, s0, lo0, tw, mtw, s0 + st - 2);
            __syncthreads();
        }
        if (st == 1) {
            smem_stage1<S, CPLX, true>(buf, ncol, colstride, lgH, lgL, s0, lo0, tw, mtw, s0);
            __syncthreads();
        }
    }
}

}  // namespace

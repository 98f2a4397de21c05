// Element-wise evaluation of the library's own arithmetic building blocks, so that tests can check
// their error bounds against FP64 references: the FP64 reciprocal of the per-frequency solvers and the
// double-float operations of the FP32-transform solve and of the double-float kernel values.
#include "freq_solve.cuh"
#include "kernel_df.cuh"

namespace {

__global__ void k_selftest_arith(int op, long long n, const double* __restrict__ x, const double* __restrict__ y,
                                 double* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = x[i], b = y ? y[i] : 0.0;
        double r = 0.0;
        switch (op) {
            case 0: r = fast_rcp(a); break;
            case 1: r = df_to_double(df_from_double(a)); break;
            case 2: r = df_to_double(df_rcp(df_from_double(a))); break;
            case 3: r = df_to_double(df_mul(df_from_double(a), df_from_double(b))); break;
            case 4: r = df_to_double(df_add(df_from_double(a), df_from_double(b))); break;
            case 5: r = df_to_double(df_fms(df_from_double(a), df_from_double(b), df_from_double(b))); break;
            case 7: r = df_to_double(dsi2_scaled_df((uint32_t)a)); break;
            case 8: r = df_to_double(si2_df((uint32_t)a, si2_consts((int)b))); break;
            case 6: {
                // log of the product of x over each warp's 32 consecutive elements (DFLogAcc and its
                // double-float logarithm), in the warp's first element; the other elements receive 0
                DFLogAcc acc;
                acc.init();
                acc.mul(df_from_double(a));
                acc.warp_product();
                r = (threadIdx.x & 31) == 0 ? df_to_double(acc.log_df()) : 0.0;
            }
        }
        out[i] = r;
    }
}

}  // namespace

extern "C" int mtgp_selftest_arith(int op, long long n, const double* x, const double* y, double* out,
                                   cudaStream_t stream) {
    if (op < 0 || op > 8 || n < 0 || (n > 0 && (!x || !out)) || ((op == 3 || op == 4 || op == 5 || op == 8) && n > 0 && !y)) {
        mtgp_set_error("mtgp_selftest_arith: bad arguments");
        return MTGP_ERR_INVALID_ARG;
    }
    if (op == 6 && n % 32 != 0) {
        mtgp_set_error("mtgp_selftest_arith: op 6 needs a multiple of 32 elements");
        return MTGP_ERR_INVALID_ARG;
    }
    if (n == 0) return MTGP_OK;
    // op 6 keeps whole warps on consecutive elements: one pass, blocks of 256 threads
    long long blocks = (n + 255) / 256;
    if (op != 6 && blocks > 4096) blocks = 4096;
    k_selftest_arith<<<(unsigned)blocks, 256, 0, stream>>>(op, n, x, y, out);
    return cudaGetLastError() == cudaSuccess ? MTGP_OK : MTGP_ERR_CUDA;
}

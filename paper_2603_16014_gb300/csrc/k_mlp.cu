// Small MLP with BF16 weights and FP32 accumulation: forward, backward and Adam, all on the GPU.
//
// It maps a fit's spectral summary to initial hyper-parameters (the learned proposal).  Layers
// h_{l+1} = act(h_l W_l^T + b_l), ReLU on hidden layers.  GEMMs are C = A B^T with A (M x K) and
// B (N x K) BF16 row-major and FP32 accumulation on the tensor cores (mma.sync m16n8k16); all
// dimensions are padded on the host to the tile sizes (M, N to 64, K to 32) with zero rows and
// columns, so the kernels need no bounds tests and padded entries stay exactly zero.
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "mtgp_internal.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 32;
constexpr int SKP = TK + 8;  // padded smem row (bf16) to spread banks

__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

// C[M x N] = A[M x K] B[N x K]^T (+ bias[N]) (ReLU) ; writes FP32 C and optionally a BF16 copy
__global__ void __launch_bounds__(128)
k_gemm_nt(const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B, int ldb,
          float* __restrict__ C, int ldc, __nv_bfloat16* __restrict__ Cb, int ldcb, const float* __restrict__ bias,
          int relu, int K) {
    __shared__ __align__(16) __nv_bfloat16 sA[TM][SKP];
    __shared__ __align__(16) __nv_bfloat16 sB[TN][SKP];
    const int bm = blockIdx.y * TM, bn = blockIdx.x * TN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // warp tile 32 x 32
    const int g = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = 0; k0 < K; k0 += TK) {
        // 64 x 32 bf16 per operand = 1024 pairs; 128 threads x 8 pairs
        for (int e = threadIdx.x; e < TM * TK / 2; e += blockDim.x) {
            const int r = e / (TK / 2), c = (e % (TK / 2)) * 2;
            *reinterpret_cast<unsigned*>(&sA[r][c]) = ld_pair(A + (long long)(bm + r) * lda + k0 + c);
            *reinterpret_cast<unsigned*>(&sB[r][c]) = ld_pair(B + (long long)(bn + r) * ldb + k0 + c);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; kk += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r0 = wm + i * 16;
                af[i][0] = ld_pair(&sA[r0 + g][kk + tq * 2]);
                af[i][1] = ld_pair(&sA[r0 + g + 8][kk + tq * 2]);
                af[i][2] = ld_pair(&sA[r0 + g][kk + 8 + tq * 2]);
                af[i][3] = ld_pair(&sA[r0 + g + 8][kk + 8 + tq * 2]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c0 = wn + j * 8;
                bf[j][0] = ld_pair(&sB[c0 + g][kk + tq * 2]);
                bf[j][1] = ld_pair(&sB[c0 + g][kk + 8 + tq * 2]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                        "{%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = bm + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int col = bn + wn + j * 8 + tq * 2 + (r & 1);
                float v = acc[i][j][r];
                if (bias) v += bias[col];
                if (relu) v = v > 0.f ? v : 0.f;
                C[(long long)row * ldc + col] = v;
                if (Cb) Cb[(long long)row * ldcb + col] = __float2bfloat16(v);
            }
}

// out[c][r] = in[r][c] (rows x cols, FP32 or BF16 in, BF16 out)
template <typename Tin>
__global__ void k_transpose_bf16(const Tin* __restrict__ in, int ldi, __nv_bfloat16* __restrict__ out, int ldo, int rows,
                                 int cols) {
    __shared__ float tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? (float)in[(long long)r * ldi + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[(long long)c * ldo + r] = __float2bfloat16(tile[threadIdx.x][i]);
    }
}

// out row r = standardised input row (sel ? sel[r] : r), zero in the padded columns
__global__ void k_to_bf16(const float* __restrict__ in, int ldi, const int* __restrict__ sel,
                          __nv_bfloat16* __restrict__ out, int ldo, int rows, int cols, int cols_pad,
                          const float* __restrict__ mu, const float* __restrict__ isd) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * cols_pad;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols_pad), c = (int)(e % cols_pad);
        float v = 0.f;
        if (c < cols) {
            const long long src = sel ? sel[r] : r;
            v = (in[src * ldi + c] - mu[c]) * isd[c];
        }
        out[(long long)r * ldo + c] = __float2bfloat16(v);
    }
}

// per input column: mean and 1 / max(standard deviation, 1e-3) over rows (FP64 sums)
__global__ void k_scaling(const float* __restrict__ x, int rows, int cols, float* __restrict__ mu,
                          float* __restrict__ isd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0, q = 0.0;
    for (int r = 0; r < rows; ++r) {
        const double v = x[(long long)r * cols + c];
        s += v;
        q += v * v;
    }
    const double mean = s / rows;
    double var = q / rows - mean * mean;
    var = var > 0.0 ? var : 0.0;
    const double sd = sqrt(var);
    mu[c] = (float)mean;
    isd[c] = (float)(1.0 / (sd > 1e-3 ? sd : 1e-3));
}

// dZ = 2 mask (out - target) / count over the real batch rows and output columns (padded rows 0);
// one block; also the loss
__global__ void k_loss_grad(const float* __restrict__ out, int ldo, const float* __restrict__ tgt,
                            const float* __restrict__ mask, const int* __restrict__ sel, int rows, int cols,
                            int rows_pad, int cols_pad, float* __restrict__ dz, __nv_bfloat16* __restrict__ dzb,
                            float* loss) {
    __shared__ float s_cnt[32], s_l[32];
    float cnt = 0.f, l = 0.f;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
        const int r = e / cols, c = e % cols;
        const long long src = (sel ? (long long)sel[r] : (long long)r) * cols + c;
        const float m = mask[src];
        const float df = out[(long long)r * ldo + c] - tgt[src];
        cnt += m;
        l += m * df * df;
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
        l += __shfl_down_sync(0xffffffffu, l, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_cnt[threadIdx.x >> 5] = cnt;
        s_l[threadIdx.x >> 5] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float c = 0.f, ll = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            c += s_cnt[w];
            ll += s_l[w];
        }
        s_cnt[0] = c > 1.f ? c : 1.f;
        if (loss) *loss = ll / s_cnt[0];
    }
    __syncthreads();
    const float inv = 1.f / s_cnt[0];
    for (int e = threadIdx.x; e < rows_pad * cols_pad; e += blockDim.x) {
        const int r = e / cols_pad, c = e % cols_pad;
        float g = 0.f;
        if (r < rows && c < cols) {
            const long long src = (sel ? (long long)sel[r] : (long long)r) * cols + c;
            g = 2.f * mask[src] * (out[(long long)r * ldo + c] - tgt[src]) * inv;
        }
        dz[e] = g;
        dzb[e] = __float2bfloat16(g);
    }
}

// dZ = dH * (Z > 0)
__global__ void k_relu_back(const float* __restrict__ dh, const float* __restrict__ z, float* __restrict__ dz,
                            __nv_bfloat16* __restrict__ dzb, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float g = z[e] > 0.f ? dh[e] : 0.f;
        dz[e] = g;
        dzb[e] = __float2bfloat16(g);
    }
}

// db[c] = sum_r dz[r][c]
__global__ void k_colsum(const float* __restrict__ dz, int rows, int cols, float* __restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(long long)r * cols + c];
    db[c] = s;
}

// Adam on FP32 masters; refreshes the BF16 weight copy and its transpose (real rows x cols inside the
// padded (rows_pad x cols_pad) arrays)
__global__ void k_adam_layer(float* __restrict__ w, const float* __restrict__ gw, float* __restrict__ m1,
                             float* __restrict__ m2, int rows, int cols, int cols_pad, int rows_pad,
                             __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ wtb, float lr, float c1, float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)rows * cols;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const long long p = (long long)r * cols_pad + c;
        const float g = gw[p];
        const float a = b1 * m1[e] + (1.f - b1) * g;
        const float b = b2 * m2[e] + (1.f - b2) * g * g;
        m1[e] = a;
        m2[e] = b;
        const float x = w[p] - lr * (a / c1) / (sqrtf(b / c2) + eps);
        w[p] = x;
        if (wb) wb[p] = __float2bfloat16(x);
        if (wtb) wtb[(long long)c * rows_pad + r] = __float2bfloat16(x);
    }
}

int pad(int x, int q) { return (x + q - 1) / q * q; }

}  // namespace

struct mtgp_mlp_s {
    int L = 0, maxB = 0, maxBp = 0;
    std::vector<int> w, wp;  // real and padded (to 64) widths
    std::vector<float*> W, b, gW, gb, m1W, m2W, m1b, m2b;  // FP32 masters / grads (padded rows x cols)
    std::vector<__nv_bfloat16*> Wb, Wtb;                    // BF16 copies (padded) and transposes
    std::vector<float*> Z;                                  // pre-activations per layer (maxBp x wp[l+1])
    std::vector<__nv_bfloat16*> Hb;                         // BF16 activations per layer input (maxBp x wp[l])
    std::vector<float*> dZ;
    std::vector<__nv_bfloat16*> dZb, dZtb, Htb;
    float *dH = nullptr, *mu = nullptr, *isd = nullptr, *loss = nullptr;
    int step = 0;
};

namespace {

int mfail(int code, const char* msg) {
    mtgp_set_error(msg);
    return code;
}

template <typename T>
bool al(T** p, size_t n) {
    if (cudaMalloc(p, n * sizeof(T) + 16) != cudaSuccess) return false;
    cudaMemset(*p, 0, n * sizeof(T) + 16);
    return true;
}

void gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, __nv_bfloat16* Cb,
          int ldcb, const float* bias, int relu, int M, int N, int K, cudaStream_t st) {
    dim3 grid(N / TN, M / TM);
    k_gemm_nt<<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, Cb, ldcb, bias, relu, K);
}

void transpose_f32(const float* in, int ldi, __nv_bfloat16* out, int ldo, int rows, int cols, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), blk(32, 8);
    k_transpose_bf16<float><<<grid, blk, 0, st>>>(in, ldi, out, ldo, rows, cols);
}
void transpose_bf(const __nv_bfloat16* in, int ldi, __nv_bfloat16* out, int ldo, int rows, int cols, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), blk(32, 8);
    k_transpose_bf16<__nv_bfloat16><<<grid, blk, 0, st>>>(in, ldi, out, ldo, rows, cols);
}

int blocks_for(long long n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

// forward pass for Bp (padded) rows; input rows (sel[r] or r, of B x w[0] floats) are standardised
// into Hb[0]
void forward(mtgp_mlp_s* m, int B, const float* x, const int* sel, cudaStream_t st) {
    const int Bp = pad(B, TM);
    const long long n0 = (long long)B * m->wp[0];
    k_to_bf16<<<blocks_for(n0), 256, 0, st>>>(x, m->w[0], sel, m->Hb[0], m->wp[0], B, m->w[0], m->wp[0], m->mu, m->isd);
    if (Bp > B) cudaMemsetAsync(m->Hb[0] + (long long)B * m->wp[0], 0, sizeof(__nv_bfloat16) * (size_t)(Bp - B) * m->wp[0], st);
    for (int l = 0; l < m->L; ++l) {
        const bool last = l == m->L - 1;
        gemm(m->Hb[l], m->wp[l], m->Wb[l], m->wp[l], m->Z[l], m->wp[l + 1], last ? nullptr : m->Hb[l + 1], m->wp[l + 1],
             m->b[l], last ? 0 : 1, Bp, m->wp[l + 1], m->wp[l], st);
    }
}

// gradients of the masked loss into gW / gb (padded layouts)
void backward(mtgp_mlp_s* m, int B, const float* tgt, const float* mask, const int* sel, cudaStream_t st) {
    const int Bp = pad(B, TM);
    const int Lr = m->L;
    k_loss_grad<<<1, 1024, 0, st>>>(m->Z[Lr - 1], m->wp[Lr], tgt, mask, sel, B, m->w[Lr], Bp, m->wp[Lr], m->dZ[Lr - 1],
                                    m->dZb[Lr - 1], m->loss);
    for (int l = Lr - 1; l >= 0; --l) {
        const int K = m->wp[l], N = m->wp[l + 1];
        // dW_l = dZ_l^T H_l : (N x Bp) x (Bp x K) as NT with A = dZ^T (N x Bp), B = H^T (K x Bp)
        transpose_f32(m->dZ[l], N, m->dZtb[l], Bp, Bp, N, st);
        transpose_bf(m->Hb[l], K, m->Htb[l], Bp, Bp, K, st);
        gemm(m->dZtb[l], Bp, m->Htb[l], Bp, m->gW[l], K, nullptr, 0, nullptr, 0, N, K, Bp, st);
        k_colsum<<<(N + 127) / 128, 128, 0, st>>>(m->dZ[l], Bp, N, m->gb[l]);
        if (l == 0) break;
        // dH_l = dZ_l W_l : (Bp x N) x (N x K) as NT with B = W^T (K x N)
        gemm(m->dZb[l], N, m->Wtb[l], N, m->dH, K, nullptr, 0, nullptr, 0, Bp, K, N, st);
        const long long n = (long long)Bp * K;
        k_relu_back<<<blocks_for(n), 256, 0, st>>>(m->dH, m->Z[l - 1], m->dZ[l - 1], m->dZb[l - 1], n);
    }
}

}  // namespace

// input width, output width and largest batch of a network (for callers inside the library)
void mlp_shape(const mtgp_mlp_t* m, int* in_width, int* out_width, int* max_batch) {
    *in_width = m->w[0];
    *out_width = m->w[m->L];
    *max_batch = m->maxB;
}

extern "C" {

int mtgp_mlp_create(mtgp_mlp_t** out, int nlayers, const int* widths, int max_batch) {
    if (!out || nlayers < 1 || nlayers > 16 || !widths || max_batch < 1) return mfail(MTGP_ERR_INVALID_ARG, "bad MLP shape");
    for (int l = 0; l <= nlayers; ++l)
        if (widths[l] < 1 || widths[l] > 4096) return mfail(MTGP_ERR_INVALID_ARG, "widths must be in [1, 4096]");
    auto* m = new mtgp_mlp_s();
    m->L = nlayers;
    m->maxB = max_batch;
    m->maxBp = pad(max_batch, TM);
    for (int l = 0; l <= nlayers; ++l) {
        m->w.push_back(widths[l]);
        m->wp.push_back(pad(widths[l], TN));  // every width is an M/N tile multiple and hence a K multiple
    }
    bool ok = al(&m->dH, (size_t)m->maxBp * 4096) && al(&m->mu, m->wp[0]) && al(&m->isd, m->wp[0]) && al(&m->loss, 1);
    for (int l = 0; l < nlayers && ok; ++l) {
        const size_t wsz = (size_t)m->wp[l + 1] * m->wp[l];
        float *W, *b, *gW, *gb, *m1W, *m2W, *m1b, *m2b, *Z, *dZ;
        __nv_bfloat16 *Wb, *Wtb, *Hb, *dZb, *dZtb, *Htb;
        ok = al(&W, wsz) && al(&b, m->wp[l + 1]) && al(&gW, wsz) && al(&gb, m->wp[l + 1]) &&
             al(&m1W, (size_t)m->w[l + 1] * m->w[l]) && al(&m2W, (size_t)m->w[l + 1] * m->w[l]) &&
             al(&m1b, m->w[l + 1]) && al(&m2b, m->w[l + 1]) && al(&Wb, wsz) && al(&Wtb, wsz) &&
             al(&Z, (size_t)m->maxBp * m->wp[l + 1]) && al(&Hb, (size_t)m->maxBp * m->wp[l]) &&
             al(&dZ, (size_t)m->maxBp * m->wp[l + 1]) && al(&dZb, (size_t)m->maxBp * m->wp[l + 1]) &&
             al(&dZtb, (size_t)m->maxBp * m->wp[l + 1]) && al(&Htb, (size_t)m->maxBp * m->wp[l]);
        if (!ok) break;
        m->W.push_back(W); m->b.push_back(b); m->gW.push_back(gW); m->gb.push_back(gb);
        m->m1W.push_back(m1W); m->m2W.push_back(m2W); m->m1b.push_back(m1b); m->m2b.push_back(m2b);
        m->Wb.push_back(Wb); m->Wtb.push_back(Wtb); m->Z.push_back(Z); m->Hb.push_back(Hb);
        m->dZ.push_back(dZ); m->dZb.push_back(dZb); m->dZtb.push_back(dZtb); m->Htb.push_back(Htb);
    }
    if (!ok) {
        mtgp_mlp_destroy(m);
        return mfail(MTGP_ERR_CUDA, "MLP allocation failed");
    }
    std::vector<float> one(m->wp[0], 1.f);
    cudaMemcpy(m->isd, one.data(), sizeof(float) * m->wp[0], cudaMemcpyHostToDevice);
    *out = m;
    return MTGP_OK;
}

int mtgp_mlp_destroy(mtgp_mlp_t* m) {
    if (!m) return MTGP_OK;
    cudaDeviceSynchronize();
    for (int l = 0; l < (int)m->W.size(); ++l) {
        void* ps[] = {m->W[l], m->b[l], m->gW[l], m->gb[l], m->m1W[l], m->m2W[l], m->m1b[l], m->m2b[l], m->Wb[l],
                      m->Wtb[l], m->Z[l], m->Hb[l], m->dZ[l], m->dZb[l], m->dZtb[l], m->Htb[l]};
        for (void* p : ps) cudaFree(p);
    }
    cudaFree(m->dH);
    cudaFree(m->mu);
    cudaFree(m->isd);
    cudaFree(m->loss);
    delete m;
    return MTGP_OK;
}

int mtgp_mlp_set_params(mtgp_mlp_t* m, const float* params, const float* mu, const float* sd) {
    if (!m || !params) return mfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    long long off = 0;
    for (int l = 0; l < m->L; ++l) {
        const int o = m->w[l + 1], i = m->w[l], ip = m->wp[l], op = m->wp[l + 1];
        std::vector<float> Wp((size_t)op * ip, 0.f), bp(op, 0.f);
        for (int r = 0; r < o; ++r)
            for (int c = 0; c < i; ++c) Wp[(size_t)r * ip + c] = params[off + (long long)r * i + c];
        off += (long long)o * i;
        for (int r = 0; r < o; ++r) bp[r] = params[off + r];
        off += o;
        cudaMemcpy(m->W[l], Wp.data(), sizeof(float) * Wp.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(m->b[l], bp.data(), sizeof(float) * bp.size(), cudaMemcpyHostToDevice);
        std::vector<__nv_bfloat16> Wb(Wp.size()), Wt(Wp.size());
        for (int r = 0; r < op; ++r)
            for (int c = 0; c < ip; ++c) {
                Wb[(size_t)r * ip + c] = __float2bfloat16(Wp[(size_t)r * ip + c]);
                Wt[(size_t)c * op + r] = __float2bfloat16(Wp[(size_t)r * ip + c]);
            }
        cudaMemcpy(m->Wb[l], Wb.data(), sizeof(__nv_bfloat16) * Wb.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(m->Wtb[l], Wt.data(), sizeof(__nv_bfloat16) * Wt.size(), cudaMemcpyHostToDevice);
        cudaMemset(m->m1W[l], 0, sizeof(float) * (size_t)o * i);
        cudaMemset(m->m2W[l], 0, sizeof(float) * (size_t)o * i);
        cudaMemset(m->m1b[l], 0, sizeof(float) * o);
        cudaMemset(m->m2b[l], 0, sizeof(float) * o);
    }
    std::vector<float> mv(m->wp[0], 0.f), sv(m->wp[0], 1.f);
    for (int c = 0; c < m->w[0]; ++c) {
        if (mu) mv[c] = mu[c];
        if (sd) sv[c] = sd[c] > 0.f ? 1.f / sd[c] : 1.f;
    }
    cudaMemcpy(m->mu, mv.data(), sizeof(float) * mv.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(m->isd, sv.data(), sizeof(float) * sv.size(), cudaMemcpyHostToDevice);
    m->step = 0;
    return cudaDeviceSynchronize() == cudaSuccess ? MTGP_OK : mfail(MTGP_ERR_CUDA, "parameter upload failed");
}

int mtgp_mlp_get_params(mtgp_mlp_t* m, float* params, float* mu, float* sd) {
    if (!m || !params) return mfail(MTGP_ERR_INVALID_ARG, "NULL argument");
    if (cudaDeviceSynchronize() != cudaSuccess) return mfail(MTGP_ERR_CUDA, "device error before parameter read");
    long long off = 0;
    for (int l = 0; l < m->L; ++l) {
        const int o = m->w[l + 1], i = m->w[l], ip = m->wp[l], op = m->wp[l + 1];
        std::vector<float> Wp((size_t)op * ip), bp(op);
        cudaMemcpy(Wp.data(), m->W[l], sizeof(float) * Wp.size(), cudaMemcpyDeviceToHost);
        cudaMemcpy(bp.data(), m->b[l], sizeof(float) * bp.size(), cudaMemcpyDeviceToHost);
        for (int r = 0; r < o; ++r)
            for (int c = 0; c < i; ++c) params[off + (long long)r * i + c] = Wp[(size_t)r * ip + c];
        off += (long long)o * i;
        for (int r = 0; r < o; ++r) params[off + r] = bp[r];
        off += o;
    }
    if (mu || sd) {
        std::vector<float> mv(m->w[0]), iv(m->w[0]);
        cudaMemcpy(mv.data(), m->mu, sizeof(float) * m->w[0], cudaMemcpyDeviceToHost);
        cudaMemcpy(iv.data(), m->isd, sizeof(float) * m->w[0], cudaMemcpyDeviceToHost);
        for (int c = 0; c < m->w[0]; ++c) {
            if (mu) mu[c] = mv[c];
            if (sd) sd[c] = 1.f / iv[c];
        }
    }
    return MTGP_OK;
}

int mtgp_mlp_fit_scaling(mtgp_mlp_t* m, int rows, const float* x, cudaStream_t st) {
    if (!m || !x || rows < 1) return mfail(MTGP_ERR_INVALID_ARG, "bad scaling arguments");
    k_scaling<<<(m->w[0] + 127) / 128, 128, 0, st>>>(x, rows, m->w[0], m->mu, m->isd);
    return cudaGetLastError() == cudaSuccess ? MTGP_OK : mfail(MTGP_ERR_CUDA, "kernel launch");
}

int mtgp_mlp_forward(mtgp_mlp_t* m, int B, const float* x, float* y, cudaStream_t st) {
    if (!m || !x || !y || B < 1 || B > m->maxB) return mfail(MTGP_ERR_INVALID_ARG, "bad forward arguments");
    forward(m, B, x, nullptr, st);
    const int Lr = m->L;
    cudaMemcpy2DAsync(y, sizeof(float) * m->w[Lr], m->Z[Lr - 1], sizeof(float) * m->wp[Lr], sizeof(float) * m->w[Lr], B,
                      cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? MTGP_OK : mfail(MTGP_ERR_CUDA, "kernel launch");
}

int mtgp_mlp_gradients(mtgp_mlp_t* m, int B, const float* x, const float* target, const float* mask, const int* rows,
                       float* grads, float* loss, cudaStream_t st) {
    if (!m || !x || !target || !mask || B < 1 || B > m->maxB) return mfail(MTGP_ERR_INVALID_ARG, "bad arguments");
    forward(m, B, x, rows, st);
    backward(m, B, target, mask, rows, st);
    if (loss) cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (grads) {
        long long off = 0;
        for (int l = 0; l < m->L; ++l) {
            const int o = m->w[l + 1], i = m->w[l];
            cudaMemcpy2DAsync(grads + off, sizeof(float) * i, m->gW[l], sizeof(float) * m->wp[l], sizeof(float) * i, o,
                              cudaMemcpyDeviceToDevice, st);
            off += (long long)o * i;
            cudaMemcpyAsync(grads + off, m->gb[l], sizeof(float) * o, cudaMemcpyDeviceToDevice, st);
            off += o;
        }
    }
    return cudaGetLastError() == cudaSuccess ? MTGP_OK : mfail(MTGP_ERR_CUDA, "kernel launch");
}

int mtgp_mlp_train_step(mtgp_mlp_t* m, int B, const float* x, const float* target, const float* mask, const int* rows,
                        float lr, float* loss, cudaStream_t st) {
    int rc = mtgp_mlp_gradients(m, B, x, target, mask, rows, nullptr, loss, st);
    if (rc) return rc;
    m->step += 1;
    const float c1 = 1.f - powf(0.9f, (float)m->step), c2 = 1.f - powf(0.999f, (float)m->step);
    for (int l = 0; l < m->L; ++l) {
        const int o = m->w[l + 1], i = m->w[l];
        k_adam_layer<<<blocks_for((long long)o * i), 256, 0, st>>>(m->W[l], m->gW[l], m->m1W[l], m->m2W[l], o, i, m->wp[l],
                                                                   m->wp[l + 1], m->Wb[l], m->Wtb[l], lr, c1, c2);
        k_adam_layer<<<blocks_for(o), 256, 0, st>>>(m->b[l], m->gb[l], m->m1b[l], m->m2b[l], 1, o, o, 1, nullptr, nullptr,
                                                    lr, c1, c2);
    }
    return cudaGetLastError() == cudaSuccess ? MTGP_OK : mfail(MTGP_ERR_CUDA, "kernel launch");
}

}  // extern "C"

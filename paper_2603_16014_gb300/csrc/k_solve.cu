// Per-frequency solves of Lambda-tilde (FP64) and the gradient weights.
//
// Equal sizes (Corollary "equal sizes"): Lambda is block diagonal over frequencies f; each block is
//   Lambda(f) = R o M(f) + sigma2 I,  M(f)_{tu} = mu_{tu}(f) (first-column transforms),
// factorised as L D L^H per thread.  tau_t is the sample mean, so rhat(0) = 0.
//
// Unequal nested sizes (Algorithm 1): entries couple (t, f) and (u, g) only when f = g mod
// min(n_t, n_u), so each residue class rho mod n_T is independent.  Eliminating tasks in order
// t = 1..T (the paper's order) makes the Schur complement of every task-t frequency a scalar --
// Algorithm 1's diagonal S_t.  This file keeps Lambda^-1 in factored form instead of the explicit
// block inverse A: the pivots are the same S_t (so log|Lambda| = sum_t log|S_t|), the factor has
// no fill (the class graph is a tree of nested residues) and the entries of Lambda^-1 the gradient
// needs -- those on Lambda's own sparsity pattern -- come from the selected-inversion recurrence
// Z = D^-1 L^-1 + (I - L^H) Z restricted to ancestor chains.
//
// Gradient (tau held at its optimum): dL = sum over pattern G_{ji} dLambda_{ij},
//   G = Lambda^-1 - alpha alpha^H, alpha = Lambda^-1 rhat.
#include "freq_solve.cuh"

namespace {

template <typename S, bool CPLX>
__device__ __forceinline__ Vt<CPLX> load_spec(const void* p, long long i) { return load_elem<S, CPLX>(p, i); }
template <typename S, bool CPLX>
__device__ __forceinline__ void store_spec(void* p, long long i, Vt<CPLX> v) { store_elem<S, CPLX>(p, i, v); }

struct SolveParams {
    int T, s, nT;
    int grad, clamp, store_alpha, gcv;  // gcv: 1 loss value, 2 gradient (needs gcv_ab)
    int pt;                             // per-task noise
    const double* gcv_ab;               // [A, B] of the GCV loss (device), for gcv = 2
    long long n[MTGP_TMAX];
    int order[MTGP_TMAX];
    int colidx[MTGP_TMAX][MTGP_TMAX];
    long long coloff[MTGP_MAX_COLS];
    long long yoff[MTGP_TMAX];
};

// R = W W^T + diag(v) in sorted task order
__device__ void load_R(double* sR, const SolveParams& p, const ThetaPtrs& th) {
    for (int e = threadIdx.x; e < p.T * p.T; e += blockDim.x) {
        int t = e / p.T, u = e % p.T;
        int tc = p.order[t], uc = p.order[u];
        double r = 0.0;
        for (int k = 0; k < th.s; ++k) r += th.W[tc * th.s + k] * th.W[uc * th.s + k];
        if (t == u) r += th.v[tc];
        sR[e] = r;
    }
}

constexpr int kEqThreads = 128;

// GCV gradient at one frequency: with Z = Lambda(f)^-1, alpha = Z rhat, beta = Z alpha and the totals
// A = sum ||alpha||^2, B = sum trace Z (c1 = 1 / B^2, c2 = 2 A / B^3), the loss differential is
// trace(G dLambda) with G = -c1 (alpha beta^H + beta alpha^H) + c2 Z^2; G is contracted and turned
// into adjoint weights exactly as the MLE path does with G = Z - alpha alpha^H.
template <int T, bool CPLX>
__device__ void gcv_grad_freq(Vt<CPLX> (&mu)[T][T], const Vt<CPLX> (&rh)[T], const double* sR, double sig, bool clamp,
                              double c1, double c2, double* acc, Vt<CPLX> (&w)[T][T], int& bad,
                              const double* sigv) {
    using V = Vt<CPLX>;
    double mu0 = creal(mu[0][0]);
    double ind0 = 1.0;
    if (clamp && mu0 < 0.0) {
        mu0 = 0.0;
        ind0 = 0.0;
    }
    V S[T][T], L[T][T];
    double D[T], iD[T];
    for (int i = 0; i < T; ++i) {
        D[i] = sR[i * T + i] * mu0 + (sigv ? sigv[i] : sig);
        for (int j = 0; j < i; ++j) S[i][j] = vscale(cconj(mu[j][i]), sR[j * T + i]);
    }
    for (int k = 0; k < T; ++k) {
        if (!(D[k] > 0.0) || !isfinite(D[k])) {
            bad = 1;
            D[k] = 1.0;
        }
        iD[k] = 1.0 / D[k];
        for (int i = k + 1; i < T; ++i) L[i][k] = vscale(S[i][k], iD[k]);
        for (int i = k + 1; i < T; ++i) {
            D[i] -= creal(vmul(L[i][k], cconj(S[i][k])));
            for (int j = k + 1; j < i; ++j) S[i][j] = vsub(S[i][j], vmul(L[i][k], cconj(S[j][k])));
        }
    }
    // Z by columns: L D L^H z = e_c
    V Z[T][T];
    for (int c = 0; c < T; ++c) {
        V x[T];
        for (int k = 0; k < T; ++k) {
            V r = (k == c) ? cfromreal<V>(1.0) : czero<V>();
            for (int j = 0; j < k; ++j) r = vsub(r, vmul(L[k][j], x[j]));
            x[k] = r;
        }
        for (int k = 0; k < T; ++k) x[k] = vscale(x[k], iD[k]);
        for (int k = T - 1; k >= 0; --k)
            for (int i = k + 1; i < T; ++i) x[k] = vsub(x[k], vmul(cconj(L[i][k]), x[i]));
        for (int k = 0; k < T; ++k) Z[k][c] = x[k];
    }
    V al[T], be[T];
    for (int i = 0; i < T; ++i) {
        V a = czero<V>();
        for (int k = 0; k < T; ++k) a = vadd(a, vmul(Z[i][k], rh[k]));
        al[i] = a;
    }
    for (int i = 0; i < T; ++i) {
        V b = czero<V>();
        for (int k = 0; k < T; ++k) b = vadd(b, vmul(Z[i][k], al[k]));
        be[i] = b;
    }
    double wdiag = 0.0;
    int q = 3;
    for (int t = 0; t < T; ++t) {
        for (int uu = t; uu < T; ++uu) {
            V z2 = czero<V>();
            for (int k = 0; k < T; ++k) z2 = vadd(z2, vmul(Z[uu][k], Z[k][t]));
            const V ga = vadd(vmul(al[uu], cconj(be[t])), vmul(be[uu], cconj(al[t])));
            const V g = vsub(vscale(z2, c2), vscale(ga, c1));
            if (uu == t) {
                const double gd = creal(g);
                acc[2] += gd;
                if (sigv) acc[3 + T * (T + 1) / 2 + t] += gd;
                acc[q] = fma(gd, mu0, acc[q]);
                wdiag = fma(sR[t * T + t], gd, wdiag);
            } else {
                acc[q] += creal(vmul(g, mu[t][uu]));
                w[t][uu] = vscale(g, 2.0 * sR[t * T + uu]);
            }
            ++q;
        }
    }
    w[0][0] = cfromreal<V>(wdiag * ind0);
}

template <int T, bool CPLX, typename S>
__global__ void __launch_bounds__(kEqThreads)
k_solve_equal(const void* spec, void* wgt, const double* yhat, SolveParams p, ThetaPtrs th, double* partials,
              double* alpha_out, int* status) {
    using V = Vt<CPLX>;
    constexpr int NG = T * (T + 1) / 2;
    constexpr int NQX = 3 + NG + T;          // with per-task noise traces
    const int NQ = 3 + NG + (p.pt ? T : 0);
    __shared__ double sR[T * T];
    __shared__ double s_sig;
    __shared__ double s_sigv[T];
    __shared__ double s_red[kEqThreads / 32][NQX];
    load_R(sR, p, th);
    if (threadIdx.x == 0) s_sig = th.sigma2[0];
    if (threadIdx.x < T) s_sigv[threadIdx.x] = noise_of(th, p.order, threadIdx.x);
    __syncthreads();
    const double sig = s_sig;
    const double* sigv = p.pt ? s_sigv : nullptr;
    const long long n = p.n[0];
    double acc[NQX];
#pragma unroll
    for (int q = 0; q < NQX; ++q) acc[q] = 0.0;
    LogAcc lacc;
    lacc.init();
    int bad = 0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < n; f += (long long)gridDim.x * blockDim.x) {
        V mu[T][T], w[T][T], al[T], rh[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
#pragma unroll
            for (int u = t; u < T; ++u) mu[t][u] = load_spec<S, CPLX>(spec, p.coloff[p.colidx[t][u]] + f);
            rh[t] = (f == 0) ? czero<V>() : ld<CPLX>(yhat, p.yoff[t] + f);
        }
        if (p.gcv == 2) {
            const double A = p.gcv_ab[0], B = p.gcv_ab[1];
            gcv_grad_freq<T, CPLX>(mu, rh, sR, sig, p.clamp != 0, 1.0 / (B * B), 2.0 * A / (B * B * B), acc, w, bad,
                                   sigv);
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int u = t; u < T; ++u)
                    if (u != t || t == 0) store_spec<S, CPLX>(wgt, p.coloff[p.colidx[t][u]] + f, w[t][u]);
            continue;
        }
        if (p.gcv) {
            // ||Lambda(f)^-1 rhat(f)||^2 and trace Lambda(f)^-1: the gradient pass yields
            // sum_t G_tt = trace Z - ||alpha||^2 in its third accumulator
            double scr[NQX];
#pragma unroll
            for (int q = 0; q < NQX; ++q) scr[q] = 0.0;
            solve_freq<T, CPLX>(mu, rh, sR, sig, p.clamp != 0, true, lacc, scr, w, al, true, bad, sigv);
            double a2 = 0.0;
#pragma unroll
            for (int t = 0; t < T; ++t) a2 += cabs2(al[t]);
            acc[1] += scr[1];
            acc[2] += a2;
            acc[3] += scr[2] + a2;
            continue;
        }
        solve_freq<T, CPLX>(mu, rh, sR, sig, p.clamp != 0, p.grad != 0, lacc, acc, w, al, p.store_alpha != 0, bad, sigv);
        if (p.store_alpha) {
#pragma unroll
            for (int k = 0; k < T; ++k) st<CPLX>(alpha_out, p.yoff[k] + f, al[k]);
        }
        if (p.grad) {
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
                for (int u = t; u < T; ++u)
                    if (u != t || t == 0) store_spec<S, CPLX>(wgt, p.coloff[p.colidx[t][u]] + f, w[t][u]);
        }
    }
    acc[0] = lacc.log_value();
    if (bad) set_status(status, ST_NOT_PD);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQX; ++q) {
        if (q >= NQ) break;
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < kEqThreads / 32; ++w) v += s_red[w][q];
        partials[(long long)blockIdx.x * NQ + q] = v;
    }
}

// --------------------------------------------------------------------------- tree solver

constexpr int kTreeThreads = 256;
constexpr int kTreeWarps = kTreeThreads / 32;
// A CTA owns kTreeCW consecutive residue classes; lane l works on class l mod kTreeCW in slot
// (warp, l / kTreeCW), and the kTreeSlots slots of a class split its nodes.
constexpr int kTreeCW = 8;
constexpr int kTreeSlots = kTreeThreads / kTreeCW;

struct TreeParams {
    int T, s, grad, clamp, gcv, pt;
    double* pi_out;  // when set: Pi = E K~^-1 E^T (sorted order, T x T) from class 0
    long long nT;
    long long n[MTGP_TMAX];
    long long po[MTGP_TMAX][MTGP_TMAX];  // pair (t <= u) element offset in spec / wgt / S / Z
    long long yoff[MTGP_TMAX];
    int order[MTGP_TMAX];
};

__device__ void load_R_tree(double* sR, const TreeParams& p, const ThetaPtrs& th) {
    for (int e = threadIdx.x; e < p.T * p.T; e += blockDim.x) {
        int t = e / p.T, u = e % p.T;
        int tc = p.order[t], uc = p.order[u];
        double r = 0.0;
        for (int k = 0; k < th.s; ++k) r += th.W[tc * th.s + k] * th.W[uc * th.s + k];
        if (t == u) r += th.v[tc];
        sR[e] = r;
    }
}

__device__ __forceinline__ int gidx(int t, int u, int T) { return t * T - t * (t - 1) / 2 + (u - t); }

// Parts a reduction of rr terms for each of ma targets is split into, so that ma * parts fills the
// kTreeSlots slots of a class when ma is small (all sizes are powers of two).
__device__ __forceinline__ int split_parts(long long ma, long long rr) {
    if (ma >= kTreeSlots) return 1;
    long long P = kTreeSlots / ma;
    return (int)(P < rr ? P : rr);
}

// Forward solve L u = r on the class graph (right-looking), accumulating sum |u_j|^2 / D_j.
// Node (t, f) is eliminated at stage t; its ancestor in task a > t is (a, f mod n_a) and
// L[(a, .), (t, f)] = conj(S_{ta}[f]) / D_{(t,f)}.  The diagonal slot of S holds 1 / D.
template <bool CPLX>
__device__ void tree_forward(const TreeParams& p, const double* Sb, double* rb, long long rho, bool act, int slot,
                             double& quad, Vt<CPLX> (*s_part)[kTreeSlots][MTGP_TMAX]) {
    using V = Vt<CPLX>;
    const long long nT = p.nT;
    const int cls = (int)(rho % kTreeCW);
    for (int t = 0; t < p.T; ++t) {
        const long long mt = p.n[t] / nT;
        if (act) {
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                quad += cabs2(ld<CPLX>(rb, p.yoff[t] + f)) * creal(ld<CPLX>(Sb, p.po[t][t] + f));
            }
        }
        for (int a = t + 1; a < p.T; ++a) {
            const long long ma = p.n[a] / nT, rr = p.n[t] / p.n[a];
            const int P = split_parts(ma, rr);
            for (long long u = slot; u < ma * P; u += kTreeSlots) {
                if (!act) break;
                const long long gi = u / P, part = u % P, q0 = part * (rr / P), q1 = q0 + rr / P;
                V acc = czero<V>();
                for (long long q = q0; q < q1; ++q) {
                    long long f = rho + (gi + q * ma) * nT;
                    const double iD = creal(ld<CPLX>(Sb, p.po[t][t] + f));
                    acc = vadd(acc, vmul(cconj(ld<CPLX>(Sb, p.po[t][a] + f)), vscale(ld<CPLX>(rb, p.yoff[t] + f), iD)));
                }
                if (P == 1) {
                    long long g = rho + gi * nT;
                    st<CPLX>(rb, p.yoff[a] + g, vsub(ld<CPLX>(rb, p.yoff[a] + g), acc));
                } else {
                    s_part[cls][u][0] = acc;
                }
            }
            if (P > 1) {
                __syncthreads();
                if (act && slot < ma) {
                    V acc = czero<V>();
                    for (int part = 0; part < P; ++part) acc = vadd(acc, s_part[cls][slot * P + part][0]);
                    long long g = rho + slot * nT;
                    st<CPLX>(rb, p.yoff[a] + g, vsub(ld<CPLX>(rb, p.yoff[a] + g), acc));
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }
}

// Backward solve L^H alpha = D^-1 u (top-down) and, when wantZ, the selected inverse on the
// pattern:  Z[j, a'] = -sum_{a in anc(j)} conj(L[a, j]) Z[a, a']  (a' in anc(j)),
//           Z[j, j]  = 1/D_j - sum_{a in anc(j)} conj(L[a, j]) Z[a, j].
// Z is stored like S: Z_{ta'}[f] = Z[(t, f), (a', f mod n_a')].  The diagonal slot of S holds 1 / D.
template <bool CPLX>
__device__ void tree_backward(const TreeParams& p, const double* Sb, double* Zb, const double* rb, double* ab,
                              long long rho, bool act, int slot, bool wantZ, bool mir = false) {
    using V = Vt<CPLX>;
    const long long nT = p.nT;
    for (int t = p.T - 1; t >= 0; --t) {
        const long long mt = p.n[t] / nT;
        if (act) {
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                const double invD = creal(ld<CPLX>(Sb, p.po[t][t] + f));
                V l[MTGP_TMAX];
#pragma unroll
                for (int a1 = 0; a1 < MTGP_TMAX; ++a1)
                    l[a1] = (a1 > t && a1 < p.T) ? vscale(ld<CPLX>(Sb, p.po[t][a1] + f), invD) : czero<V>();
                V a = vscale(ld<CPLX>(rb, p.yoff[t] + f), invD);
#pragma unroll
                for (int a2 = 0; a2 < MTGP_TMAX; ++a2)
                    if (a2 > t && a2 < p.T) a = vsub(a, vmul(l[a2], ld<CPLX>(ab, p.yoff[a2] + (f & (p.n[a2] - 1)))));
                st<CPLX>(ab, p.yoff[t] + f, a);
                // the conjugate class holds the conjugate solution at the mirrored frequencies
                if (mir) st<CPLX>(ab, p.yoff[t] + ((p.n[t] - f) & (p.n[t] - 1)), cconj(a));
                if (wantZ) {
                    double zd = invD;
#pragma unroll
                    for (int a2 = 0; a2 < MTGP_TMAX; ++a2) {
                        if (a2 > t && a2 < p.T) {
                            V z = czero<V>();
#pragma unroll
                            for (int a1 = 0; a1 < MTGP_TMAX; ++a1) {
                                if (a1 > t && a1 < p.T) {
                                    V zz = (a1 <= a2) ? ld<CPLX>(Zb, p.po[a1][a2] + (f & (p.n[a1] - 1)))
                                                      : cconj(ld<CPLX>(Zb, p.po[a2][a1] + (f & (p.n[a2] - 1))));
                                    z = vsub(z, vmul(l[a1], zz));
                                }
                            }
                            st<CPLX>(Zb, p.po[t][a2] + f, z);
                            zd -= creal(vmul(l[a2], cconj(z)));
                        }
                    }
                    st<CPLX>(Zb, p.po[t][t] + f, cfromreal<V>(zd));
                }
            }
        }
        __syncthreads();
    }
}

// A CTA owns kTreeCW consecutive residue classes rho mod n_T; the kTreeSlots slots of a class split
// its nodes, so a warp's accesses touch runs of kTreeCW consecutive frequencies.  The first class (rho = 0)
// also carries the optimal means (theorem item 4): it is solved once with yhat to get Pi and
// E K~^-1 y, then every class is solved with rhat.
template <bool CPLX, typename S>
__global__ void __launch_bounds__(kTreeThreads)
k_solve_tree(const void* spec, void* wgt, const double* yhat, double* Sb, double* Zb, double* rb, double* ab,
             double* tau_out, TreeParams p, ThetaPtrs th, double* partials, int* status, double* Hb) {
    using V = Vt<CPLX>;
    const int T = p.T;
    const int NG = T * (T + 1) / 2;
    const int NQ = 3 + NG + (p.pt ? T : 0);
    __shared__ double sR[MTGP_TMAX * MTGP_TMAX];
    __shared__ double s_sigv[MTGP_TMAX];
    __shared__ double s_tau[MTGP_TMAX];
    __shared__ double s_red[kTreeWarps][3 + MTGP_MAX_COLS + MTGP_TMAX];
    load_R_tree(sR, p, th);
    if (threadIdx.x < T) s_sigv[threadIdx.x] = noise_of(th, p.order, threadIdx.x);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = warp * (32 / kTreeCW) + lane / kTreeCW;
    const long long nT = p.nT;
    const int cls = lane % kTreeCW;
    const long long rho = (long long)blockIdx.x * kTreeCW + cls;
    // lattices (complex spectra of real data): class nT - rho is the conjugate of class rho, so only
    // rho = 0 .. nT/2 are solved; a class with a distinct conjugate counts twice and writes the
    // conjugate solution and weights at the mirrored frequencies
    const long long ncls = (CPLX && nT >= 2) ? nT / 2 + 1 : nT;
    const bool act = rho < ncls;
    const bool mir = CPLX && act && rho != 0 && 2 * rho != nT;
    __shared__ V s_part[kTreeCW][kTreeSlots][MTGP_TMAX];  // partial sums of split reductions
    double acc[3 + MTGP_MAX_COLS + MTGP_TMAX];
    for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
    int bad = 0;

    // Lambda entries of the class: S_{tu}[f] = Lambda[(t, f), (u, f mod n_u)]
    for (int t = 0; t < T; ++t) {
        const long long mt = p.n[t] / nT;
        for (int u = t; u < T; ++u) {
            const double sc = sqrt((double)p.n[u] / (double)p.n[t]) * sR[t * T + u];
            if (!act) continue;
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                V mu = load_spec<S, CPLX>(spec, p.po[t][u] + f);
                V val;
                if (t == u) {
                    double m0 = creal(mu);
                    if (p.clamp && m0 < 0.0) m0 = 0.0;
                    val = cfromreal<V>(sR[t * T + t] * m0 + s_sigv[t]);
                } else {
                    val = vscale(mu, sc);
                }
                st<CPLX>(Sb, p.po[t][u] + f, val);
            }
        }
    }
    __syncthreads();

    // elimination in task order: pivots are the Schur complements S_t of Algorithm 1.  A pivot's
    // diagonal slot is replaced by 1 / D once its log is taken; for each target node (a, g) the
    // factors L = conj(S_{ta}) / D of the rr nodes above it are formed once and applied to every
    // a2 >= a.
    // pivots multiplied into a mantissa / exponent accumulator: one log per thread at the end
    LogAcc lacc;
    lacc.init();
    for (int t = 0; t < T; ++t) {
        const long long mt = p.n[t] / nT;
        if (act) {
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                double D = creal(ld<CPLX>(Sb, p.po[t][t] + f));
                if (!pos_finite(D)) {
                    bad = 1;
                    D = 1.0;
                }
                lacc.mul(D);
                st<CPLX>(Sb, p.po[t][t] + f, cfromreal<V>(fast_rcp(D)));
            }
        }
        __syncthreads();
        for (int a = t + 1; a < T; ++a) {
            const long long ma = p.n[a] / nT, rr = p.n[t] / p.n[a];
            const int P = split_parts(ma, rr);
            for (long long u = slot; u < ma * P; u += kTreeSlots) {
                if (!act) break;
                const long long gi = u / P, part = u % P, q0 = part * (rr / P), q1 = q0 + rr / P;
                V sacc[MTGP_TMAX];
#pragma unroll
                for (int a2 = 0; a2 < MTGP_TMAX; ++a2) sacc[a2] = czero<V>();
                for (long long q = q0; q < q1; ++q) {
                    long long f = rho + (gi + q * ma) * nT;
                    const double iD = creal(ld<CPLX>(Sb, p.po[t][t] + f));
                    const V l = vscale(cconj(ld<CPLX>(Sb, p.po[t][a] + f)), iD);
#pragma unroll
                    for (int a2 = 0; a2 < MTGP_TMAX; ++a2)
                        if (a2 >= a && a2 < T) sacc[a2] = vadd(sacc[a2], vmul(l, ld<CPLX>(Sb, p.po[t][a2] + f)));
                }
                if (P == 1) {
                    long long g = rho + gi * nT;
#pragma unroll
                    for (int a2 = 0; a2 < MTGP_TMAX; ++a2)
                        if (a2 >= a && a2 < T) st<CPLX>(Sb, p.po[a][a2] + g, vsub(ld<CPLX>(Sb, p.po[a][a2] + g), sacc[a2]));
                } else {
#pragma unroll
                    for (int a2 = 0; a2 < MTGP_TMAX; ++a2)
                        if (a2 >= a && a2 < T) s_part[cls][u][a2] = sacc[a2];
                }
            }
            if (P > 1) {
                // parts of one target added in order by the target's slot
                __syncthreads();
                if (act && slot < ma) {
                    long long g = rho + slot * nT;
                    for (int a2 = a; a2 < T; ++a2) {
                        V acc = czero<V>();
                        for (int part = 0; part < P; ++part) acc = vadd(acc, s_part[cls][slot * P + part][a2]);
                        st<CPLX>(Sb, p.po[a][a2] + g, vsub(ld<CPLX>(Sb, p.po[a][a2] + g), acc));
                    }
                }
                __syncthreads();
            }
        }
        __syncthreads();
    }

    // optimal means from the first class
    if (blockIdx.x == 0) {
        const bool act0 = act && rho == 0;
        if (act0) {
            for (int t = 0; t < T; ++t) {
                const long long mt = p.n[t] / nT;
                for (long long k = slot; k < mt; k += kTreeSlots)
                    st<CPLX>(rb, p.yoff[t] + k * nT, ld<CPLX>(yhat, p.yoff[t] + k * nT));
            }
        }
        __syncthreads();
        double qd = 0.0;
        tree_forward<CPLX>(p, Sb, rb, rho, act0, slot, qd, s_part);
        tree_backward<CPLX>(p, Sb, Zb, rb, ab, rho, act0, slot, true);
        // GCV: the class-0 columns c_t = Lambda_0^-1 e_(t,0) (rows 0..T-1 of Hb) and
        // Lambda_0^-1 yhat_0 (row T), over the class-0 nodes (t, k nT) flattened task by task
        long long P0 = 0, off0[MTGP_TMAX];
        for (int t = 0; t < T; ++t) {
            off0[t] = P0;
            P0 += p.n[t] / nT;
        }
        auto save_row = [&](int row) {
            if (!act0) return;
            for (int t = 0; t < T; ++t)
                for (long long k = slot; k < p.n[t] / nT; k += kTreeSlots)
                    st<CPLX>(Hb, (long long)row * P0 + off0[t] + k, ld<CPLX>(ab, p.yoff[t] + k * nT));
        };
        if (p.gcv) {
            save_row(T);
            for (int c = 0; c < T; ++c) {
                __syncthreads();
                if (act0) {
                    for (int t = 0; t < T; ++t)
                        for (long long k = slot; k < p.n[t] / nT; k += kTreeSlots)
                            st<CPLX>(rb, p.yoff[t] + k * nT, (t == c && k == 0) ? cfromreal<V>(1.0) : czero<V>());
                }
                __syncthreads();
                tree_forward<CPLX>(p, Sb, rb, rho, act0, slot, qd, s_part);
                tree_backward<CPLX>(p, Sb, Zb, rb, ab, rho, act0, slot, false);
                save_row(c);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double Pi[MTGP_TMAX][MTGP_TMAX], b[MTGP_TMAX];
            if (!p.gcv) {
                // Pi = E K~^-1 E^T and E K~^-1 yhat from class 0 (Theorem FMTGP item 4)
                for (int t = 0; t < T; ++t) {
                    b[t] = sqrt((double)p.n[t]) * creal(ld<CPLX>(ab, p.yoff[t]));
                    for (int u = 0; u < T; ++u) {
                        double z = (t <= u) ? creal(ld<CPLX>(Zb, p.po[t][u])) : creal(ld<CPLX>(Zb, p.po[u][t]));
                        Pi[t][u] = sqrt((double)p.n[t] * (double)p.n[u]) * z;
                    }
                }
            } else {
                // H H^* and E K~^-2 yhat with H_{t,k} = sqrt(n_t) conj(c_t[k]) (Theorem FMTGP item 4)
                for (int t = 0; t < T; ++t) {
                    double bt = 0.0;
                    for (long long q = 0; q < P0; ++q)
                        bt += creal(vmul(cconj(ld<CPLX>(Hb, (long long)t * P0 + q)), ld<CPLX>(Hb, (long long)T * P0 + q)));
                    b[t] = sqrt((double)p.n[t]) * bt;
                    for (int u = 0; u <= t; ++u) {
                        double hh = 0.0;
                        for (long long q = 0; q < P0; ++q)
                            hh += creal(vmul(cconj(ld<CPLX>(Hb, (long long)t * P0 + q)), ld<CPLX>(Hb, (long long)u * P0 + q)));
                        Pi[t][u] = Pi[u][t] = sqrt((double)p.n[t] * (double)p.n[u]) * hh;
                    }
                }
            }
            if (p.pi_out && !p.gcv)
                for (int t = 0; t < T; ++t)
                    for (int u = 0; u < T; ++u) p.pi_out[t * T + u] = Pi[t][u];
            // Pi tau = b by Cholesky (Pi = E K~^-1 E^T is SPD)
            for (int k = 0; k < T; ++k) {
                double dk = Pi[k][k];
                for (int j = 0; j < k; ++j) dk -= Pi[k][j] * Pi[k][j];
                if (!(dk > 0.0)) {
                    bad = 1;
                    dk = 1.0;
                }
                dk = sqrt(dk);
                Pi[k][k] = dk;
                for (int i = k + 1; i < T; ++i) {
                    double a = Pi[i][k];
                    for (int j = 0; j < k; ++j) a -= Pi[i][j] * Pi[k][j];
                    Pi[i][k] = a / dk;
                }
            }
            for (int k = 0; k < T; ++k) {
                double a = b[k];
                for (int j = 0; j < k; ++j) a -= Pi[k][j] * b[j];
                b[k] = a / Pi[k][k];
            }
            for (int k = T - 1; k >= 0; --k) {
                double a = b[k];
                for (int i = k + 1; i < T; ++i) a -= Pi[i][k] * b[i];
                b[k] = a / Pi[k][k];
            }
            for (int t = 0; t < T; ++t) {
                s_tau[t] = b[t];
                tau_out[t] = b[t];
            }
        }
        __syncthreads();
    }

    // rhat = yhat - V^dagger E^T tau: only the zero frequency of each task changes
    if (act) {
        for (int t = 0; t < T; ++t) {
            const long long mt = p.n[t] / nT;
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                V y = ld<CPLX>(yhat, p.yoff[t] + f);
                if (f == 0) y = vsub(y, cfromreal<V>(sqrt((double)p.n[t]) * s_tau[t]));
                st<CPLX>(rb, p.yoff[t] + f, y);
            }
        }
    }
    __syncthreads();
    tree_forward<CPLX>(p, Sb, rb, rho, act, slot, acc[1], s_part);
    tree_backward<CPLX>(p, Sb, Zb, rb, ab, rho, act, slot, p.grad != 0 || p.gcv != 0, mir);

    if (p.gcv && act) {
        // ||Lambda~^-1 rhat||^2 and trace Lambda~^-1 over this class's nodes
        for (int t = 0; t < T; ++t) {
            const long long mt = p.n[t] / nT;
            for (long long k = slot; k < mt; k += kTreeSlots) {
                long long f = rho + k * nT;
                acc[2] += cabs2(ld<CPLX>(ab, p.yoff[t] + f));
                acc[3] += creal(ld<CPLX>(Zb, p.po[t][t] + f));
            }
        }
    }

    if (p.grad && act) {
        for (int t = 0; t < T; ++t) {
            const long long mt = p.n[t] / nT;
            for (int u = t; u < T; ++u) {
                const double sc = sqrt((double)p.n[u] / (double)p.n[t]);
                const int q = 3 + gidx(t, u, T);
                for (long long k = slot; k < mt; k += kTreeSlots) {
                    long long f = rho + k * nT;
                    V at = ld<CPLX>(ab, p.yoff[t] + f);
                    V au = ld<CPLX>(ab, p.yoff[u] + (f & (p.n[u] - 1)));
                    V g = vsub(cconj(ld<CPLX>(Zb, p.po[t][u] + f)), vmul(au, cconj(at)));
                    V mu = load_spec<S, CPLX>(spec, p.po[t][u] + f);
                    if (u == t) {
                        double gd = creal(g);
                        double m0 = creal(mu);
                        double ind = 1.0;
                        if (p.clamp && m0 < 0.0) {
                            m0 = 0.0;
                            ind = 0.0;
                        }
                        acc[2] += gd;
                        if (p.pt) acc[3 + NG + t] += gd;
                        acc[q] += gd * m0;
                        const V wv = cfromreal<V>(sR[t * T + t] * gd * ind);
                        store_spec<S, CPLX>(wgt, p.po[t][u] + f, wv);
                        if (mir) store_spec<S, CPLX>(wgt, p.po[t][u] + ((p.n[t] - f) & (p.n[t] - 1)), wv);
                    } else {
                        acc[q] += sc * creal(vmul(g, mu));
                        const V wv = vscale(g, 2.0 * sR[t * T + u] * sc);
                        store_spec<S, CPLX>(wgt, p.po[t][u] + f, wv);
                        if (mir) store_spec<S, CPLX>(wgt, p.po[t][u] + ((p.n[t] - f) & (p.n[t] - 1)), cconj(wv));
                    }
                }
            }
        }
    }
    if (bad) set_status(status, ST_NOT_PD);
    acc[0] = lacc.log_value();
    if (mir)
        for (int q = 0; q < NQ; ++q) acc[q] *= 2.0;
    for (int q = 0; q < NQ; ++q) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < kTreeWarps; ++w) v += s_red[w][q];
        partials[(long long)blockIdx.x * NQ + q] = v;
    }
}

// --------------------------------------------------------------------------- finalize

struct FinParams {
    int T, d, s, equal, cplx, NQ, nsolve, neta, grad, gcv, pt;
    int mix;  // DSI mixture: 4 dL/db entries follow the d eta entries of each eta partial row
    long long N;
    long long n0;
    int order[MTGP_TMAX];
    int rank[MTGP_TMAX];
    long long yoff[MTGP_TMAX];
};

// Column sums of a (nrows x ncols) partial array into out[q], by the whole block in a fixed order:
// warp w takes columns w, w + nw, ...; lane l adds rows l, l + 32, ... (the loads of 8 rows are in
// flight together), then a shuffle tree.
__device__ void block_column_sums(const double* part, int nrows, int ncols, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < ncols; q += nw) {
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
        if (lane == 0) out[q] = v;
    }
}

// one block: totals of the solver and eta partials, then every output by its own thread
__global__ void k_finalize(const double* partials, const double* eta_partials, const double* yhat,
                           const double* tau_sorted, FinParams p, ThetaPtrs th, double* out, double* tau,
                           double* g_eta, double* g_W, double* g_v, double* g_s2, double* g_b) {
    __shared__ double tot[3 + MTGP_MAX_COLS + MTGP_TMAX];
    __shared__ double etot[MTGP_MAX_DIM + 4];
    __shared__ double s_W[MTGP_TMAX * MTGP_TMAX];
    const int tid = threadIdx.x, T = p.T;
    block_column_sums(partials, p.nsolve, p.NQ, tot);
    if (p.grad) {
        block_column_sums(eta_partials, p.neta, p.d + (p.mix ? 4 : 0), etot);
        for (int e = tid; e < T * p.s; e += blockDim.x) s_W[e] = th.W[e];
    }
    __syncthreads();
    const double LOG2PI = 1.8378770664093453;
    if (tid == 0) {
        if (p.gcv == 2) {
            // GCV gradient pass: the loss was written by the value pass
        } else if (p.gcv) {
            // GCV loss ||Lambda~^-1 rhat||^2 / trace(Lambda~^-1)^2, its numerator and the trace
            out[0] = tot[2] / (tot[3] * tot[3]);
            out[1] = tot[2];
            out[2] = tot[3];
        } else {
            out[0] = 0.5 * (tot[0] + tot[1] + (double)p.N * LOG2PI);
            out[1] = tot[1];
            out[2] = tot[0];
        }
    }
    if (tau && tid < T) {
        double tv;
        if (p.equal) tv = yhat[(p.cplx ? 2 : 1) * p.yoff[tid]] / sqrt((double)p.n0);
        else tv = tau_sorted[tid];
        tau[p.order[tid]] = tv;
    }
    if (!p.grad) return;
    // MLE: gradients of NLL = L / 2; GCV: gradients of the loss itself
    const double sc = (p.gcv == 2) ? 2.0 : 1.0;
    if (p.pt) {
        if (tid < T) g_s2[tid] = 0.5 * sc * tot[3 + T * (T + 1) / 2 + p.rank[tid]];
    } else if (tid == 0) {
        g_s2[0] = 0.5 * sc * tot[2];
    }
    if (tid < p.d) g_eta[tid] = 0.5 * sc * etot[tid];
    if (p.mix && tid < 4) g_b[tid] = 0.5 * sc * etot[p.d + tid];
    for (int e = tid; e < T * p.s; e += blockDim.x) {
        const int tc = e / p.s, k = e - tc * p.s;
        const int t = p.rank[tc];
        double g = 0.0;
        for (int uc = 0; uc < T; ++uc) {
            const int u = p.rank[uc];
            const double G = (t <= u) ? tot[3 + gidx(t, u, T)] : tot[3 + gidx(u, t, T)];
            g += G * s_W[uc * p.s + k];
        }
        g_W[e] = sc * g;
    }
    if (tid < T) g_v[tid] = 0.5 * sc * tot[3 + gidx(p.rank[tid], p.rank[tid], T)];
}

// Posterior variance, unequal sizes: for B queries the quadratic forms kappa^H Lambda~^-1 kappa of the
// transformed rows (one N-vector per query in the observation layout), class by class through the
// factor the tree solver left in S: forward elimination u = L^-1 kappa with sum_j |u_j|^2 / D_j.
// Lattices: classes 0 .. nT/2 only, a class with a distinct conjugate counted twice (the rows are
// transforms of real vectors).  part[b * gridDim.x + blockIdx.x] = the sum of this CTA's classes.
template <bool CPLX>
__global__ void __launch_bounds__(kTreeThreads)
k_var_tree(const double* Sb, double* rows, long long N, TreeParams p, double* part) {
    using V = Vt<CPLX>;
    __shared__ V s_part[kTreeCW][kTreeSlots][MTGP_TMAX];
    __shared__ double s_red[kTreeWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = warp * (32 / kTreeCW) + lane / kTreeCW;
    const int cls = lane % kTreeCW;
    const long long nT = p.nT;
    const long long rho = (long long)blockIdx.x * kTreeCW + cls;
    const long long ncls = (CPLX && nT >= 2) ? nT / 2 + 1 : nT;
    const bool act = rho < ncls;
    const bool mir = CPLX && act && rho != 0 && 2 * rho != nT;
    double* rb = rows + (long long)blockIdx.y * N * (CPLX ? 2 : 1);
    double quad = 0.0;
    tree_forward<CPLX>(p, Sb, rb, rho, act, slot, quad, s_part);
    if (mir) quad *= 2.0;
    for (int o = 16; o > 0; o >>= 1) quad += __shfl_down_sync(0xffffffffu, quad, o);
    if (lane == 0) s_red[warp] = quad;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < kTreeWarps; ++w) v += s_red[w];
        part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = v;
    }
}

int eq_blocks(const Handle* h) {
    long long b = (h->n[0] + kEqThreads - 1) / kEqThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (int)b;
}

}  // namespace

int solve_equal_blocks(const Handle* h) { return eq_blocks(h); }
int solve_tree_blocks(const Handle* h) {
    const long long nT = h->n[h->T - 1];
    const long long ncls = (h->cplx && nT >= 2) ? nT / 2 + 1 : nT;  // conjugate classes (lattices)
    return (int)((ncls + kTreeCW - 1) / kTreeCW);
}

template <int T, bool CPLX, typename S>
static void run_eq(const Handle* h, ThetaPtrs th, SolveParams sp, double* partials, cudaStream_t st) {
    k_solve_equal<T, CPLX, S><<<eq_blocks(h), kEqThreads, 0, st>>>(h->spec, h->wgt, h->yhat, sp, th, partials, h->alpha,
                                                                   h->status);
}

template <bool CPLX, typename S>
static void dispatch_eq(const Handle* h, ThetaPtrs th, SolveParams sp, double* partials, cudaStream_t st) {
    switch (h->T) {
        case 1: run_eq<1, CPLX, S>(h, th, sp, partials, st); break;
        case 2: run_eq<2, CPLX, S>(h, th, sp, partials, st); break;
        case 3: run_eq<3, CPLX, S>(h, th, sp, partials, st); break;
        case 4: run_eq<4, CPLX, S>(h, th, sp, partials, st); break;
        case 5: run_eq<5, CPLX, S>(h, th, sp, partials, st); break;
        case 6: run_eq<6, CPLX, S>(h, th, sp, partials, st); break;
        case 7: run_eq<7, CPLX, S>(h, th, sp, partials, st); break;
        default: run_eq<8, CPLX, S>(h, th, sp, partials, st); break;
    }
}

void launch_solve_equal(const Handle* h, ThetaPtrs th, bool grad, double* partials, cudaStream_t st, int gcv,
                        const double* gcv_ab) {
    SolveParams sp;
    sp.T = h->T;
    sp.s = th.s;
    sp.nT = 0;
    sp.grad = (grad && !gcv) ? 1 : 0;
    sp.gcv = gcv;
    sp.gcv_ab = gcv_ab;
    sp.pt = h->noise_pt ? 1 : 0;
    sp.clamp = h->fp32 ? 1 : 0;
    sp.store_alpha = 1;
    for (int t = 0; t < MTGP_TMAX; ++t) {
        sp.n[t] = t < h->T ? h->n[t] : 0;
        sp.order[t] = t < h->T ? h->order[t] : 0;
        sp.yoff[t] = t < h->T ? h->yoff[t] : 0;
        for (int u = 0; u < MTGP_TMAX; ++u) sp.colidx[t][u] = (t < h->T && u < h->T && t <= u) ? h->col_of[t][u] : 0;
    }
    for (int c = 0; c < MTGP_MAX_COLS; ++c) sp.coloff[c] = c < h->ncols ? h->cols[c].off : 0;
    if (h->fp32) {
        if (h->cplx) dispatch_eq<true, float>(h, th, sp, partials, st);
        else dispatch_eq<false, float>(h, th, sp, partials, st);
    } else {
        if (h->cplx) dispatch_eq<true, double>(h, th, sp, partials, st);
        else dispatch_eq<false, double>(h, th, sp, partials, st);
    }
}

static TreeParams tree_params(const Handle* h, int s, bool grad, bool gcv) {
    TreeParams tp;
    tp.T = h->T;
    tp.s = s;
    tp.grad = (grad && !gcv) ? 1 : 0;
    tp.gcv = gcv ? 1 : 0;
    tp.pt = h->noise_pt ? 1 : 0;
    tp.pi_out = h->pi_buf;
    tp.clamp = h->fp32 ? 1 : 0;
    tp.nT = h->n[h->T - 1];
    for (int t = 0; t < MTGP_TMAX; ++t) {
        tp.n[t] = t < h->T ? h->n[t] : 1;
        tp.order[t] = t < h->T ? h->order[t] : 0;
        tp.yoff[t] = t < h->T ? h->yoff[t] : 0;
        for (int u = 0; u < MTGP_TMAX; ++u)
            tp.po[t][u] = (t < h->T && u < h->T && t <= u) ? h->cols[h->col_of[t][u]].off : 0;
    }
    return tp;
}

void launch_var_tree(const Handle* h, double* rows, int B, double* part, cudaStream_t st) {
    const TreeParams tp = tree_params(h, 1, false, false);
    dim3 grid((unsigned)solve_tree_blocks(h), (unsigned)B);
    if (h->cplx) k_var_tree<true><<<grid, kTreeThreads, 0, st>>>(h->S, rows, h->N, tp, part);
    else k_var_tree<false><<<grid, kTreeThreads, 0, st>>>(h->S, rows, h->N, tp, part);
}

void launch_solve_tree(const Handle* h, ThetaPtrs th, bool grad, double* partials, cudaStream_t st, bool gcv) {
    const TreeParams tp = tree_params(h, th.s, grad, gcv);
    int blocks = solve_tree_blocks(h);
    if (h->fp32) {
        if (h->cplx) k_solve_tree<true, float><<<blocks, kTreeThreads, 0, st>>>(h->spec, h->wgt, h->yhat, h->S, h->Z, h->r, h->alpha, h->tau, tp, th, partials, h->status, h->gcv_h);
        else k_solve_tree<false, float><<<blocks, kTreeThreads, 0, st>>>(h->spec, h->wgt, h->yhat, h->S, h->Z, h->r, h->alpha, h->tau, tp, th, partials, h->status, h->gcv_h);
    } else {
        if (h->cplx) k_solve_tree<true, double><<<blocks, kTreeThreads, 0, st>>>(h->spec, h->wgt, h->yhat, h->S, h->Z, h->r, h->alpha, h->tau, tp, th, partials, h->status, h->gcv_h);
        else k_solve_tree<false, double><<<blocks, kTreeThreads, 0, st>>>(h->spec, h->wgt, h->yhat, h->S, h->Z, h->r, h->alpha, h->tau, tp, th, partials, h->status, h->gcv_h);
    }
}

void launch_finalize(const Handle* h, ThetaPtrs th, bool grad, const double* partials, int nsolve,
                     const double* eta_partials, int neta, double* out, double* tau, double* g_eta, double* g_W,
                     double* g_v, double* g_s2, cudaStream_t st, int gcv) {
    FinParams fp;
    fp.gcv = gcv;
    fp.T = h->T;
    fp.d = h->d;
    fp.s = th.s;
    fp.equal = h->equal ? 1 : 0;
    fp.cplx = h->cplx ? 1 : 0;
    fp.NQ = solve_nq(h);
    fp.pt = h->noise_pt ? 1 : 0;
    fp.mix = h->dsi_mix ? 1 : 0;
    fp.nsolve = nsolve;
    fp.neta = neta;
    fp.grad = grad ? 1 : 0;
    fp.N = h->N;
    fp.n0 = h->n[0];
    for (int t = 0; t < MTGP_TMAX; ++t) {
        fp.order[t] = t < h->T ? h->order[t] : 0;
        fp.rank[t] = t < h->T ? h->rank[t] : 0;
        fp.yoff[t] = t < h->T ? h->yoff[t] : 0;
    }
    k_finalize<<<1, 256, 0, st>>>(partials, eta_partials, h->yhat, h->tau, fp, th, out, tau, g_eta, g_W, g_v, g_s2,
                                 h->dsi_mix ? h->bmix + 4 : nullptr);
}

"""The fast-MTGP structure and Algorithm 1, on the CPU in FP64 (numpy), for sizes the dense oracle cannot hold.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. 3.3 of the paper:
  * V_m^dagger a = FFT(bitrev(a)) / sqrt(2^m) (lattice) or FWHT(a) / sqrt(2^m) (digital net)
    (Theorem "fast MTGP computations", closing sentence).
  * tall case n_t >= n_t': lambda_{tt'} = Lambda_{tt'} 1 = sqrt(n_t') V_{m_t}^dagger (K~_{tt'})_{:,0}
    (same theorem, item 3); Lambda_{tt'}[f, f'] = lambda_{tt'}[f] when f' = f mod n_t', else 0.
  * Algorithm 1: Lambda^-1 and log|Lambda| by block bordering over tasks sorted n_1 >= ... >= n_T,
    executed in the paper's step order (D, A, rho; then per task: D, B, L, F, S, rho, G, H, J, M, A).
  * optimal mean: Pi tau = E K~^-1 y with Pi_{tt'} = sqrt(n_t n_t') (Lambda^-1)_{N_{t-1}, N_{t'-1}}
    (same theorem, item 4).
Two solvers that use only the structure stated by that theorem serve the largest sizes:
  * equal sizes: Lambda is block diagonal over frequencies (Corollary "equal sizes"), one T x T
    Cholesky per frequency;
  * unequal sizes: entries of Lambda couple (t, f) and (t', f') only when f = f' mod min(n_t, n_t'),
    so each residue class mod n_T is an independent dense Hermitian system (dense Cholesky per class).
"""
from __future__ import annotations

import numpy as np

from .design import design_points, product_kernel, task_covariance


# ---------------------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------------------

def bitrev_perm(m: int) -> np.ndarray:
    n = 1 << m
    j = np.arange(n)
    r = np.zeros(n, dtype=np.int64)
    for p in range(m):
        r |= ((j >> p) & 1) << (m - 1 - p)
    return r


def fwht(a: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform (Sylvester order) along the last axis."""
    a = np.array(a, dtype=np.result_type(a, np.float64), copy=True)
    n = a.shape[-1]
    h = 1
    while h < n:
        b = a.reshape(a.shape[:-1] + (n // (2 * h), 2, h))
        x = b[..., 0, :].copy()
        y = b[..., 1, :].copy()
        b[..., 0, :] = x + y
        b[..., 1, :] = x - y
        a = b.reshape(a.shape)
        h *= 2
    return a


def vdag(kind: str, a: np.ndarray, m: int) -> np.ndarray:
    """V_m^dagger a along the last axis."""
    n = 1 << m
    if kind == "lattice":
        return np.fft.fft(np.asarray(a)[..., bitrev_perm(m)], axis=-1) / np.sqrt(n)
    return fwht(a) / np.sqrt(n)


def vmul(kind: str, b: np.ndarray, m: int) -> np.ndarray:
    """V_m b along the last axis (inverse of vdag, V unitary)."""
    n = 1 << m
    if kind == "lattice":
        out = np.fft.ifft(np.asarray(b), axis=-1) * np.sqrt(n)
        inv = np.empty(n, dtype=np.int64)
        inv[bitrev_perm(m)] = np.arange(n)
        return out[..., inv]
    return fwht(b) / np.sqrt(n)


# ---------------------------------------------------------------------------------------
# Lambda-tilde
# ---------------------------------------------------------------------------------------

def sorted_order(m):
    """Task order with n_1 >= ... >= n_T (Cond. 3.1 reindexing), ties by user index."""
    return sorted(range(len(m)), key=lambda t: (-int(m[t]), t))


def lambda_blocks(kind, X_sorted, eta, R_sorted, sigma2):
    """lam[(t, u)] for t <= u in sorted order: the length-n_t vector Lambda_{tu} 1 (tall case)."""
    T = len(X_sorted)
    lam = {}
    for t in range(T):
        nt = len(X_sorted[t])
        mt = nt.bit_length() - 1
        for u in range(t, T):
            nu = len(X_sorted[u])
            col = R_sorted[t, u] * product_kernel(kind, X_sorted[t], X_sorted[u][0][None, :], eta)
            if t == u:
                col = col.copy()
                col[0] += sigma2
            lam[(t, u)] = np.sqrt(nu) * vdag(kind, col.astype(np.complex128), mt)
    return lam


def lambda_dense(lam, n):
    """Assemble the full N x N Lambda-tilde (for small checks)."""
    T = len(n)
    off = np.concatenate([[0], np.cumsum(n)])
    L = np.zeros((off[-1], off[-1]), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            f = np.arange(n[t])
            L[off[t] + f, off[u] + (f % n[u])] = lam[(t, u)]
            if u != t:
                L[off[u] + (f % n[u]), off[t] + f] = np.conj(lam[(t, u)])
    return L


# ---------------------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------------------

def _refine(A, r):
    """Re-express a p x p block matrix of n-diagonal blocks (shape (p, p, n)) with (n/r)-diagonal
    blocks: block row (t', j) becomes rows (t', j r + q), q < r, since f = (j r + q)(n/r) + rho."""
    p, _, n = A.shape
    nn = n // r
    out = np.zeros((p * r, p * r, nn), dtype=A.dtype)
    Ar = A.reshape(p, p, r, nn)
    for q in range(r):
        out[q::r, q::r, :] = Ar[:, :, q, :]
    return out


def algorithm1(lam, n):
    """Inverse and log-determinant of Lambda-tilde, Algorithm 1, step by step.

    Block matrices whose blocks are n_t x n_t diagonal are stored as arrays (rows, cols, n_t).
    Block row b of stage t stands for task t' = owner(b) and frequencies f = j n_t + rho.
    Returns (A, rho) with A the (P, P, n_T) representation of Lambda^-1 and rho = log|Lambda|.
    """
    T = len(n)
    D = lam[(0, 0)].real.reshape(1, 1, n[0])                 # D <- Lambda_11
    A = (1.0 / D).astype(np.complex128)                       # A <- D^-1
    rho = float(np.sum(np.log(D)))                            # rho <- log|D|
    for t in range(1, T):
        A = _refine(A, n[t - 1] // n[t])                      # same matrix, n_t-diagonal blocks
        D = lam[(t, t)].real.reshape(1, 1, n[t])              # D <- Lambda_tt
        B = np.concatenate([lam[(u, t)].reshape(n[u] // n[t], 1, n[t]) for u in range(t)], axis=0)
        Lm = np.einsum("abk,bck->ack", A, B)                  # L <- A B
        F = np.einsum("bak,bck->ack", np.conj(B), Lm)         # F <- B^dagger L
        S = D - F.real                                        # S <- D - F (Schur complement, diagonal)
        if np.any(S <= 0):
            raise np.linalg.LinAlgError("Schur complement not positive")
        rho += float(np.sum(np.log(S)))                       # rho <- rho + log|S|
        G = 1.0 / S                                           # G <- S^-1
        H = Lm * G                                            # H <- L G
        J = np.einsum("ak,bk->abk", H[:, 0, :], np.conj(Lm[:, 0, :]))   # J <- H L^dagger
        M = A + J                                             # M <- A + J
        p = A.shape[0]
        An = np.empty((p + 1, p + 1, n[t]), dtype=np.complex128)
        An[:p, :p] = M                                        # A <- [[M, -H], [-H^dagger, G]]
        An[:p, p] = -H[:, 0, :]
        An[p, :p] = -np.conj(H[:, 0, :])
        An[p, p] = G[0, 0]
        A = An
    return A, rho


def block_rows(n):
    """(task, j) of each block row of Algorithm 1's final representation (n_T-diagonal blocks)."""
    rows = []
    for t in range(len(n)):
        rows += [(t, j) for j in range(n[t] // n[-1])]
    return rows


def apply_inverse(A, n, vecs):
    """Lambda^-1 applied to a vector given per task (list of length-n_t arrays), via Algorithm 1's A."""
    nT = n[-1]
    rows = block_rows(n)
    flat = np.stack([vecs[t][j * nT:(j + 1) * nT] for (t, j) in rows])   # (P, n_T)
    res = np.einsum("abk,bk->ak", A, flat)
    out = [np.zeros(n[t], dtype=np.complex128) for t in range(len(n))]
    for b, (t, j) in enumerate(rows):
        out[t][j * nT:(j + 1) * nT] = res[b]
    return out


def nll_algorithm1(kind, gen, shift, m, y, eta, W, v, sigma2):
    """MLE loss (Eq. 3.3) via Theorem (fast MTGP computations) and Algorithm 1."""
    order = sorted_order(m)
    n_user = [1 << int(x) for x in m]
    offs = np.concatenate([[0], np.cumsum(n_user)])
    X = [design_points(kind, gen, shift[t], n_user[t]) for t in order]
    ys = [np.asarray(y[offs[t]:offs[t + 1]], dtype=np.float64) for t in order]
    R = task_covariance(W, v)[np.ix_(order, order)]
    n = [n_user[t] for t in order]
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    A, rho = algorithm1(lam, n)
    yhat = [vdag(kind, ys[t].astype(np.complex128), int(np.log2(n[t]))) for t in range(len(n))]
    # optimal mean (theorem item 4): Pi tau = E K^-1 y
    rows = block_rows(n)
    first = [rows.index((t, 0)) for t in range(len(n))]
    Pi = np.array([[np.sqrt(n[t] * n[u]) * A[first[t], first[u], 0] for u in range(len(n))]
                   for t in range(len(n))]).real
    Ly = apply_inverse(A, n, yhat)
    b = np.array([np.sqrt(n[t]) * Ly[t][0] for t in range(len(n))]).real
    tau_s = np.linalg.solve(Pi, b)
    rhat = [yh.copy() for yh in yhat]
    for t in range(len(n)):
        rhat[t][0] -= np.sqrt(n[t]) * tau_s[t]
    Lr = apply_inverse(A, n, rhat)
    quad = float(sum(np.vdot(rhat[t], Lr[t]).real for t in range(len(n))))
    tau = np.empty(len(n))
    tau[order] = tau_s
    N = sum(n)
    return dict(L=quad + rho, nll=0.5 * (quad + rho + N * np.log(2 * np.pi)), quad=quad, logdet=rho, tau=tau)


# ---------------------------------------------------------------------------------------
# per-frequency (equal sizes) and per-residue-class (unequal sizes) solvers
# ---------------------------------------------------------------------------------------

def class_matrix(lam, n, rho):
    """Dense Hermitian system of residue class rho mod n_T; node list [(t, f)]."""
    T = len(n)
    nT = n[-1]
    nodes = [(t, f) for t in range(T) for f in range(rho, n[t], nT)]
    idx = {nd: i for i, nd in enumerate(nodes)}
    P = len(nodes)
    M = np.zeros((P, P), dtype=np.complex128)
    for (t, f), i in idx.items():
        for u in range(t, T):
            j = idx[(u, f % n[u])]
            val = lam[(t, u)][f]
            if u == t:
                M[i, i] = val.real
            else:
                M[i, j] = val
                M[j, i] = np.conj(val)
    return nodes, M


def nll_by_class(kind, gen, shift, m, y, eta, W, v, sigma2, want_alpha=False):
    """MLE loss via independent dense Cholesky per residue class mod n_T (equal sizes: per frequency)."""
    order = sorted_order(m)
    n_user = [1 << int(x) for x in m]
    offs = np.concatenate([[0], np.cumsum(n_user)])
    X = [design_points(kind, gen, shift[t], n_user[t]) for t in order]
    ys = [np.asarray(y[offs[t]:offs[t + 1]], dtype=np.float64) for t in order]
    R = task_covariance(W, v)[np.ix_(order, order)]
    n = [n_user[t] for t in order]
    T = len(n)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    yhat = [vdag(kind, ys[t].astype(np.complex128), int(np.log2(n[t]))) for t in range(T)]
    nT = n[-1]
    # class 0 carries the optimal mean
    nodes0, M0 = class_matrix(lam, n, 0)
    Minv0 = np.linalg.inv(M0)
    pos0 = [nodes0.index((t, 0)) for t in range(T)]
    Pi = np.array([[np.sqrt(n[t] * n[u]) * Minv0[pos0[t], pos0[u]] for u in range(T)] for t in range(T)]).real
    yv0 = np.array([yhat[t][f] for (t, f) in nodes0])
    sol0 = Minv0 @ yv0
    b = np.array([np.sqrt(n[t]) * sol0[pos0[t]] for t in range(T)]).real
    tau_s = np.linalg.solve(Pi, b)
    rhat = [yh.copy() for yh in yhat]
    for t in range(T):
        rhat[t][0] -= np.sqrt(n[t]) * tau_s[t]
    quad = 0.0
    logdet = 0.0
    alpha = [np.zeros(n[t], dtype=np.complex128) for t in range(T)]
    for rho in range(nT):
        nodes, M = class_matrix(lam, n, rho)
        Lc = np.linalg.cholesky(M)
        d = np.real(np.diag(Lc))
        if np.any(d <= 0) or not np.all(np.isfinite(d)):
            raise np.linalg.LinAlgError("class matrix not positive definite")
        logdet += 2.0 * float(np.sum(np.log(d)))
        rv = np.array([rhat[t][f] for (t, f) in nodes])
        z = np.linalg.solve(Lc, rv)
        quad += float(np.vdot(z, z).real)
        if want_alpha:
            a = np.linalg.solve(Lc.conj().T, z)
            for (t, f), val in zip(nodes, a):
                alpha[t][f] = val
    tau = np.empty(T)
    tau[order] = tau_s
    N = sum(n)
    out = dict(L=quad + logdet, nll=0.5 * (quad + logdet + N * np.log(2 * np.pi)), quad=quad,
               logdet=logdet, tau=tau)
    if want_alpha:
        out.update(alpha=alpha, order=order, n_sorted=n, X_sorted=X, R_sorted=R, lam=lam)
    return out


def nll_equal(kind, gen, shift, m, y, eta, W, v, sigma2):
    """Equal sizes: per-frequency T x T Cholesky (Corollary 'equal sizes'); vectorised over frequencies."""
    T = len(m)
    if len(set(int(x) for x in m)) != 1:
        raise ValueError("equal sizes required")
    mm = int(m[0])
    n = 1 << mm
    X = [design_points(kind, gen, shift[t], n) for t in range(T)]
    R = task_covariance(W, v)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    Lam = np.zeros((n, T, T), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            Lam[:, t, u] = lam[(t, u)]
            Lam[:, u, t] = np.conj(lam[(t, u)])
        Lam[:, t, t] = lam[(t, t)].real
    ys = np.asarray(y, dtype=np.float64).reshape(T, n)
    yhat = vdag(kind, ys.astype(np.complex128), mm)          # (T, n)
    tau = yhat[:, 0].real / np.sqrt(n)                         # sample means (Pi = n Lambda(0)^-1)
    rhat = yhat.copy()
    rhat[:, 0] = 0.0
    Lc = np.linalg.cholesky(Lam)
    dg = np.real(np.diagonal(Lc, axis1=1, axis2=2))
    if np.any(dg <= 0):
        raise np.linalg.LinAlgError("frequency matrix not positive definite")
    logdet = 2.0 * float(np.sum(np.log(dg)))
    z = np.linalg.solve(Lc, rhat.T[:, :, None])[:, :, 0]
    quad = float(np.sum(np.abs(z) ** 2))
    N = T * n
    return dict(L=quad + logdet, nll=0.5 * (quad + logdet + N * np.log(2 * np.pi)), quad=quad,
                logdet=logdet, tau=tau)


def gcv_by_class(kind, gen, shift, m, y, eta, W, v, sigma2):
    """GCV loss via the residue classes mod n_T: tau_GCV from (H H^*) tau = E K~^-2 y with
    H = (sqrt(n_t) (Lambda~^-1)_{(t,0), k}) over the nodes k of class 0 (Theorem FMTGP item 4),
    then num = ||Lambda~^-1 rhat||^2 and trace = trace(Lambda~^-1) summed over classes."""
    order = sorted_order(m)
    n_user = [1 << int(x) for x in m]
    offs = np.concatenate([[0], np.cumsum(n_user)])
    X = [design_points(kind, gen, shift[t], n_user[t]) for t in order]
    ys = [np.asarray(y[offs[t]:offs[t + 1]], dtype=np.float64) for t in order]
    R = task_covariance(W, v)[np.ix_(order, order)]
    n = [n_user[t] for t in order]
    T = len(n)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    yhat = [vdag(kind, ys[t].astype(np.complex128), int(np.log2(n[t]))) for t in range(T)]
    nT = n[-1]
    nodes0, M0 = class_matrix(lam, n, 0)
    Minv0 = np.linalg.inv(M0)
    pos0 = [nodes0.index((t, 0)) for t in range(T)]
    H = np.array([np.sqrt(n[t]) * Minv0[pos0[t], :] for t in range(T)])
    yv0 = np.array([yhat[t][f] for (t, f) in nodes0])
    HH = (H @ H.conj().T).real
    b = (H @ (Minv0 @ yv0)).real
    tau_s = np.linalg.solve(HH, b)
    rhat = [yh.copy() for yh in yhat]
    for t in range(T):
        rhat[t][0] -= np.sqrt(n[t]) * tau_s[t]
    num = 0.0
    tr = 0.0
    for rho in range(nT):
        nodes, M = class_matrix(lam, n, rho)
        Minv = np.linalg.inv(M)
        rv = np.array([rhat[t][f] for (t, f) in nodes])
        a = Minv @ rv
        num += float(np.vdot(a, a).real)
        tr += float(np.trace(Minv).real)
    tau = np.empty(T)
    tau[order] = tau_s
    return dict(L=num / tr ** 2, num=num, trace=tr, tau=tau)


def gcv_equal(kind, gen, shift, m, y, eta, W, v, sigma2):
    """Equal sizes: tau_GCV is the vector of sample means (Pi-like matrix n Lambda(0)^-2) and the
    per-frequency T x T inverses give num = sum_f ||Lambda(f)^-1 rhat(f)||^2, trace = sum_f tr."""
    T = len(m)
    mm = int(m[0])
    n = 1 << mm
    X = [design_points(kind, gen, shift[t], n) for t in range(T)]
    R = task_covariance(W, v)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    Lam = np.zeros((n, T, T), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            Lam[:, t, u] = lam[(t, u)]
            Lam[:, u, t] = np.conj(lam[(t, u)])
        Lam[:, t, t] = lam[(t, t)].real
    ys = np.asarray(y, dtype=np.float64).reshape(T, n)
    yhat = vdag(kind, ys.astype(np.complex128), mm)
    tau = yhat[:, 0].real / np.sqrt(n)
    rhat = yhat.copy()
    rhat[:, 0] = 0.0
    Z = np.linalg.inv(Lam)
    a = (Z @ rhat.T[:, :, None])[:, :, 0]
    num = float(np.sum(np.abs(a) ** 2))
    tr = float(np.sum(np.real(np.trace(Z, axis1=1, axis2=2))))
    return dict(L=num / tr ** 2, num=num, trace=tr, tau=tau)


def posterior_by_class(kind, gen, shift, m, y, eta, W, v, sigma2, Xq, task_q):
    """Posterior mean / variance (Eq. 3.2) at a few queries using the per-class solver for K~^-1."""
    out = nll_by_class(kind, gen, shift, m, y, eta, W, v, sigma2, want_alpha=True)
    order, n, X, R, lam = out["order"], out["n_sorted"], out["X_sorted"], out["R_sorted"], out["lam"]
    T = len(n)
    alpha = out["alpha"]
    beta = [vmul(kind, alpha[t], int(np.log2(n[t]))).real for t in range(T)]   # K~^-1 r per task
    pos = {u: i for i, u in enumerate(order)}                                 # user -> sorted
    tau = out["tau"]
    nT = n[-1]
    mean = np.empty(len(task_q))
    var = np.empty(len(task_q))
    for qi in range(len(task_q)):
        ts = pos[int(task_q[qi])]
        kv = [R[ts, u] * product_kernel(kind, X[u], Xq[qi][None, :], eta) for u in range(T)]
        mean[qi] = tau[int(task_q[qi])] + sum(float(kv[u] @ beta[u]) for u in range(T))
        kh = [vdag(kind, kv[u].astype(np.complex128), int(np.log2(n[u]))) for u in range(T)]
        acc = 0.0
        for rho in range(nT):
            nodes, M = class_matrix(lam, n, rho)
            kvec = np.array([kh[t][f] for (t, f) in nodes])
            acc += float(np.vdot(kvec, np.linalg.solve(M, kvec)).real)
        prior = R[ts, ts] * float(product_kernel(kind, Xq[qi], Xq[qi], eta))
        var[qi] = prior - acc
    return mean, var


def posterior_mean_equal(kind, gen, shift, m, y, eta, W, v, sigma2, Xq, task_q):
    """Posterior mean (Eq. 3.2) for equal sizes: alpha(f) = Lambda(f)^-1 rhat(f) per frequency,
    beta_t = V alpha_t (= K~^-1 r per task), mean_t(x) = tau_t + sum_u R_tu sum_i Q(x, x_ui) beta_u[i]."""
    T = len(m)
    mm = int(m[0])
    n = 1 << mm
    X = [design_points(kind, gen, shift[t], n) for t in range(T)]
    R = task_covariance(W, v)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    Lam = np.zeros((n, T, T), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            Lam[:, t, u] = lam[(t, u)]
            Lam[:, u, t] = np.conj(lam[(t, u)])
        Lam[:, t, t] = lam[(t, t)].real
    ys = np.asarray(y, dtype=np.float64).reshape(T, n)
    yhat = vdag(kind, ys.astype(np.complex128), mm)
    tau = yhat[:, 0].real / np.sqrt(n)
    rhat = yhat.copy()
    rhat[:, 0] = 0.0
    alpha = np.linalg.solve(Lam, rhat.T[:, :, None])[:, :, 0].T        # (T, n)
    beta = vmul(kind, alpha, mm).real
    mean = np.empty(len(task_q))
    for qi in range(len(task_q)):
        t = int(task_q[qi])
        mean[qi] = tau[t] + sum(R[t, u] * float(product_kernel(kind, X[u], Xq[qi][None, :], eta) @ beta[u])
                                for u in range(T))
    return mean


def posterior_var_equal(kind, gen, shift, m, eta, W, v, sigma2, Xq, task_q):
    """Posterior variance (Eq. 3.2) for equal sizes, query by query: kappa_u = R_{t u} V^dagger q_u(x)
    with q_u(x)[i] = Q(x, x_ui), var = R_tt Q(x, x) - sum_f kappa(f)^H Lambda(f)^-1 kappa(f)."""
    T = len(m)
    mm = int(m[0])
    n = 1 << mm
    X = [design_points(kind, gen, shift[t], n) for t in range(T)]
    R = task_covariance(W, v)
    lam = lambda_blocks(kind, X, eta, R, sigma2)
    Lam = np.zeros((n, T, T), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            Lam[:, t, u] = lam[(t, u)]
            Lam[:, u, t] = np.conj(lam[(t, u)])
        Lam[:, t, t] = lam[(t, t)].real
    var = np.empty(len(task_q))
    for qi in range(len(task_q)):
        t = int(task_q[qi])
        kap = np.stack([R[t, u] * vdag(kind, product_kernel(kind, X[u], Xq[qi][None, :], eta).astype(np.complex128), mm)
                        for u in range(T)], axis=1)                        # (n, T)
        sol = np.linalg.solve(Lam, kap[:, :, None])[:, :, 0]
        prior = R[t, t] * float(product_kernel(kind, Xq[qi], Xq[qi], eta))
        var[qi] = prior - float(np.sum(np.conj(kap) * sol).real)
    return var


def nll_grad_equal(kind, gen, shift, m, y, eta, W, v, sigma2, alpha=2):
    """Equal sizes: L (Eq. 3.3) and its gradient by per-frequency traces, dL/dtheta = sum_f tr(G(f) dLambda(f)),
    G(f) = Lambda(f)^-1 - alpha(f) alpha(f)^H, every dLambda(f)/dtheta formed explicitly:
      dLambda/d eta_j = R o dM_j(f)  (dM_j = transforms of the columns' eta_j derivatives),
      dLambda/d W_ts  = (e_t W_s^T + W_s e_t^T) o M(f),  dLambda/d v_t = e_t e_t^T o M(f),  dLambda/d sigma2 = I.
    Returns (out, g_eta, g_W, g_v, g_sigma2) for L (the NLL gradient is half of it).  With the four DSI
    mixture weights b of Eq. 2.6 as ``alpha`` (digital nets), also g_b (4,) last, from
      dLambda/d b_a = R o dB_a(f),  dB_a = transforms of sum_j eta_j K_a(x_j) prod_{l != j} (1 + eta_l K(x_l))."""
    from .design import kernel_1d
    mix = np.ndim(alpha) > 0
    T = len(m)
    mm = int(m[0])
    n = 1 << mm
    X = [design_points(kind, gen, shift[t], n) for t in range(T)]
    R = task_covariance(W, v)
    d = len(eta)
    M = np.zeros((n, T, T), dtype=np.complex128)
    dM = np.zeros((d, n, T, T), dtype=np.complex128)
    dB = np.zeros((4, n, T, T), dtype=np.complex128)
    for t in range(T):
        for u in range(t, T):
            K1 = [kernel_1d(kind, X[t][:, j], np.full(n, X[u][0, j], dtype=np.uint64), alpha) for j in range(d)]
            fac = [1.0 + eta[j] * K1[j] for j in range(d)]
            col = np.prod(fac, axis=0)
            mu = np.sqrt(n) * vdag(kind, col.astype(np.complex128), mm)
            M[:, t, u] = mu
            M[:, u, t] = np.conj(mu)
            for j in range(d):
                dcol = K1[j] * np.prod([fac[l] for l in range(d) if l != j], axis=0) if d > 1 else K1[j]
                dmu = np.sqrt(n) * vdag(kind, dcol.astype(np.complex128), mm)
                dM[j, :, t, u] = dmu
                dM[j, :, u, t] = np.conj(dmu)
            if mix:
                for a_ in range(1, 5):
                    dcol = np.zeros(n)
                    for j in range(d):
                        Ka = kernel_1d(kind, X[t][:, j], np.full(n, X[u][0, j], dtype=np.uint64), a_)
                        dcol += eta[j] * Ka * np.prod([fac[l] for l in range(d) if l != j], axis=0) if d > 1 \
                            else eta[j] * Ka
                    dmu = np.sqrt(n) * vdag(kind, dcol.astype(np.complex128), mm)
                    dB[a_ - 1, :, t, u] = dmu
                    dB[a_ - 1, :, u, t] = np.conj(dmu)
    for t in range(T):
        M[:, t, t] = M[:, t, t].real
        dM[:, :, t, t] = dM[:, :, t, t].real
        dB[:, :, t, t] = dB[:, :, t, t].real
    Lam = R[None, :, :] * M + sigma2 * np.eye(T)[None, :, :]
    ys = np.asarray(y, dtype=np.float64).reshape(T, n)
    rhat = vdag(kind, ys.astype(np.complex128), mm).T.copy()     # (n, T)
    tau = rhat[0].real / np.sqrt(n)
    rhat[0] = 0.0
    Lc = np.linalg.cholesky(Lam)
    logdet = 2.0 * float(np.sum(np.log(np.real(np.diagonal(Lc, axis1=1, axis2=2)))))
    Z = np.linalg.inv(Lam)
    a = np.einsum("fab,fb->fa", Z, rhat)
    quad = float(np.einsum("fa,fa->", np.conj(rhat), a).real)
    G = Z - a[:, :, None] * np.conj(a[:, None, :])

    def tr(dLam):
        return float(np.einsum("fba,fab->", G, dLam).real)

    g_eta = np.array([tr(R[None] * dM[j]) for j in range(d)])
    s = W.shape[1]
    g_W = np.zeros_like(W)
    for t in range(T):
        for k in range(s):
            e = np.zeros(T)
            e[t] = 1.0
            dR = np.outer(e, W[:, k]) + np.outer(W[:, k], e)
            g_W[t, k] = tr(dR[None] * M)
    g_v = np.array([tr(np.diag(np.eye(T)[t])[None] * M) for t in range(T)])
    g_s2 = float(np.einsum("faa->", G).real)
    N = T * n
    out = dict(L=quad + logdet, nll=0.5 * (quad + logdet + N * np.log(2 * np.pi)), quad=quad, logdet=logdet, tau=tau)
    if mix:
        return out, g_eta, g_W, g_v, g_s2, np.array([tr(R[None] * dB[a_]) for a_ in range(4)])
    return out, g_eta, g_W, g_v, g_s2


def grad_by_class(kind, gen, shift, m, y, eta, W, v, sigma2, loss="mle"):
    """Gradient of L (Eq. 3.3, MLE or GCV form) through the residue classes mod n_T (unequal nested
    sizes; any sizes), tau held at the loss's own optimum.  With M_rho the class matrix and every
    dM_rho/dtheta assembled from the transformed first columns of the derivative kernels exactly as
    M_rho is assembled from the kernel's (theorem item 3):
      MLE: dL = sum_rho Re tr(G_rho dM_rho),  G = M^-1 - a a^H,  a = M^-1 rhat;
      GCV: G = -(a b^H + b a^H) / B^2 + (2 A / B^3) M^-2,  b = M^-1 a,
           A = sum_rho ||a||^2, B = sum_rho tr M^-1.
    One shared sigma2.  Returns (L, g_eta, g_W, g_v, g_sigma2), W and v in user task order."""
    from .design import kernel_1d
    order = sorted_order(m)
    n_user = [1 << int(x) for x in m]
    offs = np.concatenate([[0], np.cumsum(n_user)])
    X = [design_points(kind, gen, shift[t], n_user[t]) for t in order]
    ys = [np.asarray(y[offs[t]:offs[t + 1]], dtype=np.float64) for t in order]
    Ru = task_covariance(W, v)
    R = Ru[np.ix_(order, order)]
    n = [n_user[t] for t in order]
    T, d = len(n), len(eta)
    if np.ndim(sigma2) != 0:
        raise NotImplementedError("one shared noise variance (per-task noise: the dense oracle)")
    sig = np.full(T, float(sigma2))
    ref = (nll_by_class if loss == "mle" else gcv_by_class)(kind, gen, shift, m, y, eta, W, v, float(sigma2))
    tau_s = np.asarray(ref["tau"])[order]
    mt = [int(np.log2(x)) for x in n]
    yhat = [vdag(kind, ys[t].astype(np.complex128), mt[t]) for t in range(T)]
    rhat = [yh.copy() for yh in yhat]
    for t in range(T):
        rhat[t][0] -= np.sqrt(n[t]) * tau_s[t]
    # transformed first columns of Q and of its eta derivatives (sorted pairs t <= u)
    lamQ, dlamQ = {}, {}
    for t in range(T):
        for u in range(t, T):
            K1 = [kernel_1d(kind, X[t][:, j], np.full(n[t], X[u][0, j], dtype=np.uint64)) for j in range(d)]
            fac = [1.0 + eta[j] * K1[j] for j in range(d)]
            sc = np.sqrt(n[u])
            lamQ[(t, u)] = sc * vdag(kind, np.prod(fac, axis=0).astype(np.complex128), mt[t])
            dlamQ[(t, u)] = [sc * vdag(kind, (K1[j] * np.prod([fac[l] for l in range(d) if l != j], axis=0)
                                              if d > 1 else K1[j]).astype(np.complex128), mt[t]) for j in range(d)]

    def blocks(dR=None, eta_j=None, noise=None):
        out = {}
        for t in range(T):
            for u in range(t, T):
                if eta_j is not None:
                    val = R[t, u] * dlamQ[(t, u)][eta_j]
                elif dR is not None:
                    val = dR[t, u] * lamQ[(t, u)]
                else:
                    val = np.zeros(n[t], dtype=np.complex128)
                if noise is not None and t == u:
                    val = val + noise[t]
                out[(t, u)] = val
        return out

    lam = blocks(dR=R, noise=sig)
    classes = []
    A = Bt = 0.0
    for rho in range(n[-1]):
        nodes, M = class_matrix(lam, n, rho)
        Minv = np.linalg.inv(M)
        a = Minv @ np.array([rhat[t][f] for (t, f) in nodes])
        classes.append((rho, Minv, a))
        A += float(np.vdot(a, a).real)
        Bt += float(np.trace(Minv).real)

    def contract(blk):
        tot = 0.0
        for rho, Minv, a in classes:
            _, dM = class_matrix(blk, n, rho)
            if loss == "mle":
                G = Minv - np.outer(a, a.conj())
            else:
                b = Minv @ a
                G = -(np.outer(a, b.conj()) + np.outer(b, a.conj())) / Bt ** 2 + (2.0 * A / Bt ** 3) * (Minv @ Minv)
            tot += float(np.sum(G * dM.T).real)           # tr(G dM)
        return tot

    g_eta = np.array([contract(blocks(eta_j=j)) for j in range(d)])
    s = W.shape[1]
    g_W = np.zeros_like(W)
    for tc in range(T):
        for k in range(s):
            e = np.zeros(T)
            e[tc] = 1.0
            dRu = np.outer(e, W[:, k]) + np.outer(W[:, k], e)
            g_W[tc, k] = contract(blocks(dR=dRu[np.ix_(order, order)]))
    g_v = np.zeros(T)
    for tc in range(T):
        dRu = np.zeros((T, T))
        dRu[tc, tc] = 1.0
        g_v[tc] = contract(blocks(dR=dRu[np.ix_(order, order)]))
    g_s2 = contract(blocks(noise=np.ones(T)))
    return ref["L"], g_eta, g_W, g_v, g_s2

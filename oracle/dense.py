"""The plain definition of the multitask GP quantities: dense Gram matrix and dense Cholesky.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Everything follows Sec. 3.1 of the paper directly, with no structure exploited:
  * Gram matrix  K~_{tt'} = R_{tt'} Q(X_t, X_t') + delta_{tt'} xi I  (Eq. 3.1 and the text after Eq. 3.2),
    a single noise xi = sigma2 for all tasks, gamma = 1.
  * optimal means  (E K~^-1 E^T) tau = E K~^-1 y                        (Eq. 3.4, MLE)
  * loss           L = (y - E^T tau)^T K~^-1 (y - E^T tau) + log|K~|    (Eq. 3.3, MLE)
  * NLL            = (L + N log 2 pi) / 2
  * gradient       dL/dtheta = tr(K~^-1 dK~) - a^T dK~ a, a = K~^-1 r, at tau fixed (tau minimises L)
  * posterior      mean_t(x) = tau_t + k(t,x)^T K~^-1 r,  var_t(x) = K((t,x),(t,x)) - k^T K~^-1 k  (Eq. 3.2)
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .design import design_points, product_kernel, task_covariance, kernel_1d


def all_points(kind, gen, shift, m):
    """Design points of every task (Cond. 3.1: common generator, per-task shift)."""
    return [design_points(kind, gen, shift[t], 1 << int(m[t])) for t in range(len(m))]


def gram(kind, X_tasks, eta, R, sigma2, alpha=2):
    """Dense K~ (N x N), tasks in the given order, each in radical-inverse order (alpha: SI smoothness)."""
    T = len(X_tasks)
    n = [len(X) for X in X_tasks]
    off = np.concatenate([[0], np.cumsum(n)])
    K = np.empty((off[-1], off[-1]))
    for t in range(T):
        for u in range(T):
            Q = product_kernel(kind, X_tasks[t][:, None, :], X_tasks[u][None, :, :], eta, alpha=alpha)
            K[off[t]:off[t + 1], off[u]:off[u + 1]] = R[t, u] * Q
    # noise: one variance sigma2, or one per task (xi_t of Eq. 3.1's data model) when given T values
    sig = np.asarray(sigma2, dtype=np.float64)
    if sig.ndim == 0:
        K[np.diag_indices_from(K)] += float(sig)
    else:
        for t in range(T):
            idx = np.arange(off[t], off[t + 1])
            K[idx, idx] += sig[t]
    return K


def summing_matrix(n):
    """E in R^{T x N}: row t has ones on task t's block (text after Eq. 3.2)."""
    T = len(n)
    E = np.zeros((T, sum(n)))
    off = 0
    for t in range(T):
        E[t, off:off + n[t]] = 1.0
        off += n[t]
    return E


def nll(kind, X_tasks, y, eta, W, v, sigma2, alpha=2):
    """Returns dict with L (Eq. 3.3), nll, quad, logdet, tau (Eq. 3.4) by dense Cholesky."""
    R = task_covariance(W, v)
    K = gram(kind, X_tasks, eta, R, sigma2, alpha)
    n = [len(X) for X in X_tasks]
    N = sum(n)
    E = summing_matrix(n)
    cf = sla.cho_factor(K, lower=True)
    Kinv_Et = sla.cho_solve(cf, E.T)
    Kinv_y = sla.cho_solve(cf, y)
    Pi = E @ Kinv_Et
    tau = np.linalg.solve(Pi, E @ Kinv_y)
    r = y - E.T @ tau
    a = sla.cho_solve(cf, r)
    quad = float(r @ a)
    logdet = float(2.0 * np.sum(np.log(np.diag(cf[0]))))
    L = quad + logdet
    return dict(L=L, nll=0.5 * (L + N * np.log(2 * np.pi)), quad=quad, logdet=logdet,
                tau=tau, alpha=a, Pi=Pi)


def gcv(kind, X_tasks, y, eta, W, v, sigma2, alpha=2):
    """GCV loss (Eq. 3.3, second form) at the GCV mean (Eq. 3.4, second form), by dense inverses:
    tau solves (E K~^-2 E^T) tau = E K~^-2 y, r = y - E^T tau, L = r^T K~^-2 r / trace(K~^-1)^2.
    Returns dict L, num (r^T K~^-2 r), trace (trace K~^-1), tau."""
    R = task_covariance(W, v)
    K = gram(kind, X_tasks, eta, R, sigma2, alpha)
    n = [len(X) for X in X_tasks]
    E = summing_matrix(n)
    Kinv = np.linalg.inv(K)
    Kinv = 0.5 * (Kinv + Kinv.T)
    K2 = Kinv @ Kinv
    tau = np.linalg.solve(E @ K2 @ E.T, E @ K2 @ y)
    r = y - E.T @ tau
    num = float(r @ K2 @ r)
    tr = float(np.trace(Kinv))
    return dict(L=num / tr ** 2, num=num, trace=tr, tau=tau)


def _param_contractions(kind, X_tasks, eta, W, R, K, contract, alpha=2, sigma2_shape=0.0):
    """contract(dK~/dtheta) for every parameter: eta (d), W (T x s), v (T), sigma2, with the dense
    derivatives of K~ written out (see nll_grad)."""
    T = len(X_tasks)
    n = [len(X) for X in X_tasks]
    off = np.concatenate([[0], np.cumsum(n)])
    d = len(eta)
    # univariate kernel blocks per dimension
    K1 = [[None] * T for _ in range(T)]
    for t in range(T):
        for u in range(T):
            K1[t][u] = [kernel_1d(kind, X_tasks[t][:, None, j], X_tasks[u][None, :, j], alpha) for j in range(d)]
    g_eta = np.zeros(d)
    for j in range(d):
        dK = np.zeros_like(K)
        for t in range(T):
            for u in range(T):
                blk = K1[t][u][j].copy()
                for l in range(d):
                    if l != j:
                        blk = blk * (1.0 + eta[l] * K1[t][u][l])
                dK[off[t]:off[t + 1], off[u]:off[u + 1]] = R[t, u] * blk
        g_eta[j] = contract(dK)
    Qfull = gram(kind, X_tasks, eta, np.ones((T, T)), 0.0, alpha)

    def blockwise(dR):
        dK = np.empty_like(K)
        for t in range(T):
            for u in range(T):
                dK[off[t]:off[t + 1], off[u]:off[u + 1]] = dR[t, u] * Qfull[off[t]:off[t + 1], off[u]:off[u + 1]]
        return dK

    s = W.shape[1]
    g_W = np.zeros_like(W)
    for t in range(T):
        for k in range(s):
            e = np.zeros(T)
            e[t] = 1.0
            dR = np.outer(e, W[:, k]) + np.outer(W[:, k], e)
            g_W[t, k] = contract(blockwise(dR))
    g_v = np.zeros(T)
    for t in range(T):
        dR = np.zeros((T, T))
        dR[t, t] = 1.0
        g_v[t] = contract(blockwise(dR))
    if np.ndim(sigma2_shape) == 0:
        g_s2 = contract(np.eye(K.shape[0]))
    else:
        g_s2 = np.zeros(T)
        for t in range(T):
            dK = np.zeros_like(K)
            idx = np.arange(off[t], off[t + 1])
            dK[idx, idx] = 1.0
            g_s2[t] = contract(dK)
    return g_eta, g_W, g_v, g_s2


def _gcv_weights(kind, X_tasks, y, eta, W, v, sigma2, alpha=2):
    """The GCV loss and the dense matrix G with dL_GCV = sum(G * dK~) (see gcv_grad)."""
    out = gcv(kind, X_tasks, y, eta, W, v, sigma2, alpha)
    R = task_covariance(W, v)
    K = gram(kind, X_tasks, eta, R, sigma2, alpha)
    n = [len(X) for X in X_tasks]
    E = summing_matrix(n)
    Kinv = np.linalg.inv(K)
    Kinv = 0.5 * (Kinv + Kinv.T)
    r = y - E.T @ out["tau"]
    a = Kinv @ r
    b = Kinv @ a
    A, B = float(a @ a), float(np.trace(Kinv))
    G = -(np.outer(a, b) + np.outer(b, a)) / B ** 2 + (2.0 * A / B ** 3) * (Kinv @ Kinv)
    return out, R, K, G


def gcv_grad(kind, X_tasks, y, eta, W, v, sigma2, alpha=2):
    """Analytic gradient of the GCV loss (Eq. 3.3, second form) at the GCV mean (fixed by the envelope
    theorem: tau_GCV minimises the numerator, the trace does not depend on tau).  With a = K~^-1 r,
    b = K~^-1 a, A = a^T a, B = trace K~^-1:
        dL = dA / B^2 - 2 A dB / B^3,  dA = -2 a^T dK~ b,  dB = -trace(K~^-2 dK~),
    i.e. dL = sum(G * dK~) with G = -(a b^T + b a^T) / B^2 + (2 A / B^3) K~^-2.
    Returns (gcv dict, g_eta, g_W, g_v, g_sigma2)."""
    out, R, K, G = _gcv_weights(kind, X_tasks, y, eta, W, v, sigma2, alpha)

    def contract(dK):
        return float(np.sum(G * dK))

    g_eta, g_W, g_v, g_s2 = _param_contractions(kind, X_tasks, eta, W, R, K, contract, alpha, sigma2)
    return out, g_eta, g_W, g_v, g_s2


def nll_grad(kind, X_tasks, y, eta, W, v, sigma2, alpha=2):
    """Analytic gradient of L (Eq. 3.3) w.r.t. eta (d), W (T x s), v (T), sigma2, at the optimal tau.

    dL/dtheta = tr(K~^-1 dK~/dtheta) - a^T (dK~/dtheta) a, each dK~ written out densely:
      dK~/d eta_j   = R_{tt'} K(x_j, x'_j) prod_{l != j} (1 + eta_l K(x_l, x'_l))
      dK~/d W_{ts}  = (dR/dW_{ts})_{tt'} Q,   dR/dW_{ts} = e_t W_{:,s}^T + W_{:,s} e_t^T
      dK~/d v_t     = (e_t e_t^T)_{tt'} Q
      dK~/d sigma2  = I
    Returns (out_dict_of_nll, g_eta, g_W, g_v, g_sigma2) for L (the NLL gradient is half of it).
    """
    out = nll(kind, X_tasks, y, eta, W, v, sigma2, alpha)
    R = task_covariance(W, v)
    K = gram(kind, X_tasks, eta, R, sigma2, alpha)
    Kinv = np.linalg.inv(K)
    Kinv = 0.5 * (Kinv + Kinv.T)
    a = out["alpha"]

    def contract(dK):
        return float(np.sum(Kinv * dK) - a @ dK @ a)

    g_eta, g_W, g_v, g_s2 = _param_contractions(kind, X_tasks, eta, W, R, K, contract, alpha, sigma2)
    return out, g_eta, g_W, g_v, g_s2


def posterior(kind, X_tasks, y, eta, W, v, sigma2, Xq, task_q, alpha=2):
    """Posterior mean and variance of f(t, x) at fixed-point queries Xq (nq x d), Eq. 3.2.

    tau is the MLE optimal mean (Eq. 3.4), plugged in as the prior mean.
    """
    out = nll(kind, X_tasks, y, eta, W, v, sigma2, alpha)
    R = task_covariance(W, v)
    K = gram(kind, X_tasks, eta, R, sigma2, alpha)
    cf = sla.cho_factor(K, lower=True)
    T = len(X_tasks)
    nq = Xq.shape[0]
    kq = np.empty((nq, K.shape[0]))
    off = 0
    Qs = []
    for u in range(T):
        Qs.append(product_kernel(kind, Xq[:, None, :], X_tasks[u][None, :, :], eta, alpha=alpha))
    for i in range(nq):
        row = np.concatenate([R[task_q[i], u] * Qs[u][i] for u in range(T)])
        kq[i] = row
    mean = out["tau"][task_q] + kq @ out["alpha"]
    Kinv_kq = sla.cho_solve(cf, kq.T)
    prior = np.array([R[task_q[i], task_q[i]] * product_kernel(kind, Xq[i], Xq[i], eta, alpha=alpha)
                      for i in range(nq)])
    var = prior - np.einsum("ij,ji->i", kq, Kinv_kq)
    return mean, var, prior


def cubature(kind, X_tasks, y, eta, W, v, sigma2, gamma=1.0, alpha=2):
    """Multitask Bayesian cubature (Sec. 3.5, multitask cubature theorem) for the task integrals
    mu_t = int f(t, x) dx, with int Q(x, x') dx' = gamma: at tau = tau_MLE,
        mu_hat = tau + gamma R E K~^-1 (y - E^T tau),   Sigma = gamma R - gamma^2 R Pi R,
    Pi = E K~^-1 E^T, written out with dense solves.  Returns (mu_hat, Sigma, tau)."""
    out = nll(kind, X_tasks, y, eta, W, v, sigma2, alpha)
    R = task_covariance(W, v)
    n = [len(X) for X in X_tasks]
    E = summing_matrix(n)
    tau = out["tau"]
    mu = tau + gamma * R @ (E @ out["alpha"])
    Sigma = gamma * R - gamma ** 2 * R @ out["Pi"] @ R
    return mu, Sigma, tau


def dsi_weights_grad(kind, X_tasks, y, eta, W, v, sigma2, b, loss="mle"):
    """Gradient of L (Eq. 3.3, MLE or GCV form) with respect to the DSI mixture weights b of Eq. 2.6,
    K(x, x') = sum_a b_a K_a(x XOR x'), with the dense derivative written out:
      dK~/db_a = R_{tt'} sum_j eta_j K_a(x_j, x'_j) prod_{l != j} (1 + eta_l K(x_l, x'_l)).
    Returns (loss dict, g_b (4,)) for L (the NLL gradient is half of the MLE one)."""
    b = np.asarray(b, dtype=np.float64)
    R = task_covariance(W, v)
    if loss == "mle":
        out = nll(kind, X_tasks, y, eta, W, v, sigma2, b)
        K = gram(kind, X_tasks, eta, R, sigma2, b)
        Kinv = np.linalg.inv(K)
        Kinv = 0.5 * (Kinv + Kinv.T)
        a = out["alpha"]

        def contract(dK):
            return float(np.sum(Kinv * dK) - a @ dK @ a)
    elif loss == "gcv":
        out, R, K, G = _gcv_weights(kind, X_tasks, y, eta, W, v, sigma2, b)

        def contract(dK):
            return float(np.sum(G * dK))
    else:
        raise ValueError(loss)
    T = len(X_tasks)
    n = [len(X) for X in X_tasks]
    off = np.concatenate([[0], np.cumsum(n)])
    d = len(eta)
    g_b = np.zeros(4)
    for a_ in range(1, 5):
        dK = np.zeros_like(K)
        for t in range(T):
            for u in range(T):
                Xa, Xb = X_tasks[t][:, None, :], X_tasks[u][None, :, :]
                mix = [kernel_1d(kind, Xa[..., j], Xb[..., j], b) for j in range(d)]
                blk = np.zeros((n[t], n[u]))
                for j in range(d):
                    term = eta[j] * kernel_1d(kind, Xa[..., j], Xb[..., j], a_)
                    for l in range(d):
                        if l != j:
                            term = term * (1.0 + eta[l] * mix[l])
                    blk += term
                dK[off[t]:off[t + 1], off[u]:off[u + 1]] = R[t, u] * blk
        g_b[a_ - 1] = contract(dK)
    return out, g_b

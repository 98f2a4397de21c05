"""Pins for the cubature oracle: the closed forms against the definitions they come from,
mu_hat = int E[f(t, x) | y] dx and Sigma = int int Cov[f(t, x), f(u, x') | y] dx dx', both integrated
numerically over a fine independent point set; gamma = 1 for the product kernels; mu_hat = tau_MLE."""
import numpy as np
import pytest

from oracle import dense, design
from paper_2603_16014_gb300 import inputs


@pytest.mark.parametrize("kind,m", [("lattice", (5, 4)), ("dnet", (4, 4, 3))])
def test_cubature_matches_integrated_posterior(kind, m):
    p = inputs.make_problem(kind, 2, m, seed=31, eta=0.8, v=0.2, sigma2=1e-3)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    mu, Sigma, tau = dense.cubature(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    # at the MLE mean the correction term vanishes (E K~^-1 (y - E^T tau) = 0)
    assert np.allclose(mu, tau, rtol=1e-9, atol=1e-12)
    # numerical integration: a 2^12-point rank-1 lattice of the unit square (its own generator),
    # exact for the smooth periodic integrands up to ~1e-6 here
    M = 1 << 12
    g = np.array([1, 1487], dtype=np.uint64)
    i = np.arange(M, dtype=np.uint64)
    Xq = ((i[:, None] * g[None, :]) % M * (1 << 20)).astype(np.uint32)   # (i g mod M) / M in fixed point
    if kind == "dnet":
        Xq = Xq ^ np.uint32(0x9E3779B9)          # the DSI kernel is not periodic: shift the grid
    T = p.T
    for t in range(T):
        mean, var, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, np.full(M, t))
        assert mean.mean() == pytest.approx(mu[t], abs=2e-4 * (abs(mu[t]) + np.sqrt(Sigma[t, t]) + 1))
    # Sigma from the double integral of the posterior covariance over two independent random point
    # sets (a grid shared by x and x' would bias the digital-net kernel, whose argument x xor x'
    # falls back onto the grid)
    Mc = 1024
    rng = np.random.default_rng(5)
    A = rng.integers(0, 1 << 32, size=(Mc, 2), dtype=np.uint64).astype(np.uint32)
    B = rng.integers(0, 1 << 32, size=(Mc, 2), dtype=np.uint64).astype(np.uint32)
    R = dense.task_covariance(p.W, p.v)
    K = dense.gram(p.kind, X, p.eta, R, p.sigma2)
    Kinv = np.linalg.inv(K)
    Qab = design.product_kernel(p.kind, A[:, None, :], B[None, :, :], p.eta)

    def kx(P, t):
        return np.concatenate([R[t, u] * design.product_kernel(p.kind, P[:, None, :], X[u][None, :, :], p.eta)
                               for u in range(T)], axis=1)

    for t in range(T):
        for u in range(T):
            cov = R[t, u] * Qab - kx(A, t) @ Kinv @ kx(B, u).T
            assert cov.mean() == pytest.approx(Sigma[t, u], abs=1e-2 * np.sqrt(R[t, t] * R[u, u]))
    assert np.all(np.linalg.eigvalsh(Sigma) > -1e-12)


def test_product_kernels_integrate_to_one():
    # gamma = int Q(x, x') dx' = 1: each univariate kernel integrates to 0 over a full period
    for kind in ("lattice", "dnet"):
        M = 1 << 16
        x = (np.arange(M, dtype=np.uint64) * (1 << 16)).astype(np.uint32)
        k = design.kernel_1d(kind, x, np.zeros_like(x))
        assert abs(k.mean()) < 1e-4          # left-point rule on 2^16 points (the exact integral is 0)

"""Pins for the spectral oracle: the theorem's structure, Algorithm 1 and the per-class solvers
against the dense plain definition and against closed forms."""
import os

import numpy as np
import pytest

from oracle import dense, design, spectral
from paper_2603_16014_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sorted_setup(p):
    order = spectral.sorted_order(p.m)
    X = [design.design_points(p.kind, p.gen, p.shift[t], 1 << p.m[t]) for t in order]
    R = design.task_covariance(p.W, p.v)[np.ix_(order, order)]
    return order, X, R


def _vblock(kind, n):
    """Dense V = diag(V_{m_t}) built column by column from vmul (V e_k)."""
    N = sum(n)
    V = np.zeros((N, N), dtype=np.complex128)
    off = 0
    for nt in n:
        mt = nt.bit_length() - 1
        V[off:off + nt, off:off + nt] = spectral.vmul(kind, np.eye(nt, dtype=np.complex128), mt).T
        off += nt
    return V


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_transform_unitary_constant_row(kind):
    # Theorem "fast MTGP computations", item 1: V unitary with constant zeroth row and column
    for m in (0, 1, 3, 6):
        n = 1 << m
        V = spectral.vmul(kind, np.eye(n, dtype=np.complex128), m).T
        assert np.allclose(V.conj().T @ V, np.eye(n), atol=1e-13)
        assert np.allclose(V[:, 0], 1 / np.sqrt(n)) and np.allclose(V[0, :], 1 / np.sqrt(n))
        a = np.random.default_rng(m).standard_normal(n)
        assert np.allclose(spectral.vdag(kind, a, m), V.conj().T @ a, atol=1e-12)


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_theorem_block_structure_T3_example(kind):
    # the paper's worked example n = (8, 4, 2): V^dagger K~ V equals Lambda-tilde assembled from the
    # tall-case first-column transforms, with the golden sparsity pattern
    p = inputs.make_problem(kind, 2, (3, 2, 1), seed=4, eta=0.7, v=0.3, sigma2=1e-3)
    order, X, R = _sorted_setup(p)
    n = [len(x) for x in X]
    K = dense.gram(kind, X, p.eta, R, p.sigma2)
    V = _vblock(kind, n)
    Lam_true = V.conj().T @ K @ V
    lam = spectral.lambda_blocks(kind, X, p.eta, R, p.sigma2)
    Lam = spectral.lambda_dense(lam, n)
    assert np.allclose(Lam, Lam_true, atol=1e-12 * np.abs(Lam_true).max())
    pat = np.array([[int(c) for c in l.strip()] for l in open(os.path.join(GOLDEN, "lambda_pattern_T3_8_4_2.txt"))
                    if not l.startswith("#") and l.strip()])
    assert np.all(np.abs(Lam_true[pat == 0]) < 1e-12 * np.abs(Lam_true).max())
    # Hermitian (item 5)
    assert np.allclose(Lam_true, Lam_true.conj().T, atol=1e-12)


@pytest.mark.parametrize("kind,m", [("lattice", (4, 4)), ("dnet", (5, 3, 2)), ("lattice", (6, 3, 5, 2))])
def test_eigenvalues_equal_transform_spectrum(kind, m):
    # P1: eigenvalues of the dense Gram = eigenvalues of the assembled Lambda-tilde
    p = inputs.make_problem(kind, 3, m, seed=9, eta=0.5, v=0.2, sigma2=1e-4)
    order, X, R = _sorted_setup(p)
    n = [len(x) for x in X]
    K = dense.gram(kind, X, p.eta, R, p.sigma2)
    Lam = spectral.lambda_dense(spectral.lambda_blocks(kind, X, p.eta, R, p.sigma2), n)
    assert np.allclose(np.linalg.eigvalsh(K), np.linalg.eigvalsh(Lam), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("m", [4, 8, 10])
def test_lattice_1d_closed_form_spectrum(m):
    # P2: single task, d = 1, odd g: eigenvalues are n [f = 0] + n eta A(f), A the aliased
    # Fourier coefficients of the order-2 Bernoulli kernel (multiset over f)
    n = 1 << m
    eta = 0.7
    p = inputs.make_problem("lattice", 1, (m,), seed=m, eta=eta, W=np.zeros((1, 1)), v=1.0, sigma2=0.0)
    order, X, R = _sorted_setup(p)
    lam = spectral.lambda_blocks("lattice", X, p.eta, R, 0.0)[(0, 0)]
    f = np.arange(1, n)
    A = np.empty(n)
    A[0] = np.pi ** 4 / (45 * n ** 4)
    A[1:] = np.pi ** 4 * (1 + 2 * np.cos(np.pi * f / n) ** 2) / (3 * np.sin(np.pi * f / n) ** 4) / n ** 4
    ref = n * eta * A
    ref[0] += n
    assert np.max(np.abs(lam.imag)) < 1e-9 * n
    assert np.allclose(np.sort(lam.real), np.sort(ref), rtol=1e-8, atol=1e-11)


@pytest.mark.parametrize("kind,m", [("lattice", (3, 2, 1)), ("dnet", (5, 3, 2)), ("lattice", (4, 4, 2)),
                                    ("dnet", (6, 6, 6)), ("lattice", (2, 5, 3, 4))])
def test_algorithm1_inverse_and_logdet_vs_dense(kind, m):
    # P11: Algorithm 1's Lambda^-1 and log|Lambda| against dense inverse / slogdet
    p = inputs.make_problem(kind, 2, m, seed=13, eta=0.9, v=0.15, sigma2=1e-3)
    order, X, R = _sorted_setup(p)
    n = [len(x) for x in X]
    lam = spectral.lambda_blocks(kind, X, p.eta, R, p.sigma2)
    Lam = spectral.lambda_dense(lam, n)
    A, rho = spectral.algorithm1(lam, n)
    sgn, ld = np.linalg.slogdet(Lam)
    assert abs(rho - ld) < 1e-10 * max(1, abs(ld))
    # assemble A densely
    nT = n[-1]
    offs = np.concatenate([[0], np.cumsum(n)])
    rows = spectral.block_rows(n)
    Ad = np.zeros_like(Lam)
    for a, (t, j) in enumerate(rows):
        for b, (u, k) in enumerate(rows):
            for r in range(nT):
                Ad[offs[t] + j * nT + r, offs[u] + k * nT + r] = A[a, b, r]
    Linv = np.linalg.inv(Lam)
    assert np.allclose(Ad, Linv, atol=1e-10 * np.abs(Linv).max())


@pytest.mark.parametrize("kind,m", [("lattice", (5, 5)), ("dnet", (5, 3, 2)), ("lattice", (4, 6, 3)),
                                    ("dnet", (4, 4, 4, 4)), ("lattice", (1, 0)), ("dnet", (0, 0, 0))])
def test_fast_nll_matches_dense(kind, m):
    # P5: every spectral route equals the dense Cholesky NLL and the dense optimal means
    p = inputs.make_problem(kind, 3, m, seed=17, eta=0.6, v=0.1, sigma2=1e-4, s=2)
    X = dense.all_points(kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref = dense.nll(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    args = (kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    a1 = spectral.nll_algorithm1(*args)
    bc = spectral.nll_by_class(*args)
    for out in (a1, bc):
        assert abs(out["L"] - ref["L"]) < 1e-9 * max(1, abs(ref["L"]))
        assert np.allclose(out["tau"], ref["tau"], atol=1e-9 * (1 + np.abs(ref["tau"]).max()))
    if len(set(m)) == 1:
        eq = spectral.nll_equal(*args)
        assert abs(eq["L"] - ref["L"]) < 1e-9 * max(1, abs(ref["L"]))
        # equal sizes: optimal means are the per-task sample means (theorem item 4 with Pi = n Lambda(0)^-1)
        n = 1 << m[0]
        assert np.allclose(eq["tau"], y.reshape(len(m), n).mean(axis=1), atol=1e-12)


def test_pi_formula_matches_dense():
    # P7: Pi_{tt'} = sqrt(n_t n_t') (Lambda^-1)_{N_{t-1}, N_{t'-1}} equals E K~^-1 E^T
    p = inputs.make_problem("dnet", 2, (5, 3, 4), seed=23, eta=0.6, v=0.1, sigma2=1e-3)
    order, X, R = _sorted_setup(p)
    n = [len(x) for x in X]
    K = dense.gram("dnet", X, p.eta, R, p.sigma2)
    E = dense.summing_matrix(n)
    Pi_dense = E @ np.linalg.solve(K, E.T)
    lam = spectral.lambda_blocks("dnet", X, p.eta, R, p.sigma2)
    A, _ = spectral.algorithm1(lam, n)
    rows = spectral.block_rows(n)
    first = [rows.index((t, 0)) for t in range(len(n))]
    Pi = np.array([[np.sqrt(n[t] * n[u]) * A[first[t], first[u], 0] for u in range(3)] for t in range(3)])
    assert np.allclose(Pi, Pi_dense, rtol=1e-10)


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_spectrum_nonnegative(kind):
    # PSD product kernels: every first-column transform of a diagonal block is >= 0 (up to roundoff)
    p = inputs.make_problem(kind, 4, (10,), seed=3, eta=1.5, v=1.0, W=np.zeros((1, 1)), sigma2=0.0)
    order, X, R = _sorted_setup(p)
    lam = spectral.lambda_blocks(kind, X, p.eta, R, 0.0)[(0, 0)]
    assert np.min(lam.real) > -1e-10 * np.max(lam.real)


@pytest.mark.parametrize("kind,m", [("lattice", (5, 4)), ("dnet", (4, 4, 3))])
def test_posterior_by_class_matches_dense(kind, m):
    p = inputs.make_problem(kind, 2, m, seed=29, eta=0.6, v=0.1, sigma2=1e-4)
    X = dense.all_points(kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    Xq, _, tq = inputs.query_points(6, 2, seed=4, tasks=len(m))
    mean_d, var_d, _ = dense.posterior(kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    mean_s, var_s = spectral.posterior_by_class(kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    assert np.allclose(mean_s, mean_d, atol=1e-9)
    assert np.allclose(var_s, var_d, atol=1e-9)


@pytest.mark.parametrize("kind,m,d", [("lattice", (5, 5), 2), ("dnet", (4, 4, 4), 3), ("dnet", (6,), 2),
                                      ("lattice", (3, 3, 3, 3), 1)])
def test_equal_spectral_gradient_matches_dense(kind, m, d):
    p = inputs.make_problem(kind, d, m, seed=31, eta=0.7, v=0.2, sigma2=1e-3, s=min(2, len(m)))
    X = dense.all_points(kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref = dense.nll_grad(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    got = spectral.nll_grad_equal(kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    assert abs(got[0]["L"] - ref[0]["L"]) < 1e-9 * abs(ref[0]["L"])
    for a, b in zip(got[1:], ref[1:]):
        assert np.allclose(a, b, rtol=1e-8, atol=1e-8 * (1 + np.abs(np.asarray(ref[1])).max()))


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_posterior_mean_equal_matches_dense(kind):
    p = inputs.make_problem(kind, 2, (5, 5, 5), seed=17, eta=0.6, v=0.1, sigma2=1e-4)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    Xq, xq, tq = inputs.query_points(9, 2, seed=3, tasks=3)
    mean_ref, _, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    mean = spectral.posterior_mean_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    assert np.allclose(mean, mean_ref, rtol=0, atol=1e-9 * prior.max())
    _, var_ref, _ = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    var = spectral.posterior_var_equal(p.kind, p.gen, p.shift, p.m, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    assert np.allclose(var, var_ref, rtol=0, atol=1e-9 * prior.max())

"""Pins for the dense (plain-definition) oracle: exact determinants, closed forms, identities, FD."""
import numpy as np
import pytest

from oracle import dense, design, exact, spectral
from paper_2603_16014_gb300 import inputs


def _setup(problem):
    X = dense.all_points(problem.kind, problem.gen, problem.shift, problem.m)
    y = inputs.synth_y(problem, X)
    return X, y


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_logdet_matches_exact_bareiss(kind):
    # N <= 64: dense Cholesky log-det vs the exact rational determinant of the same float matrix
    p = inputs.make_problem(kind, 2, (5, 4), seed=11, eta=0.8, v=0.2, sigma2=1e-3)
    X, y = _setup(p)
    R = design.task_covariance(p.W, p.v)
    K = dense.gram(kind, X, p.eta, R, p.sigma2)
    out = dense.nll(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    assert K.shape[0] == 48
    assert abs(out["logdet"] - exact.exact_logdet(K)) < 1e-10 * max(1.0, abs(out["logdet"]))


def test_exact_det_small_integer_matrix():
    A = np.array([[2.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 4.0]])
    D, E = exact.exact_det_scaled(A)
    assert D == 18 and E == 0
    B = np.array([[0.5, 0.25], [0.25, 0.5]])
    D, E = exact.exact_det_scaled(B)
    assert D / 2 ** (2 * E) == 0.1875


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_single_task_mean_is_sample_mean(kind):
    # Theorem "fast GP computations", item 4: tau_MLE = sample mean under the SI-LAT / DSI-DSEQ pairing.
    # (Fails for an unstructured design or a kernel that is not (digitally) shift invariant.)
    p = inputs.make_problem(kind, 3, (7,), seed=5, eta=0.9, v=0.3, sigma2=1e-4)
    X, y = _setup(p)
    out = dense.nll(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    assert abs(out["tau"][0] - y.mean()) < 1e-10 * (1 + abs(y.mean()))


def test_single_task_mean_not_sample_mean_for_random_design():
    # control: with i.i.d. points the identity above does not hold
    p = inputs.make_problem("lattice", 3, (6,), seed=5, eta=0.9, v=0.3, sigma2=1e-4)
    rng = np.random.default_rng(0)
    X = [rng.integers(0, 1 << 32, size=(64, 3), dtype=np.uint64).astype(np.uint32)]
    y = inputs.synth_y(p, X)
    out = dense.nll("lattice", X, y, p.eta, p.W, p.v, p.sigma2)
    assert abs(out["tau"][0] - y.mean()) > 1e-6


@pytest.mark.parametrize("kind,m", [("lattice", (5, 5)), ("dnet", (5, 4, 3)), ("lattice", (4, 5, 3))])
def test_gradient_matches_central_differences(kind, m):
    p = inputs.make_problem(kind, 3, m, seed=21, eta=0.7, v=0.2, sigma2=1e-3, s=2)
    X, y = _setup(p)
    out, g_eta, g_W, g_v, g_s2 = dense.nll_grad(kind, X, y, p.eta, p.W, p.v, p.sigma2)

    def L(eta, W, v, s2):
        return dense.nll(kind, X, y, eta, W, v, s2)["L"]

    h = 1e-6
    for j in range(p.d):
        e = np.zeros(p.d)
        e[j] = h
        fd = (L(p.eta + e, p.W, p.v, p.sigma2) - L(p.eta - e, p.W, p.v, p.sigma2)) / (2 * h)
        assert abs(fd - g_eta[j]) < 1e-5 * (1 + abs(g_eta[j]))
    for t in range(p.T):
        for k in range(p.W.shape[1]):
            E = np.zeros_like(p.W)
            E[t, k] = h
            fd = (L(p.eta, p.W + E, p.v, p.sigma2) - L(p.eta, p.W - E, p.v, p.sigma2)) / (2 * h)
            assert abs(fd - g_W[t, k]) < 1e-5 * (1 + abs(g_W[t, k]))
        e = np.zeros(p.T)
        e[t] = h
        fd = (L(p.eta, p.W, p.v + e, p.sigma2) - L(p.eta, p.W, p.v - e, p.sigma2)) / (2 * h)
        assert abs(fd - g_v[t]) < 1e-5 * (1 + abs(g_v[t]))
    hs = 1e-3 * p.sigma2
    fd = (L(p.eta, p.W, p.v, p.sigma2 + hs) - L(p.eta, p.W, p.v, p.sigma2 - hs)) / (2 * hs)
    assert abs(fd - g_s2) < 1e-5 * (1 + abs(g_s2))


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_mean_estimate_zero_residual_sum(kind):
    # Eq. 3.4 at the MLE: E K~^-1 (y - E^T tau) = 0 (multitask cubature theorem, last statement)
    p = inputs.make_problem(kind, 2, (5, 4, 4), seed=2, eta=0.6, v=0.1, sigma2=1e-4)
    X, y = _setup(p)
    out = dense.nll(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    n = [len(x) for x in X]
    E = dense.summing_matrix(n)
    assert np.max(np.abs(E @ out["alpha"])) < 1e-7 * np.max(np.abs(out["alpha"])) * max(n)


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_posterior_identities_at_design_points(kind):
    # at a design point x_ti:  mean = y_ti - sigma2 a_ti,  var = sigma2 - sigma2^2 (K~^-1)_{ii}
    p = inputs.make_problem(kind, 2, (5, 4), seed=8, eta=0.6, v=0.1, sigma2=1e-2)
    X, y = _setup(p)
    n = [len(x) for x in X]
    Xq = np.concatenate(X)
    tq = np.concatenate([np.full(n[t], t) for t in range(len(n))])
    mean, var, _ = dense.posterior(kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    out = dense.nll(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    R = design.task_covariance(p.W, p.v)
    Kinv = np.linalg.inv(dense.gram(kind, X, p.eta, R, p.sigma2))
    assert np.allclose(mean, y - p.sigma2 * out["alpha"], atol=1e-9)
    assert np.allclose(var, p.sigma2 - p.sigma2 ** 2 * np.diag(Kinv), atol=1e-9)
    # away from the design the variance lies in [0, prior]
    Xr, _, tr = inputs.query_points(20, 2, seed=3, tasks=2)
    _, v2, prior = dense.posterior(kind, X, y, p.eta, p.W, p.v, p.sigma2, Xr, tr)
    assert np.all(v2 >= -1e-12) and np.all(v2 <= prior + 1e-12)


@pytest.mark.parametrize("alpha", [1, 3, 4])
def test_gradient_other_si_smoothness_matches_central_differences(alpha):
    p = inputs.make_problem("lattice", 2, (4, 3), seed=22, eta=0.7, v=0.2, sigma2=1e-3, s=2)
    X, y = _setup(p)
    out, g_eta, g_W, g_v, g_s2 = dense.nll_grad("lattice", X, y, p.eta, p.W, p.v, p.sigma2, alpha)

    def L(eta, W, v, s2):
        return dense.nll("lattice", X, y, eta, W, v, s2, alpha)["L"]

    h = 1e-6
    for j in range(p.d):
        e = np.zeros(p.d)
        e[j] = h
        fd = (L(p.eta + e, p.W, p.v, p.sigma2) - L(p.eta - e, p.W, p.v, p.sigma2)) / (2 * h)
        assert abs(fd - g_eta[j]) < 1e-5 * (1 + abs(g_eta[j]))
    E = np.zeros_like(p.W)
    E[1, 0] = h
    fd = (L(p.eta, p.W + E, p.v, p.sigma2) - L(p.eta, p.W - E, p.v, p.sigma2)) / (2 * h)
    assert abs(fd - g_W[1, 0]) < 1e-5 * (1 + abs(g_W[1, 0]))
    # the smoothness changes the kernel: alpha = 2 gives a different loss
    assert abs(out["L"] - dense.nll("lattice", X, y, p.eta, p.W, p.v, p.sigma2)["L"]) > 1e-6


def test_per_task_noise_reduces_to_scalar_and_matches_differences():
    p = inputs.make_problem("dnet", 2, (4, 3, 3), seed=23, eta=0.7, v=0.2, sigma2=1e-3, s=2)
    X, y = _setup(p)
    xi = np.full(p.T, p.sigma2)
    a = dense.nll_grad("dnet", X, y, p.eta, p.W, p.v, p.sigma2)
    b = dense.nll_grad("dnet", X, y, p.eta, p.W, p.v, xi)
    assert b[0]["L"] == pytest.approx(a[0]["L"], rel=1e-13)
    assert np.sum(b[4]) == pytest.approx(a[4], rel=1e-11)          # per-task traces add up
    xi = np.array([1e-3, 3e-3, 5e-4])
    out, ge, gW, gv, gs = dense.nll_grad("dnet", X, y, p.eta, p.W, p.v, xi)
    for t in range(p.T):
        h = 1e-4 * xi[t]
        e = np.zeros(p.T)
        e[t] = h
        fd = (dense.nll("dnet", X, y, p.eta, p.W, p.v, xi + e)["L"] - dense.nll("dnet", X, y, p.eta, p.W, p.v, xi - e)["L"]) / (2 * h)
        assert fd == pytest.approx(gs[t], rel=1e-5)
    g = dense.gcv_grad("dnet", X, y, p.eta, p.W, p.v, xi)
    h = 1e-4 * xi[1]
    e = np.array([0.0, h, 0.0])
    fd = (dense.gcv("dnet", X, y, p.eta, p.W, p.v, xi + e)["L"] - dense.gcv("dnet", X, y, p.eta, p.W, p.v, xi - e)["L"]) / (2 * h)
    assert fd == pytest.approx(g[4][1], rel=1e-5)

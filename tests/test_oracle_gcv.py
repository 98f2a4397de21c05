"""Pins for the GCV oracle (Eq. 3.3 second form, Eq. 3.4 second form): scale invariance, the
closed form when K~ = sigma2 I, stationarity of the numerator at tau_GCV, sample means for equal
sizes, and the spectral routes against the dense definition."""
import numpy as np
import pytest

from oracle import dense, spectral
from paper_2603_16014_gb300 import inputs


def _setup(kind, d, m, seed):
    p = inputs.make_problem(kind, d, m, seed=seed, eta=0.7, v=0.2, sigma2=1e-3)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    return p, X, inputs.synth_y(p, X)


def test_gcv_scale_invariance_and_sigma_only_closed_form():
    p, X, y = _setup("lattice", 2, (5, 4), 1)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    c = 7.3
    g2 = dense.gcv(p.kind, X, y, p.eta, p.W * np.sqrt(c), p.v * c, p.sigma2 * c)
    assert g2["L"] == pytest.approx(g["L"], rel=1e-11)
    # R = 0: K~ = sigma2 I, tau = task sample means, L = sum (y - ybar_t)^2 / N^2
    z = dense.gcv(p.kind, X, y, p.eta, np.zeros_like(p.W), np.zeros(p.T), 0.5)
    offs = np.concatenate([[0], np.cumsum(p.n)])
    means = [y[offs[t]:offs[t + 1]].mean() for t in range(p.T)]
    ss = sum(((y[offs[t]:offs[t + 1]] - means[t]) ** 2).sum() for t in range(p.T))
    assert np.allclose(z["tau"], means, rtol=1e-12)
    assert z["L"] == pytest.approx(ss / p.N ** 2, rel=1e-12)


def test_gcv_mean_minimises_numerator():
    p, X, y = _setup("dnet", 2, (5, 3, 3), 2)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    R = dense.task_covariance(p.W, p.v)
    K = dense.gram(p.kind, X, p.eta, R, p.sigma2)
    Ki = np.linalg.inv(K)
    E = dense.summing_matrix(p.n)

    def num(tau):
        r = y - E.T @ tau
        return r @ Ki @ Ki @ r

    h = 1e-4
    for t in range(p.T):
        e = np.zeros(p.T)
        e[t] = h
        assert abs(num(g["tau"] + e) - num(g["tau"] - e)) <= 1e-6 * num(g["tau"])
        assert num(g["tau"] + e) > num(g["tau"])


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_gcv_equal_sizes_sample_means_and_spectral(kind):
    p, X, y = _setup(kind, 3, (5, 5, 5), 3)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    means = y.reshape(p.T, -1).mean(axis=1)
    assert np.allclose(g["tau"], means, rtol=1e-9, atol=1e-12)
    s = spectral.gcv_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    for k in ("L", "num", "trace"):
        assert s[k] == pytest.approx(g[k], rel=1e-9), k
    c = spectral.gcv_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    assert c["L"] == pytest.approx(g["L"], rel=1e-9)


@pytest.mark.parametrize("kind,m", [("lattice", (6, 4, 2)), ("dnet", (5, 5, 3)), ("lattice", (3, 5, 4))])
def test_gcv_unequal_sizes_by_class(kind, m):
    p, X, y = _setup(kind, 2, m, 4)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    c = spectral.gcv_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    for k in ("L", "num", "trace"):
        assert c[k] == pytest.approx(g[k], rel=1e-9), k
    assert np.allclose(c["tau"], g["tau"], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("kind,m", [("lattice", (4, 4)), ("dnet", (4, 3, 3))])
def test_gcv_gradient_matches_central_differences(kind, m):
    p, X, y = _setup(kind, 2, m, 5)
    out, ge, gW, gv, gs = dense.gcv_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)

    def L(eta, W, v, s2):
        return dense.gcv(p.kind, X, y, eta, W, v, s2)["L"]

    h = 1e-4          # relative step: truncation ~1e-8, roundoff eps L / (h theta) well below 1e-5
    for j in range(p.d):
        e = np.zeros(p.d)
        e[j] = h * p.eta[j]
        fd = (L(p.eta + e, p.W, p.v, p.sigma2) - L(p.eta - e, p.W, p.v, p.sigma2)) / (2 * e[j])
        assert fd == pytest.approx(ge[j], rel=1e-5, abs=1e-9 * out["L"])
    for (t, k) in [(0, 0), (p.T - 1, 1)]:
        E = np.zeros_like(p.W)
        E[t, k] = h
        fd = (L(p.eta, p.W + E, p.v, p.sigma2) - L(p.eta, p.W - E, p.v, p.sigma2)) / (2 * h)
        assert fd == pytest.approx(gW[t, k], rel=1e-5, abs=1e-9 * out["L"])
    for t in range(p.T):
        e = np.zeros(p.T)
        e[t] = h * p.v[t]
        fd = (L(p.eta, p.W, p.v + e, p.sigma2) - L(p.eta, p.W, p.v - e, p.sigma2)) / (2 * e[t])
        assert fd == pytest.approx(gv[t], rel=1e-5, abs=1e-9 * out["L"])
    hs = h * p.sigma2
    fd = (L(p.eta, p.W, p.v, p.sigma2 + hs) - L(p.eta, p.W, p.v, p.sigma2 - hs)) / (2 * hs)
    assert fd == pytest.approx(gs, rel=1e-5, abs=1e-9 * out["L"])


@pytest.mark.parametrize("kind,m", [("lattice", (5, 3, 2)), ("dnet", (4, 4, 2)), ("lattice", (3, 5))])
@pytest.mark.parametrize("loss", ["mle", "gcv"])
def test_per_class_gradient_matches_dense(kind, m, loss):
    # the residue-class gradient (any sizes) against the dense analytic gradient, itself pinned by
    # central differences: same loss, same gradient for eta, W, v, sigma2
    p = inputs.make_problem(kind, 2, m, seed=91, eta=0.6, v=0.2, sigma2=1e-3, s=2)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    L, ge, gW, gv, gs = spectral.grad_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, loss)
    f = dense.nll_grad if loss == "mle" else dense.gcv_grad
    out, re, rW, rv, rs = f(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    assert L == pytest.approx(out["L"], rel=1e-11)
    got = np.concatenate([ge, gW.ravel(), gv, [gs]])
    exp = np.concatenate([re, rW.ravel(), rv, [rs]])
    assert np.abs(got - exp).max() <= 1e-9 * np.abs(exp).max()

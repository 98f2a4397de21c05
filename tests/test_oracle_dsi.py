"""Pins for the adaptive-smoothness DSI kernel of Eq. 2.6 (orders 1-4 and the mixture weights b).

The closed forms are checked against their Walsh series, written independently of them: with
k = 2^{a_1 - 1} + 2^{a_2 - 1} + ... (a_1 > a_2 > ...) and mu_alpha(k) = a_1 + ... + a_min(v, alpha),
  K_alpha(x) = sum_{k >= 1} r_alpha(k) wal_k(x),  r_alpha(k) = 2^{-mu_alpha(k)} (alpha = 2, 3, 4),
  K_1(x)     = sum_{k >= 1} 4^{-a_1(k)} / 3 wal_k(x)  (the order-one Walsh kernel).
The series has no constant term (mean zero) and non-negative coefficients (positive semi-definite);
a wrong constant, sign or digit index in any closed form breaks the agreement.  The mixture gradient
is pinned by central differences of the dense loss.
"""
import numpy as np
import pytest

from oracle import dense, design
from paper_2603_16014_gb300 import inputs


def walsh_series(X, alpha, P=64):
    """sum_k r_alpha(k) wal_k(x) for x = X / 2^32, by a recursion over the digit positions p = P..1:
    state j = how many of k's alpha leading bits were placed; once all are placed the remaining
    lower bits are free (their sum over both values gives 1 + (-1)^{x_p})."""
    X = np.asarray(X, dtype=np.uint64)
    f = np.zeros((alpha + 1, X.size))
    f[0] = 1.0
    for p in range(P, 0, -1):
        if p <= 32:
            xp = ((X >> np.uint64(32 - p)) & np.uint64(1)).astype(np.float64)
        else:
            xp = np.zeros(X.size)
        s = 1.0 - 2.0 * xp
        w = 2.0 ** -p if alpha >= 2 else 4.0 ** -p / 3.0
        g = f.copy()
        for j in range(1, alpha):
            g[j] = f[j] + f[j - 1] * w * s
        g[alpha] = f[alpha] * (1.0 + s) + f[alpha - 1] * w * s
        f = g
    return f[1:].sum(axis=0)


def _words():
    rng = np.random.default_rng(5)
    edge = [0, 1, 2, 3, 7, 1 << 16, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, 3 << 30, (1 << 32) - 1]
    return np.concatenate([np.array(edge, dtype=np.uint64),
                           rng.integers(0, 1 << 32, size=400, dtype=np.uint64),
                           rng.integers(0, 1 << 12, size=100, dtype=np.uint64)])


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_closed_form_equals_walsh_series(alpha):
    X = _words()
    got = design.dsi_kernel_1d(X, alpha)
    ref = walsh_series(X, alpha)
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("alpha", [1, 2, 3, 4])
def test_kernel_at_zero_is_coefficient_sum(alpha):
    # K_alpha(0) = sum_k r_alpha(k); for alpha = 1 this is sum_a 2^{a-1} 4^{-a} / 3 = 1/6, for alpha = 2
    # 3/2; alpha = 3 and 4 follow from the constant terms of Eq. 2.6 (-1 + 43/18 and -1 + 701/294).
    expect = {1: 1.0 / 6.0, 2: 1.5, 3: 25.0 / 18.0, 4: 407.0 / 294.0}[alpha]
    assert design.dsi_kernel_1d(np.array([0], dtype=np.uint64), alpha)[0] == pytest.approx(expect, rel=1e-15)
    assert walsh_series(np.array([0], dtype=np.uint64), alpha)[0] == pytest.approx(expect, rel=1e-14)


def test_walsh_gram_spectrum_nonnegative_for_mixture():
    # positive weights of positive semi-definite DSI kernels: the Walsh spectrum of the first column
    # of the Gram matrix on the dyadic grid is non-negative (Sec. 2.2, DSI-DSEQ pairing)
    m = 8
    X = (np.arange(1 << m, dtype=np.uint64) << np.uint64(32 - m))
    b = np.array([0.3, 1.0, 0.5, 0.2])
    col = design.kernel_1d("dnet", X, np.zeros_like(X), b)
    H = np.array([[1.0]])
    for _ in range(m):
        H = np.block([[H, H], [H, -H]])
    # natural-order Walsh: wal_k(i / 2^m) with the digit order reversed between k and i
    rev = np.array([int(format(i, f"0{m}b")[::-1], 2) for i in range(1 << m)])
    lam = H[rev] @ col          # aliased sums of the non-negative Walsh coefficients
    assert lam.min() > 0.0


def test_mixture_is_the_weighted_sum_and_order_two_is_the_default():
    X = _words()
    b = np.array([0.3, 1.0, 0.5, 0.2])
    mix = design.kernel_1d("dnet", X, np.zeros_like(X), b)
    ref = sum(b[a - 1] * walsh_series(X, a) for a in range(1, 5))
    assert np.max(np.abs(mix - ref)) < 1e-13
    p = inputs.make_problem("dnet", 2, (3, 3), seed=31, eta=0.6, v=0.2, sigma2=1e-3)
    Xt = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, Xt)
    a = dense.nll("dnet", Xt, y, p.eta, p.W, p.v, p.sigma2)["L"]
    e2 = dense.nll("dnet", Xt, y, p.eta, p.W, p.v, p.sigma2, np.array([0.0, 1.0, 0.0, 0.0]))["L"]
    assert e2 == pytest.approx(a, rel=1e-14)


@pytest.mark.parametrize("loss", ["mle", "gcv"])
def test_mixture_weight_gradient_matches_central_differences(loss):
    p = inputs.make_problem("dnet", 2, (4, 3), seed=32, eta=0.6, v=0.2, sigma2=1e-3, s=2)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    b = np.array([0.3, 1.0, 0.5, 0.2])
    out, g_b = dense.dsi_weights_grad("dnet", X, y, p.eta, p.W, p.v, p.sigma2, b, loss)
    f = dense.nll if loss == "mle" else dense.gcv

    def L(bb):
        return f("dnet", X, y, p.eta, p.W, p.v, p.sigma2, bb)["L"]

    assert out["L"] == pytest.approx(L(b), rel=1e-13)
    for a in range(4):
        h = 1e-5
        e = np.zeros(4)
        e[a] = h
        fd = (L(b + e) - L(b - e)) / (2 * h)
        assert abs(fd - g_b[a]) < 1e-5 * (1 + abs(g_b[a]))
    # the eta gradient with a mixture kernel (dense dK/deta_j with the mixed univariate kernel)
    grad = dense.nll_grad if loss == "mle" else dense.gcv_grad
    _, g_eta, g_W, _, _ = grad("dnet", X, y, p.eta, p.W, p.v, p.sigma2, b)
    for j in range(p.d):
        h = 1e-6
        e = np.zeros(p.d)
        e[j] = h
        fd = (f("dnet", X, y, p.eta + e, p.W, p.v, p.sigma2, b)["L"]
              - f("dnet", X, y, p.eta - e, p.W, p.v, p.sigma2, b)["L"]) / (2 * h)
        assert abs(fd - g_eta[j]) < 1e-5 * (1 + abs(g_eta[j]))
    # homogeneity: scaling b by c and eta by 1/c leaves K unchanged, so b.g_b = eta.g_eta
    assert float(b @ g_b) == pytest.approx(float(p.eta @ g_eta), rel=1e-9, abs=1e-9)


def test_spectral_mixture_gradient_matches_dense():
    from oracle import spectral
    p = inputs.make_problem("dnet", 3, (5, 5, 5), seed=33, eta=0.6, v=0.2, sigma2=1e-3, s=2)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    b = np.array([0.3, 1.0, 0.5, 0.2])
    out, ge, gW, gv, gs, gb = spectral.nll_grad_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, b)
    ref, re, rW, rv, rs = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, b)
    _, rb = dense.dsi_weights_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, b)
    assert out["L"] == pytest.approx(ref["L"], rel=1e-11)
    got = np.concatenate([ge, gW.ravel(), gv, [gs], gb])
    exp = np.concatenate([re, rW.ravel(), rv, [rs], rb])
    assert np.allclose(got, exp, rtol=1e-8, atol=1e-9 * np.abs(exp).max())


def test_dsi_order2_is_exact_dyadic():
    """Eq. 2.6, order 2: with x = X / 2^32 and beta = -floor(log2 x), 2^33 K_2(x) = 2^33 (-1 - beta x +
    5/2 (1 - 2^-beta)) = 3 2^32 - 2 beta X - 5 2^(32 - beta), an integer below 2^34 (3 2^32 at X = 0); the
    oracle's floating-point evaluation agrees with it to FP64 rounding at every tested word (this exact form
    is what lets the kernels evaluate K_2 without rounding)."""
    import numpy as np
    from oracle import design
    rng = np.random.default_rng(9)
    X = np.concatenate([[0, 1, 2, 3, (1 << 31) - 1, 1 << 31, (1 << 32) - 1],
                        [1 << k for k in range(32)],
                        rng.integers(0, 1 << 32, size=5000, dtype=np.uint64),
                        rng.integers(0, 1 << 32, size=5000, dtype=np.uint64) >> rng.integers(0, 32, size=5000).astype(np.uint64)])
    X = X.astype(np.uint64)
    k = design.dsi_kernel_1d(X, alpha=2)
    for x, kv in zip(X.tolist(), k.tolist()):
        if x == 0:
            exact = 3 << 32
        else:
            b = 33 - int(x).bit_length()
            exact = (3 << 32) - 2 * b * int(x) - 5 * (1 << (32 - b))
        assert abs(exact) < 1 << 34
        assert abs(kv * 2.0 ** 33 - exact) <= 4.0 * 2.0 ** 33 * 2.0 ** -52, (x, kv, exact)

"""The adaptive-smoothness DSI kernel (Eq. 2.6: orders 1-4, mixture weights b) on the GPU against the
dense and spectral oracles: MLE loss and gradient including dL/db, single orders through
mtgp_set_smoothness, posterior, GCV and its gradient, cubature; equal and nested sizes, FP64 and
FP32 transforms, and the full-size digital-net shape."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense, spectral  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

B = np.array([0.3, 1.0, 0.5, 0.2])
TOL = {"fp64": (1e-8, 1e-6), "fp32": (1e-5, 1e-3)}   # (relative NLL, normwise gradient)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _setup(m, seed, precision="fp64", d=2):
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("dnet", d, m, seed=seed, eta=0.6, v=0.2, sigma2=1e-4, recipe="walshcos32",
                            mmax=max(max(m), 8))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    model = MTGP.from_problem(p, precision)
    model.set_y(torch.from_numpy(y))
    return p, X, y, model


def _grad_vec(ge, gW, gv, gs, gb=None):
    parts = [np.asarray(ge).ravel(), np.asarray(gW).ravel(), np.asarray(gv).ravel(), np.atleast_1d(gs)]
    if gb is not None:
        parts.append(np.asarray(gb).ravel())
    return np.concatenate(parts)


@pytest.mark.parametrize("m,precision", [((5, 5, 5), "fp64"), ((6, 4, 3), "fp64"), ((5, 3, 3, 2), "fp64"),
                                         ((6, 6), "fp32"), ((6, 5, 3), "fp32")])
def test_mixture_nll_grad(m, precision):
    p, X, y, model = _setup(m, 71, precision)
    model.set_dsi_weights(B)
    ref, ge, gW, gv, gs = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, B)
    _, gb = dense.dsi_weights_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, B)
    out, tau, e_, W_, v_, s_ = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    g_b = model.dsi_weights_grad()
    model.sync()
    tn, tg = TOL[precision]
    assert abs(out[0].item() - ref["nll"]) <= tn * abs(ref["nll"])
    assert np.allclose(tau.cpu().numpy(), ref["tau"], rtol=0, atol=tn * (1 + np.abs(ref["tau"]).max()))
    gref = 0.5 * _grad_vec(ge, gW, gv, gs, gb)
    got = _grad_vec(e_.cpu(), W_.cpu(), v_.cpu(), s_.cpu(), g_b.cpu())
    assert np.abs(got - gref).max() <= tg * (1 + np.abs(gref).max()), (got, gref)
    model.close()


@pytest.mark.parametrize("alpha", [1, 3, 4])
@pytest.mark.parametrize("m", [(6, 6, 6), (6, 4, 3)])
def test_single_order_through_set_smoothness(alpha, m):
    p, X, y, model = _setup(m, 72)
    model.set_smoothness(alpha)
    ref, ge, gW, gv, gs = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, alpha)
    out, _, e_, W_, v_, s_ = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"])
    gref = 0.5 * _grad_vec(ge, gW, gv, gs)
    got = _grad_vec(e_.cpu(), W_.cpu(), v_.cpu(), s_.cpu())
    assert np.abs(got - gref).max() <= 1e-6 * (1 + np.abs(gref).max())
    # back to the order-2 default (fused kernels for equal sizes)
    model.set_smoothness(2)
    ref2 = dense.nll(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    out2, _ = model.nll(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out2[0].item() - ref2["nll"]) <= 1e-8 * abs(ref2["nll"])
    assert abs(ref2["nll"] - ref["nll"]) > 1e-6 * abs(ref["nll"])        # the order matters
    model.close()


@pytest.mark.parametrize("m", [(5, 5, 5), (6, 4, 3)])
def test_mixture_posterior_gcv_cubature(m):
    p, X, y, model = _setup(m, 73)
    model.set_dsi_weights(B)
    equal = len(set(m)) == 1
    Xq, xq, tq = inputs.query_points(7, 2, seed=4, tasks=len(m))
    mean_ref, var_ref, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq, B)
    mean, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq),
                                variance=True)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, B)
    gout, _ = model.gcv(p.eta, p.W, p.v, p.sigma2)
    mu_ref, S_ref, _ = dense.cubature(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, alpha=B)
    mu, S = model.cubature(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=1e-8 * prior.max())
    assert abs(gout[0].item() - g["L"]) <= 1e-8 * abs(g["L"])
    R = dense.task_covariance(p.W, p.v)
    assert np.allclose(mu.cpu().numpy(), mu_ref, rtol=0, atol=1e-8 * (np.abs(mu_ref).max() + 1))
    assert np.allclose(S.cpu().numpy(), S_ref, rtol=0, atol=1e-8 * np.abs(R).max())
    assert np.allclose(var.cpu().numpy(), var_ref, rtol=0, atol=1e-8 * prior.max())
    if equal:
        _, _, ge, gW, gv, gs = model.gcv_grad(p.eta, p.W, p.v, p.sigma2)
        g_b = model.dsi_weights_grad()
        model.sync()
        r = dense.gcv_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, B)
        _, rb = dense.dsi_weights_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, B, "gcv")
        gref = _grad_vec(r[1], r[2], r[3], r[4], rb)
        got = _grad_vec(ge.cpu(), gW.cpu(), gv.cpu(), gs.cpu(), g_b.cpu())
        assert np.allclose(got, gref, rtol=1e-6, atol=1e-8 * np.abs(gref).max())
    model.close()


def test_mixture_full_dnet_d8_T4_n65536_vs_spectral_oracle():
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.dnet_equal()
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2, g_b = spectral.nll_grad_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v,
                                                               p.sigma2, B)
    model = MTGP.from_problem(p, "fp64")
    model.set_y(torch.from_numpy(y))
    model.set_dsi_weights(B)
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    gb = model.dsi_weights_grad()
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"])
    gref = 0.5 * _grad_vec(g_eta, g_W, g_v, g_s2, g_b)
    got = _grad_vec(ge.cpu(), gW.cpu(), gv.cpu(), gs.cpu(), gb.cpu())
    assert np.abs(got - gref).max() <= 1e-7 * (1 + np.abs(gref).max()), (got, gref)
    model.close()


def test_mixture_weights_argument_checks():
    from paper_2603_16014_gb300._lib import MTGPError
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("lattice", 2, (4, 4), seed=74)
    lat = MTGP.from_problem(p, "fp64")
    with pytest.raises(MTGPError) as ei:
        lat.set_dsi_weights(B)
    assert ei.value.code == 5                       # MTGP_ERR_UNSUPPORTED
    lat.close()
    p, X, y, model = _setup((4, 4), 75)
    with pytest.raises(MTGPError) as ei:
        model.dsi_weights_grad()                    # no weights set
    assert ei.value.code == 1                       # MTGP_ERR_INVALID_ARG
    model.set_dsi_weights(np.array([0.1, -1.0, 0.0, 0.0]))
    with pytest.raises(MTGPError) as ei:
        model.nll(p.eta, p.W, p.v, p.sigma2)
        model.sync()
    assert ei.value.code == 3                       # MTGP_ERR_NUMERIC: negative weight
    model.sync()
    # clearing the weights returns to the order-2 kernel
    model.set_dsi_weights(None)
    ref = dense.nll(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    out, _ = model.nll(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"])
    model.close()

"""Per-task noise variances (MTGP_NOISE_PER_TASK) on the GPU against the dense oracle: MLE loss and
gradient (one noise derivative per task), posterior, GCV and its gradient, cubature; equal and
nested sizes, both designs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _setup(kind, m, seed):
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem(kind, 2, m, seed=seed, eta=0.6, v=0.2, sigma2=1e-4,
                            recipe="walshcos32" if kind == "dnet" else "cos16", mmax=max(max(m), 8))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    xi = np.array([1e-4, 5e-4, 2e-3, 3e-5][:len(m)])
    model = MTGP.from_problem(p, "fp64", noise_per_task=True)
    model.set_y(torch.from_numpy(y))
    return p, X, y, xi, model


@pytest.mark.parametrize("kind,m", [("dnet", (5, 5, 5)), ("lattice", (6, 6)), ("lattice", (6, 4, 3)),
                                    ("dnet", (5, 3, 3, 2))])
def test_per_task_noise_nll_grad(kind, m):
    p, X, y, xi, model = _setup(kind, m, 61)
    ref, ge, gW, gv, gs = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, xi)
    out, tau, e_, W_, v_, s_ = model.nll_grad(p.eta, p.W, p.v, xi)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"])
    gref = 0.5 * np.concatenate([ge, gW.ravel(), gv, gs])
    got = np.concatenate([e_.cpu().numpy(), W_.cpu().numpy().ravel(), v_.cpu().numpy(), s_.cpu().numpy()])
    assert np.allclose(got, gref, rtol=1e-6, atol=1e-8 * np.abs(gref).max())
    model.close()


@pytest.mark.parametrize("kind,m", [("dnet", (5, 5, 5)), ("lattice", (6, 4, 3))])
def test_per_task_noise_posterior_gcv_cubature(kind, m):
    p, X, y, xi, model = _setup(kind, m, 62)
    equal = len(set(m)) == 1
    Xq, xq, tq = inputs.query_points(7, 2, seed=2, tasks=len(m))
    mean_ref, var_ref, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, xi, Xq, tq)
    mean, var = model.posterior(p.eta, p.W, p.v, xi, torch.from_numpy(xq), torch.from_numpy(tq), variance=True)
    g = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, xi)
    gout, _ = model.gcv(p.eta, p.W, p.v, xi)
    mu_ref, S_ref, _ = dense.cubature(p.kind, X, y, p.eta, p.W, p.v, xi)
    mu, S = model.cubature(p.eta, p.W, p.v, xi)
    model.sync()
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=1e-8 * prior.max())
    assert np.allclose(var.cpu().numpy(), var_ref, rtol=0, atol=1e-8 * prior.max())
    if equal:
        _, _, ge, gW, gv, gs = model.gcv_grad(p.eta, p.W, p.v, xi)
        model.sync()
        r = dense.gcv_grad(p.kind, X, y, p.eta, p.W, p.v, xi)
        gref = np.concatenate([r[1], r[2].ravel(), r[3], r[4]])
        got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
        assert np.allclose(got, gref, rtol=1e-6, atol=1e-8 * np.abs(gref).max())
    assert abs(gout[0].item() - g["L"]) <= 1e-8 * abs(g["L"])
    R = dense.task_covariance(p.W, p.v)
    assert np.allclose(mu.cpu().numpy(), mu_ref, rtol=0, atol=1e-8 * (np.abs(mu_ref).max() + 1))
    assert np.allclose(S.cpu().numpy(), S_ref, rtol=0, atol=1e-8 * np.abs(R).max())
    model.close()


def test_per_task_noise_refused_by_batch_and_static():
    from paper_2603_16014_gb300._lib import NOISE_PER_TASK, FP64, MTGPError, check, lib
    import ctypes
    h = ctypes.c_void_p()
    kind = (ctypes.c_int * 1)(1)
    one = (ctypes.c_int * 1)(2)
    m = (ctypes.c_int * 1)(5)
    gen = (ctypes.c_uint32 * 64)(*([1 << 31] * 64))
    gcols = (ctypes.c_int * 1)(32)
    shift = (ctypes.c_uint32 * 4)()
    prec = (ctypes.c_int * 1)(FP64 | NOISE_PER_TASK)
    rc = lib().mtgp_batch_create(ctypes.byref(h), 1, kind, one, one, m, gen, gcols, shift, 1, prec)
    assert rc == 5

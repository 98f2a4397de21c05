"""GCV loss and GCV mean on the GPU (C ABI mtgp_gcv) against the dense definition and the spectral
forms of the oracle: equal and nested unequal sizes, both designs, FP64 and FP32 transforms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense, spectral  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

TOL = {"fp64": 1e-8, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _run(p, y, precision):
    from paper_2603_16014_gb300.mtgp import MTGP
    model = MTGP.from_problem(p, precision)
    model.set_y(torch.from_numpy(y))
    out, tau = model.gcv(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    res = out.cpu().numpy(), tau.cpu().numpy()
    model.close()
    return res


@pytest.mark.parametrize("kind,m,precision", [
    ("lattice", (6, 6), "fp64"), ("dnet", (5, 5, 5), "fp64"), ("dnet", (6, 6, 6, 6), "fp32"),
    ("lattice", (6, 4, 2), "fp64"), ("dnet", (5, 5, 3), "fp64"), ("lattice", (3, 5, 4), "fp64"),
    ("dnet", (6, 3, 3, 1), "fp64")])
def test_gcv_vs_dense(kind, m, precision):
    p = inputs.make_problem(kind, 3, m, seed=21, eta=0.7, v=0.2, sigma2=1e-4,
                            recipe="walshcos32" if kind == "dnet" else "cos16", mmax=max(max(m), 8))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref = dense.gcv(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    out, tau = _run(p, y, precision)
    tol = TOL[precision]
    assert abs(out[0] - ref["L"]) <= tol * abs(ref["L"]), (out[0], ref["L"])
    assert abs(out[1] - ref["num"]) <= tol * abs(ref["num"])
    assert abs(out[2] - ref["trace"]) <= tol * abs(ref["trace"])
    assert np.allclose(tau, ref["tau"], rtol=tol, atol=tol * np.abs(ref["tau"]).max())


def test_gcv_full_size_digital_net_equal():
    p = inputs.dnet_equal(fp32_transform=False)
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref = spectral.gcv_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    out, tau = _run(p, y, "fp64")
    assert abs(out[0] - ref["L"]) <= 1e-8 * abs(ref["L"])
    assert np.allclose(tau, ref["tau"], rtol=1e-10, atol=1e-12)


def test_gcv_nested_lattice_d16_vs_class_oracle():
    p = inputs.lattice_nested(m=(12, 10, 8, 6, 4))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref = spectral.gcv_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    out, tau = _run(p, y, "fp64")
    assert abs(out[0] - ref["L"]) <= 1e-8 * abs(ref["L"]), (out[0], ref["L"])
    assert abs(out[2] - ref["trace"]) <= 1e-8 * abs(ref["trace"])
    assert np.allclose(tau, ref["tau"], rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("kind,m,precision", [("lattice", (6, 6), "fp64"), ("dnet", (5, 5, 5), "fp64"),
                                              ("dnet", (6, 6, 6, 6), "fp32")])
def test_gcv_gradient_vs_dense(kind, m, precision):
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem(kind, 3, m, seed=22, eta=0.7, v=0.2, sigma2=1e-4,
                            recipe="walshcos32" if kind == "dnet" else "cos16", mmax=max(max(m), 8))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    ref, ge, gW, gv, gs = dense.gcv_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    model = MTGP.from_problem(p, precision)
    model.set_y(torch.from_numpy(y))
    out, tau, e_, W_, v_, s_ = model.gcv_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    tol = 1e-7 if precision == "fp64" else 1e-4
    gref = np.concatenate([ge, gW.ravel(), gv, [gs]])
    got = np.concatenate([e_.cpu().numpy(), W_.cpu().numpy().ravel(), v_.cpu().numpy(), s_.cpu().numpy()])
    assert abs(out[0].item() - ref["L"]) <= TOL[precision] * abs(ref["L"])
    assert np.allclose(got, gref, rtol=tol, atol=tol * np.abs(gref).max()), np.max(np.abs(got - gref) / np.abs(gref).max())
    model.close()


def test_gcv_gradient_unequal_sizes_unsupported():
    from paper_2603_16014_gb300._lib import MTGPError
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("lattice", 2, (5, 3), seed=2)
    model = MTGP.from_problem(p, "fp64")
    model.set_y(torch.zeros(p.N, dtype=torch.float64))
    with pytest.raises(MTGPError) as ei:
        model.gcv_grad(p.eta, p.W, p.v, p.sigma2)
    assert ei.value.code == 5
    model.close()

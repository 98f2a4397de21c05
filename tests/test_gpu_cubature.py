"""Multitask Bayesian cubature on the GPU (C ABI mtgp_cubature) against the dense oracle: equal and
nested unequal sizes, both designs, FP64 and FP32 transforms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

TOL = {"fp64": 1e-8, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


@pytest.mark.parametrize("kind,m,precision", [
    ("lattice", (6, 6), "fp64"), ("dnet", (5, 5, 5), "fp64"), ("dnet", (6, 6, 6, 6), "fp32"),
    ("lattice", (6, 4, 2), "fp64"), ("dnet", (5, 5, 3), "fp64"), ("lattice", (3, 5, 4), "fp64")])
def test_cubature_vs_dense(kind, m, precision):
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem(kind, 3, m, seed=23, eta=0.7, v=0.2, sigma2=1e-4,
                            recipe="walshcos32" if kind == "dnet" else "cos16", mmax=max(max(m), 8))
    X = dense.all_points(p.kind, p.gen, p.shift, p.m)
    y = inputs.synth_y(p, X)
    mu_ref, S_ref, tau_ref = dense.cubature(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    model = MTGP.from_problem(p, precision)
    model.set_y(torch.from_numpy(y))
    mu, S = model.cubature(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    mu, S = mu.cpu().numpy(), S.cpu().numpy()
    R = dense.task_covariance(p.W, p.v)
    scale = np.abs(R).max()
    tol = TOL[precision]
    assert np.allclose(mu, mu_ref, rtol=0, atol=tol * (np.abs(mu_ref).max() + np.sqrt(scale)))
    assert np.allclose(S, S_ref, rtol=0, atol=tol * scale)
    assert np.allclose(S, S.T, rtol=0, atol=1e-12 * scale)
    model.close()

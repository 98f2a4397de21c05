"""GPU parity: the CUDA path through the C ABI against the CPU oracle on identical seeded inputs.

Tolerances: NLL within 1e-8 relative in FP64 mode and 1e-5 in FP32-transform mode.  Gradients:
within 1e-7 (FP64) / 1e-4 (FP32) of the gradient's max-norm scale.  Posterior: |delta mean| and
|delta var| within 1e-8 (FP64) / 1e-5 (FP32) of the largest prior variance R_tt Q(x, x).
FP32-transform mode is exercised on digital nets, the designs it is specified for: the SI lattice
spectrum decays like f^-4, so its small eigenvalues fall below the FP32 transform noise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense, design, spectral  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

TOL_NLL = {"fp64": 1e-8, "fp32": 1e-5}
TOL_GRAD = {"fp64": 1e-7, "fp32": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _model(p, precision):
    from paper_2603_16014_gb300.mtgp import MTGP
    return MTGP.from_problem(p, precision)


def _points_oracle(p):
    return dense.all_points(p.kind, p.gen, p.shift, p.m)


SMALL = [
    ("lattice", 2, (5, 5)), ("dnet", 3, (6, 6, 6)), ("lattice", 2, (6, 4, 3)), ("dnet", 2, (7, 5, 5, 3)),
    ("lattice", 3, (3, 6, 4)), ("dnet", 2, (4, 0)), ("lattice", 2, (0, 0)), ("lattice", 1, (7,)),
    ("dnet", 4, (6,)), ("dnet", 2, (3,) * 8), ("lattice", 2, (2, 2, 2, 2, 2)), ("dnet", 3, (5, 5, 3, 3)),
]


@pytest.mark.parametrize("kind,d,m", SMALL)
def test_points_bit_exact(kind, d, m):
    p = inputs.make_problem(kind, d, m, seed=41)
    model = _model(p, "fp64")
    got = model.points().cpu().numpy().view(np.uint32)
    ref = np.concatenate(_points_oracle(p))
    assert np.array_equal(got, ref)


CASES = [(k, d, m, "fp64") for (k, d, m) in SMALL] + [(k, d, m, "fp32") for (k, d, m) in SMALL if k == "dnet"]


@pytest.mark.parametrize("kind,d,m,precision", CASES)
def test_nll_and_grad_vs_dense_oracle(kind, d, m, precision):
    p = inputs.make_problem(kind, d, m, seed=43, eta=0.6, v=0.1, sigma2=1e-4, s=min(2, len(m)))
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2 = dense.nll_grad(kind, X, y, p.eta, p.W, p.v, p.sigma2)
    model = _model(p, precision)
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    out = out.cpu().numpy()
    tol = TOL_NLL[precision]
    assert abs(out[0] - ref["nll"]) <= tol * abs(ref["nll"]), (out[0], ref["nll"])
    assert abs(out[1] + out[2] - ref["L"]) <= tol * max(abs(ref["quad"]) + abs(ref["logdet"]), 1.0)
    assert np.allclose(tau.cpu().numpy(), ref["tau"], rtol=0, atol=10 * tol * (1 + np.abs(ref["tau"]).max()))
    gref = np.concatenate([0.5 * g_eta, 0.5 * g_W.ravel(), 0.5 * g_v, [0.5 * g_s2]])
    got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
    scale = 1.0 + np.abs(gref).max()
    err = np.abs(got - gref).max()
    assert err <= TOL_GRAD[precision] * scale, (err, scale, got, gref)
    # NLL-only entry point agrees with the NLL of the gradient call
    out2, tau2 = model.nll(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out2.cpu().numpy()[0] - out[0]) <= 1e-12 * abs(out[0])


@pytest.mark.parametrize("kind,d,m,precision", [("lattice", 2, (6, 6), "fp64"), ("dnet", 3, (5, 5, 5), "fp64"),
                                                ("lattice", 2, (6, 4, 3), "fp64"), ("dnet", 2, (6, 3), "fp64"),
                                                ("dnet", 3, (5, 5, 5), "fp32"), ("dnet", 2, (6, 3), "fp32")])
def test_posterior_vs_dense_oracle(kind, d, m, precision):
    p = inputs.make_problem(kind, d, m, seed=47, eta=0.6, v=0.1, sigma2=1e-4)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    Xq, xq, tq = inputs.query_points(37, d, seed=5, tasks=len(m))
    mean_ref, var_ref, prior = dense.posterior(kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    model = _model(p, precision)
    model.set_y(torch.from_numpy(y))
    mean, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=True)
    model.sync()
    tol = TOL_NLL[precision]
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=tol * prior.max())
    assert np.allclose(var.cpu().numpy(), var_ref, rtol=0, atol=tol * prior.max())


@pytest.mark.parametrize("nq", [1, 2, 257, 4099])
def test_posterior_mean_slicing_edge_cases(nq):
    """The mean splits queries and design points over CTAs: one query (every point slice in its own
    CTA), ragged query counts, per-task slices of unequal tasks with partial last slices."""
    p = inputs.make_problem("lattice", 3, (9, 7, 5), seed=48, eta=0.6, v=0.1, sigma2=1e-4)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    Xq, xq, tq = inputs.query_points(nq, 3, seed=6, tasks=3)
    mean_ref, _, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq)
    model = _model(p, "fp64")
    model.set_y(torch.from_numpy(y))
    mean, _ = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=False)
    model.sync()
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=TOL_NLL["fp64"] * prior.max())


def test_errors_surface_through_status():
    p = inputs.make_problem("dnet", 2, (5, 5), seed=3, sigma2=1e-4)
    from paper_2603_16014_gb300._lib import MTGPError
    model = _model(p, "fp64")
    with pytest.raises(MTGPError):                 # NLL before set_y
        model.nll(p.eta, p.W, p.v, p.sigma2)
    y = np.zeros(p.N)
    y[3] = np.nan
    model.set_y(torch.from_numpy(y))
    with pytest.raises(MTGPError) as ei:
        model.sync()
    assert ei.value.code == 3                       # MTGP_ERR_NUMERIC
    model.set_y(torch.zeros(p.N, dtype=torch.float64))
    model.sync()
    # an indefinite task covariance (v < 0 and W = 0) makes a pivot negative
    with pytest.raises(MTGPError):
        model.nll(p.eta, np.zeros_like(p.W), -np.ones(p.T), 1e-6)
        model.sync()
    model.sync()
    # a non-finite parameter is flagged by the fused kernels' own check
    with pytest.raises(MTGPError) as ei:
        model.nll_grad(np.r_[np.nan, p.eta[1:]], p.W, p.v, p.sigma2)
        model.sync()
    assert ei.value.code == 3
    model.sync()
    out, _ = model.nll(p.eta, p.W, p.v, p.sigma2)  # and the handle stays usable
    model.sync()
    assert np.isfinite(out[0].item())


# ----------------------------------------------------------------------------- full sizes

def test_full_lattice_d2_T2_n1024_vs_dense():
    p = inputs.lattice_small()
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2 = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
    model = _model(p, "fp64")
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"])
    gref = np.concatenate([0.5 * g_eta, 0.5 * g_W.ravel(), 0.5 * g_v, [0.5 * g_s2]])
    got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
    assert np.abs(got - gref).max() <= 1e-7 * (1 + np.abs(gref).max())


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_dnet_d8_T4_n65536_vs_spectral_oracle(precision):
    p = inputs.dnet_equal()
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2 = spectral.nll_grad_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    model = _model(p, precision)
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= TOL_NLL[precision] * abs(ref["nll"])
    assert np.allclose(tau.cpu().numpy(), ref["tau"], atol=1e-12)
    gref = np.concatenate([0.5 * g_eta, 0.5 * g_W.ravel(), 0.5 * g_v, [0.5 * g_s2]])
    got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
    assert np.abs(got - gref).max() <= TOL_GRAD[precision] * (1 + np.abs(gref).max()), (got, gref)
    if precision == "fp64":
        # central differences (sigma2 = 1e-8 moves the NLL below FP64 resolution: checked above only)
        _check_fd(model, p, ge, gW, gv, gs, idx_eta=[0, 5], idx_W=[(1, 0), (3, 1)], idx_v=[2], nll=out[0].item(),
                  with_sigma2=False)


def _check_fd(model, p, ge, gW, gv, gs, idx_eta, idx_W, idx_v, nll, with_sigma2=True, h=1e-6, rtol=1e-5):
    """Central differences with step h (relative, in log space, for eta, v, sigma2; absolute for W).
    Allowed error = rtol (|g| + 1) + roundoff of the difference quotient, 16 eps |NLL| / h."""
    eps = np.finfo(np.float64).eps
    rnd = 16 * eps * abs(nll) / h

    def f(eta, W, v, s2):
        out, _ = model.nll(eta, W, v, s2)
        return out[0].item()

    def ok(fd, g):
        return abs(fd - g) <= rtol * (abs(g) + 1) + rnd
    for j in idx_eta:
        e1, e2 = p.eta.copy(), p.eta.copy()
        e1[j] *= np.exp(h)
        e2[j] *= np.exp(-h)
        fd = (f(e1, p.W, p.v, p.sigma2) - f(e2, p.W, p.v, p.sigma2)) / (2 * h) / p.eta[j]
        assert ok(fd, ge[j].item()), (j, fd, ge[j].item(), rnd)
    for (t, k) in idx_W:
        W1, W2 = p.W.copy(), p.W.copy()
        W1[t, k] += h
        W2[t, k] -= h
        fd = (f(p.eta, W1, p.v, p.sigma2) - f(p.eta, W2, p.v, p.sigma2)) / (2 * h)
        assert ok(fd, gW[t, k].item()), (t, k, fd, gW[t, k].item(), rnd)
    for t in idx_v:
        v1, v2 = p.v.copy(), p.v.copy()
        v1[t] *= np.exp(h)
        v2[t] *= np.exp(-h)
        fd = (f(p.eta, p.W, v1, p.sigma2) - f(p.eta, p.W, v2, p.sigma2)) / (2 * h) / p.v[t]
        assert ok(fd, gv[t].item()), (t, fd, gv[t].item(), rnd)
    if with_sigma2:
        fd = (f(p.eta, p.W, p.v, p.sigma2 * np.exp(h)) - f(p.eta, p.W, p.v, p.sigma2 * np.exp(-h))) / (2 * h) / p.sigma2
        assert abs(fd - gs[0].item()) <= rtol * (abs(gs[0].item()) + 1) + rnd / p.sigma2, (fd, gs[0].item())


def test_full_lattice_d16_T5_nested_vs_class_oracle():
    p = inputs.lattice_nested()
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    model = _model(p, "fp64")
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    ref = spectral.nll_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"]), (out[0].item(), ref["nll"])
    assert np.allclose(tau.cpu().numpy(), ref["tau"], atol=1e-8 * (1 + np.abs(ref["tau"]).max()))
    nll = out[0].item()
    allW = [(t, k) for t in range(5) for k in range(2)]
    # the finite-difference step of the workload definition (1e-6) ...
    _check_fd(model, p, ge, gW, gv, gs, idx_eta=list(range(16)), idx_W=allW, idx_v=list(range(5)), nll=nll,
              with_sigma2=False)
    # ... and a tighter check at a step where truncation (h^2) and roundoff (1/h) are both small
    _check_fd(model, p, ge, gW, gv, gs, idx_eta=list(range(16)), idx_W=allW, idx_v=list(range(5)), nll=nll,
              with_sigma2=True, h=1e-4, rtol=1e-6)


# (d = 2, T = 8 at sigma2 = 1e-6 is outside FP32-transform mode: FP32 columns rounded exactly and transformed
# in FP32 already miss 1e-5 there, 1.5e-5 on the CPU)
RT_CASES = [(3, 1, 10), (9, 2, 11), (16, 3, 12), (5, 4, 13), (12, 6, 10), (3, 8, 11), (8, 4, 18)]


@pytest.mark.parametrize("d,T,m", RT_CASES)
def test_register_tile_path_vs_oracle(d, T, m):
    """Equal-size digital nets with FP32 transforms at sizes the register-tile kernels take (both tile
    sizes in 2^5..2^9, d <= 16): NLL and gradient against the per-frequency oracle, with the
    double-float solve (default) and with the FP64 solve; the two solves see the same FP32 spectra and
    agree to far better than the FP32-mode tolerance."""
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("dnet", d, (m,) * T, seed=70 + m + T, s=min(2, T), eta=(0.3, 1.2), v=0.1, sigma2=1e-6,
                            recipe="walshcos32", mmax=max(m, 16))
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2 = spectral.nll_grad_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    gref = 0.5 * np.concatenate([g_eta, np.ravel(g_W), g_v, [g_s2]])
    res = {}
    for solve in ("df", "fp64"):
        model = MTGP.from_problem(p, "fp32", solve=solve)
        model.set_y(torch.from_numpy(y))
        out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
        o2, _ = model.nll(p.eta, p.W, p.v, p.sigma2)
        model.sync()
        got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
        nll = out[0].item()
        assert abs(nll - ref["nll"]) <= TOL_NLL["fp32"] * abs(ref["nll"]), (solve, nll, ref["nll"])
        assert o2[0].item() == pytest.approx(nll, rel=1e-12, abs=0)
        assert np.all(np.abs(got - gref) <= TOL_GRAD["fp32"] * np.abs(gref).max()), (solve, got, gref)
        res[solve] = (nll, got)
        model.close()
    # the adjoint weights of both solves are rounded to FP32 before the FP32 adjoint transforms, so the
    # gradients agree to the transforms' amplification of one rounding (1e-5 of the largest entry)
    assert abs(res["df"][0] - res["fp64"][0]) <= 1e-10 * abs(res["fp64"][0])
    assert np.all(np.abs(res["df"][1] - res["fp64"][1]) <= 1e-5 * np.abs(res["fp64"][1]).max())


def test_double_float_solve_falls_back_to_fp64_outside_its_range():
    """sigma2 = 1e-20 with a spectrum below the FP32 transform noise (d = 8, eta = 0.1): the clamped
    frequencies have pivots far below the double-float working range (2^-50) and are solved by the FP64
    recurrences; the result equals the FP64-solve handle's."""
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem("dnet", 8, (11,) * 3, seed=81, s=2, eta=0.1, v=0.1, sigma2=1e-20, recipe="walshcos32",
                            mmax=16)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    outs = {}
    for solve in ("df", "fp64"):
        model = MTGP.from_problem(p, "fp32", solve=solve)
        model.set_y(torch.from_numpy(y))
        out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
        model.sync()
        outs[solve] = (out.cpu().numpy(), np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(),
                                                          gv.cpu().numpy(), gs.cpu().numpy()]))
        model.close()
    assert np.all(np.isfinite(outs["df"][0])) and np.all(np.isfinite(outs["df"][1]))
    assert abs(outs["df"][0][0] - outs["fp64"][0][0]) <= 1e-10 * abs(outs["fp64"][0][0])
    assert np.all(np.abs(outs["df"][1] - outs["fp64"][1]) <= 1e-5 * np.abs(outs["fp64"][1]).max())


@pytest.mark.parametrize("kind", ["lattice", "dnet"])
def test_medium_nested_gradient_vs_class_oracle(kind):
    """Nested sizes n = 2^12, 2^10, 2^8 (tree solver, FP64): every gradient entry against the residue-class
    oracle's gradient (sum over classes of tr(G dM), built independently of the dense matrix)."""
    p = inputs.make_problem(kind, 4, (12, 10, 8), seed=61, s=2, eta=(0.3, 1.5), v=0.1, sigma2=1e-6)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    model = _model(p, "fp64")
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    L, g_eta, g_W, g_v, g_s2 = spectral.grad_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
    N = sum(1 << x for x in p.m)
    assert abs(out[0].item() - 0.5 * (L + N * np.log(2 * np.pi))) <= 1e-8 * abs(out[0].item())
    gref = 0.5 * np.concatenate([g_eta, g_W.ravel(), g_v, [g_s2]])
    got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
    scale = np.abs(gref).max()
    assert np.all(np.abs(got - gref) <= TOL_GRAD["fp64"] * scale), (got, gref)


def test_autograd_function_gradient_vs_dense_oracle():
    """torch.autograd through mtgp.NLLFunction (the hand-written adjoint behind the autograd interface):
    d(3 NLL + 2)/d(eta, W, v, sigma2) against 3/2 times the dense oracle's analytic gradient of L."""
    from paper_2603_16014_gb300.mtgp import nll as nll_fn
    for kind, d, m in (("lattice", 2, (6, 4)), ("dnet", 3, (5, 5, 5))):
        p = inputs.make_problem(kind, d, m, seed=62, s=2, eta=0.6, v=0.2, sigma2=1e-4)
        X = _points_oracle(p)
        y = inputs.synth_y(p, X)
        ref, g_eta, g_W, g_v, g_s2 = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2)
        model = _model(p, "fp64")
        model.set_y(torch.from_numpy(y))
        th = [torch.as_tensor(np.asarray(a, dtype=np.float64)).cuda().requires_grad_()
              for a in (p.eta, p.W, p.v, [p.sigma2])]
        loss = 3.0 * nll_fn(model, *th) + 2.0
        grads = torch.autograd.grad(loss, th)
        model.sync()
        assert abs(loss.item() - (3.0 * ref["nll"] + 2.0)) <= 1e-8 * abs(3.0 * ref["nll"] + 2.0)
        gref = 1.5 * np.concatenate([g_eta, g_W.ravel(), g_v, [g_s2]])
        got = np.concatenate([g.detach().cpu().numpy().ravel() for g in grads])
        assert grads[1].shape == th[1].shape and grads[3].shape == th[3].shape
        assert np.all(np.abs(got - gref) <= TOL_GRAD["fp64"] * np.abs(gref).max()), (kind, got, gref)
        model.close()


# ----------------------------------------------------------------------------- full sizes, bench launch shapes

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_posterior_sampled_outputs(precision):
    """The d = 8, T = 4, n = 2^16 net fit with the bench's query counts (2^16 means, 2^10 variances);
    sampled outputs against the per-frequency oracle."""
    p = inputs.dnet_equal(fp32_transform=(precision == "fp32"))
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    model = _model(p, precision)
    model.set_y(torch.from_numpy(y))
    Xq, xq, tq = inputs.query_points(1 << 16, p.d, seed=3, tasks=p.T)
    mean, _ = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=False)
    Xv, xv, tv = inputs.query_points(1 << 10, p.d, seed=4, tasks=p.T)
    _, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xv), torch.from_numpy(tv), variance=True)
    model.sync()
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    pick = np.array([0, 1, 4097, 65535, 31337])
    ref = spectral.posterior_mean_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2, Xq[pick], tq[pick])
    R = design.task_covariance(p.W, p.v)
    prior = np.array([R[t, t] * design.product_kernel(p.kind, Xq[i], Xq[i], p.eta) for i, t in zip(pick, tq[pick])])
    tol = TOL_NLL[precision]
    assert np.all(np.abs(mean[pick] - ref) <= tol * prior), np.max(np.abs(mean[pick] - ref) / prior)
    vpick = np.array([0, 511, 1023])
    vref = spectral.posterior_var_equal(p.kind, p.gen, p.shift, p.m, p.eta, p.W, p.v, p.sigma2, Xv[vpick], tv[vpick])
    vprior = np.array([R[t, t] * design.product_kernel(p.kind, Xv[i], Xv[i], p.eta) for i, t in zip(vpick, tv[vpick])])
    assert np.all(np.abs(var[vpick] - vref) <= tol * vprior), np.max(np.abs(var[vpick] - vref) / vprior)


LATTICE_SAMPLE = (0, 77, 200, 255)
DNET_SAMPLE = (256, 300, 401, 511)


def test_full_size_batch_sampled_fits():
    """The 512-fit mixed batch of the bench, in its precisions (digital nets with FP32 transforms,
    lattices with FP64 transforms): sampled fits of both halves, NLL and gradient against the
    per-frequency oracle at the precision's tolerance."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2603_16014_gb300.mtgp import Batch
    probs = bench.batch_problems(512)
    sample = LATTICE_SAMPLE + DNET_SAMPLE
    ys = [inputs.synth_y(q, dense.all_points(q.kind, q.gen, q.shift, q.m)) if i in sample else
          np.random.default_rng(i).standard_normal(q.N) for i, q in enumerate(probs)]
    b = Batch(probs, s=2, precision="auto")
    assert all(b.precision[f] == "fp64" for f in LATTICE_SAMPLE)
    assert all(b.precision[f] == "fp32" for f in DNET_SAMPLE)
    b.set_y(torch.from_numpy(np.concatenate(ys)))
    th = [bench.default_theta(q) for q in probs]
    b.set_theta(torch.from_numpy(b.pack(th)))
    nll, g = b.nll_grad()
    torch.cuda.synchronize()
    nll, g = nll.cpu().numpy(), g.cpu().numpy()
    for f in sample:
        q = probs[f]
        assert q.kind == ("lattice" if f in LATTICE_SAMPLE else "dnet")
        out, ge, gW, gv, gs = spectral.nll_grad_equal(q.kind, q.gen, q.shift, q.m, ys[f], *th[f])
        gref = 0.5 * np.concatenate([ge, np.ravel(gW), gv, [gs]])
        o0, o1 = b.param_offsets[f], b.param_offsets[f + 1]
        err = np.abs(g[o0:o1] - gref).max() / np.abs(gref).max()
        if q.kind == "lattice":
            # FP64 mode: 1e-8 relative NLL; gradient normwise 1e-7
            assert abs(nll[f] - out["nll"]) <= 1e-8 * abs(out["nll"]), (f, nll[f], out["nll"])
            assert err <= 1e-7, (f, err)
        else:
            assert abs(nll[f] - out["nll"]) <= 1e-5 * abs(out["nll"]), (f, nll[f], out["nll"])
            # FP32 transforms of up to 29 columns of 2^16 entries: normwise 1e-3 (the eta entries are sums
            # over C n terms of FP32-transformed adjoint weights; 1.8e-4 measured at T = 8)
            assert err <= 1e-3, (f, err)
    b.close()


# ----------------------------------------------------------------------------- SI smoothness

@pytest.mark.parametrize("alpha", [1, 3, 4])
@pytest.mark.parametrize("m", [(6, 6), (6, 4, 3)])
def test_si_smoothness_nll_grad_posterior_vs_dense(alpha, m):
    """Lattice handles with the SI kernel of smoothness 1, 3, 4 (Eq. 2.5): equal sizes (fused
    kernels) and nested sizes (tree solver), against the dense oracle with the same kernel."""
    p = inputs.make_problem("lattice", 2, m, seed=51, eta=0.6, v=0.2, sigma2=1e-4)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    ref, g_eta, g_W, g_v, g_s2 = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, alpha)
    model = _model(p, "fp64")
    model.set_smoothness(alpha)
    model.set_y(torch.from_numpy(y))
    out, tau, ge, gW, gv, gs = model.nll_grad(p.eta, p.W, p.v, p.sigma2)
    model.sync()
    assert abs(out[0].item() - ref["nll"]) <= 1e-8 * abs(ref["nll"]), (out[0].item(), ref["nll"])
    gref = 0.5 * np.concatenate([g_eta, g_W.ravel(), g_v, [g_s2]])
    got = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
    assert np.allclose(got, gref, rtol=1e-6, atol=1e-8 * np.abs(gref).max())
    Xq, xq, tq = inputs.query_points(9, 2, seed=8, tasks=len(m))
    mean_ref, var_ref, prior = dense.posterior(p.kind, X, y, p.eta, p.W, p.v, p.sigma2, Xq, tq, alpha)
    equal = len(set(m)) == 1
    mean, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=equal)
    model.sync()
    assert np.allclose(mean.cpu().numpy(), mean_ref, rtol=0, atol=1e-8 * prior.max())
    if equal:
        assert np.allclose(var.cpu().numpy(), var_ref, rtol=0, atol=1e-8 * prior.max())


def test_smoothness_argument_checks():
    from paper_2603_16014_gb300._lib import MTGPError
    p = inputs.make_problem("dnet", 2, (5, 5), seed=3)
    model = _model(p, "fp64")
    for bad in (0, 5):
        with pytest.raises(MTGPError) as ei:
            model.set_smoothness(bad)
        assert ei.value.code == 1
    q = inputs.make_problem("lattice", 2, (5, 5), seed=3)
    mq = _model(q, "fp64")
    with pytest.raises(MTGPError) as ei:
        mq.set_smoothness(7)
    assert ei.value.code == 1


@pytest.mark.parametrize("kind,d,m,pt", [("dnet", 3, (6, 6, 6), False), ("lattice", 2, (6, 4, 3), False),
                                         ("dnet", 2, (5, 5), True)])
def test_host_buffer_entry_point_matches_device_call(kind, d, m, pt):
    # mtgp_nll_grad_host: packed host theta in, packed host results out, same values as the device call
    from paper_2603_16014_gb300.mtgp import MTGP
    p = inputs.make_problem(kind, d, m, seed=81, eta=0.6, v=0.2, sigma2=1e-4, s=2)
    X = _points_oracle(p)
    y = inputs.synth_y(p, X)
    model = MTGP.from_problem(p, "fp64", noise_per_task=pt)
    model.set_y(torch.from_numpy(y))
    s2 = np.array([1e-4, 3e-4, 2e-4][:p.T]) if pt else p.sigma2
    ref = [t.cpu().numpy() for t in model.nll_grad(p.eta, p.W, p.v, s2)]
    h_th = model.pack_theta(p.eta, p.W, p.v, s2)
    h_out = model.host_out(p.W.shape[1])
    h_out.fill_(np.nan)
    model.nll_grad_host(h_th, h_out, p.W.shape[1])
    model.sync()
    got = [t.numpy() for t in model.unpack_out(h_out, p.W.shape[1])]
    for a, b in zip(got, ref):
        assert np.array_equal(a.reshape(-1), b.reshape(-1))
    dref, ge, gW, gv, gs = dense.nll_grad(p.kind, X, y, p.eta, p.W, p.v, s2)
    assert abs(got[0][0] - dref["nll"]) <= 1e-8 * abs(dref["nll"])
    # later calls replay the captured sequence and read the host buffer's current contents
    v2 = p.v * 1.5
    h_th.copy_(model.pack_theta(p.eta, p.W, v2, s2, pin=False))
    model.nll_grad_host(h_th, h_out, p.W.shape[1])
    model.sync()
    ref2 = [t.cpu().numpy() for t in model.nll_grad(p.eta, p.W, v2, s2)]
    for a, b in zip(model.unpack_out(h_out, p.W.shape[1]), ref2):
        assert np.array_equal(a.numpy().reshape(-1), b.reshape(-1))
    # a kernel-configuration change takes effect (digital nets: order 3 of Eq. 2.6)
    if kind == "dnet":
        model.set_smoothness(3)
        model.nll_grad_host(h_th, h_out, p.W.shape[1])
        model.sync()
        ref3 = [t.cpu().numpy() for t in model.nll_grad(p.eta, p.W, v2, s2)]
        for a, b in zip(model.unpack_out(h_out, p.W.shape[1]), ref3):
            assert np.array_equal(a.numpy().reshape(-1), b.reshape(-1))
        assert abs(ref3[0][0] - ref2[0][0]) > 1e-6 * abs(ref2[0][0])
    # pageable host buffers take the direct launches
    p_th = model.pack_theta(p.eta, p.W, v2, s2, pin=False)
    p_out = model.host_out(p.W.shape[1], pin=False)
    model.nll_grad_host(p_th, p_out, p.W.shape[1])
    model.sync()
    assert np.array_equal(p_out.numpy(), h_out.numpy())
    with pytest.raises(Exception):
        model.nll_grad_host(h_th, h_out, p.T + 1)    # s out of range: refused before any device work
    model.close()


@pytest.mark.parametrize("nq", [1, 3, 130])
def test_nested_posterior_variance_batches_and_medium_size(nq):
    """Unequal sizes: the variance through the tree solver's factor (rows of a query batch, per-task
    transforms, class-by-class forward elimination), at a size with 256 residue classes, against
    the per-class dense oracle; query counts below, at and above the batch edges."""
    p = inputs.make_problem("lattice", 4, (12, 10, 8), seed=49, eta=0.6, v=0.1, sigma2=1e-4)
    model = _model(p, "fp64")
    X = model.points().cpu().numpy().view(np.uint32)
    offs = np.concatenate([[0], np.cumsum(p.n)])
    y = inputs.synth_y(p, [X[offs[t]:offs[t + 1]] for t in range(p.T)])
    model.set_y(torch.from_numpy(y))
    Xq, xq, tq = inputs.query_points(nq, 4, seed=7, tasks=3)
    mean, var = model.posterior(p.eta, p.W, p.v, p.sigma2, torch.from_numpy(xq), torch.from_numpy(tq), variance=True)
    model.sync()
    k = min(nq, 3)
    mean_ref, var_ref = spectral.posterior_by_class(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2,
                                                    Xq[:k], tq[:k])
    R = dense.task_covariance(p.W, p.v)
    scale = np.abs(R).max() * (1 + 0.6 * np.pi ** 4 / 45) ** 4     # prior bound: R_tt prod_j (1 + eta_j K(0))
    assert np.allclose(var.cpu().numpy()[:k], var_ref, rtol=0, atol=1e-8 * scale)
    assert np.allclose(mean.cpu().numpy()[:k], mean_ref, rtol=0, atol=1e-8 * scale)
    v = var.cpu().numpy()
    assert np.all(v > -1e-9 * scale)

"""Batched fits (mtgp_batch_*): per-fit results equal the single-fit entry points, Adam steps equal a
host-side Adam over single-fit gradients, and graph replay equals eager launches."""
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


def _fits(seed, count, ms=(5, 7, 8, 10), precision="fp32"):
    """Mixed fits; with precision "fp32" all digital nets (FP32 transforms are specified for digital
    nets), with "fp64" or "auto" alternating lattices and nets."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = "lattice" if i % 2 == 0 else "dnet"
        if precision == "fp32":
            kind = "dnet"
        T = int(rng.choice([2, 3, 5, 8]))
        d = int(rng.choice([2, 5, 9, 12]))
        m = int(rng.choice(ms))
        p = inputs.make_problem(kind, d, (m,) * T, seed=1000 * seed + i, s=2, eta=(0.3, 1.0), v=0.1, sigma2=1e-4,
                                recipe="walshcos32" if kind == "dnet" else "cos16", mmax=max(m, 12))
        out.append(p)
    return out


def _theta(p, rng):
    return (p.eta * np.exp(0.2 * rng.standard_normal(p.d)), p.W + 0.1 * rng.standard_normal(p.W.shape),
            p.v * np.exp(0.2 * rng.standard_normal(p.T)), p.sigma2)


def _ys(probs):
    ys = []
    for p in probs:
        X = dense.all_points(p.kind, p.gen, p.shift, p.m)
        ys.append(inputs.synth_y(p, X))
    return ys


@pytest.mark.parametrize("precision", ["fp32", "fp64", "auto"])
def test_batch_nll_grad_equals_single_fit(precision):
    """Batched NLL and gradient equal the single-fit entry point bit for bit; "auto" mixes FP64-transform
    lattices and FP32-transform nets in one batch (separate kernel classes)."""
    from paper_2603_16014_gb300.mtgp import MTGP, Batch
    probs = _fits({"fp32": 3, "fp64": 4, "auto": 5}[precision], 10, precision=precision)
    ys = _ys(probs)
    rng = np.random.default_rng(11)
    thetas = [_theta(p, rng) for p in probs]
    b = Batch(probs, s=2, precision=precision)
    b.set_y(torch.from_numpy(np.concatenate(ys)))
    b.set_theta(torch.from_numpy(b.pack(thetas)))
    nll, g = b.nll_grad()
    torch.cuda.synchronize()
    nll, g = nll.cpu().numpy(), g.cpu().numpy()
    if precision == "auto":
        assert b.precision == ["fp64" if p.kind == "lattice" else "fp32" for p in probs]
    for f, (p, y, th) in enumerate(zip(probs, ys, thetas)):
        m = MTGP.from_problem(p, b.precision[f])
        m.set_y(torch.from_numpy(y))
        out, tau, ge, gW, gv, gs = m.nll_grad(*th)
        m.sync()
        gref = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
        o0, o1 = b.param_offsets[f], b.param_offsets[f + 1]
        # same kernels, same split, same reduction order: identical results
        assert nll[f] == out[0].item(), (f, nll[f], out[0].item())
        assert np.array_equal(g[o0:o1], gref), f
        m.close()
    if precision != "fp32":
        # and the dense oracle on a lattice and a net (FP64 lattice: 1e-8; "auto" net: FP32 1e-5)
        for f in (0, 1):
            p, y, th = probs[f], ys[f], thetas[f]
            X = dense.all_points(p.kind, p.gen, p.shift, p.m)
            ref = dense.nll(p.kind, X, y, *th)
            tol = 1e-8 if b.precision[f] == "fp64" else 1e-5
            assert abs(nll[f] - ref["nll"]) <= tol * abs(ref["nll"])
    # autotuned splits change rounding only
    b.autotune(reps=2)
    nll2, _ = b.nll_grad()
    torch.cuda.synchronize()
    tol = np.array([1e-5 if q == "fp32" else 1e-10 for q in b.precision])
    assert np.all(np.abs(nll2.cpu().numpy() - nll) <= tol * np.abs(nll))
    b.close()


def test_batch_adam_matches_host_adam_and_graph_replay():
    from paper_2603_16014_gb300.mtgp import MTGP, Batch
    probs = _fits(7, 6, ms=(6, 8), precision="fp32")
    ys = _ys(probs)
    rng = np.random.default_rng(5)
    thetas = [_theta(p, rng) for p in probs]
    y_all = torch.from_numpy(np.concatenate(ys))
    steps, lr = 6, 0.05
    traces = []
    finals = []
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for graph in (False, True):
            b = Batch(probs, s=2, precision="fp32")
            b.set_y(y_all)
            b.set_theta(torch.from_numpy(b.pack(thetas)))
            trace = torch.zeros(steps * len(probs), dtype=torch.float64, device="cuda")
            b.adam(steps, lr, graph=graph, trace=trace)
            stream.synchronize()
            traces.append(trace.cpu().numpy().reshape(steps, len(probs)))
            finals.append(b.get_theta().cpu().numpy())
            b.close()
    assert np.array_equal(traces[0], traces[1])
    assert np.array_equal(finals[0], finals[1])
    # host Adam over single-fit gradients (log parameters for eta, v, sigma2)
    b1, b2, eps = 0.9, 0.999, 1e-8
    for f, (p, y, th) in enumerate(zip(probs, ys, thetas)):
        m = MTGP.from_problem(p, "fp32")
        m.set_y(torch.from_numpy(y))
        eta, W, v, s2 = [np.array(x, dtype=np.float64) for x in th]
        x = np.concatenate([np.log(eta), W.ravel(), np.log(v), [np.log(s2)]])
        islog = np.concatenate([np.ones(p.d), np.zeros(W.size), np.ones(p.T), [1.0]]).astype(bool)
        m1 = np.zeros_like(x)
        m2 = np.zeros_like(x)
        for k in range(steps):
            nat = np.where(islog, np.exp(x), x)
            e_, W_, v_, s_ = nat[:p.d], nat[p.d:p.d + W.size].reshape(W.shape), nat[p.d + W.size:-1], nat[-1]
            out, tau, ge, gW, gv, gs = m.nll_grad(e_, W_, v_, s_)
            gnat = np.concatenate([ge.cpu().numpy(), gW.cpu().numpy().ravel(), gv.cpu().numpy(), gs.cpu().numpy()])
            assert abs(out[0].item() - traces[0][k, f]) <= 1e-12 * abs(out[0].item())
            gl = np.where(islog, gnat * nat, gnat)
            m1 = b1 * m1 + (1 - b1) * gl
            m2 = b2 * m2 + (1 - b2) * gl * gl
            x = x - lr * (m1 / (1 - b1 ** (k + 1))) / (np.sqrt(m2 / (1 - b2 ** (k + 1))) + eps)
        nat = np.where(islog, np.exp(x), x)
        o0, o1 = 0, 0
        from paper_2603_16014_gb300.mtgp import Batch as _B  # noqa: F401
        m.close()
        fin = finals[0]
        # locate the fit's slice from the packing order (eta, W, v, sigma2)
        sizes = [q.d + len(q.m) * 2 + len(q.m) + 1 for q in probs]
        o0 = int(np.sum(sizes[:f]))
        o1 = o0 + sizes[f]
        assert np.allclose(fin[o0:o1], nat, rtol=1e-10, atol=1e-14), f


def test_batch_fit_entry_point_equals_composed_calls():
    """mtgp_batch_fit (one C call: theta0, steps, lr, graph flag -> final parameters and NLL) equals
    set_theta + adam + nll_grad + get_theta; theta0 = NULL continues from the current state."""
    from paper_2603_16014_gb300 import _lib
    from paper_2603_16014_gb300.mtgp import Batch, _ptr, _stream
    probs = _fits(21, 6, ms=(6, 8), precision="auto")
    ys = _ys(probs)
    rng = np.random.default_rng(2)
    thetas = [_theta(p, rng) for p in probs]
    y_all = torch.from_numpy(np.concatenate(ys))
    steps, lr = 7, 0.05
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b1 = Batch(probs, s=2, precision="auto")
        theta0 = torch.from_numpy(b1.pack(thetas)).cuda()
        b1.set_y(y_all)
        tr1 = torch.zeros(steps * len(probs), dtype=torch.float64, device="cuda")
        th1, nll1 = b1.fit(theta0, steps, lr, graph=True, trace=tr1)
        # the same through the raw C ABI with host-side ctypes arguments, and continued by 3 steps
        th1b = torch.empty_like(th1)
        _lib.check(_lib.lib().mtgp_batch_fit(b1._h, None, 3, lr, 0, _ptr(th1b), None, None, _stream()),
                   "mtgp_batch_fit")
        b2 = Batch(probs, s=2, precision="auto")
        b2.set_y(y_all)
        b2.set_theta(theta0)
        tr2 = torch.zeros(steps * len(probs), dtype=torch.float64, device="cuda")
        b2.adam(steps, lr, graph=False, trace=tr2)
        nll2, _ = b2.nll_grad()
        th2 = b2.get_theta()
        b2.adam(3, lr, graph=False)
        th2b = b2.get_theta()
        stream.synchronize()
    assert torch.equal(tr1, tr2)
    assert torch.equal(th1, th2) and torch.equal(nll1, nll2)
    assert torch.equal(th1b, th2b)
    assert np.all(nll1.cpu().numpy() < tr1.view(steps, -1)[0].cpu().numpy())
    with pytest.raises(_lib.MTGPError):
        b1.fit(theta0, 0, lr)
    b1.close()
    b2.close()

"""Learned proposal on the GPU: the BF16 MLP against the FP64 oracle MLP within a rounding-error bound
derived per element, Adam, training, and the feature / target / parameter maps against the
proposal oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense, mlp as omlp, proposal as oprop  # noqa: E402
from paper_2603_16014_gb300 import inputs  # noqa: E402

U_BF16 = 2.0 ** -8      # unit roundoff of round-to-nearest BF16 (8 significant bits)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    build.build()


def _bf(a):
    """Round to the nearest BF16 value (returned as float64)."""
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _net(rng, widths, wscale=0.1):
    """BF16-exact weights; hidden biases +-1 so that no hidden pre-activation is near 0."""
    Ws, bs = [], []
    for l in range(len(widths) - 1):
        Ws.append(_bf(rng.standard_normal((widths[l + 1], widths[l])) * wscale / np.sqrt(widths[l])))
        if l < len(widths) - 2:
            bs.append(np.where(rng.uniform(size=widths[l + 1]) < 0.5, -1.0, 1.0))
        else:
            bs.append(_bf(rng.standard_normal(widths[l + 1]) * 0.5))
    return Ws, bs


def _pack(Ws, bs):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in zip(Ws, bs)]).astype(np.float32)


def _fwd_bound(Ws, bs, acts):
    """Elementwise bound on |h_l(GPU) - h_l(FP64)|: FP32 accumulation (K 2^-22 of sum |w h|) and BF16
    storage of hidden activations (2^-8 |h|); the ReLU pattern is the same on both sides."""
    e = np.zeros_like(acts[0])
    out = [e]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        K = W.shape[1]
        ez = e @ np.abs(W).T + K * 2.0 ** -22 * (np.abs(acts[l]) @ np.abs(W).T + np.abs(b))
        e = ez + (U_BF16 * np.abs(acts[l + 1]) if l < len(Ws) - 1 else 2.0 ** -23 * np.abs(acts[l + 1]))
        out.append(e)
    return out


def test_mlp_forward_matches_oracle_within_bf16_bound():
    from paper_2603_16014_gb300.proposal import MLP
    rng = np.random.default_rng(0)
    widths = [40, 64, 96, 24]
    B = 70                                   # two row tiles, ragged; K and N padded
    Ws, bs = _net(rng, widths)
    x = _bf(rng.standard_normal((B, widths[0])))
    out, acts, pre = omlp.forward(x, Ws, bs)
    assert min(np.abs(z).min() for z in pre[:-1]) > 0.25
    net = MLP(widths, max_batch=128)
    net.set_params(_pack(Ws, bs))
    y = net.forward(torch.from_numpy(x.astype(np.float32))).cpu().numpy().astype(np.float64)
    bound = _fwd_bound(Ws, bs, acts)[-1]
    assert np.all(np.abs(y - out) <= 2 * bound + 1e-7), np.max(np.abs(y - out) / (bound + 1e-7))
    # the bound is not vacuous: it is small against the output scale
    assert bound.max() < 0.02 * np.abs(out).max()
    net.close()


def test_mlp_forward_bench_shape_within_bf16_bound():
    """The proposal network's own shape (258-256-256-256-37) at its largest batch (1024 rows)."""
    from paper_2603_16014_gb300.proposal import MLP, WIDTHS
    rng = np.random.default_rng(7)
    widths = list(WIDTHS)
    Ws, bs = _net(rng, widths)
    x = _bf(rng.standard_normal((1024, widths[0])))
    out, acts, pre = omlp.forward(x, Ws, bs)
    assert min(np.abs(z).min() for z in pre[:-1]) > 0.25
    net = MLP(widths, max_batch=1024)
    net.set_params(_pack(Ws, bs))
    y = net.forward(torch.from_numpy(x.astype(np.float32))).cpu().numpy().astype(np.float64)
    bound = _fwd_bound(Ws, bs, acts)[-1]
    pick = np.random.default_rng(8).integers(0, 1024, 64)
    assert np.all(np.abs(y - out) <= 2 * bound + 1e-7), np.max(np.abs(y - out) / (bound + 1e-7))
    assert np.all(np.abs(y[pick] - out[pick]) <= 2 * bound[pick] + 1e-7)
    net.close()


def test_mlp_gradients_match_oracle_within_bound():
    from paper_2603_16014_gb300.proposal import MLP
    rng = np.random.default_rng(1)
    widths = [40, 64, 24]
    B = 70
    Ws, bs = _net(rng, widths)
    x = _bf(rng.standard_normal((B, widths[0])))
    tgt = rng.standard_normal((B, widths[-1]))
    mask = (rng.uniform(size=tgt.shape) < 0.7).astype(np.float64)
    L, dWs, dbs = omlp.backward(x, Ws, bs, tgt, mask)
    out, acts, pre = omlp.forward(x, Ws, bs)
    assert np.abs(pre[0]).min() > 0.25
    net = MLP(widths, max_batch=128)
    net.set_params(_pack(Ws, bs))
    f32 = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32))  # noqa: E731
    loss, g = net.gradients(f32(x), f32(tgt), f32(mask))
    loss, g = float(loss.item()), g.cpu().numpy().astype(np.float64)
    gW, gb = net.split(g)
    # propagate the forward bound through dZ2 = 2 m (out - t) / cnt, the BF16 copies of dZ and H, and
    # the FP32 GEMM / column sums
    ef = _fwd_bound(Ws, bs, acts)
    cnt = mask.sum()
    dZ2 = 2 * mask * (out - tgt) / cnt
    e_dz2 = 2 * mask * ef[2] / cnt + 2.0 ** -23 * np.abs(dZ2)
    E2 = e_dz2 + U_BF16 * np.abs(dZ2)
    gam = B * 2.0 ** -22
    H1 = acts[1]
    bW2 = E2.T @ np.abs(H1) + np.abs(dZ2).T @ ef[1] + E2.T @ ef[1] + gam * np.abs(dZ2).T @ np.abs(H1)
    bb2 = e_dz2.sum(0) + gam * np.abs(dZ2).sum(0)
    dH1 = dZ2 @ Ws[1]
    e_dh1 = E2 @ np.abs(Ws[1]) + widths[2] * 2.0 ** -22 * np.abs(dZ2) @ np.abs(Ws[1])
    dZ1 = dH1 * (pre[0] > 0)
    E1 = e_dh1 * (pre[0] > 0) + U_BF16 * np.abs(dZ1)
    bW1 = E1.T @ np.abs(x) + gam * np.abs(dZ1).T @ np.abs(x)
    bb1 = (e_dh1 * (pre[0] > 0)).sum(0) + gam * np.abs(dZ1).sum(0)
    for got, ref, bd in ((gW[1], dWs[1], bW2), (gb[1], dbs[1], bb2), (gW[0], dWs[0], bW1), (gb[0], dbs[0], bb1)):
        assert np.all(np.abs(got - ref) <= 2 * bd + 1e-9), np.max(np.abs(got - ref) / (bd + 1e-9))
    lb = np.sum(mask * 2 * np.abs(out - tgt) * ef[2]) / cnt + 1e-6 * L
    assert abs(loss - L) <= 2 * lb
    net.close()


def test_mlp_adam_step_and_weight_copies():
    from paper_2603_16014_gb300.proposal import MLP
    rng = np.random.default_rng(2)
    widths = [258, 256, 256, 256, 37]
    net = MLP(widths, max_batch=256)
    p0 = net.init_params(3)
    x = torch.from_numpy(rng.standard_normal((200, 258)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((200, 37)).astype(np.float32)).cuda()
    mk = torch.from_numpy((rng.uniform(size=(200, 37)) < 0.8).astype(np.float32)).cuda()
    net.set_params(p0)
    _, g = net.gradients(x, t, mk)
    g = g.cpu().numpy().astype(np.float64)
    rows = torch.arange(200, dtype=torch.int32, device="cuda")
    lr = 1e-2
    net.train_step(x, t, mk, rows, lr)
    p1, _, _ = net.get_params()
    # first Adam step: m = 0.1 g, v = 0.001 g^2, bias corrections 0.1 and 0.001
    ref = p0 - lr * (0.1 * g / 0.1) / (np.sqrt(0.001 * g * g / 0.001) + 1e-8)
    assert np.allclose(p1, ref, rtol=2e-6, atol=2e-7)
    # the BF16 copies (and transposes) used by forward and backward were refreshed by the step
    y_a = net.forward(x).cpu().numpy()
    _, g_a = net.gradients(x, t, mk)
    net.set_params(p1)
    y_b = net.forward(x).cpu().numpy()
    _, g_b = net.gradients(x, t, mk)
    assert np.array_equal(y_a, y_b)
    assert torch.equal(g_a, g_b)
    # selected rows: same as passing those rows contiguously
    sel = torch.from_numpy(rng.permutation(200)[:150].astype(np.int32)).cuda()
    l_s, g_s = net.gradients(x, t, mk, rows=sel)
    l_c, g_c = net.gradients(x[sel.long()].contiguous(), t[sel.long()].contiguous(), mk[sel.long()].contiguous())
    assert torch.equal(g_s, g_c) and torch.equal(l_s, l_c)
    net.close()


def test_mlp_training_reduces_loss():
    from paper_2603_16014_gb300.proposal import MLP, train
    rng = np.random.default_rng(4)
    teacher_W, teacher_b = _net(rng, [258, 64, 37], wscale=1.0)
    x = rng.standard_normal((2048, 258))
    tgt, _, _ = omlp.forward(x, teacher_W, teacher_b)
    mask = (rng.uniform(size=tgt.shape) < 0.8).astype(np.float64)
    net = MLP(max_batch=256)
    net.set_params(net.init_params(5))
    f32 = lambda a: torch.from_numpy(np.asarray(a, dtype=np.float32)).cuda()  # noqa: E731
    losses = train(net, f32(x), f32(tgt), f32(mask), steps=400, batch=256, lr=1e-3, seed=6).cpu().numpy()
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean()
    net.close()


def _fits(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = "lattice" if i % 2 == 0 else "dnet"
        T = int(rng.choice([2, 3, 5, 8]))
        d = int(rng.choice([2, 7, 12]))
        m = int(rng.choice([4, 5, 8, 10]))
        out.append(inputs.make_problem(kind, d, (m,) * T, seed=100 * seed + i, s=2, eta=(0.3, 1.5), v=0.1,
                                       sigma2=1e-4, recipe="walshcos32" if kind == "dnet" else "cos16",
                                       mmax=max(m, 12)))
    return out


def _ys(probs):
    return [inputs.synth_y(p, dense.all_points(p.kind, p.gen, p.shift, p.m)) for p in probs]


def test_features_targets_and_proposal_map_match_oracle():
    from paper_2603_16014_gb300.mtgp import Batch
    probs = _fits(8, 12)
    ys = _ys(probs)
    b = Batch(probs, s=2, precision="fp64")
    b.set_y(torch.from_numpy(np.concatenate(ys)))
    feat = b.features().cpu().numpy().astype(np.float64)
    for f, (p, y) in enumerate(zip(probs, ys)):
        n = 1 << p.m[0]
        ref = oprop.features(p.kind, [y[t * n:(t + 1) * n] for t in range(len(p.m))], p.m[0], p.d)
        assert np.all(np.abs(feat[f] - ref) <= 4 * 2.0 ** -24 * np.abs(ref) + 1e-9), f
    rng = np.random.default_rng(9)
    thetas = []
    for p in probs:
        T = len(p.m)
        thetas.append((np.exp(rng.uniform(-2, 0.7, p.d)), rng.standard_normal((T, 2)), np.exp(rng.uniform(-4, 0, T)),
                       float(np.exp(rng.uniform(-18, -9)))))
    thetas[3] = (thetas[3][0], thetas[3][1], np.r_[thetas[3][2][:-1], np.nan], thetas[3][3])  # a diverged fit
    b.set_theta(torch.from_numpy(b.pack(thetas)))
    tg, mk = b.targets()
    tg, mk = tg.cpu().numpy().astype(np.float64), mk.cpu().numpy()
    for f, th in enumerate(thetas):
        rt, rm = oprop.targets(*th)
        assert np.array_equal(mk[f], rm.astype(np.float32)), f
        assert (f == 3) == (rm.sum() == 0)
        assert np.all(np.abs(tg[f] - rt) <= 2.0 ** -23 * np.abs(rt) + 1e-14), f
    pred = rng.standard_normal((len(probs), 37)).astype(np.float32) * 2
    pred[0, 0] = -100.0                       # clamped at the lower end
    b.set_theta_proposal(torch.from_numpy(pred))
    got = b.unpack(b.get_theta().cpu().numpy())
    for f, p in enumerate(probs):
        e, W, v, s2 = oprop.theta_from_prediction(pred[f].astype(np.float64), p.d, len(p.m))
        ge, gW, gv, gs = got[f]
        assert np.allclose(ge, e, rtol=1e-15) and np.array_equal(gW, W)
        assert np.allclose(gv, v, rtol=1e-15) and gs == pytest.approx(s2, rel=1e-15)
    b.close()


def test_proposal_pipeline_on_training_fits():
    """Labels from the batched optimiser, a network fitted to them, proposals closer than the default."""
    from paper_2603_16014_gb300.mtgp import Batch
    from paper_2603_16014_gb300.proposal import MLP, propose, train
    probs = _fits(10, 48)
    ys = _ys(probs)
    b = Batch(probs, s=2, precision="fp64")
    b.set_y(torch.from_numpy(np.concatenate(ys)))
    theta0 = b.pack([(np.ones(p.d), 0.1 * np.ones((len(p.m), 2)), np.ones(len(p.m)), 1e-4) for p in probs])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.set_theta(torch.from_numpy(theta0))
        nll0, _ = b.nll_grad()
        b.adam(200, 0.05, graph=True)
        nll_lab, _ = b.nll_grad()
        tg, mk = b.targets()
        feats = b.features()
        net = MLP(max_batch=64)
        net.set_params(net.init_params(0))
        train(net, feats, tg, mk, steps=600, batch=48, lr=2e-3, seed=1)
        propose(b, net)
        nll_p, _ = b.nll_grad()
        stream.synchronize()
    nll0, nll_lab, nll_p = (t.cpu().numpy() for t in (nll0, nll_lab, nll_p))
    assert np.all(np.isfinite(nll_p))
    closer = np.abs(nll_p - nll_lab) < np.abs(nll0 - nll_lab)
    assert closer.mean() >= 0.75, (closer.mean(), nll0[:4], nll_p[:4], nll_lab[:4])
    net.close()
    b.close()


def test_propose_entry_point_equals_composed_calls():
    """mtgp_propose (features -> MLP forward -> parameter map in one C call) equals the three calls
    made one by one, for a batch larger than the network's max_batch (chunked forward passes)."""
    from paper_2603_16014_gb300 import _lib
    from paper_2603_16014_gb300.mtgp import Batch
    from paper_2603_16014_gb300.proposal import MLP, propose
    probs = _fits(12, 20)
    ys = _ys(probs)
    b = Batch(probs, s=2, precision="auto")
    b.set_y(torch.from_numpy(np.concatenate(ys)))
    net = MLP(max_batch=8)
    net.set_params(net.init_params(3))
    net.fit_scaling(b.features())
    pred, _ = propose(b, net)
    th_prop = b.get_theta()
    ref_pred = net.forward(b.features())
    b.set_theta_proposal(ref_pred)
    th_ref = b.get_theta()
    torch.cuda.synchronize()
    assert torch.equal(pred, ref_pred)
    assert torch.equal(th_prop, th_ref)
    # a network of the wrong shape is refused
    bad = MLP(widths=(258, 64, 36), max_batch=8)
    with pytest.raises(_lib.MTGPError):
        propose(b, bad)
    # and so is an unknown judge mode
    with pytest.raises(_lib.MTGPError):
        propose(b, net, judge=3)
    bad.close()
    net.close()
    b.close()


def test_judged_proposal_on_heldout_fits():
    """Held-out fits (seeds not used in training): the judged proposal (mtgp_propose with the exact-NLL
    judge) starts no fit worse than the plain fixed start and most strictly better, and reaches the plain
    optimiser's best NLL in fewer steps, its own cost (five batched evaluations and the network)
    included, on most fits; the same for the two-candidate blend judge (judge = 2)."""
    from paper_2603_16014_gb300.mtgp import Batch
    from paper_2603_16014_gb300.proposal import MLP, propose, train
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    lr, S = 0.05, 400
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        train_fits = _fits(20, 128)
        bt = Batch(train_fits, s=2, precision="auto")
        bt.set_y(torch.from_numpy(np.concatenate(_ys(train_fits))))
        th0 = torch.from_numpy(bt.pack([bench.default_theta(p) for p in train_fits])).cuda()
        bt.fit(th0, 400, lr, graph=True, final_nll=False)
        tg, mk = bt.targets()
        feats = bt.features()
        net = MLP(max_batch=128)
        net.set_params(net.init_params(0))
        train(net, feats, tg, mk, steps=800, batch=64, lr=2e-3, seed=1, lr_final=1e-4)
        held = _fits(21, 32)
        b = Batch(held, s=2, precision="auto")
        b.set_y(torch.from_numpy(np.concatenate(_ys(held))))
        theta0 = torch.from_numpy(b.pack([bench.default_theta(p) for p in held])).cuda()
        traces = {}
        for name in ("plain", "proposal", "proposal_blend"):
            b.set_theta(theta0)
            if name == "proposal":
                _, chosen = propose(b, net, judge=True)
            elif name == "proposal_blend":
                _, chosen2 = propose(b, net, judge=2)
            tr = torch.zeros(S * len(held), dtype=torch.float64, device="cuda")
            b.fit(None, S, lr, graph=False, trace=tr, final_nll=False)
            traces[name] = tr.view(S, -1).cpu().numpy()
        stream.synchronize()
    plain, prop = traces["plain"], traces["proposal"]
    assert np.all(prop[0] <= plain[0]), (prop[0], plain[0])
    better = prop[0] < plain[0]
    assert better.mean() >= 0.75, (better.mean(), chosen.cpu().numpy())
    target = np.nanmin(plain, axis=0)
    k_plain = bench.steps_to_target(plain, target) + 1
    k_prop = bench.steps_to_target(prop, target)
    faster = (k_prop >= 0) & (k_prop + 1 + 6 < k_plain)
    assert faster.mean() >= 0.75, (faster.mean(), k_plain, k_prop)
    # the blend judge: candidates (p + 3 c) / 4 and c only
    blend = traces["proposal_blend"]
    c2 = chosen2.cpu().numpy()
    assert np.all((c2 == 3) | (c2 == 4)), c2
    assert np.all(blend[0] <= plain[0]), (blend[0], plain[0])
    k_bl = bench.steps_to_target(blend, target)
    faster_bl = (k_bl >= 0) & (k_bl + 1 + 3 < k_plain)
    assert faster_bl.mean() >= 0.75, (faster_bl.mean(), k_plain, k_bl)
    net.close()
    bt.close()
    b.close()


def test_training_early_stopping_keeps_lowest_held_out_loss():
    """proposal.train with a held-out share: the held-out rows are not trained on, and the network ends
    with the parameters whose held-out loss is the lowest of the checkpoints."""
    from paper_2603_16014_gb300.mtgp import Batch
    from paper_2603_16014_gb300.proposal import MLP, train
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    fits = _fits(23, 48)
    b = Batch(fits, s=2, precision="auto")
    b.set_y(torch.from_numpy(np.concatenate(_ys(fits))))
    th0 = torch.from_numpy(b.pack([bench.default_theta(p) for p in fits])).cuda()
    b.fit(th0, 100, 0.05, graph=False, final_nll=False)
    tg, mk = b.targets()
    feats = b.features()
    net = MLP(max_batch=64)
    net.set_params(net.init_params(0))
    train(net, feats, tg, mk, steps=600, batch=16, lr=3e-3, seed=2, lr_final=1e-3, val_fraction=0.25, eval_every=50)
    val = net.val_rows.cpu().numpy()
    assert len(val) == 12 and len(np.unique(val)) == 12
    hist = net.val_history
    assert [s for s, _ in hist] == list(range(50, 601, 50))
    vl, _ = net.gradients(feats, tg, mk, rows=net.val_rows)
    assert float(vl.item()) == min(v for _, v in hist), (float(vl.item()), hist)
    net.close()
    b.close()

"""Pins for the proposal oracle (features, bins, canonical W, targets) against brute force, Parseval's
identity, a single Walsh mode and orthogonal invariance."""
import numpy as np
import pytest

from oracle import proposal, spectral


def _bin_bruteforce(f, m):
    bits = bin(f)[2:]
    L = len(bits) - 1
    frac3 = int((bits[1:4] + "000")[:3], 2)
    return (4 * (8 * L + frac3)) // m


@pytest.mark.parametrize("m", [4, 5, 8, 11, 16])
def test_bins_bruteforce_cover_and_log_spacing(m):
    n = 1 << m
    f = np.arange(1, n)
    b = proposal.bin_index(f, m)
    assert np.array_equal(b, [_bin_bruteforce(int(x), m) for x in f])
    assert b[0] == 0 and b.min() >= 0 and b.max() <= 31
    assert np.all(np.diff(b) >= 0)              # contiguous, log-ordered bins
    # floor of a piecewise-linear log2 that under-estimates log2 by less than 0.22 octave
    gap = 32 * np.log2(f) / m - b
    assert gap.min() >= -1e-12 and gap.max() < 1 + 32 * 0.22 / m
    for k in range(m):                          # octave boundaries
        assert b[(1 << k) - 1] == (32 * k) // m


@pytest.mark.parametrize("kind,m", [("lattice", 8), ("dnet", 8), ("lattice", 10), ("dnet", 10)])
def test_features_parseval(kind, m):
    rng = np.random.default_rng(m)
    ys = [rng.standard_normal(1 << m) * (t + 1) + 3.0 for t in range(3)]
    feat, cnt = proposal.features(kind, ys, m, d=5, with_counts=True)
    for t, y in enumerate(ys):
        energy = np.sum(cnt * np.exp(feat[t * 32:(t + 1) * 32]) * (cnt > 0))
        assert abs(energy - np.sum((y - y.mean()) ** 2)) <= 1e-9 * energy
    assert np.all(feat[3 * 32:8 * 32] == 0)
    assert feat[256] == m and feat[257] == 5


def test_features_single_walsh_mode():
    m, f0 = 9, 77
    n = 1 << m
    i = np.arange(n)
    y = np.array([(-1) ** bin(int(k) & f0).count("1") for k in i], dtype=float)
    feat, cnt = proposal.features("dnet", [y], m, d=2, with_counts=True)
    b0 = proposal.bin_index(np.array([f0]), m)[0]
    # |V^dagger y|^2 = n at f0 alone
    assert abs(feat[b0] - np.log(n / cnt[b0] + 1e-30)) < 1e-12
    others = [k for k in range(32) if k != b0 and cnt[k] > 0]
    assert all(feat[k] == pytest.approx(np.log(1e-30)) for k in others)
    # the oracle transform really puts the mode at index f0
    assert np.argmax(np.abs(spectral.vdag("dnet", y, m))) == f0


def test_canonical_w_invariance():
    rng = np.random.default_rng(3)
    for T in (2, 3, 8):
        W = rng.standard_normal((T, 2))
        C = proposal.canonical_w(W)
        assert C[0, 1] == 0.0 and C[0, 0] >= 0 and C[1, 1] >= 0
        assert np.allclose(C @ C.T, W @ W.T, rtol=0, atol=1e-12)
        for refl in (False, True):
            th = rng.uniform(0, 2 * np.pi)
            Q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
            if refl:
                Q = Q @ np.diag([1.0, -1.0])
            assert np.allclose(proposal.canonical_w(W @ Q), C, rtol=0, atol=1e-12)


def test_targets_round_trip_and_mask():
    rng = np.random.default_rng(4)
    d, T = 5, 3
    eta = np.exp(rng.uniform(-2, 0.7, d))
    W = rng.standard_normal((T, 2))
    v = np.exp(rng.uniform(-4, 0, T))
    s2 = 1e-6
    t, mk = proposal.targets(eta, W, v, s2)
    assert t.shape == (37,) and mk.sum() == d + 2 * T + T + 1
    assert np.all(mk[d:12] == 0) and np.all(mk[12 + 2 * T:28] == 0) and np.all(mk[28 + T:36] == 0)
    e2, W2, v2, s22 = proposal.theta_from_prediction(t, d, T)
    assert np.allclose(e2, eta, rtol=1e-14) and np.allclose(v2, v, rtol=1e-14)
    assert np.allclose(W2, proposal.canonical_w(W), atol=1e-15) and s22 == pytest.approx(s2, rel=1e-14)
    # a diverged fit (non-finite parameter) is left out entirely
    t_bad, m_bad = proposal.targets(np.r_[eta[:-1], np.nan], W, v, s2)
    assert np.all(t_bad == 0) and np.all(m_bad == 0)
    t_bad, m_bad = proposal.targets(eta, W, np.r_[v[:-1], 0.0], s2)      # log 0
    assert np.all(t_bad == 0) and np.all(m_bad == 0)

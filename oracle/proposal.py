"""Inputs and targets of the learned hyper-parameter proposal, in plain numpy (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper fits each model by first-order optimisation of the MLE loss (Sec. 4.1) from a fixed start;
a learned proposal replaces that start by a prediction from a fixed-size summary of the data.  The
paper gives no such summary, so this module states the one used here (its definitions are readings,
not the paper's):

  * features (258 values): for each of up to 8 tasks (caller order; absent tasks are zero) and each of
    32 frequency bins, log(mean |yhat_t(f)|^2 + 1e-30) over the frequencies f in 1..n-1 of the bin,
    where yhat_t = V^dagger y_t (the transform of Sec. 3.3 with its 1/sqrt(n) factor); then log2 n and
    d.  An empty bin repeats the previous bin's value (bin 0 always holds f = 1).
  * bin(f) = floor(4 q(f) / m) with q(f) = 8 floor(log2 f) + (the three bits of f after its leading
    one, zero-filled for f < 8): a piecewise-linear log2 in eighth octaves, so bins are log-spaced
    and the assignment is integer arithmetic only.
  * targets (37 values): 12 x log eta_j, 8 x 2 entries of W, 8 x log v_t, log sigma2, with a mask that
    is 0 for j >= d and for tasks t >= T.  R = W W^T + diag(v) does not change when W is multiplied on
    the right by an orthogonal 2 x 2 matrix, so W is first brought to the canonical form with
    W[0, 1] = 0, W[0, 0] >= 0, W[1, 1] >= 0 (a rotation, then the sign of column 1).  A fit whose
    parameters give a non-finite entry (a diverged optimiser run) is left out: target 0, mask 0.
"""
from __future__ import annotations

import numpy as np

NT, NB, DMAXP = 8, 32, 12
NFEAT = NT * NB + 2
NOUT = DMAXP + 2 * NT + NT + 1


def bin_index(f: np.ndarray, m: int) -> np.ndarray:
    """Frequency bin of each f in 1..2^m - 1 (integer arithmetic)."""
    f = np.asarray(f, dtype=np.int64)
    L = np.floor(np.log2(f)).astype(np.int64)
    # exact floor(log2) for integers (guard the float rounding)
    L = np.where((1 << (L + 1)) <= f, L + 1, L)
    L = np.where((1 << L) > f, L - 1, L)
    frac3 = np.where(L >= 3, (f >> np.maximum(L - 3, 0)) & 7, (f << np.maximum(3 - L, 0)) & 7)
    q = 8 * L + frac3
    return (4 * q) // m


def features(kind: str, y_tasks, m: int, d: int, with_counts: bool = False):
    """258 features of a fit with equal task sizes 2^m from its observations (radical-inverse order)."""
    from .spectral import vdag
    n = 1 << m
    feat = np.zeros(NFEAT)
    f = np.arange(1, n)
    b = bin_index(f, m)
    cnt = np.bincount(b, minlength=NB).astype(np.float64)
    for t, y in enumerate(y_tasks):
        yh = vdag(kind, np.asarray(y, dtype=np.float64), m)
        e = np.abs(yh[1:]) ** 2
        s = np.bincount(b, weights=e, minlength=NB)
        prev = np.log(s[0] / max(cnt[0], 1.0) + 1e-30)
        for k in range(NB):
            if cnt[k] > 0:
                prev = np.log(s[k] / cnt[k] + 1e-30)
            feat[t * NB + k] = prev
    feat[NT * NB] = m
    feat[NT * NB + 1] = d
    return (feat, cnt) if with_counts else feat


def canonical_w(W: np.ndarray) -> np.ndarray:
    """W Q for the orthogonal Q that makes W[0, 1] = 0, W[0, 0] >= 0, W[1, 1] >= 0 (W is T x 2)."""
    W = np.array(W, dtype=np.float64)
    a, b = W[0, 0], W[0, 1]
    r = np.sqrt(a * a + b * b)
    if r > 0:
        c, s = a / r, b / r
        W = W @ np.array([[c, -s], [s, c]])
        W[0, 1] = 0.0
    if W.shape[0] > 1 and W[1, 1] < 0:
        W[:, 1] = -W[:, 1]
    return W


def targets(eta, W, v, sigma2):
    """(target[37], mask[37]) of one fit's hyper-parameters (caller task order)."""
    eta = np.asarray(eta, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    d, T = len(eta), len(v)
    t = np.zeros(NOUT)
    mk = np.zeros(NOUT)
    with np.errstate(divide="ignore", invalid="ignore"):
        t[:d] = np.log(eta)
        mk[:d] = 1
        Wc = canonical_w(W)
        t[DMAXP:DMAXP + 2 * T] = Wc.ravel()
        mk[DMAXP:DMAXP + 2 * T] = 1
        t[DMAXP + 2 * NT:DMAXP + 2 * NT + T] = np.log(v)
        mk[DMAXP + 2 * NT:DMAXP + 2 * NT + T] = 1
        t[-1] = np.log(sigma2)
        mk[-1] = 1
    if not np.all(np.isfinite(t)):
        return np.zeros(NOUT), np.zeros(NOUT)
    return t, mk


LOG_LO, LOG_HI = -40.0, 20.0


def theta_from_prediction(p, d: int, T: int):
    """(eta, W, v, sigma2) from a 37-vector: exp of the clamped log entries, W as predicted."""
    p = np.asarray(p, dtype=np.float64)
    ex = lambda z: np.exp(np.clip(z, LOG_LO, LOG_HI))  # noqa: E731
    eta = ex(p[:d])
    W = p[DMAXP:DMAXP + 2 * T].reshape(T, 2).copy()
    v = ex(p[DMAXP + 2 * NT:DMAXP + 2 * NT + T])
    s2 = float(ex(p[-1]))
    return eta, W, v, s2

"""Seeded synthetic inputs for the fast multitask GP (MTGP) hot path.

This module draws everything a fit consumes from a seed: generating vectors or
generating matrices, per-task shifts, hyper-parameters, query points and the
coefficients of synthetic response functions.  It holds none of the method's
arithmetic: design points are not generated here.  The response ``y`` is a test
function evaluated at design points that the caller supplies as 32-bit
fixed-point coordinates (value = X / 2^32), so the CUDA path and the CPU oracle
both receive bit-identical inputs from whichever side produced the points.

Workloads (sizes follow the benchmark configurations of the fast-MTGP paper's
setting, Section 4; the paper's own test functions and QGP data are not used):

* ``lat_d2_T2_n2^10``     rank-1 lattice, d=2,  T=2, n=2^10 each (N=2048), SI order-2 kernel.
* ``dnet_d8_T4_n2^16``    digital net,    d=8,  T=4, n=2^16 each (N=262144), DSI order-2 kernel.
* ``lat_d16_T5_nested``   lattice,        d=16, T=5, n=2^20,2^18,2^16,2^14,2^12 (N=1396736).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

LATTICE = "lattice"
DNET = "dnet"

#: kernel identifiers: shift-invariant Bernoulli kernel of smoothness alpha=2
#: (Eq. SI_kernel_1d_ex) and digitally-shift-invariant order-2 kernel (Eq. DSI_kernel_1d_ex, b=(0,1,0,0)).
KERNEL_FOR_KIND = {LATTICE: "si2", DNET: "dsi2"}


@dataclass
class Problem:
    """One multitask GP fit: design, hyper-parameters and synthetic-response recipe."""

    kind: str                 # "lattice" or "dnet"
    d: int
    m: tuple                  # log2 n_t per task, user order
    gen: np.ndarray           # lattice: (d,) odd uint32; dnet: (d, mmax) uint32 generating-matrix columns
    shift: np.ndarray         # (T, d) uint32 (lattice: shift mod 1; dnet: digital shift)
    eta: np.ndarray           # (d,) product weights eta_j > 0
    W: np.ndarray             # (T, s) factor of the task covariance R = W W^T + diag(v)
    v: np.ndarray             # (T,) > 0
    sigma2: float             # noise variance
    recipe: str = "cos16"     # synthetic response recipe ("cos16" or "walshcos32")
    seed: int = 0
    name: str = ""
    fp32_transform: bool = False
    extras: dict = field(default_factory=dict)

    @property
    def T(self) -> int:
        return len(self.m)

    @property
    def n(self) -> list:
        return [1 << mt for mt in self.m]

    @property
    def N(self) -> int:
        return sum(self.n)

    @property
    def kernel(self) -> str:
        return KERNEL_FOR_KIND[self.kind]

    def theta(self):
        return self.eta.copy(), self.W.copy(), self.v.copy(), float(self.sigma2)


def _unit_upper_gf2_columns(rng: np.random.Generator, mmax: int) -> np.ndarray:
    """Columns of a random unit upper-triangular mmax x mmax matrix over GF(2).

    Row r is the binary digit of weight 2^-(r+1) (bit 31-r of the fixed-point word),
    column p multiplies bit p of the point index.  C[r][p] = 0 for r > p, C[p][p] = 1.
    """
    cols = np.zeros(mmax, dtype=np.uint64)
    for p in range(mmax):
        word = 1 << (31 - p)
        for r in range(p):
            if rng.integers(0, 2):
                word |= 1 << (31 - r)
        cols[p] = word
    return cols.astype(np.uint32)


def make_problem(kind: str, d: int, m, *, seed: int = 0, s: int | None = None,
                 eta=0.5, v=0.1, sigma2=1e-6, recipe: str = "cos16", mmax: int | None = None,
                 W=None, fp32_transform: bool = False, name: str = "") -> Problem:
    """Draw a problem from ``seed``.

    Lattice generating vector: odd integers uniform in [1, n_max) (n_max = max n_t).
    Digital net: independent unit upper-triangular GF(2) matrices, one per coordinate.
    Shifts: uniform 32-bit words per task and coordinate.  W ~ N(0,1) of shape T x s.
    ``eta`` is a scalar (all coordinates), an array, or a (lo, hi) tuple for U[lo, hi).
    """
    m = tuple(int(x) for x in m)
    T = len(m)
    rng = np.random.default_rng(seed)
    mx = max(m)
    if kind == LATTICE:
        nmax = 1 << mx
        if nmax <= 2:
            gen = np.ones(d, dtype=np.uint32)
        else:
            gen = (2 * rng.integers(0, nmax // 2, size=d) + 1).astype(np.uint32)
    elif kind == DNET:
        mm = mmax if mmax is not None else max(mx, 1)
        gen = np.stack([_unit_upper_gf2_columns(rng, mm) for _ in range(d)])
    else:
        raise ValueError(kind)
    shift = rng.integers(0, 1 << 32, size=(T, d), dtype=np.uint64).astype(np.uint32)
    if isinstance(eta, tuple):
        eta_arr = rng.uniform(eta[0], eta[1], size=d)
    else:
        eta_arr = np.broadcast_to(np.asarray(eta, dtype=np.float64), (d,)).copy()
    s = T if s is None else s
    W_arr = rng.standard_normal((T, s)) if W is None else np.asarray(W, dtype=np.float64)
    v_arr = np.broadcast_to(np.asarray(v, dtype=np.float64), (T,)).copy()
    return Problem(kind=kind, d=d, m=m, gen=gen, shift=shift, eta=eta_arr, W=W_arr, v=v_arr,
                   sigma2=float(sigma2), recipe=recipe, seed=seed, name=name,
                   fp32_transform=fp32_transform)


# --------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------

def lattice_small(seed: int = 0, m: int = 10) -> Problem:
    """Rank-1 lattice, d=2, T=2, n=2^m (2^10 gives N=2048), eta=0.5, W 2x1, v=0.1, sigma2=1e-6."""
    return make_problem(LATTICE, 2, (m, m), seed=seed, s=1, eta=0.5, v=0.1, sigma2=1e-6,
                        recipe="cos16", name=f"lat_d2_T2_n2^{m}")


def dnet_equal(seed: int = 0, m: int = 16, fp32_transform: bool = True) -> Problem:
    """Digital net, d=8, T=4, n=2^m each (2^16 gives N=262144), eta=0.5, W 4x2, v=0.05, sigma2=1e-8."""
    return make_problem(DNET, 8, (m,) * 4, seed=seed, s=2, eta=0.5, v=0.05, sigma2=1e-8,
                        recipe="walshcos32", mmax=max(m, 16), fp32_transform=fp32_transform,
                        name=f"dnet_d8_T4_n2^{m}")


def lattice_nested(seed: int = 0, m=(20, 18, 16, 14, 12)) -> Problem:
    """Lattice, d=16, T=5, nested sizes 2^20..2^12, eta~U[0.1,2), W 5x2, v=0.1, sigma2=1e-7."""
    return make_problem(LATTICE, 16, m, seed=seed, s=2, eta=(0.1, 2.0), v=0.1, sigma2=1e-7,
                        recipe="cos16", name="lat_d16_T5_nested" + "_".join(str(x) for x in m))


# --------------------------------------------------------------------------------------
# synthetic responses
# --------------------------------------------------------------------------------------

def _sparse_freq(rng, d, lo, hi, allow_neg):
    """An integer frequency vector with 1..min(3,d) active coordinates."""
    h = np.zeros(d, dtype=np.int64)
    k = int(rng.integers(1, min(3, d) + 1))
    idx = rng.choice(d, size=k, replace=False)
    for j in idx:
        val = int(rng.integers(lo, hi + 1))
        if allow_neg and rng.integers(0, 2):
            val = -val
        h[j] = val
    return h


def _task_correlation(W: np.ndarray) -> np.ndarray:
    C = W @ W.T + 0.09 * np.eye(W.shape[0])
    dd = np.sqrt(np.diag(C))
    return C / np.outer(dd, dd)


def _cos_mode(X: np.ndarray, h: np.ndarray, phi: float) -> np.ndarray:
    # phase = h . x mod 1 computed exactly on the 32-bit fixed-point words
    ph = np.zeros(X.shape[0], dtype=np.int64)
    for j in range(X.shape[1]):
        if h[j]:
            ph = (ph + int(h[j]) * X[:, j].astype(np.int64)) & 0xFFFFFFFF
    return np.cos(2.0 * np.pi * (ph.astype(np.float64) / 2.0 ** 32) + phi)


def _walsh_mode(X: np.ndarray, h: np.ndarray) -> np.ndarray:
    # wal_h(x) = (-1)^{sum_j sum_p h_{j,p} x_{j,p+1}}; digit p+1 of x_j is bit 31-p of X_j
    par = np.zeros(X.shape[0], dtype=np.int64)
    for j in range(X.shape[1]):
        hj = int(h[j])
        p = 0
        while hj:
            if hj & 1:
                par ^= (X[:, j].astype(np.int64) >> (31 - p)) & 1
            hj >>= 1
            p += 1
    return 1.0 - 2.0 * par.astype(np.float64)


def synth_y(problem: Problem, X_tasks, noise: bool = True) -> np.ndarray:
    """Synthetic responses at the given design points, concatenated over tasks (user order).

    ``X_tasks[t]`` is an (n_t, d) uint32 array of task t's design points in the order
    the response is wanted (radical-inverse order for fits).

    Recipe "cos16": y_t(x) = sum_{k=1..16} a_{tk} cos(2 pi h_k.x + phi_k), a_{.k} ~ N(0, C)/k with
    C the correlation matrix of W W^T + 0.09 I (tasks correlated, marginal N(0, 1/k^2)),
    h_k integer with 1-3 active coordinates in {+-1..+-4}, phi_k ~ U[0, 2 pi).
    Recipe "walshcos32": 32 modes, each with probability 1/2 a Walsh function wal_h
    (h_j in 1..15 on 1-3 coordinates) or a cosine as above, amplitudes (W u_j + 0.3 eps_j)/j.
    Noise: N(0, sigma2) per observation when ``noise``.
    """
    rng = np.random.default_rng([problem.seed, 7919])
    T, d = problem.T, problem.d
    ys = [np.zeros(problem.n[t]) for t in range(T)]
    if problem.recipe == "cos16":
        L = np.linalg.cholesky(_task_correlation(problem.W))
        for k in range(1, 17):
            h = _sparse_freq(rng, d, 1, 4, True)
            phi = rng.uniform(0, 2 * np.pi)
            a = (L @ rng.standard_normal(T)) / k
            for t in range(T):
                ys[t] += a[t] * _cos_mode(np.asarray(X_tasks[t]), h, phi)
    elif problem.recipe == "walshcos32":
        W = problem.W
        for k in range(1, 33):
            walsh = bool(rng.integers(0, 2))
            if walsh:
                h = _sparse_freq(rng, d, 1, 15, False)
                phi = 0.0
            else:
                h = _sparse_freq(rng, d, 1, 4, True)
                phi = rng.uniform(0, 2 * np.pi)
            a = (W @ rng.standard_normal(W.shape[1]) + 0.3 * rng.standard_normal(T)) / k
            for t in range(T):
                X = np.asarray(X_tasks[t])
                mode = _walsh_mode(X, h) if walsh else _cos_mode(X, h, phi)
                ys[t] += a[t] * mode
    else:
        raise ValueError(problem.recipe)
    if noise and problem.sigma2 > 0:
        for t in range(T):
            ys[t] += np.sqrt(problem.sigma2) * rng.standard_normal(problem.n[t])
    return np.concatenate(ys)


def query_points(nq: int, d: int, seed: int = 1, tasks: int = 1):
    """Seeded uniform query points as fixed-point words and the matching doubles, plus task ids."""
    rng = np.random.default_rng([seed, 104729])
    Xq = rng.integers(0, 1 << 32, size=(nq, d), dtype=np.uint64).astype(np.uint32)
    task = rng.integers(0, tasks, size=nq).astype(np.int32)
    return Xq, Xq.astype(np.float64) / 2.0 ** 32, task


def perturb_theta(problem: Problem, seed: int, scale: float = 0.3) -> Problem:
    """A copy of ``problem`` with log-normally perturbed eta, v, sigma2 and perturbed W."""
    rng = np.random.default_rng([seed, 31337])
    return replace(problem,
                   eta=problem.eta * np.exp(scale * rng.standard_normal(problem.d)),
                   W=problem.W + scale * rng.standard_normal(problem.W.shape),
                   v=problem.v * np.exp(scale * rng.standard_normal(problem.T)),
                   sigma2=problem.sigma2 * float(np.exp(scale * rng.standard_normal())))

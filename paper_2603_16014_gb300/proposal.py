"""Learned starting point for the fits' optimiser.

An MLP with BF16 weights and FP32 accumulation (C ABI mtgp_mlp_*) maps each fit's spectral summary
(mtgp_batch_features) to its hyper-parameters [log eta, canonical W, log v, log sigma2]
(mtgp_batch_targets / mtgp_batch_set_theta_proposal).  Training data are fits whose parameters were
found by the batched exact optimiser (Batch.adam).  This module passes pointers and sizes; the
forward pass, gradients, Adam and the feature / target maps all run in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from ._lib import check, lib
from .mtgp import _dev, _ptr, _stream

WIDTHS = (258, 256, 256, 256, 37)


class MLP:
    """Fully connected ReLU network, last layer linear.  ``widths`` = (in, hidden..., out)."""

    def __init__(self, widths=WIDTHS, max_batch: int = 1024):
        self.widths = [int(w) for w in widths]
        self.L = len(self.widths) - 1
        self.max_batch = int(max_batch)
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * len(self.widths))(*self.widths)
        check(lib().mtgp_mlp_create(ctypes.byref(h), self.L, arr, self.max_batch), "mtgp_mlp_create")
        self._h = h
        self.nparams = sum(self.widths[l + 1] * self.widths[l] + self.widths[l + 1] for l in range(self.L))

    def init_params(self, seed: int) -> np.ndarray:
        """He-normal weights (ReLU layers), a 0.1-scaled last layer, zero biases; packed."""
        rng = np.random.default_rng(seed)
        out = []
        for l in range(self.L):
            fi, fo = self.widths[l], self.widths[l + 1]
            sc = np.sqrt(2.0 / fi) if l < self.L - 1 else 0.1 / np.sqrt(fi)
            out += [rng.standard_normal((fo, fi)).ravel() * sc, np.zeros(fo)]
        return np.concatenate(out).astype(np.float32)

    def split(self, packed):
        """Packed parameters -> ([W_l], [b_l]) as numpy arrays."""
        packed = np.asarray(packed)
        Ws, bs, o = [], [], 0
        for l in range(self.L):
            fi, fo = self.widths[l], self.widths[l + 1]
            Ws.append(packed[o:o + fo * fi].reshape(fo, fi))
            o += fo * fi
            bs.append(packed[o:o + fo])
            o += fo
        return Ws, bs

    def set_params(self, params, mu=None, sd=None):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        assert p.size == self.nparams
        mu_a = None if mu is None else np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
        sd_a = None if sd is None else np.ascontiguousarray(np.asarray(sd, dtype=np.float32))
        c = lambda a: None if a is None else a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        check(lib().mtgp_mlp_set_params(self._h, c(p), c(mu_a), c(sd_a)), "mtgp_mlp_set_params")

    def get_params(self):
        p = np.empty(self.nparams, dtype=np.float32)
        mu = np.empty(self.widths[0], dtype=np.float32)
        sd = np.empty(self.widths[0], dtype=np.float32)
        check(lib().mtgp_mlp_get_params(self._h, p.ctypes.data_as(ctypes.c_void_p), mu.ctypes.data_as(ctypes.c_void_p),
                                        sd.ctypes.data_as(ctypes.c_void_p)), "mtgp_mlp_get_params")
        return p, mu, sd

    def fit_scaling(self, x, stream=None):
        x = _dev(x, torch.float32)
        check(lib().mtgp_mlp_fit_scaling(self._h, x.shape[0], _ptr(x), _stream(stream)), "mtgp_mlp_fit_scaling")

    def forward(self, x, stream=None) -> torch.Tensor:
        x = _dev(x, torch.float32)
        y = torch.empty((x.shape[0], self.widths[-1]), dtype=torch.float32, device="cuda")
        for r0 in range(0, x.shape[0], self.max_batch):
            r1 = min(r0 + self.max_batch, x.shape[0])
            check(lib().mtgp_mlp_forward(self._h, r1 - r0, _ptr(x[r0:r1]), _ptr(y[r0:r1]), _stream(stream)),
                  "mtgp_mlp_forward")
        return y

    def gradients(self, x, target, mask, rows=None, stream=None):
        """(loss, packed gradient) of the masked squared error on the batch (device tensors)."""
        x, target, mask = _dev(x, torch.float32), _dev(target, torch.float32), _dev(mask, torch.float32)
        B = x.shape[0] if rows is None else int(rows.numel())
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda")
        check(lib().mtgp_mlp_gradients(self._h, B, _ptr(x), _ptr(target), _ptr(mask), _ptr(rows), _ptr(g), _ptr(loss),
                                       _stream(stream)), "mtgp_mlp_gradients")
        return loss, g

    def train_step(self, x, target, mask, rows, lr: float, loss_out=None, stream=None):
        """One Adam step on the rows ``rows`` (device int32) of (x, target, mask) (device FP32)."""
        check(lib().mtgp_mlp_train_step(self._h, int(rows.numel()), _ptr(x), _ptr(target), _ptr(mask), _ptr(rows),
                                        ctypes.c_float(lr), _ptr(loss_out), _stream(stream)), "mtgp_mlp_train_step")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(lib().mtgp_mlp_destroy(self._h), "mtgp_mlp_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def train(mlp: MLP, feats, targets, masks, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-4, stream=None, val_fraction: float = 0.0, eval_every: int = 100) -> torch.Tensor:
    """Adam on minibatches drawn by seeded epoch permutations; returns the per-step losses (device).

    The learning rate decays geometrically from lr to lr_final.  Input scaling comes from the
    training features.  With ``val_fraction`` > 0 a seeded share of the rows is held out: every
    ``eval_every`` steps the masked loss on it (mtgp_mlp_gradients) is taken, and the network ends with
    the parameters of the lowest held-out loss (early stopping: the network otherwise overfits the
    few thousand labelled fits, and its proposals for unseen fits get worse).  The held-out rows and
    the (step, loss) history stay on the network as ``val_rows`` and ``val_history``.
    """
    feats = _dev(feats, torch.float32)
    targets = _dev(targets, torch.float32)
    masks = _dev(masks, torch.float32)
    n = feats.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.arange(n)
    val = None
    if val_fraction > 0.0:
        perm = rng.permutation(n)
        nv = min(max(1, int(round(val_fraction * n))), mlp.max_batch, n - 1)
        val = torch.as_tensor(np.sort(perm[:nv]).astype(np.int32)).cuda()
        idx = np.sort(perm[nv:])
    batch = min(batch, len(idx), mlp.max_batch)
    order = []
    while len(order) < steps * batch:
        order.extend(idx[rng.permutation(len(idx))].tolist())
    rows = torch.as_tensor(np.asarray(order[:steps * batch], dtype=np.int32)).cuda()
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    mlp.fit_scaling(feats, stream)
    decay = (lr_final / lr) ** (1.0 / max(steps - 1, 1))
    best, best_params = np.inf, None
    mlp.val_rows, mlp.val_history = val, []
    for k in range(steps):
        mlp.train_step(feats, targets, masks, rows[k * batch:(k + 1) * batch], lr * decay ** k, losses[k:k + 1], stream)
        if val is not None and ((k + 1) % eval_every == 0 or k == steps - 1):
            vl, _ = mlp.gradients(feats, targets, masks, rows=val, stream=stream)
            v = float(vl.item())
            mlp.val_history.append((k + 1, v))
            if v < best:
                best, best_params = v, mlp.get_params()
    if best_params is not None:
        mlp.set_params(*best_params)
    return losses


def propose(batch, mlp: MLP, judge=False, stream=None):
    """Set every fit's parameters to the network's prediction from its features (mtgp_propose: features,
    forward pass and parameter map in one call).  With ``judge`` (True or 1) the exact NLL picks, per fit,
    the best of the prediction, two blends with the parameters set before the call and those parameters
    themselves; with ``judge=2`` the best of the quarter blend (p + 3 c) / 4 and the parameters set
    before the call.  Returns (prediction, chosen candidate per fit or None)."""
    mode = 1 if judge is True else int(judge or 0)
    pred = torch.empty((batch.n, mlp.widths[-1]), dtype=torch.float32, device="cuda")
    chosen = torch.empty(batch.n, dtype=torch.int32, device="cuda") if mode else None
    check(lib().mtgp_propose(batch._h, mlp._h, _ptr(pred), mode, _ptr(chosen), _stream(stream)),
          "mtgp_propose")
    return pred, chosen

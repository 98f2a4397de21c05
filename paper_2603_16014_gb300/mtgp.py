"""Python binding of the fast multitask GP library: one handle per fit, torch tensors for memory/streams.

Every computation runs in the CUDA library (libmtgp_gb300.so); this module only passes device
pointers, sizes and the current CUDA stream through the C ABI of include/mtgp.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import DNET, FP32_TRANSFORM, FP64, LATTICE, NOISE_PER_TASK, SOLVE_FP64, check, lib


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(x, dtype=torch.float64):
    t = torch.as_tensor(x, dtype=dtype)
    if not t.is_cuda:
        t = t.cuda()
    return t.contiguous()


class MTGP:
    """A fast-MTGP fit: design (lattice or digital net), per-task shifts, task sizes 2^m_t.

    ``gen``: lattice -- (d,) generating vector words; digital net -- (d, gen_cols) column words.
    ``shift``: (T, d) words.  ``precision``: "fp64" or "fp32" (FP32 kernel-column transforms).
    ``solve``: "df" (default: FP32-transform digital nets solve each frequency in double-float) or
    "fp64" (MTGP_SOLVE_FP64: FP64 per-frequency solves throughout).
    """

    def __init__(self, kind: str, d: int, m, gen, shift, precision: str = "fp64", noise_per_task: bool = False,
                 solve: str = "df"):
        self.kind = LATTICE if kind == "lattice" else DNET
        self.d = int(d)
        self.m = [int(x) for x in m]
        self.T = len(self.m)
        self.N = sum(1 << x for x in self.m)
        gen = np.ascontiguousarray(np.asarray(gen, dtype=np.uint32))
        shift = np.ascontiguousarray(np.asarray(shift, dtype=np.uint32).reshape(self.T, self.d))
        gen_cols = int(gen.shape[1]) if (self.kind == DNET and gen.ndim == 2) else 0
        m_arr = (ctypes.c_int * self.T)(*self.m)
        h = ctypes.c_void_p()
        prec = ((FP32_TRANSFORM if precision == "fp32" else FP64) | (NOISE_PER_TASK if noise_per_task else 0)
                | (SOLVE_FP64 if solve == "fp64" else 0))
        self.nsig = self.T if noise_per_task else 1
        check(lib().mtgp_create(ctypes.byref(h), self.kind, self.d, self.T, m_arr,
                                gen.ctypes.data_as(ctypes.c_void_p), gen_cols,
                                shift.ctypes.data_as(ctypes.c_void_p), prec), "mtgp_create")
        self._h = h
        self.precision = precision

    @classmethod
    def from_problem(cls, p, precision=None, noise_per_task: bool = False, solve: str = "df"):
        prec = precision or ("fp32" if p.fp32_transform else "fp64")
        return cls(p.kind, p.d, p.m, p.gen, p.shift, prec, noise_per_task, solve)

    # ------------------------------------------------------------------ calls
    def points(self, stream=None) -> torch.Tensor:
        """(N, d) int32 tensor holding the uint32 fixed-point words of the design points."""
        x = torch.empty((self.N, self.d), dtype=torch.int32, device="cuda")
        check(lib().mtgp_points(self._h, _ptr(x), _stream(stream)), "mtgp_points")
        return x

    def set_y(self, y, stream=None) -> None:
        y = _dev(y)
        assert y.numel() == self.N
        self._y = y
        check(lib().mtgp_set_y(self._h, _ptr(y), _stream(stream)), "mtgp_set_y")

    def _theta(self, eta, W, v, sigma2):
        eta = _dev(eta).reshape(-1)
        W = _dev(W).reshape(self.T, -1)
        v = _dev(v).reshape(-1)
        s2 = _dev(sigma2).reshape(self.nsig)
        return eta, W, v, s2

    def nll(self, eta, W, v, sigma2, stream=None):
        """Returns (out, tau): out = [NLL, quad, logdet] (device float64), tau (T,)."""
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        tau = torch.empty(self.T, dtype=torch.float64, device="cuda")
        check(lib().mtgp_nll(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), _ptr(out), _ptr(tau),
                             _stream(stream)), "mtgp_nll")
        return out, tau

    def nll_grad(self, eta, W, v, sigma2, stream=None, outs=None):
        """Returns (out, tau, g_eta, g_W, g_v, g_sigma2) with gradients of the NLL."""
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        if outs is None:
            outs = (torch.empty(3, dtype=torch.float64, device="cuda"),
                    torch.empty(self.T, dtype=torch.float64, device="cuda"),
                    torch.empty(self.d, dtype=torch.float64, device="cuda"),
                    torch.empty_like(W), torch.empty(self.T, dtype=torch.float64, device="cuda"),
                    torch.empty(self.nsig, dtype=torch.float64, device="cuda"))
        out, tau, ge, gW, gv, gs = outs
        check(lib().mtgp_nll_grad(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), _ptr(out), _ptr(tau),
                                  _ptr(ge), _ptr(gW), _ptr(gv), _ptr(gs), _stream(stream)), "mtgp_nll_grad")
        return outs

    def set_smoothness(self, alpha: int) -> None:
        """Kernel smoothness alpha (1..4): the SI kernel of Eq. 2.5 (lattices) or the single order
        K_alpha of the DSI kernel of Eq. 2.6 (digital nets)."""
        check(lib().mtgp_set_smoothness(self._h, int(alpha)), "mtgp_set_smoothness")

    def set_dsi_weights(self, b, stream=None) -> None:
        """Mixture weights b (4, >= 0) of the adaptive-smoothness DSI kernel (Eq. 2.6, digital nets);
        None returns to the order-2 kernel alone."""
        if b is None:
            self._b = None
            check(lib().mtgp_set_dsi_weights(self._h, None, _stream(stream)), "mtgp_set_dsi_weights")
            return
        b = _dev(b).reshape(4)
        self._b = b
        check(lib().mtgp_set_dsi_weights(self._h, _ptr(b), _stream(stream)), "mtgp_set_dsi_weights")

    def dsi_weights_grad(self, stream=None) -> torch.Tensor:
        """Gradient with respect to b (4,) from the last nll_grad (of the NLL) or gcv_grad call."""
        g = torch.empty(4, dtype=torch.float64, device="cuda")
        check(lib().mtgp_dsi_weights_grad(self._h, _ptr(g), _stream(stream)), "mtgp_dsi_weights_grad")
        return g

    def gcv(self, eta, W, v, sigma2, stream=None):
        """Returns (out, tau): out = [L_GCV, r^T K~^-2 r, trace K~^-1] (device float64), tau (T,) at
        the GCV mean."""
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        tau = torch.empty(self.T, dtype=torch.float64, device="cuda")
        check(lib().mtgp_gcv(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), _ptr(out), _ptr(tau),
                             _stream(stream)), "mtgp_gcv")
        return out, tau

    def gcv_grad(self, eta, W, v, sigma2, stream=None):
        """Returns (out, tau, g_eta, g_W, g_v, g_sigma2): the GCV loss and its gradient (equal sizes)."""
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        tau = torch.empty(self.T, dtype=torch.float64, device="cuda")
        ge = torch.empty(self.d, dtype=torch.float64, device="cuda")
        gW = torch.empty_like(W)
        gv = torch.empty(self.T, dtype=torch.float64, device="cuda")
        gs = torch.empty(self.nsig, dtype=torch.float64, device="cuda")
        check(lib().mtgp_gcv_grad(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), _ptr(out), _ptr(tau),
                                  _ptr(ge), _ptr(gW), _ptr(gv), _ptr(gs), _stream(stream)), "mtgp_gcv_grad")
        return out, tau, ge, gW, gv, gs

    def cubature(self, eta, W, v, sigma2, stream=None):
        """Returns (mu_hat (T,), Sigma (T, T)): posterior mean and covariance of the task integrals."""
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        mu = torch.empty(self.T, dtype=torch.float64, device="cuda")
        Sigma = torch.empty((self.T, self.T), dtype=torch.float64, device="cuda")
        check(lib().mtgp_cubature(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), _ptr(mu), _ptr(Sigma),
                                  _stream(stream)), "mtgp_cubature")
        return mu, Sigma

    # ------------------------------------------------------------ host-buffer entry point
    def pack_theta(self, eta, W, v, sigma2, pin=True) -> torch.Tensor:
        """Packed host theta of mtgp_nll_grad_host: eta | W (T x s) | v | sigma2 (1 or T)."""
        parts = [np.asarray(eta, dtype=np.float64).reshape(-1), np.asarray(W, dtype=np.float64).reshape(-1),
                 np.asarray(v, dtype=np.float64).reshape(-1), np.asarray(sigma2, dtype=np.float64).reshape(self.nsig)]
        t = torch.from_numpy(np.concatenate(parts))
        return t.pin_memory() if pin else t

    def host_out(self, s, pin=True) -> torch.Tensor:
        """Host output buffer of mtgp_nll_grad_host for W with s columns."""
        n = 3 + self.T + self.d + self.T * s + self.T + self.nsig
        t = torch.empty(n, dtype=torch.float64)
        return t.pin_memory() if pin else t

    def unpack_out(self, out, s):
        """(out3, tau, g_eta, g_W, g_v, g_sigma2) views of a filled host output buffer."""
        T, d = self.T, self.d
        sizes = [3, T, d, T * s, T, self.nsig]
        o = torch.split(out, sizes)
        return o[0], o[1], o[2], o[3].view(T, s), o[4], o[5]

    def nll_grad_host(self, theta, out, s, stream=None) -> None:
        """NLL and gradient with host buffers (theta packed as pack_theta, out as host_out): copy in,
        evaluate, copy out, all in stream order; call sync() before reading ``out``."""
        assert theta.device.type == "cpu" and out.device.type == "cpu"
        assert theta.dtype == torch.float64 and out.dtype == torch.float64
        check(lib().mtgp_nll_grad_host(self._h, ctypes.c_void_p(theta.data_ptr()), int(s),
                                       ctypes.c_void_p(out.data_ptr()), _stream(stream)), "mtgp_nll_grad_host")

    def posterior(self, eta, W, v, sigma2, xq, task, variance=True, stream=None):
        eta, W, v, s2 = self._theta(eta, W, v, sigma2)
        xq = _dev(xq).reshape(-1, self.d)
        task = _dev(task, torch.int32).reshape(-1)
        nq = xq.shape[0]
        mean = torch.empty(nq, dtype=torch.float64, device="cuda")
        var = torch.empty(nq, dtype=torch.float64, device="cuda") if variance else None
        check(lib().mtgp_posterior(self._h, _ptr(eta), _ptr(W), W.shape[1], _ptr(v), _ptr(s2), nq, _ptr(xq),
                                   _ptr(task), _ptr(mean), _ptr(var), _stream(stream)), "mtgp_posterior")
        return mean, var

    def sync(self, stream=None) -> None:
        check(lib().mtgp_sync(self._h, _stream(stream)), "mtgp_sync")

    def profile(self, enable: bool) -> None:
        """Bracket every kernel the handle launches with CUDA events (off by default)."""
        check(lib().mtgp_profile(self._h, 1 if enable else 0), "mtgp_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read; synchronises on the events."""
        cap = 64
        names = ctypes.create_string_buffer(32 * cap)
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_int * cap)()
        n = ctypes.c_int()
        check(lib().mtgp_profile_read(self._h, cap, names, ms, cnt, ctypes.byref(n)), "mtgp_profile_read")
        out = {}
        for i in range(min(n.value, cap)):
            nm = names.raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (ms[i], cnt[i])
        return out

    def workspace_bytes(self) -> int:
        return int(lib().mtgp_workspace_bytes(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            check(lib().mtgp_destroy(self._h), "mtgp_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nll_equal_static(kind: str, d: int, T: int, m: int, gen, shift, y, eta, W, v, sigma2, precision="fp64",
                     stream=None):
    """NLL of an equal-size fit through mtgp_nll_equal_static, which allocates no device memory
    (for callers that cannot call cudaMalloc); returns (out [NLL, quad, logdet], tau, status)."""
    k = LATTICE if kind == "lattice" else DNET
    gen = np.ascontiguousarray(np.asarray(gen, dtype=np.uint32))
    shift = np.ascontiguousarray(np.asarray(shift, dtype=np.uint32).reshape(T, d))
    gen_cols = int(gen.shape[1]) if (k == DNET and gen.ndim == 2) else 0
    y = _dev(y)
    eta, W, v, s2 = _dev(eta).reshape(-1), _dev(W).reshape(T, -1), _dev(v).reshape(-1), _dev(sigma2).reshape(1)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    tau = torch.empty(T, dtype=torch.float64, device="cuda")
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    check(lib().mtgp_nll_equal_static(k, d, T, m, gen.ctypes.data_as(ctypes.c_void_p), gen_cols,
                                      shift.ctypes.data_as(ctypes.c_void_p),
                                      FP32_TRANSFORM if precision == "fp32" else FP64, _ptr(y), _ptr(eta), _ptr(W),
                                      W.shape[1], _ptr(v), _ptr(s2), _ptr(out), _ptr(tau), _ptr(status),
                                      _stream(stream)), "mtgp_nll_equal_static")
    return out, tau, status


def _carr(ctype, vals):
    return (ctype * len(vals))(*vals)


class Batch:
    """Many independent equal-size fits evaluated / optimised together (C ABI mtgp_batch_*).

    ``problems``: objects with kind, d, m (equal sizes), gen, shift (e.g. inputs.Problem).
    Parameters are packed per fit as [eta, W (T x s), v, sigma2].
    ``precision``: "fp32" or "fp64" for every fit, "auto" (FP32 transforms for digital nets, FP64 for
    lattices, whose spectra decay below FP32 transform noise), or one of those per fit (a list).
    """

    def __init__(self, problems, s: int = 2, precision="fp32", solve: str = "df"):
        self.problems = list(problems)
        n = len(self.problems)
        kind = [LATTICE if p.kind == "lattice" else DNET for p in self.problems]
        if isinstance(precision, str):
            precision = [precision] * n
        precision = [("fp64" if k == LATTICE else "fp32") if q == "auto" else q for q, k in zip(precision, kind)]
        assert len(precision) == n and all(q in ("fp32", "fp64") for q in precision), precision
        self.precision = precision
        d = [int(p.d) for p in self.problems]
        T = [len(p.m) for p in self.problems]
        m = [int(p.m[0]) for p in self.problems]
        gens, gcols, shifts = [], [], []
        for p, k in zip(self.problems, kind):
            g = np.asarray(p.gen, dtype=np.uint32)
            gens.append(g.ravel())
            gcols.append(int(g.shape[1]) if (k == DNET and g.ndim == 2) else 0)
            shifts.append(np.asarray(p.shift, dtype=np.uint32).ravel())
        gen = np.ascontiguousarray(np.concatenate(gens))
        shift = np.ascontiguousarray(np.concatenate(shifts))
        h = ctypes.c_void_p()
        check(lib().mtgp_batch_create(ctypes.byref(h), n, _carr(ctypes.c_int, kind), _carr(ctypes.c_int, d),
                                      _carr(ctypes.c_int, T), _carr(ctypes.c_int, m),
                                      gen.ctypes.data_as(ctypes.c_void_p), _carr(ctypes.c_int, gcols),
                                      shift.ctypes.data_as(ctypes.c_void_p), s,
                                      _carr(ctypes.c_int, [(FP32_TRANSFORM if q == "fp32" else FP64)
                                                           | (SOLVE_FP64 if solve == "fp64" else 0) for q in precision])),
              "mtgp_batch_create")
        self._h = h
        self.n, self.s = n, s
        po = (ctypes.c_longlong * (n + 1))()
        yo = (ctypes.c_longlong * (n + 1))()
        check(lib().mtgp_batch_layout(self._h, po, yo), "mtgp_batch_layout")
        self.param_offsets = list(po)
        self.y_offsets = list(yo)
        self.nparams = self.param_offsets[-1]

    def pack(self, thetas) -> np.ndarray:
        """[(eta, W, v, sigma2), ...] -> packed natural parameters."""
        return np.concatenate([np.concatenate([np.ravel(e), np.ravel(W), np.ravel(v), np.ravel([s2])])
                               for (e, W, v, s2) in thetas]).astype(np.float64)

    def unpack(self, packed):
        out = []
        packed = np.asarray(packed)
        for f, p in enumerate(self.problems):
            o, d, T = self.param_offsets[f], p.d, len(p.m)
            x = packed[o:self.param_offsets[f + 1]]
            out.append((x[:d], x[d:d + T * self.s].reshape(T, self.s), x[d + T * self.s:d + T * self.s + T],
                        float(x[-1])))
        return out

    def set_y(self, y, stream=None):
        self._y = _dev(y)
        check(lib().mtgp_batch_set_y(self._h, _ptr(self._y), _stream(stream)), "mtgp_batch_set_y")

    def set_theta(self, packed, stream=None):
        self._t = _dev(packed)
        check(lib().mtgp_batch_set_theta(self._h, _ptr(self._t), _stream(stream)), "mtgp_batch_set_theta")

    def get_theta(self, stream=None) -> torch.Tensor:
        t = torch.empty(self.nparams, dtype=torch.float64, device="cuda")
        check(lib().mtgp_batch_get_theta(self._h, _ptr(t), _stream(stream)), "mtgp_batch_get_theta")
        return t

    def nll_grad(self, stream=None):
        nll = torch.empty(self.n, dtype=torch.float64, device="cuda")
        g = torch.empty(self.nparams, dtype=torch.float64, device="cuda")
        check(lib().mtgp_batch_nll_grad(self._h, _ptr(nll), _ptr(g), _stream(stream)), "mtgp_batch_nll_grad")
        return nll, g

    def adam(self, steps: int, lr: float, graph: bool = True, trace=None, stream=None):
        check(lib().mtgp_batch_adam(self._h, steps, lr, 1 if graph else 0, _ptr(trace), _stream(stream)),
              "mtgp_batch_adam")

    def fit(self, theta0, steps: int, lr: float, graph: bool = True, trace=None, final_nll: bool = True,
            stream=None):
        """mtgp_batch_fit: ``steps`` Adam steps from theta0 (packed natural parameters, or None to continue
        from the current parameters, e.g. after propose()); returns (final packed parameters, NLL at
        them or None)."""
        t0 = None if theta0 is None else _dev(theta0)
        self._t = t0
        th = torch.empty(self.nparams, dtype=torch.float64, device="cuda")
        nll = torch.empty(self.n, dtype=torch.float64, device="cuda") if final_nll else None
        check(lib().mtgp_batch_fit(self._h, _ptr(t0), int(steps), float(lr), 1 if graph else 0, _ptr(th), _ptr(nll),
                                   _ptr(trace), _stream(stream)), "mtgp_batch_fit")
        return th, nll

    def autotune(self, reps: int = 3, stream=None):
        chosen = (ctypes.c_int * self.n)()
        check(lib().mtgp_batch_autotune(self._h, reps, chosen, _stream(stream)), "mtgp_batch_autotune")
        return list(chosen)

    def features(self, stream=None) -> torch.Tensor:
        """(nfits, 258) FP32 spectral summaries (mtgp_batch_features)."""
        f = torch.empty((self.n, 258), dtype=torch.float32, device="cuda")
        check(lib().mtgp_batch_features(self._h, _ptr(f), _stream(stream)), "mtgp_batch_features")
        return f

    def targets(self, stream=None):
        """(target, mask), each (nfits, 37) FP32, from the current parameters (mtgp_batch_targets)."""
        t = torch.empty((self.n, 37), dtype=torch.float32, device="cuda")
        mk = torch.empty((self.n, 37), dtype=torch.float32, device="cuda")
        check(lib().mtgp_batch_targets(self._h, _ptr(t), _ptr(mk), _stream(stream)), "mtgp_batch_targets")
        return t, mk

    def set_theta_proposal(self, pred, stream=None):
        """Parameters from a (nfits, 37) prediction (mtgp_batch_set_theta_proposal)."""
        self._pred = _dev(pred, torch.float32)
        check(lib().mtgp_batch_set_theta_proposal(self._h, _ptr(self._pred), _stream(stream)),
              "mtgp_batch_set_theta_proposal")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            check(lib().mtgp_batch_destroy(self._h), "mtgp_batch_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NLLFunction(torch.autograd.Function):
    """NLL as a differentiable function of (eta, W, v, sigma2) through the hand-written adjoint."""

    @staticmethod
    def forward(ctx, model: MTGP, eta, W, v, sigma2):
        out, tau, ge, gW, gv, gs = model.nll_grad(eta, W, v, sigma2)
        ctx.save_for_backward(ge, gW.reshape(W.shape), gv, gs.reshape(sigma2.shape))
        return out[0]

    @staticmethod
    def backward(ctx, g):
        ge, gW, gv, gs = ctx.saved_tensors
        return None, g * ge, g * gW, g * gv, g * gs


def nll(model: MTGP, eta, W, v, sigma2):
    return NLLFunction.apply(model, eta, W, v, sigma2)

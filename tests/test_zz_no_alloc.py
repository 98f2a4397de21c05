"""mtgp_nll_equal_static: the NLL entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc (allocation forbidden or unsafe where they run); all
of its intermediates live in one fixed-size device array inside the library.  These tests check
that it gives the same NLL as the handle-based entry point (mtgp_create + mtgp_nll) on the same
inputs, on consecutive calls that reuse the shared array, and that oversized problems are refused
before any device work.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import dense
from paper_2603_16014_gb300 import inputs

TOL = {"fp64": 1e-8, "fp32": 1e-5}


def _problems():
    return [
        (inputs.make_problem("dnet", 8, (12,) * 4, seed=5, s=2, eta=0.5, v=0.05, sigma2=1e-8, recipe="walshcos32",
                             mmax=16), "fp32"),
        (inputs.make_problem("lattice", 2, (10, 10), seed=6, s=1, eta=0.5, v=0.1, sigma2=1e-6), "fp64"),
        (inputs.make_problem("dnet", 3, (8, 8, 8), seed=7, s=2, eta=0.7, v=0.1, sigma2=1e-4), "fp64"),
    ]


def _static_nll(p, y, precision):
    from paper_2603_16014_gb300.mtgp import nll_equal_static
    out, tau, status = nll_equal_static(p.kind, p.d, p.T, p.m[0], p.gen, p.shift, y, p.eta, p.W, p.v, p.sigma2,
                                        precision=precision)
    return out.cpu().numpy(), tau.cpu().numpy(), int(status.item())


@pytest.mark.gpu
def test_static_nll_matches_handle_nll_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_16014_gb300 import build
    from paper_2603_16014_gb300.mtgp import MTGP
    build.build()
    from oracle import spectral
    cases = []
    for p, prec in _problems():
        X = dense.all_points(p.kind, p.gen, p.shift, p.m)
        y = inputs.synth_y(p, X)
        model = MTGP.from_problem(p, prec)
        model.set_y(torch.from_numpy(y))
        ref, tau_ref = model.nll(p.eta, p.W, p.v, p.sigma2)
        model.sync()
        cases.append((p, prec, y, ref.cpu().numpy(), tau_ref.cpu().numpy()))
        model.close()
        # the oracle on the same inputs (per-frequency Cholesky of the CPU oracle), so the comparison
        # does not rest on the handle-based path alone
        orc = spectral.nll_equal(p.kind, p.gen, p.shift, p.m, y, p.eta, p.W, p.v, p.sigma2)
        out, _, status = _static_nll(p, y, prec)
        assert status == 0
        assert abs(out[0] - orc["nll"]) <= TOL[prec] * abs(orc["nll"]), (out[0], orc["nll"])
    # two passes over all problems: every call after the first finds the array holding another
    # problem's intermediates
    for _ in range(2):
        for p, prec, y, ref, tau_ref in cases:
            out, tau, status = _static_nll(p, y, prec)
            assert status == 0
            assert abs(out[0] - ref[0]) <= TOL[prec] * abs(ref[0]), (out, ref)
            assert abs(out[1] + out[2] - (ref[1] + ref[2])) <= TOL[prec] * (abs(ref[1]) + abs(ref[2]))
            assert np.allclose(tau, tau_ref, rtol=0, atol=1e-12 * (1 + np.abs(tau_ref).max()))


def test_static_nll_rejects_problems_beyond_the_scratch_array():
    from paper_2603_16014_gb300 import _lib
    from paper_2603_16014_gb300 import build
    build.build()
    L = _lib.lib()
    T, d, m = 4, 4, 18          # FP64 digital net: ~18 MB of intermediates, more than the 8 MiB array
    gen = (ctypes.c_uint32 * (d * 32))(*([1 << 31] * (d * 32)))
    shift = (ctypes.c_uint32 * (T * d))()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check fails first
    rc = L.mtgp_nll_equal_static(1, d, T, m, gen, 32, shift, 0, dummy, dummy, dummy, 1, dummy, dummy, dummy,
                                 None, None, None)
    assert rc == 1   # MTGP_ERR_INVALID_ARG
    assert b"static scratch array holds" in L.mtgp_last_error_string()

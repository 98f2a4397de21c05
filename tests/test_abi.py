"""Host-side checks of the C ABI library (no GPU needed): it loads and exports every declared symbol."""
import ctypes
import os

import pytest

from paper_2603_16014_gb300 import _lib


@pytest.fixture(scope="module")
def built():
    from paper_2603_16014_gb300 import build
    build.build()
    return _lib.lib()


def test_exports_every_declared_symbol(built):
    names = _lib.declared_symbols()
    assert "mtgp_create" in names and "mtgp_nll_grad" in names
    for n in names:
        assert hasattr(built, n), n


def test_invalid_arguments_rejected_on_host(built):
    L = built
    h = ctypes.c_void_p()
    m = (ctypes.c_int * 2)(4, 4)
    gen = (ctypes.c_uint32 * 2)(1, 3)
    sh = (ctypes.c_uint32 * 4)(0, 0, 0, 0)
    # bad kind / dimension / task count / size / precision: rejected before any device work
    assert L.mtgp_create(ctypes.byref(h), 7, 2, 2, m, gen, 0, sh, 0) == 1
    assert L.mtgp_create(ctypes.byref(h), 0, 0, 2, m, gen, 0, sh, 0) == 1
    assert L.mtgp_create(ctypes.byref(h), 0, 2, 0, m, gen, 0, sh, 0) == 1
    assert L.mtgp_create(ctypes.byref(h), 0, 2, 9, m, gen, 0, sh, 0) == 1
    bad_m = (ctypes.c_int * 2)(4, 25)
    assert L.mtgp_create(ctypes.byref(h), 0, 2, 2, bad_m, gen, 0, sh, 0) == 1
    assert L.mtgp_create(ctypes.byref(h), 0, 2, 2, m, gen, 0, sh, 5) == 1
    # digital nets need enough generating-matrix columns
    assert L.mtgp_create(ctypes.byref(h), 1, 2, 2, m, gen, 2, sh, 0) == 1
    assert b"gen_cols" in L.mtgp_last_error_string()
    assert L.mtgp_create(None, 0, 2, 2, m, gen, 0, sh, 0) == 1
    # NULL handle calls
    assert L.mtgp_sync(None, None) == 1
    assert L.mtgp_destroy(None) == 0


def test_oracle_not_imported_by_product_modules():
    here = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2603_16014_gb300")
    for f in os.listdir(here):
        if f.endswith(".py"):
            src = open(os.path.join(here, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f


def test_host_buffer_layout_round_trip():
    # packed layouts of mtgp_nll_grad_host (host logic only): theta = eta | W (T x s) | v | sigma2,
    # out = [NLL, quad, logdet] | tau | g_eta | g_W | g_v | g_sigma2
    import numpy as np
    from paper_2603_16014_gb300.mtgp import MTGP
    m = MTGP.__new__(MTGP)
    m.T, m.d = 3, 4
    for nsig in (1, 3):
        m.nsig = nsig
        eta = np.arange(4.0) + 1
        W = np.arange(6.0).reshape(3, 2) + 10
        v = np.array([0.1, 0.2, 0.3])
        s2 = np.full(nsig, 1e-4) * (1 + np.arange(nsig))
        th = m.pack_theta(eta, W, v, s2, pin=False)
        assert th.numel() == 4 + 6 + 3 + nsig
        assert np.array_equal(th.numpy(), np.concatenate([eta, W.ravel(), v, s2]))
        out = m.host_out(2, pin=False)
        assert out.numel() == 3 + 3 + 4 + 6 + 3 + nsig
        out.copy_(__import__("torch").arange(out.numel(), dtype=out.dtype))
        o3, tau, ge, gW, gv, gs = m.unpack_out(out, 2)
        assert o3.tolist() == [0, 1, 2] and tau.tolist() == [3, 4, 5] and ge.tolist() == [6, 7, 8, 9]
        assert gW.shape == (3, 2) and gW[0, 0].item() == 10 and gW[2, 1].item() == 15
        assert gv.tolist() == [16, 17, 18] and gs.numel() == nsig and gs[0].item() == 19

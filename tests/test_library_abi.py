"""The C-ABI library loads and exports every call include/sps.h declares (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sps.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sps_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1304_4333_b300 import _native as N
    if not os.path.exists(N.LIB_PATH):
        from paper_1304_4333_b300.build import build
        build()
    return N.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sps_init", "sps_loglik", "sps_loglik_grad", "sps_cphase", "sps_sphase",
                     "sps_mphase", "sps_run", "sps_destroy", "sps_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1304_4333_b300 import _native as N
    assert sorted(N.SIGNATURES) == _declared()


def test_options_default_are_the_papers_constants(lib):
    from paper_1304_4333_b300 import _native as N
    o = N.SpsOptions()
    lib.sps_options_default(C.byref(o))
    assert (o.ess_fraction, o.h_init, o.h_step, o.h_min, o.h_max) == (0.5, 0.5, 0.01, 0.1, 1.0)
    assert (o.target_accept, o.rne_cycle, o.rne_final) == (0.25, 0.35, 0.9)
    assert o.precision == N.PREC_SPLIT and o.mkernel == N.MKERNEL_RW


def test_status_strings(lib):
    for s in range(9):
        assert lib.sps_status_string(s)


def test_init_rejects_bad_arguments_without_touching_the_device(lib):
    # argument checks run before any CUDA call
    from paper_1304_4333_b300 import _native as N
    import numpy as np
    X = np.ones((4, 2))
    y = np.array([0, 1, 2, 1], np.int32)   # outcome 2 out of range for C = 2
    sd = np.array([5.0])
    pr = N.SpsPrior(N.PRIOR_ISO, None, sd.ctypes.data_as(C.POINTER(C.c_double)))
    ctx = C.c_void_p()
    st = lib.sps_init(C.byref(ctx), C.c_void_p(X.ctypes.data), 4, 2, C.c_void_p(y.ctypes.data), 2,
                      C.byref(pr), None)
    assert st == 1 and not ctx.value

"""The C-ABI library loads and exports every entry point of include/fmm_vortex.h (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmm_vortex.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1106_5273_gb300 import binding
    return binding.lib


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fmm_plan_create", "fmm_eval_velocity_stretching", "fmm_plan_destroy", "fmm_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_and_errors_without_gpu(lib):
    from paper_1106_5273_gb300 import binding
    q = binding.Params.default()
    assert (q.p, round(q.theta, 6), q.ncrit, q.periodic, q.images) == (10, 0.4, 64, 0, 3)
    assert binding._strerror(0) == "ok" and "invalid" in binding._strerror(-1)
    # parameter validation happens before any CUDA call
    h = ctypes.c_void_p()
    for bad in (dict(p=0), dict(p=17), dict(theta=1.5), dict(ncrit=0), dict(periodic=1, box_len=0.0),
                dict(periodic=1, images=0), dict(m2l_mode=7)):
        qq = binding.Params.default(**bad)
        assert lib.fmm_plan_create(ctypes.byref(qq), 100, ctypes.byref(h)) == -1
    assert lib.fmm_plan_create(ctypes.byref(q), -1, ctypes.byref(h)) == -1
    # batched entry point: argument checks before any CUDA call
    off = (ctypes.c_int64 * 3)(0, 10, 20)
    assert lib.fmm_eval_batch(None, 2, off, None, None, None, None, None, None, None, None) == -1
    assert lib.fmm_plan_device_bytes(None) == 0

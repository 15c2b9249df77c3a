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
    assert (q.sigma_rule, q.p2p_pair_max, q.m2l_mode) == (0, 0, 0)
    assert binding._strerror(0) == "ok" and "invalid" in binding._strerror(-1)
    # parameter validation happens before any CUDA call
    h = ctypes.c_void_p()
    for bad in (dict(p=0), dict(p=17), dict(theta=1.5), dict(ncrit=0), dict(periodic=1, box_len=0.0),
                dict(periodic=1, images=0), dict(m2l_mode=7), dict(m2l_mode=64), dict(sigma_rule=2),
                dict(p2p_pair_max=-1),
                dict(split_tie=2), dict(p2p_tpl=3)):
        qq = binding.Params.default(**bad)
        assert lib.fmm_plan_create(ctypes.byref(qq), 100, ctypes.byref(h)) == -1
    assert lib.fmm_plan_create(ctypes.byref(q), -1, ctypes.byref(h)) == -1
    # batched entry point: argument checks before any CUDA call
    off = (ctypes.c_int64 * 3)(0, 10, 20)
    assert lib.fmm_eval_batch(None, 2, off, None, None, None, None, None, None, None, None) == -1
    assert lib.fmm_plan_device_bytes(None) == 0


def test_struct_layouts_match_the_header(lib, tmp_path):
    """ctypes mirrors of the header's structs have the C sizes (gcc on this host)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "fmm_vortex.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu",'
                   'sizeof(fmm_params), sizeof(fmm_stats), sizeof(fmm_server_params), sizeof(fmm_request),'
                   'sizeof(fmm_request_result), sizeof(fmm_server_counters));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    from paper_1106_5273_gb300 import binding as b
    assert sizes == [ctypes.sizeof(t) for t in (b.Params, b.Stats, b.ServerParams, b.Request, b.RequestResult,
                                                 b.ServerCounters)]


def test_server_params_validated_without_gpu(lib):
    from paper_1106_5273_gb300 import binding as b
    h = ctypes.c_void_p()
    for bad in (dict(workers=0), dict(workers=17), dict(batching=2), dict(hbm_budget_bytes=0),
                dict(max_batch_problems=0), dict(theta=1.0), dict(ncrit=-1), dict(images=0)):
        q = b.ServerParams.default(**bad)
        assert lib.fmm_server_create(ctypes.byref(q), ctypes.byref(h)) == -1
    assert lib.fmm_server_submit(None, None, None) == -1


def test_noalloc_binding_rejects_bad_outputs_before_the_call(lib):
    """morton_order_noalloc checks shapes, devices and dtypes in Python, so a
    wrong output never reaches the kernels (checked here with CPU tensors)."""
    import torch
    from paper_1106_5273_gb300 import binding as b
    pos = torch.zeros((8, 3), dtype=torch.float32)
    keys = torch.zeros(8, dtype=torch.int64)
    order = torch.zeros(8, dtype=torch.int32)
    with pytest.raises(ValueError):
        b.morton_order_noalloc(torch.zeros((8, 2), dtype=torch.float32), keys, order)
    with pytest.raises(ValueError):
        b.morton_order_noalloc(torch.zeros(24, dtype=torch.float32), keys, order)
    with pytest.raises(TypeError):  # CPU outputs
        b.morton_order_noalloc(pos, keys, order)


def test_lattice_operator_host_build_without_gpu(lib):
    """fmm_lattice_operator's host build runs without a device; bad arguments are refused."""
    import numpy as np
    from paper_1106_5273_gb300 import binding as b
    a = b.lattice_operator(3, 2, on_device=False)
    assert a.shape == (9, 9) and np.isfinite(a).all() and np.abs(a).max() > 0
    out = np.zeros(1)
    assert lib.fmm_lattice_operator(0, 3, 0, out.ctypes.data) == -1
    assert lib.fmm_lattice_operator(4, 9, 0, out.ctypes.data) == -1
    assert lib.fmm_lattice_operator(4, 3, 0, None) == -1

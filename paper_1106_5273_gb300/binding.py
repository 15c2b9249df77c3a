"""ctypes binding of include/fmm_vortex.h (argument marshalling only).

Every computation runs in the CUDA library; there is no CPU fallback.  The
library must have been built (``__graft_entry__.build()`` or
``python -m paper_1106_5273_gb300.build``); importing this module raises if
it is missing.  Device arrays are torch CUDA tensors (float32, contiguous),
passed by ``data_ptr()``; host arrays for the ``_host`` entry point are numpy.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "_lib", "libfmm_vortex.so")

FMM_OK = 0
FMM_M2L_AUTO, FMM_M2L_SIMT, FMM_M2L_TENSOR = 0, 1, 2
FMM_M2L_SORT_STEPS = 8
FMM_M2L_FULL_SPLIT = 16
FMM_M2L_CHUNK_STAGES = 32
FMM_SIGMA_SOURCE, FMM_SIGMA_MIXED = 0, 1
FMM_SPLIT_SOURCE, FMM_SPLIT_TARGET = 0, 1
FMM_OUT_VELOCITY, FMM_OUT_STRETCHING, FMM_OUT_STRETCHING_TRANSPOSE = 1, 2, 4


class FmmError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s (%d)" % (what, _strerror(code), code))
        self.code = code


if not os.path.exists(library_path):
    raise ImportError("CUDA library %s is missing: run __graft_entry__.build() "
                      "(python -m paper_1106_5273_gb300.build)" % library_path)
lib = ctypes.CDLL(library_path)


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("theta", ctypes.c_float), ("ncrit", ctypes.c_int32),
                ("periodic", ctypes.c_int32), ("images", ctypes.c_int32),
                ("box_min", ctypes.c_double * 3), ("box_len", ctypes.c_double),
                ("sigma_sep", ctypes.c_float), ("outputs", ctypes.c_int32),
                ("m2l_mode", ctypes.c_int32), ("sigma_rule", ctypes.c_int32),
                ("p2p_pair_max", ctypes.c_int32), ("split_tie", ctypes.c_int32), ("p2p_tpl", ctypes.c_int32)]

    @classmethod
    def default(cls, **kw):
        q = cls()
        lib.fmm_params_default(ctypes.byref(q))
        for k, v in kw.items():
            if k == "box_min":
                for i in range(3):
                    q.box_min[i] = float(v[i])
            else:
                setattr(q, k, v)
        return q


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ncells", ctypes.c_int64), ("nleaves", ctypes.c_int64),
                ("nlevels", ctypes.c_int32), ("m2l_tensor", ctypes.c_int32),
                ("p2p_cell_pairs", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("m2l_steps", ctypes.c_int64),
                ("m2l_keys", ctypes.c_int64), ("m2l_built", ctypes.c_int64),
                ("p2p_pairs_near", ctypes.c_int64), ("p2p_pairs_mid", ctypes.c_int64),
                ("p2p_pairs_far", ctypes.c_int64), ("ms_tree", ctypes.c_double),
                ("ms_upward", ctypes.c_double), ("ms_traverse", ctypes.c_double),
                ("ms_m2l", ctypes.c_double), ("ms_downward", ctypes.c_double),
                ("ms_p2p", ctypes.c_double), ("ms_total", ctypes.c_double), ("traversal_runs", ctypes.c_int64),
                ("m2l_split_coefs", ctypes.c_int64), ("m2l_stage_chunks", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
lib.fmm_params_default.argtypes = [ctypes.POINTER(Params)]
lib.fmm_params_default.restype = None
lib.fmm_strerror.argtypes = [ctypes.c_int]
lib.fmm_strerror.restype = ctypes.c_char_p
lib.fmm_plan_create.argtypes = [ctypes.POINTER(Params), _i64, ctypes.POINTER(_vp)]
lib.fmm_plan_destroy.argtypes = [_vp]
lib.fmm_plan_destroy.restype = None
for _name in ("fmm_eval_velocity_stretching", "fmm_eval_velocity_stretching_host"):
    getattr(lib, _name).argtypes = [_vp, _i64, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp]
lib.fmm_direct_velocity_stretching.argtypes = [_i64, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp]
lib.fmm_eval_targets.argtypes = [_vp, _i64, _vp, _vp, _vp, ctypes.c_float, _i64, _vp, _vp, _vp]
lib.fmm_autotune_plan.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32,
                                  _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp]
lib.fmm_autotune_ncrit.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                                   ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp]
lib.fmm_plan_set_timing.argtypes = [_vp, ctypes.c_int]
lib.fmm_plan_set_list_capacity.argtypes = [_vp, _i64, _i64, _i64]
lib.fmm_selftest_bounded_wait.argtypes = [_i64, ctypes.c_int, _vp]
lib.fmm_eval_batch.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
lib.fmm_plan_device_bytes.argtypes = [_vp]
lib.fmm_plan_device_bytes.restype = _i64
lib.fmm_morton_order_noalloc.argtypes = [_i64, _vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp, _vp]
lib.fmm_eval_strengths.argtypes = [_vp, _vp, _vp, _vp, _vp]
lib.fmm_plan_status.argtypes = [_vp, _vp]
lib.fmm_graph_capture.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]
lib.fmm_graph_launch.argtypes = [_vp, _vp]
lib.fmm_graph_kernel_count.argtypes = [_vp]
lib.fmm_graph_kernel_count.restype = _i64
lib.fmm_graph_destroy.argtypes = [_vp]
lib.fmm_graph_destroy.restype = None
lib.fmm_lattice_operator.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp]
lib.fmm_probe_fp32_rate.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     _vp]
lib.fmm_kernel_launch_count.argtypes = []
lib.fmm_kernel_launch_count.restype = ctypes.c_int64
lib.fmm_plan_get_stats.argtypes = [_vp, ctypes.POINTER(Stats)]
lib.fmm_plan_get_order.argtypes = [_vp, _vp, _vp]
lib.fmm_plan_get_cells.argtypes = [_vp] + [_vp] * 8
lib.fmm_plan_get_lists.argtypes = [_vp, _vp, _vp]


def _strerror(code):
    return lib.fmm_strerror(code).decode()


def _check(code, what):
    if code != FMM_OK:
        raise FmmError(code, what)


def _dptr(t, n=None, name="array"):
    """Device pointer of a float32 contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float32":
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """An FMM plan (tree, lists and expansions resident on the device)."""

    def __init__(self, n_max, params=None, **kw):
        self.params = params if params is not None else Params.default(**kw)
        h = _vp()
        _check(lib.fmm_plan_create(ctypes.byref(self.params), int(n_max), ctypes.byref(h)),
               "fmm_plan_create")
        self._h = h
        self.n_max = int(n_max)

    def close(self):
        if getattr(self, "_h", None):
            lib.fmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, pos, gamma, sigma=None, sigma_uniform=0.0, vel=None, dgamma=None, stream=None,
             stretching=True):
        """fmm_eval_velocity_stretching on torch CUDA tensors; returns (vel, dgamma).
        stretching=False passes no stretching output (the velocity-only kernels run)
        and returns (vel, None)."""
        import torch
        n = pos.shape[0]
        if vel is None:
            vel = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        if dgamma is None and stretching:
            dgamma = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        if not stretching:
            dgamma = None
        _check(lib.fmm_eval_velocity_stretching(
            self._h, n, _dptr(pos, name="pos"), _dptr(gamma, name="gamma"), _dptr(sigma, name="sigma"),
            float(sigma_uniform), _dptr(vel, name="vel"), _dptr(dgamma, name="dgamma"),
            _stream_ptr(stream)), "fmm_eval_velocity_stretching")
        return vel, dgamma

    def eval_targets(self, src_pos, src_gamma, tgt_pos, sigma=None, sigma_uniform=0.0, vel=None, stream=None):
        """fmm_eval_targets on torch CUDA tensors: the velocity of the sources at the
        target points; returns vel [nt, 3]."""
        import torch
        nt = tgt_pos.shape[0]
        if vel is None:
            vel = torch.empty((nt, 3), dtype=torch.float32, device=tgt_pos.device)
        _check(lib.fmm_eval_targets(
            self._h, src_pos.shape[0], _dptr(src_pos, name="src_pos"), _dptr(src_gamma, name="src_gamma"),
            _dptr(sigma, name="sigma"), float(sigma_uniform), nt, _dptr(tgt_pos, name="tgt_pos"),
            _dptr(vel, name="vel"), _stream_ptr(stream)), "fmm_eval_targets")
        return vel

    def eval_host(self, pos, gamma, sigma=None, sigma_uniform=0.0, vel=None, dgamma=None, stream=None):
        """fmm_eval_velocity_stretching_host on numpy float32 arrays (synchronous)."""
        import numpy as np
        n = pos.shape[0]
        for a in (pos, gamma) + ((sigma,) if sigma is not None else ()):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        if vel is None:
            vel = np.empty((n, 3), np.float32)
        if dgamma is None:
            dgamma = np.empty((n, 3), np.float32)
        _check(lib.fmm_eval_velocity_stretching_host(
            self._h, n, pos.ctypes.data, gamma.ctypes.data,
            sigma.ctypes.data if sigma is not None else None, float(sigma_uniform),
            vel.ctypes.data, dgamma.ctypes.data, _stream_ptr(stream)), "fmm_eval_velocity_stretching_host")
        return vel, dgamma

    def eval_batch(self, offsets, pos, gamma, sigma=None, sigma_prob=None, boxes=None, vel=None, dgamma=None,
                   stream=None):
        """fmm_eval_batch: problems k = [offsets[k], offsets[k+1]) of the concatenated torch CUDA
        tensors; sigma_prob (one core width per problem) and boxes ([nprob, 4] periodic cubes)
        are host arrays.  Returns (vel, dgamma)."""
        import numpy as np
        import torch
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        nprob = off.shape[0] - 1
        n = pos.shape[0]
        if vel is None:
            vel = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        if dgamma is None:
            dgamma = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        sp = None if sigma_prob is None else np.ascontiguousarray(sigma_prob, dtype=np.float32)
        bx = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64)
        _check(lib.fmm_eval_batch(
            self._h, nprob, off.ctypes.data, _dptr(pos, name="pos"), _dptr(gamma, name="gamma"),
            _dptr(sigma, name="sigma"), None if sp is None else sp.ctypes.data,
            None if bx is None else bx.ctypes.data, _dptr(vel, name="vel"), _dptr(dgamma, name="dgamma"),
            _stream_ptr(stream)), "fmm_eval_batch")
        return vel, dgamma

    def eval_strengths(self, gamma, vel=None, dgamma=None, stream=None, stretching=True):
        """fmm_eval_strengths: new strengths (torch CUDA [n, 3], the caller's order) on the
        positions, core widths and tree of the last full evaluation; returns (vel, dgamma)."""
        import torch
        n = gamma.shape[0]
        if n != self.stats().n:
            raise ValueError("gamma has %d rows, the plan's last evaluation %d" % (n, self.stats().n))
        if vel is None:
            vel = torch.empty((n, 3), dtype=torch.float32, device=gamma.device)
        if dgamma is None and stretching:
            dgamma = torch.empty((n, 3), dtype=torch.float32, device=gamma.device)
        if not stretching:
            dgamma = None
        _check(lib.fmm_eval_strengths(self._h, _dptr(gamma, name="gamma"), _dptr(vel, name="vel"),
                                      _dptr(dgamma, name="dgamma"), _stream_ptr(stream)), "fmm_eval_strengths")
        return vel, dgamma

    def status(self, stream=None):
        """fmm_plan_status: 0 or the FMM_E_* raised on the device (waits for the stream)."""
        return int(lib.fmm_plan_status(self._h, _stream_ptr(stream)))

    def capture_graph(self, gamma, vel, dgamma=None):
        """fmm_graph_capture: a Graph replaying fmm_eval_strengths on these fixed tensors."""
        return Graph(self, gamma, vel, dgamma)

    def device_bytes(self):
        """Device memory the plan holds (fmm_plan_device_bytes)."""
        return int(lib.fmm_plan_device_bytes(self._h))

    def set_list_capacity(self, frontier=0, m2l=0, p2p=0):
        """fmm_plan_set_list_capacity: starting capacities of the traversal's buffers."""
        _check(lib.fmm_plan_set_list_capacity(self._h, int(frontier), int(m2l), int(p2p)),
               "fmm_plan_set_list_capacity")

    def set_timing(self, on=True):
        _check(lib.fmm_plan_set_timing(self._h, 1 if on else 0), "fmm_plan_set_timing")

    def stats(self):
        s = Stats()
        _check(lib.fmm_plan_get_stats(self._h, ctypes.byref(s)), "fmm_plan_get_stats")
        return s

    def order(self):
        import numpy as np
        n = self.stats().n
        o = np.zeros(n, np.uint32)
        k = np.zeros(n, np.uint64)
        _check(lib.fmm_plan_get_order(self._h, o.ctypes.data, k.ctypes.data), "fmm_plan_get_order")
        return o, k

    def cells(self):
        import numpy as np
        nc = self.stats().ncells
        a = {k: np.zeros(nc, np.int32) for k in ("begin", "end", "level", "parent", "child_begin", "nchild")}
        a["center"] = np.zeros((nc, 3), np.float64)
        a["radius"] = np.zeros(nc, np.float64)
        _check(lib.fmm_plan_get_cells(self._h, *[a[k].ctypes.data for k in
                                                 ("begin", "end", "level", "parent", "child_begin", "nchild",
                                                  "center", "radius")]), "fmm_plan_get_cells")
        return a

    def lists(self):
        import numpy as np
        s = self.stats()
        p2p = np.zeros((s.p2p_cell_pairs, 3), np.int32)
        m2l = np.zeros((s.m2l_pairs, 3), np.int32)
        _check(lib.fmm_plan_get_lists(self._h, p2p.ctypes.data, m2l.ctypes.data), "fmm_plan_get_lists")
        return p2p, m2l


class Graph:
    """A captured CUDA graph of fmm_eval_strengths (fmm_graph_*).  Keeps the plan and the
    tensors it reads and writes alive."""

    def __init__(self, plan, gamma, vel, dgamma=None):
        n = plan.stats().n
        for t, name in ((gamma, "gamma"), (vel, "vel")) + (((dgamma, "dgamma"),) if dgamma is not None else ()):
            if t.dim() != 2 or t.shape[0] != n or t.shape[1] != 3:
                raise ValueError("%s must have shape [%d, 3]" % (name, n))
        h = _vp()
        _check(lib.fmm_graph_capture(plan._h, _dptr(gamma, name="gamma"), _dptr(vel, name="vel"),
                                     _dptr(dgamma, name="dgamma"), ctypes.byref(h)), "fmm_graph_capture")
        self._h = h
        self._keep = (plan, gamma, vel, dgamma)

    def launch(self, stream=None):
        _check(lib.fmm_graph_launch(self._h, _stream_ptr(stream)), "fmm_graph_launch")

    def kernel_count(self):
        return int(lib.fmm_graph_kernel_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib.fmm_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NOALLOC_MAX_N = 1 << 20
BATCH_MAX = 1 << 15
BATCH_DEPTH = 16


def morton_order_noalloc(pos, keys_out, order_out, periodic=False, box_min=None, box_len=0.0, stream=None):
    """fmm_morton_order_noalloc: Morton keys + stable sort without any allocation.

    pos: float32 CUDA tensor [n,3]; keys_out: int64 CUDA tensor [n] (holds the
    uint64 keys); order_out: int32 CUDA tensor [n] (holds uint32 indices).
    """
    import torch
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("pos must have shape [n, 3]")
    n = pos.shape[0]
    for t, dt, name in ((keys_out, torch.int64, "keys_out"), (order_out, torch.int32, "order_out")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != dt:
            raise TypeError("%s must be a contiguous %s CUDA tensor" % (name, dt))
        if t.device != pos.device:
            raise ValueError("%s must be on the device of pos (%s)" % (name, pos.device))
        if t.numel() < n:
            raise ValueError("%s holds %d elements, fewer than n = %d" % (name, t.numel(), n))
    bm = (ctypes.c_double * 3)(*(box_min if box_min is not None else (0.0, 0.0, 0.0)))
    _check(lib.fmm_morton_order_noalloc(n, _dptr(pos, name="pos"), 1 if periodic else 0, bm, float(box_len),
                                        ctypes.c_void_p(keys_out.data_ptr()), ctypes.c_void_p(order_out.data_ptr()),
                                        _stream_ptr(stream)), "fmm_morton_order_noalloc")
    return keys_out, order_out


def lattice_operator(p, images, on_device=True):
    """fmm_lattice_operator: the P x P FP64 periodic lattice operator (numpy)."""
    import numpy as np
    out = np.zeros((p * p, p * p), np.float64)
    _check(lib.fmm_lattice_operator(int(p), int(images), 1 if on_device else 0, out.ctypes.data),
           "fmm_lattice_operator")
    return out


def probe_fp32_rate(launches=20, stream=None):
    """fmm_probe_fp32_rate: (TFLOP/s, ms per launch) of independent FFMA2 chains."""
    t = ctypes.c_double(0.0)
    ms = ctypes.c_double(0.0)
    _check(lib.fmm_probe_fp32_rate(int(launches), ctypes.byref(t), ctypes.byref(ms), _stream_ptr(stream)),
           "fmm_probe_fp32_rate")
    return float(t.value), float(ms.value)


def selftest_bounded_wait(spins, arrive, stream=None):
    """fmm_selftest_bounded_wait: FMM_OK (0) or FMM_E_TIMEOUT (-4)."""
    return int(lib.fmm_selftest_bounded_wait(int(spins), int(arrive), _stream_ptr(stream)))


def kernel_launch_count():
    """Kernels launched by the CUDA library since it was loaded."""
    return int(lib.fmm_kernel_launch_count())


def direct(pos, gamma, sigma=None, sigma_uniform=0.0, vel=None, dgamma=None, stream=None):
    """fmm_direct_velocity_stretching: all pairs on the device (O(n^2))."""
    import torch
    n = pos.shape[0]
    if vel is None:
        vel = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
    if dgamma is None:
        dgamma = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
    _check(lib.fmm_direct_velocity_stretching(n, _dptr(pos, name="pos"), _dptr(gamma, name="gamma"),
                                              _dptr(sigma, name="sigma"), float(sigma_uniform),
                                              _dptr(vel, name="vel"), _dptr(dgamma, name="dgamma"),
                                              _stream_ptr(stream)), "fmm_direct_velocity_stretching")
    return vel, dgamma


# ---------------------------------------------------------------- serving loop

def autotune_ncrit(params, offsets, pos, gamma, sigma_prob, boxes=None, candidates=(32, 48, 64, 96, 128, 192, 256),
                   reps=1, stream=None):
    """fmm_autotune_ncrit on a sample batch (torch CUDA tensors, host offsets /
    sigma_prob / boxes as for Plan.eval_batch); returns (best ncrit, {ncrit: ms})."""
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    sp = np.ascontiguousarray(sigma_prob, dtype=np.float32)
    bx = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64)
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    ms = np.zeros(cand.shape[0], np.float64)
    best = ctypes.c_int32(0)
    _check(lib.fmm_autotune_ncrit(ctypes.byref(params), off.shape[0] - 1, off.ctypes.data, _dptr(pos, name="pos"),
                                  _dptr(gamma, name="gamma"), sp.ctypes.data,
                                  None if bx is None else bx.ctypes.data, cand.ctypes.data, cand.shape[0],
                                  int(reps), ctypes.byref(best), ms.ctypes.data, _stream_ptr(stream)),
           "fmm_autotune_ncrit")
    return int(best.value), {int(c): float(m) for c, m in zip(cand, ms)}


def autotune_plan(params, offsets, pos, gamma, sigma_prob, boxes=None, ncrit=(32, 48, 64, 96, 128, 192, 256),
                  tpl=(1, 2), reps=1, stream=None):
    """fmm_autotune_plan: the fastest (ncrit, p2p_tpl) on a sample batch; returns
    (ncrit, tpl, {(ncrit, tpl): ms})."""
    import numpy as np
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    sp = np.ascontiguousarray(sigma_prob, dtype=np.float32)
    bx = None if boxes is None else np.ascontiguousarray(boxes, dtype=np.float64)
    nc = np.ascontiguousarray(ncrit, dtype=np.int32)
    tp = np.ascontiguousarray(tpl, dtype=np.int32)
    ms = np.zeros(nc.shape[0] * tp.shape[0], np.float64)
    bn, bt = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib.fmm_autotune_plan(ctypes.byref(params), off.shape[0] - 1, off.ctypes.data, _dptr(pos, name="pos"),
                                 _dptr(gamma, name="gamma"), sp.ctypes.data, None if bx is None else bx.ctypes.data,
                                 nc.ctypes.data, nc.shape[0], tp.ctypes.data, tp.shape[0], int(reps), ctypes.byref(bn),
                                 ctypes.byref(bt), ms.ctypes.data, _stream_ptr(stream)), "fmm_autotune_plan")
    table = {(int(a), int(b)): float(ms[i * tp.shape[0] + j]) for i, a in enumerate(nc) for j, b in enumerate(tp)}
    return int(bn.value), int(bt.value), table


class ServerParams(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("batching", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("max_batch_particles", ctypes.c_int64), ("max_batch_problems", ctypes.c_int32),
                ("theta", ctypes.c_float), ("ncrit", ctypes.c_int32), ("sigma_sep", ctypes.c_float),
                ("images", ctypes.c_int32), ("m2l_mode", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("model_bytes_per_particle", ctypes.c_int64)]

    @classmethod
    def default(cls, **kw):
        q = cls()
        lib.fmm_server_params_default(ctypes.byref(q))
        for k, v in kw.items():
            setattr(q, k, v)
        return q


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("p", ctypes.c_int32), ("periodic", ctypes.c_int32),
                ("box", ctypes.c_double * 4), ("sigma", ctypes.c_float), ("pos", ctypes.c_void_p),
                ("gamma", ctypes.c_void_p), ("vel", ctypes.c_void_p), ("dgamma", ctypes.c_void_p)]


class RequestResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_problems", ctypes.c_int32), ("worker", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("batch_particles", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ServerCounters(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_int64), ("requests", ctypes.c_int64), ("particles", ctypes.c_int64),
                ("peak_bytes", ctypes.c_int64), ("memory_waits", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


lib.fmm_server_params_default.argtypes = [ctypes.POINTER(ServerParams)]
lib.fmm_server_params_default.restype = None
lib.fmm_server_create.argtypes = [ctypes.POINTER(ServerParams), ctypes.POINTER(_vp)]
lib.fmm_server_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(_i64)]
lib.fmm_server_wait.argtypes = [_vp, _i64, ctypes.c_double, ctypes.POINTER(RequestResult)]
lib.fmm_server_clock.argtypes = [_vp]
lib.fmm_server_clock.restype = ctypes.c_double
lib.fmm_server_get_counters.argtypes = [_vp, ctypes.POINTER(ServerCounters)]
lib.fmm_server_destroy.argtypes = [_vp]
lib.fmm_server_destroy.restype = None


class Server:
    """fmm_server_*: queue of host-array requests, continuous batching on the device."""

    def __init__(self, params=None, **kw):
        self.params = params if params is not None else ServerParams.default(**kw)
        h = _vp()
        _check(lib.fmm_server_create(ctypes.byref(self.params), ctypes.byref(h)), "fmm_server_create")
        self._h = h
        self._live = {}

    def submit(self, pos, gamma, p, sigma, periodic=False, box=None, vel=None, dgamma=None):
        """Queue one request (numpy float32 [n,3] arrays, kept alive until wait); returns a ticket."""
        import numpy as np
        for a in (pos, gamma):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        n = pos.shape[0]
        if vel is None:
            vel = np.empty((n, 3), np.float32)
        if dgamma is None:
            dgamma = np.empty((n, 3), np.float32)
        r = Request()
        r.n, r.p, r.periodic, r.sigma = n, int(p), 1 if periodic else 0, float(sigma)
        if box is not None:
            for k in range(4):
                r.box[k] = float(box[k])
        r.pos, r.gamma = pos.ctypes.data, gamma.ctypes.data
        r.vel = vel.ctypes.data if vel is not False else None
        r.dgamma = dgamma.ctypes.data if dgamma is not False else None
        t = _i64()
        _check(lib.fmm_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "fmm_server_submit")
        self._live[t.value] = (pos, gamma, vel, dgamma)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        """(result dict, vel, dgamma) of a ticket; raises FmmError on timeout."""
        res = RequestResult()
        _check(lib.fmm_server_wait(self._h, int(ticket), float(timeout), ctypes.byref(res)), "fmm_server_wait")
        _, _, vel, dg = self._live.pop(int(ticket))
        return res.as_dict(), vel, dg

    def clock(self):
        return float(lib.fmm_server_clock(self._h))

    def counters(self):
        c = ServerCounters()
        _check(lib.fmm_server_get_counters(self._h, ctypes.byref(c)), "fmm_server_get_counters")
        return c.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            lib.fmm_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

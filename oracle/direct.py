"""ctypes front end of the plain-C FP64 direct sum (oracle/direct.c).

Oracle, test infrastructure only.  Computes Eqs. (1)-(3) over all pairs (and
an explicit list of image shifts); see direct.c for the formulas.  The shared
library is built by ``build()`` (gcc, -ffp-contract=off so x86 and Arm hosts
give the same bits) and rebuilt on first use when it is missing.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "_liboracle_direct.so")
_lib = None


def build(force=False):
    """Compile direct.c into a shared library next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct.argtypes = [ctypes.c_int64, p, p, ctypes.c_int64, p, p, p,
                                      ctypes.c_int64, p, ctypes.c_int, ctypes.c_int, p, p]
        lib.oracle_direct.restype = None
        lib.oracle_pair_ST.argtypes = [ctypes.c_double, ctypes.c_double, p, p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def direct(xt, gt, xs, gs, sigma, images=None, skip_self=False, transpose=False):
    """u, s [nt,3] FP64 at targets xt (strengths gt) from all sources.

    sigma: scalar or [ns]; images: [nimg,3] shifts added to d (default: one
    zero shift); skip_self: targets are the sources, index for index, and the
    zero-shift self pair is left out (its exact value is zero); transpose: the
    stretching in the transpose scheme (grad u)^T gamma instead of
    (gamma . grad) u.
    """
    lib = _load()
    xt = np.ascontiguousarray(xt, np.float64).reshape(-1, 3)
    gt = np.ascontiguousarray(gt, np.float64).reshape(-1, 3)
    xs = np.ascontiguousarray(xs, np.float64).reshape(-1, 3)
    gs = np.ascontiguousarray(gs, np.float64).reshape(-1, 3)
    ns = xs.shape[0]
    sig = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.float64), (ns,)))
    if images is None:
        images = np.zeros((1, 3))
    images = np.ascontiguousarray(images, np.float64).reshape(-1, 3)
    nt = xt.shape[0]
    u = np.zeros((nt, 3))
    s = np.zeros((nt, 3))
    if nt and ns:
        lib.oracle_direct(nt, _ptr(xt), _ptr(gt), ns, _ptr(xs), _ptr(gs), _ptr(sig),
                          images.shape[0], _ptr(images), 1 if skip_self else 0, 1 if transpose else 0,
                          _ptr(u), _ptr(s))
    return u, s


def pair_ST(r2, sigma):
    """S, T of one pair from the C code (for cross-checking pairs.S_T)."""
    lib = _load()
    S = ctypes.c_double()
    T = ctypes.c_double()
    lib.oracle_pair_ST(float(r2), float(sigma), ctypes.byref(S), ctypes.byref(T))
    return S.value, T.value


def num_threads():
    return int(_load().oracle_num_threads())

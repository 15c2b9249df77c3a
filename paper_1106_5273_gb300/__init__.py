"""GB300 (sm_103a) FMM for the regularized Biot-Savart velocity and the
vortex-stretching term of N Gaussian vortex blobs (Yokota, Barba, Narumi,
Yasuoka, arXiv:1106.5273, Secs. 2-3).

The compute path is the CUDA library built from csrc/ (C ABI in
include/fmm_vortex.h); `binding` is its thin Python binding:

    from paper_1106_5273_gb300 import Params, Plan, direct

The binding is loaded on first use, so `python -m paper_1106_5273_gb300.build`
works before the library exists; using the binding without the library
raises ImportError (there is no fallback).
"""
__all__ = ["Params", "Plan", "Stats", "FmmError", "direct", "lib", "library_path", "kernel_launch_count", "morton_order_noalloc", "NOALLOC_MAX_N", "BATCH_MAX", "BATCH_DEPTH", "Server", "ServerParams",
           "FMM_M2L_AUTO", "FMM_M2L_SIMT", "FMM_M2L_TENSOR", "FMM_M2L_SORT_STEPS", "FMM_M2L_FULL_SPLIT", "FMM_M2L_CHUNK_STAGES", "FMM_SIGMA_SOURCE", "FMM_SIGMA_MIXED",
           "FMM_OUT_VELOCITY", "FMM_OUT_STRETCHING", "FMM_OUT_STRETCHING_TRANSPOSE", "autotune_ncrit",
           "FMM_SPLIT_SOURCE", "FMM_SPLIT_TARGET", "Graph", "autotune_plan"]


def __getattr__(name):
    if name in __all__:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)

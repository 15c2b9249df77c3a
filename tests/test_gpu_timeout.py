"""The bounded device wait gives up with a status instead of hanging, and the
context stays usable (no trap, no fault: the barrier is simply never completed)."""
import numpy as np
import pytest

import workloads
from gpu_common import rel_l2, run_fmm

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_1106_5273_gb300 import binding
    assert binding.selftest_bounded_wait(4096, 1) == 0          # completed barrier: FMM_OK
    assert binding.selftest_bounded_wait(4096, 0) == -4         # nothing arrives: FMM_E_TIMEOUT
    assert binding.selftest_bounded_wait(0, 0) == -1            # bad argument
    # the context is still usable: a tensor-core M2L evaluation after the timeout
    w = workloads.plummer(6000)
    w["sigma"] = np.float32(0.002)
    _, u1, _ = run_fmm(w, 8, 0.5, 32, m2l_mode=1)
    plan, u2, _ = run_fmm(w, 8, 0.5, 32, m2l_mode=2)
    assert plan.stats().m2l_tensor == 1 and rel_l2(u2, u1) < 1e-5

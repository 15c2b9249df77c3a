"""The allocation-free Morton ordering entry point against the plan's ordering.

fmm_morton_order_noalloc serves callers that cannot call cudaMalloc (code
under a memory manager that owns all device memory, or code that must not
cause the implicit device synchronization of cudaMalloc/cudaFree); its
scratch is one static device array.  Its keys and permutation must equal,
bit for bit, those fmm_eval_velocity_stretching computes, on consecutive
calls that reuse the array.  Kept in the last-collected file so a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _cases():
    w1 = workloads.jittered_lattice(16)
    w2 = workloads.plummer(100000)
    w3 = workloads.taylor_green(32)
    return [(w1, dict(p=6, theta=0.5, ncrit=32)), (w2, dict(p=4, theta=0.5, ncrit=64)),
            (w3, dict(p=4, theta=0.4, ncrit=64, periodic=1, box_min=w3["box_min"], box_len=w3["box_len"]))]


def test_noalloc_ordering_matches_plan_on_consecutive_calls():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1106_5273_gb300 import NOALLOC_MAX_N, FmmError, Params, Plan, morton_order_noalloc

    for w, kw in _cases():
        n = w["pos"].shape[0]
        pos = torch.from_numpy(w["pos"]).cuda()
        gam = torch.from_numpy(w["gamma"]).cuda()
        plan = Plan(n, Params.default(**kw))
        plan.eval(pos, gam, sigma_uniform=float(w["sigma"]))
        torch.cuda.synchronize()
        order_ref, keys_ref = plan.order()
        plan.close()
        keys = torch.empty(n, dtype=torch.int64, device="cuda")
        order = torch.empty(n, dtype=torch.int32, device="cuda")
        for _ in range(2):  # the static array keeps the previous call's contents
            keys.fill_(-1)
            order.fill_(-1)
            morton_order_noalloc(pos, keys, order, periodic=bool(kw.get("periodic")),
                                 box_min=kw.get("box_min"), box_len=kw.get("box_len", 0.0))
            torch.cuda.synchronize()
            assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_ref)
            assert np.array_equal(order.cpu().numpy().view(np.uint32), order_ref)

    # outputs of the wrong dtype or size are refused before the library is called
    pos = torch.zeros((1000, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        morton_order_noalloc(pos, torch.empty(999, dtype=torch.int64, device="cuda"),
                             torch.empty(1000, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        morton_order_noalloc(pos, torch.empty(1000, dtype=torch.int32, device="cuda"),
                             torch.empty(1000, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        morton_order_noalloc(pos, torch.empty(1000, dtype=torch.int64, device="cuda"),
                             torch.empty(2000, dtype=torch.int32, device="cuda")[::2])

    big = torch.zeros((NOALLOC_MAX_N + 1, 3), dtype=torch.float32, device="cuda")
    kb = torch.empty(NOALLOC_MAX_N + 1, dtype=torch.int64, device="cuda")
    ob = torch.empty(NOALLOC_MAX_N + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(FmmError) as err:
        morton_order_noalloc(big, kb, ob)
    assert err.value.code == -3  # FMM_E_CAPACITY: beyond the static scratch

"""Re-evaluation with new strengths on an unchanged tree (fmm_eval_strengths)
and its CUDA graph (fmm_graph_*), through the C ABI.

The vortex method puts its particles back on the same positions every step
and reuses the tree (Sec. 3.4).  A strength-only re-evaluation runs the same
kernels in the same order on the same tree, lists and operators, so it must
equal a full evaluation of the same input bit for bit; so must every replay
of the captured graph.  Marked gpu.
"""
import numpy as np
import pytest

import workloads
from gpu_common import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _gammas(n, k, seed=77):
    g = np.random.default_rng(seed)
    return [g.standard_normal((n, 3)).astype(np.float32) for _ in range(k)]


def _case(name):
    from paper_1106_5273_gb300 import Params
    if name == "taylor-green-16-tensor":
        w = workloads.taylor_green(16)
        return w, Params.default(p=10, theta=0.4, ncrit=64, periodic=1, box_min=w["box_min"],
                                 box_len=w["box_len"], m2l_mode=2), None
    w = workloads.plummer(4000, seed=12, sigma_rule="halfmass")
    if name == "plummer-simt":
        return w, Params.default(p=8, theta=0.5, ncrit=32, m2l_mode=1), None
    sig = (w["sigma"] * np.linspace(0.7, 1.3, 4000)).astype(np.float32)
    return w, Params.default(p=8, theta=0.5, ncrit=48, m2l_mode=2), sig


def _full(params, w, gam, sig):
    import torch
    from paper_1106_5273_gb300 import Plan
    plan = Plan(w["pos"].shape[0], params)
    u, s = plan.eval(to_dev(w["pos"]), to_dev(gam), sigma=to_dev(sig) if sig is not None else None,
                     sigma_uniform=float(w["sigma"]))
    torch.cuda.synchronize()
    return plan, u.cpu().numpy(), s.cpu().numpy()


@pytest.mark.parametrize("name", ["taylor-green-16-tensor", "plummer-simt", "plummer-sigma-array-tensor"])
def test_strengths_reuse_equals_full_evaluation(name):
    import torch
    w, params, sig = _case(name)
    n = w["pos"].shape[0]
    g1, g2 = _gammas(n, 2)
    plan, _, _ = _full(params, w, g1, sig)
    u2, s2 = plan.eval_strengths(to_dev(g2))
    torch.cuda.synchronize()
    assert plan.status() == 0
    _, ur, sr = _full(params, w, g2, sig)
    assert np.array_equal(u2.cpu().numpy(), ur) and np.array_equal(s2.cpu().numpy(), sr)
    # velocity only: the same velocity
    u3, s3 = plan.eval_strengths(to_dev(g2), stretching=False)
    torch.cuda.synchronize()
    assert s3 is None and np.array_equal(u3.cpu().numpy(), ur)


def test_graph_replays_equal_full_evaluations():
    import torch
    from paper_1106_5273_gb300 import FmmError, kernel_launch_count
    w, params, _ = _case("taylor-green-16-tensor")
    n = w["pos"].shape[0]
    g1, g2, g3 = _gammas(n, 3, seed=5)
    plan, _, _ = _full(params, w, g1, None)
    gbuf = to_dev(g1)
    vel = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    dg = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    graph = plan.capture_graph(gbuf, vel, dg)
    assert graph.kernel_count() > 5
    for g in (g2, g3, g2):
        gbuf.copy_(to_dev(g))
        l0 = kernel_launch_count()
        graph.launch()
        assert kernel_launch_count() - l0 == graph.kernel_count()
        torch.cuda.synchronize()
        assert plan.status() == 0
        _, ur, sr = _full(params, w, g, None)
        assert np.array_equal(vel.cpu().numpy(), ur) and np.array_equal(dg.cpu().numpy(), sr)
    # a full evaluation builds a new tree: the graph refuses to replay
    plan.eval(to_dev(w["pos"]), to_dev(g1), sigma_uniform=float(w["sigma"]))
    with pytest.raises(FmmError) as err:
        graph.launch()
    assert err.value.code == -1
    graph.close()


def test_user_stream_capture_of_strength_evaluation():
    """The caller can capture fmm_eval_strengths in its own graph (torch.cuda.graph)."""
    import torch
    w, params, _ = _case("taylor-green-16-tensor")
    n = w["pos"].shape[0]
    g1, g2 = _gammas(n, 2, seed=9)
    plan, _, _ = _full(params, w, g1, None)
    gbuf = to_dev(g1)
    vel = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    dg = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    plan.eval_strengths(gbuf, vel, dg)  # warm-up outside the capture
    torch.cuda.synchronize()
    tg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(tg, capture_error_mode="relaxed"):
        plan.eval_strengths(gbuf, vel, dg)
    gbuf.copy_(to_dev(g2))
    tg.replay()
    torch.cuda.synchronize()
    _, ur, sr = _full(params, w, g2, None)
    assert np.array_equal(vel.cpu().numpy(), ur) and np.array_equal(dg.cpu().numpy(), sr)


def test_reuse_needs_a_full_evaluation_of_the_plan_particles():
    import torch
    from paper_1106_5273_gb300 import Params, Plan
    w = workloads.plummer(2000)
    plan = Plan(4000, Params.default(p=6, theta=0.5, ncrit=32))
    g = to_dev(w["gamma"])
    from paper_1106_5273_gb300 import binding
    # nothing evaluated yet
    assert binding.lib.fmm_eval_strengths(plan._h, g.data_ptr(), None, None, None) == -1
    with pytest.raises(ValueError):
        plan.eval_strengths(g)
    tg = np.random.default_rng(1).uniform(-0.5, 0.5, (500, 3)).astype(np.float32)
    plan.eval_targets(to_dev(w["pos"]), g, to_dev(tg), sigma_uniform=float(w["sigma"]))
    torch.cuda.synchronize()
    assert binding.lib.fmm_eval_strengths(plan._h, g.data_ptr(), None, None, None) == -1
    plan.eval(to_dev(w["pos"]), g, sigma_uniform=float(w["sigma"]))
    u, s = plan.eval_strengths(g)
    torch.cuda.synchronize()
    assert plan.status() == 0 and np.isfinite(u.cpu().numpy()).all()

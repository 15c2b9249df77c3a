"""Batched evaluation (fmm_eval_batch): many independent problems in one
forest of octrees.  Each problem against the FP64 direct sum or the periodic
Fourier oracle, against the one-problem entry point, and bit-identical alone
and in the mix."""
import math

import numpy as np
import pytest

import workloads
from gpu_common import rel_l2, to_dev

pytestmark = pytest.mark.gpu

# The one-problem entry point against the same problem in a batch on the tensor
# cores: the same lists and products, but the one-problem M2L sums each tile in
# work items of at most 256 steps (partial sums added in FP32 afterwards) and
# the batch each tile in one FP32 tensor-memory accumulation; the long
# accumulation carries an error of up to ~2e-5 (measured 1.4e-6 free space,
# 1.1e-5 periodic, 2.0e-5 through the serving loop).
PLAIN_VS_BATCH = 5e-5


def _concat(probs, per_particle_sigma=False):
    off = np.zeros(len(probs) + 1, np.int64)
    for k, w in enumerate(probs):
        off[k + 1] = off[k] + w["pos"].shape[0]
    cat = lambda key: np.concatenate([w[key].reshape(-1, 3) for w in probs]) if off[-1] else np.zeros((0, 3), np.float32)
    pos, gam = cat("pos").astype(np.float32), cat("gamma").astype(np.float32)
    sig = np.array([float(w["sigma"]) for w in probs], np.float32)
    sarr = None
    if per_particle_sigma:
        sarr = np.concatenate([w["sigma_arr"] for w in probs]).astype(np.float32)
    return off, pos, gam, sig, sarr


def _run_batch(plan, off, pos, gam, sig=None, sarr=None, boxes=None):
    import torch
    u, s = plan.eval_batch(off, to_dev(pos), to_dev(gam), sigma=None if sarr is None else to_dev(sarr),
                           sigma_prob=None if sarr is not None else sig, boxes=boxes)
    torch.cuda.synchronize()
    return u.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)


def _free_problems():
    sizes = [0, 1, 40, 333, 1500, 0, 5000, 2600]
    out = []
    for k, n in enumerate(sizes):
        w = (workloads.uniform_ball if k % 2 == 0 else workloads.plummer)(n, seed=700 + k) if n else \
            dict(pos=np.zeros((0, 3), np.float32), gamma=np.zeros((0, 3), np.float32), sigma=np.float32(0.1))
        out.append(w)
    return out


@pytest.mark.parametrize("m2l_mode", [1, 2])
def test_batch_free_space_matches_direct_alone_and_plain(m2l_mode):
    from oracle import direct as od
    from paper_1106_5273_gb300 import Plan, Params
    probs = _free_problems()
    off, pos, gam, sig, _ = _concat(probs)
    prm = Params.default(p=8, theta=0.5, ncrit=32, m2l_mode=m2l_mode)
    plan = Plan(int(off[-1]), prm)
    u, s = _run_batch(plan, off, pos, gam, sig)
    st = plan.stats()
    assert st.n == off[-1] and st.m2l_pairs > 0
    for k, w in enumerate(probs):
        a, b = off[k], off[k + 1]
        n = b - a
        if n == 0:
            continue
        ud, sd = od.direct(w["pos"], w["gamma"], w["pos"], w["gamma"], float(w["sigma"]), skip_self=True)
        if n == 1:
            assert np.all(u[a:b] == 0) and np.all(s[a:b] == 0)
        else:
            assert rel_l2(u[a:b], ud) < 2e-4 and rel_l2(s[a:b], sd) < 1e-3, k
        # alone: the same problem as a batch of one gives the same bits
        ua, sa = _run_batch(plan, np.array([0, n]), w["pos"], w["gamma"], sig[k:k + 1])
        assert np.array_equal(ua, u[a:b]) and np.array_equal(sa, s[a:b]), k
    # the one-problem entry point on the largest problem (21-bit keys there;
    # on the tensor cores its M2L sums each tile in runs of at most 256 steps,
    # the batch each tile in one tensor-memory sum: FP32 accumulation order)
    k = int(np.argmax(np.diff(off)))
    w = probs[k]
    one = Plan(w["pos"].shape[0], prm)
    up, sp_ = one.eval(to_dev(w["pos"]), to_dev(w["gamma"]), sigma_uniform=float(w["sigma"]))
    tol = 1e-6 if m2l_mode == 1 else PLAIN_VS_BATCH
    assert rel_l2(u[off[k]:off[k + 1]], up.cpu().numpy()) < tol
    assert rel_l2(s[off[k]:off[k + 1]], sp_.cpu().numpy()) < tol


def test_batch_order_of_problems_does_not_matter():
    from paper_1106_5273_gb300 import Plan, Params
    probs = [p for p in _free_problems() if p["pos"].shape[0] > 1]
    off, pos, gam, sig, _ = _concat(probs)
    plan = Plan(int(off[-1]), Params.default(p=6, theta=0.5, ncrit=16))
    u, s = _run_batch(plan, off, pos, gam, sig)
    rev = probs[::-1]
    off2, pos2, gam2, sig2, _ = _concat(rev)
    u2, s2 = _run_batch(plan, off2, pos2, gam2, sig2)
    for k in range(len(probs)):
        j = len(probs) - 1 - k
        assert np.array_equal(u[off[k]:off[k + 1]], u2[off2[j]:off2[j + 1]])
        assert np.array_equal(s[off[k]:off[k + 1]], s2[off2[j]:off2[j + 1]])


def test_batch_periodic_cubes_match_fourier_and_plain():
    """Two different periodic cubes in one batch; the FMM error of each is
    measured by the CPU oracle FMM (same p, theta, ncrit) against the exact field."""
    from oracle import fmm as ofmm
    from oracle import periodic as op
    from paper_1106_5273_gb300 import Plan, Params
    L = 2 * math.pi
    P_, TH, NC = 6, 0.5, 16
    tg = workloads.taylor_green(16)
    c = workloads.random_cloud(600, seed=21, box=1.0, zero_net=True)
    g = c["gamma"] - c["gamma"].astype(np.float64).mean(0).astype(np.float32)
    cloud = dict(pos=(c["pos"] + np.float32(1.0)).astype(np.float32), gamma=g, sigma=np.float32(0.07))
    probs = [tg, cloud, tg]
    boxes = np.array([[0, 0, 0, L], [1, 1, 1, 1.0], [0, 0, 0, L]], np.float64)
    off, pos, gam, sig, _ = _concat(probs)
    prm = Params.default(p=P_, theta=TH, ncrit=NC, periodic=1, box_min=np.zeros(3), box_len=1.0, images=3)
    plan = Plan(int(off[-1]), prm)
    u, s = _run_batch(plan, off, pos, gam, sig, boxes=boxes)
    # problems 0 and 2 are the same problem: same bits
    assert np.array_equal(u[off[0]:off[1]], u[off[2]:off[3]])
    assert np.array_equal(s[off[0]:off[1]], s[off[2]:off[3]])
    # Taylor-Green against its closed form
    ut, st_ = op.taylor_green(tg["pos"].astype(np.float64), tg["gamma"].astype(np.float64), float(tg["sigma"]))
    ref = ofmm.fmm(tg["pos"], tg["gamma"], float(tg["sigma"]), P_, TH, NC, periodic=True, box_min=np.zeros(3),
                   box_len=L, images=3)
    assert rel_l2(u[off[0]:off[1]], ut) < 1.5 * rel_l2(ref.u, ut) + 2e-5
    # the cloud in the unit cube at (1,1,1) against the Fourier series
    uf, sf = op.fourier(cloud["pos"], g, cloud["pos"], g, 0.07, 1.0, 14)
    ref = ofmm.fmm(cloud["pos"], g, 0.07, P_, TH, NC, periodic=True, box_min=np.ones(3), box_len=1.0, images=3)
    assert rel_l2(u[off[1]:off[2]], uf) < 1.5 * rel_l2(ref.u, uf) + 2e-5
    assert rel_l2(s[off[1]:off[2]], sf) < 1.5 * rel_l2(ref.s, sf) + 5e-5
    # against the one-problem entry point with the same cube
    one = Plan(600, Params.default(p=P_, theta=TH, ncrit=NC, periodic=1, box_min=np.ones(3), box_len=1.0, images=3))
    up, sp_ = one.eval(to_dev(cloud["pos"]), to_dev(g), sigma_uniform=0.07)
    assert rel_l2(u[off[1]:off[2]], up.cpu().numpy()) < PLAIN_VS_BATCH
    # alone
    ua, sa = _run_batch(plan, np.array([0, 600]), cloud["pos"], g, sig[1:2], boxes=boxes[1:2])
    assert np.array_equal(ua, u[off[1]:off[2]]) and np.array_equal(sa, s[off[1]:off[2]])


def test_batch_per_particle_sigma():
    from oracle import direct as od
    from paper_1106_5273_gb300 import Plan, Params
    probs = []
    for k, n in enumerate([900, 2500]):
        w = workloads.plummer(n, seed=900 + k)
        w["sigma_arr"] = (w["sigma"] * np.linspace(0.7, 1.3, n)).astype(np.float32)
        probs.append(w)
    off, pos, gam, _, sarr = _concat(probs, per_particle_sigma=True)
    plan = Plan(int(off[-1]), Params.default(p=8, theta=0.5, ncrit=16))
    u, s = _run_batch(plan, off, pos, gam, sarr=sarr)
    for k, w in enumerate(probs):
        ud, sd = od.direct(w["pos"], w["gamma"], w["pos"], w["gamma"], w["sigma_arr"], skip_self=True)
        assert rel_l2(u[off[k]:off[k + 1]], ud) < 2e-4 and rel_l2(s[off[k]:off[k + 1]], sd) < 1e-3


def test_batch_mixed_core_width_alone_and_in_the_mix():
    """Per-particle widths with the mixed rule (FMM_SIGMA_MIXED) in a batch:
    each problem against the FP64 pair sum with the same rule, and bit-identical
    alone and in the mix."""
    from oracle import pairs
    from paper_1106_5273_gb300 import FMM_SIGMA_MIXED, Plan, Params
    probs = []
    for k, n in enumerate([700, 1800]):
        w = workloads.plummer(n, seed=950 + k)
        w["sigma_arr"] = (w["sigma"] * np.linspace(1.3, 0.7, n)).astype(np.float32)
        probs.append(w)
    off, pos, gam, _, sarr = _concat(probs, per_particle_sigma=True)
    plan = Plan(int(off[-1]), Params.default(p=8, theta=0.5, ncrit=16, sigma_rule=FMM_SIGMA_MIXED))
    u, s = _run_batch(plan, off, pos, gam, sarr=sarr)
    for k, w in enumerate(probs):
        n = w["pos"].shape[0]
        x, g, sg = (a.astype(np.float64) for a in (w["pos"], w["gamma"], w["sigma_arr"]))
        ud, sd = pairs.pair_sum(x, g, x, g, sg, None, np.eye(n, dtype=bool), sig_t=sg)
        assert rel_l2(u[off[k]:off[k + 1]], ud) < 2e-4 and rel_l2(s[off[k]:off[k + 1]], sd) < 1e-3
        ua, sa = _run_batch(plan, np.array([0, n]), w["pos"], w["gamma"], sarr=w["sigma_arr"])
        assert np.array_equal(ua, u[off[k]:off[k + 1]]) and np.array_equal(sa, s[off[k]:off[k + 1]])


def test_autotune_ncrit_picks_the_fastest_candidate():
    """fmm_autotune_ncrit times each candidate leaf size on the sample batch and
    returns the fastest; the batch evaluated with it matches the direct sum."""
    import torch
    from oracle import direct as od
    from paper_1106_5273_gb300 import Params, Plan, autotune_ncrit
    probs = _free_problems()[2:5]
    off, pos, gam, sig, _ = _concat(probs)
    prm = Params.default(p=8, theta=0.5, ncrit=64)
    best, ms = autotune_ncrit(prm, off, to_dev(pos), to_dev(gam), sig, candidates=(16, 32, 64, 128), reps=2)
    assert best in (16, 32, 64, 128) and set(ms) == {16, 32, 64, 128}
    assert all(v > 0 for v in ms.values()) and ms[best] == min(ms.values())
    plan = Plan(int(off[-1]), Params.default(p=8, theta=0.5, ncrit=best))
    u, s = plan.eval_batch(off, to_dev(pos), to_dev(gam), sigma_prob=sig)
    torch.cuda.synchronize()
    u = u.cpu().numpy()
    for k in range(len(probs)):
        a, b = int(off[k]), int(off[k + 1])
        if b - a < 2:
            continue
        ud, _ = od.direct(pos[a:b], gam[a:b], pos[a:b], gam[a:b], float(sig[k]), skip_self=True)
        assert rel_l2(u[a:b], ud) < 2e-4
    plan.close()


def test_autotune_plan_picks_leaf_size_and_p2p_tile():
    """fmm_autotune_plan times every (ncrit, p2p_tpl) pair and returns the
    fastest.  The one- and two-targets-per-lane P2P kernels evaluate the same
    pair terms (staged in chunks of 32 or 64 sources, so the sums are ordered
    differently): their results agree to FP32 rounding."""
    import torch
    from paper_1106_5273_gb300 import Params, Plan, autotune_plan
    probs = _free_problems()[2:5]
    off, pos, gam, sig, _ = _concat(probs)
    prm = Params.default(p=8, theta=0.5, ncrit=64)
    bn, bt, ms = autotune_plan(prm, off, to_dev(pos), to_dev(gam), sig, ncrit=(32, 64, 128), tpl=(1, 2), reps=2)
    assert set(ms) == {(a, b) for a in (32, 64, 128) for b in (1, 2)}
    assert all(v > 0 for v in ms.values()) and ms[(bn, bt)] == min(ms.values())
    outs = []
    for tpl in (1, 2):
        plan = Plan(int(off[-1]), Params.default(p=8, theta=0.5, ncrit=64, p2p_tpl=tpl))
        u, s = plan.eval_batch(off, to_dev(pos), to_dev(gam), sigma_prob=sig)
        torch.cuda.synchronize()
        outs.append((u.cpu().numpy(), s.cpu().numpy()))
        plan.close()
    assert rel_l2(outs[0][0], outs[1][0]) < 1e-6 and rel_l2(outs[0][1], outs[1][1]) < 1e-6


def test_batch_argument_errors():
    import torch
    from paper_1106_5273_gb300 import Plan, Params, FmmError, BATCH_MAX
    plan = Plan(100, Params.default(p=4, ncrit=8))
    x = torch.zeros((100, 3), device="cuda")
    for off in ([1, 10], [0, 20, 10], [0, 200]):
        with pytest.raises(FmmError):
            plan.eval_batch(np.array(off), x, x, sigma_prob=np.ones(len(off) - 1))
    with pytest.raises(FmmError):
        plan.eval_batch(np.array([0, 10]), x, x, sigma_prob=np.array([0.0]))
    with pytest.raises(FmmError):
        plan.eval_batch(np.zeros(BATCH_MAX + 2, np.int64), x, x, sigma_prob=np.ones(BATCH_MAX + 1))
    per = Plan(100, Params.default(p=4, ncrit=8, periodic=1, box_len=1.0))
    with pytest.raises(FmmError):
        per.eval_batch(np.array([0, 10]), x, x, sigma_prob=np.ones(1))
    # all problems empty: nothing to do
    plan.eval_batch(np.array([0, 0, 0]), x, x, sigma_prob=np.ones(2))

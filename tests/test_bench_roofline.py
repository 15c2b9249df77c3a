"""The roofline arithmetic of bench.py on synthetic counts (no GPU).

P2P: achieved = sum over classes of flops per pair x pairs / time, against
152 SMs x 128 FP32 lanes x 2 x 2070 MHz.  M2L: useful flops per pair
2 P x 3 x (3 K3 + (P - K3)); issued = every 128 x 192 x 16 MMA, 3 per K step
of 16 for the first K3 coefficients and 1 per K step after them, per row
block of 128.
"""
import types

import pytest


@pytest.fixture()
def bench(monkeypatch):
    import bench as b
    monkeypatch.setattr(b, "bf16_peak", lambda: (1000.0, "test"))
    return b


def test_p2p_roofline_counts_flops_by_class(bench):
    st = types.SimpleNamespace(p2p_pairs_near=1e9, p2p_pairs_mid=2e9, p2p_pairs_far=3e9, p2p_pairs=6e9)
    r = bench.p2p_roofline(st, 10.0)
    flops = 56 * 1e9 + 55 * 2e9 + 41 * 3e9
    assert r["achieved"] == pytest.approx(flops / 10e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


@pytest.mark.parametrize("p,k3,mmas", [(10, 64, 15), (10, 100, 21), (8, 64, 12), (12, 64, 2 * (12 + 5)),
                                       (12, 144, 2 * 27)])
def test_m2l_roofline_useful_and_issued(bench, p, k3, mmas):
    P = p * p
    st = types.SimpleNamespace(ms_m2l=4.0, m2l_tensor=1, m2l_split_coefs=k3, m2l_pairs=1e6, m2l_steps=1e4)
    r = bench.m2l_roofline(st, p)
    useful = 2.0 * P * 3 * (3 * k3 + (P - k3)) * 1e6
    assert r["achieved"] == pytest.approx(useful / 4e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert r["issued"]["mmas_per_step"] == mmas
    assert r["issued"]["achieved"] == pytest.approx(2.0 * 128 * 192 * 16 * mmas * 1e4 / 4e-3 / 1e12)


def test_m2l_roofline_absent_without_tensor_m2l(bench):
    st = types.SimpleNamespace(ms_m2l=4.0, m2l_tensor=0, m2l_split_coefs=0, m2l_pairs=1, m2l_steps=1)
    assert bench.m2l_roofline(st, 10) is None

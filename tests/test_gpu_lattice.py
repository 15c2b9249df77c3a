"""The periodic lattice operator (Sec. 3.5), built by plans on the device in
FP64: against the same sums built on the host, and through whole periodic
FMM evaluations against the oracle FMM (whose lattice sum uses Cartesian
Taylor expansions) with 3 and 5 lattice levels.  Marked gpu."""
import math

import numpy as np
import pytest

import workloads
from gpu_common import rel_l2, run_fmm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("p,images", [(4, 3), (10, 3), (10, 5), (16, 2)])
def test_device_lattice_operator_matches_host_build(p, images):
    from paper_1106_5273_gb300 import binding
    a_dev = binding.lattice_operator(p, images, on_device=True)
    a_host = binding.lattice_operator(p, images, on_device=False)
    assert np.isfinite(a_dev).all() and np.abs(a_host).max() > 0
    # the same FP64 sums in a different order of the (k, l) terms: rounding only
    assert np.abs(a_dev - a_host).max() <= 1e-12 * np.abs(a_host).max()


@pytest.mark.parametrize("images", [3, 5])
def test_periodic_cloud_with_net_dipole_matches_oracle_fmm(images):
    """A random periodic cloud whose strengths sum to zero but whose dipole
    sum x x gamma does not vanish, p=8: the GPU FMM against the oracle FMM on
    the same lists, with 3 and with 5 lattice levels."""
    from oracle import fmm as ofmm
    L = 2 * math.pi
    c = workloads.random_cloud(700, seed=33, box=L, zero_net=True)
    g = c["gamma"] - c["gamma"].astype(np.float64).mean(0).astype(np.float32)
    w = dict(pos=c["pos"], gamma=g, sigma=np.float32(0.4), periodic=True, box_min=np.zeros(3), box_len=L)
    plan, u, s = run_fmm(w, 8, 0.5, 16, m2l_mode=1, images=images)
    ref = ofmm.fmm(w["pos"], g, 0.4, 8, 0.5, 16, periodic=True, box_min=np.zeros(3), box_len=L, images=images)
    assert rel_l2(u, ref.u) < 2e-5 and rel_l2(s, ref.s) < 5e-5

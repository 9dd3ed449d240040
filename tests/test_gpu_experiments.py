"""The paper's experiments in synthetic form (Sec. V, Figs. 4-6; the Ford/KITTI data are not
available): the MI cost surface around the true pose peaks at the truth for both features,
and a coarse lattice search followed by Nelder-Mead recovers a pose several metres away.
Surface values are checked against the oracle on the same poses."""
import math

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, lowest_argmax, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()
FEATURES = {"MI-N": dict(feature=0, count_levels=7, var_levels=1),
            "MI-VARZ": dict(feature=1, count_levels=1, var_levels=15)}


@pytest.fixture(scope="module")
def pair():
    T = np.array([1.3, -0.7, 0.0, 0.0, 0.0, math.radians(4.0)])
    return scangen.lidar_pair(seed=scangen.SEED_BASE + 90, T=T, n_beams=32)


@pytest.mark.parametrize("fname", list(FEATURES))
def test_cost_surface_peaks_at_truth(pair, fname):
    """MI over (t_x, t_y) within +-4 m of the truth at 0.5 m, and over the heading within
    +-20 deg at 1 deg (other parameters at the truth), 1 m voxels (Fig. 6's setting): the
    maximum is at the truth, and the GPU values match the oracle's."""
    from paper_1709_06948_gb300 import align
    spec = scangen.lidar_grid(1.0)
    L = lib_grid(spec, **FEATURES[fname])
    align.align_set_reference(L, pair.xyzA)
    g = np.arange(-4.0, 4.0001, 0.5)
    etas = np.repeat(pair.T[None, :], len(g) * len(g), 0)
    etas[:, 0] += np.repeat(g, len(g))
    etas[:, 1] += np.tile(g, len(g))
    h = np.radians(np.arange(-20.0, 20.0001, 1.0))
    eh = np.repeat(pair.T[None, :], len(h), 0)
    eh[:, 5] += h
    G = oracle_grid(spec, **FEATURES[fname])
    symA, boxA = G.reference(pair.xyzA)
    for e, centre in ((etas, len(g) * len(g) // 2), (eh, len(h) // 2)):
        mi, am, _ = align.align_eval_mi(L, pair.xyzB, eta6=e)
        assert am == lowest_argmax(mi)
        assert am == centre, (fname, am, centre)
        mo, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(e), nthreads=NT)
        assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
        assert int(oracle.argmax(mo)) == centre


def test_search_then_nelder_mead_recovers_a_large_offset():
    """A 5 m / 6 deg offset: lattice search (+-10 m, +-25 deg yaw) then Nelder-Mead, 1 m
    voxels, z-variance feature (MI-VARZ): final translation error below 0.5 m, heading error
    below 1 deg."""
    from paper_1709_06948_gb300 import align
    T = np.array([3.0, 4.0, 0.05, 0.0, 0.0, math.radians(6.0)])
    p = scangen.lidar_pair(seed=scangen.SEED_BASE + 91, T=T, n_beams=32)
    spec = scangen.lidar_grid(1.0)
    L = lib_grid(spec, **FEATURES["MI-VARZ"])
    align.align_set_reference(L, p.xyzA)
    rngs = np.array([10.0, 10.0, 0.5, math.radians(2.0), math.radians(2.0), math.radians(25.0)])
    Ts, _, _ = align.align_search(L, p.xyzB, np.zeros(6), rngs, levels=5, counts=(12, 12, 2, 2, 2, 12))
    Tn, _, _ = align.align_refine_nm(L, p.xyzB, Ts[None, :], step=np.array([0.5, 0.5, 0.2, 0.01, 0.01, 0.03]),
                                     max_iter=60)
    assert np.linalg.norm(Tn[0][:2] - T[:2]) < 0.5
    assert abs(Tn[0][5] - T[5]) < math.radians(1.0)

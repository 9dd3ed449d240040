"""align_search (coarse-to-fine lattice standing in for Algorithm 1's Nelder-Mead loop)
against the oracle's search with the same schedule."""
import math

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()


def _both(pair, init, rng, counts, levels):
    from paper_1709_06948_gb300 import align
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    L = lib_grid(pair.grid)
    align.align_set_reference(L, pair.xyzA)
    T, mi, lb = align.align_search(L, pair.xyzB, init, rng, levels=levels, counts=counts)
    To, mio, lbo = G.search(symA, boxA, pair.xyzB, init, rng, counts=counts, levels=levels, nthreads=NT)
    return T, mi, lb, To, mio, lbo


def test_search_tiny_matches_oracle():
    T_true = np.array([0.35, -0.6, 0.1, math.radians(1.0), math.radians(-1.5), math.radians(3.0)])
    pair = scangen.tiny_pair(T=T_true)
    rng = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])
    T, mi, lb, To, mio, lbo = _both(pair, np.zeros(6), rng, (3, 3, 3, 3, 3, 3), 4)
    assert lb.tolist() == lbo.tolist()
    assert T.tolist() == To.tolist()
    assert abs(mi - mio) <= 1e-5
    assert np.all(np.abs(T[:2] - T_true[:2]) <= 0.3)


def test_search_lidar_matches_oracle_and_recovers():
    pair = scangen.lidar_pair()
    rng = np.array([2.0, 2.0, 0.25, math.radians(1.0), math.radians(1.0), math.radians(5.0)])
    T, mi, lb, To, mio, lbo = _both(pair, np.zeros(6), rng, (8, 8, 2, 2, 2, 8), 3)
    assert lb.tolist() == lbo.tolist()
    assert T.tolist() == To.tolist()
    assert abs(mi - mio) <= 1e-5
    # third level step: 4 m / 7 / 4 in x, y
    assert np.hypot(T[0] - pair.T[0], T[1] - pair.T[1]) <= 0.5


def test_search_default_counts_runs():
    from paper_1709_06948_gb300 import align
    pair = scangen.tiny_pair()
    L = lib_grid(pair.grid)
    align.align_set_reference(L, pair.xyzA)
    T, mi, _ = align.align_search(L, pair.xyzB, np.zeros(6), [1, 1, 0.5, 0.04, 0.04, 0.09], levels=2)
    assert np.all(np.isfinite(T)) and mi > 0


@pytest.mark.parametrize("counts,levels", [((3, 3, 3, 3, 3, 3), 1), ((3, 3, 3, 3, 3, 3), 2),
                                           ((2, 2, 2, 4, 4, 4), 5), ((2, 3, 1, 1, 5, 3), 3),
                                           ((1, 1, 1, 12, 12, 1), 2)])
def test_search_schedules_match_oracle(counts, levels):
    """Levels built on the device (small rotation lattices) and level by level on the host
    (a 144-rotation lattice) give the oracle's choices at every level."""
    T_true = np.array([-0.4, 0.5, -0.1, math.radians(-1.0), math.radians(2.0), math.radians(-4.0)])
    pair = scangen.tiny_pair(T=T_true)
    rng = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])
    T, mi, lb, To, mio, lbo = _both(pair, np.array([0.1, -0.1, 0.0, 0.0, 0.01, -0.02]), rng, counts, levels)
    assert lb.tolist() == lbo.tolist()
    assert T.tolist() == To.tolist()
    assert abs(mi - mio) <= 1e-5

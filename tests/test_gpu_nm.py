"""Nelder-Mead refinement (Algorithm 1's optimiser) on the GPU against the oracle's
Nelder-Mead with FP64 MI: the same vertex decisions (identical histograms give equal MI on
both sides, so ties resolve alike), hence the same final poses, and MI within 1e-5 nats.
The oracle's Nelder-Mead is itself pinned to SciPy's (tests/test_oracle_pins.py)."""
import math

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
STEP_TINY = np.array([1.0, 1.0, 0.5, 0.05, 0.05, 0.1])


def _setup(pair):
    from paper_1709_06948_gb300 import align
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    L = lib_grid(pair.grid)
    align.align_set_reference(L, pair.xyzA)
    return G, symA, boxA, L


def test_nm_tiny_matches_oracle():
    from paper_1709_06948_gb300 import align
    pair = scangen.tiny_pair(T=np.array([0.35, -0.6, 0.1, math.radians(1.0), math.radians(-1.5),
                                         math.radians(3.0)]))
    G, symA, boxA, L = _setup(pair)
    starts = np.array([[0, 0, 0, 0, 0, 0], [0.3, -0.3, 0, 0, 0, 0.02], [-0.4, 0.2, 0.1, 0.01, 0, -0.03]],
                      dtype=np.float64)
    T, mi, it = align.align_refine_nm(L, pair.xyzB, starts, step=STEP_TINY, max_iter=25)
    for k in range(len(starts)):
        To, mio, ito = G.nm(symA, boxA, pair.xyzB, starts[k], STEP_TINY, 25)
        assert it[k] == ito == 25
        assert T[k].tolist() == To.tolist()
        assert abs(float(mi[k]) - mio) <= mi_tolerance()


def test_nm_ftol_stop_and_improvement():
    from paper_1709_06948_gb300 import align
    pair = scangen.tiny_pair(T=np.array([0.35, -0.6, 0.1, math.radians(1.0), math.radians(-1.5),
                                         math.radians(3.0)]))
    G, symA, boxA, L = _setup(pair)
    starts = np.zeros((2, 6))
    T, mi, it = align.align_refine_nm(L, pair.xyzB, starts, step=STEP_TINY, max_iter=400, ftol=1e-7)
    To, mio, ito = G.nm(symA, boxA, pair.xyzB, starts[0], STEP_TINY, 400, ftol=1e-7)
    assert it[0] == it[1] and it[0] < 400 and it[0] == ito
    assert T[0].tolist() == To.tolist()
    mi0, _, _ = align.align_eval_mi(L, pair.xyzB, eta6=np.zeros((1, 6)))
    assert mi[0] >= mi0[0]
    assert np.hypot(T[0][0] - 0.35, T[0][1] + 0.6) < 0.5


def test_nm_lidar_matches_oracle_from_lattice_argmax():
    """Seeded from a coarse lattice search, as a refinement stage would be."""
    from paper_1709_06948_gb300 import align
    pair = scangen.lidar_pair(seed=scangen.SEED_BASE + 71, n_beams=32)
    G, symA, boxA, L = _setup(pair)
    rng = np.array([2.0, 2.0, 0.25, math.radians(1.0), math.radians(1.0), math.radians(5.0)])
    T0, _, _ = align.align_search(L, pair.xyzB, np.zeros(6), rng, levels=2)
    step = np.array([0.3, 0.3, 0.1, 0.005, 0.005, 0.02])
    T, mi, it = align.align_refine_nm(L, pair.xyzB, T0[None, :], step=step, max_iter=12)
    To, mio, ito = G.nm(symA, boxA, pair.xyzB, T0, step, 12)
    assert T[0].tolist() == To.tolist()
    assert abs(float(mi[0]) - mio) <= mi_tolerance()


def test_nm_zero_simplices_and_errors():
    from paper_1709_06948_gb300 import align
    pair = scangen.tiny_pair()
    _, _, _, L = _setup(pair)
    T, mi, it = align.align_refine_nm(L, pair.xyzB, np.zeros((0, 6)))
    assert T.shape == (0, 6)
    with pytest.raises(align.AlignError) as e:
        align.align_refine_nm(L, pair.xyzB, np.full((1, 6), np.nan))
    assert e.value.status == align.ALIGN_E_INVALID

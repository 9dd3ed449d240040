"""Serving (align_server_*): requests admitted into slots as they free up, each slot running
its request's device-pipelined search on its own stream.  Each request's result is the same
alone and in a mix of concurrent requests, and the same as align_search_ex on its own grid
(itself pinned to the oracle's search); the tiny request also against the oracle directly.
Admission by slots and by the device memory budget; polling semantics."""
import math
import time

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()
COUNTS = (4, 4, 2, 2, 2, 4)
RNG_L = np.array([2.0, 2.0, 0.25, math.radians(1.0), math.radians(1.0), math.radians(5.0)])
RNG_T = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])


class World:
    def __init__(self):
        rng = np.random.default_rng(61)
        self.tiny = scangen.tiny_pair(T=np.array([0.35, -0.6, 0.1, math.radians(1.0), math.radians(-1.5),
                                                   math.radians(3.0)]))
        self.lp = scangen.lidar_pair(seed=scangen.SEED_BASE + 62, n_beams=32)
        self.refs = [(self.tiny.xyzA, self.tiny.grid), (self.lp.xyzA, scangen.lidar_grid(1.0)),
                     (self.lp.xyzA, scangen.lidar_grid(0.5))]
        # requests: (ref index, B, init, range, levels)
        self.reqs = [(0, self.tiny.xyzB, np.zeros(6), RNG_T, 3)]
        for k in range(7):
            ref = 1 + k % 2
            n = int(rng.integers(8000, 30000))
            B = scangen.subsample(self.lp.xyzB, n, rng)
            init = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 0, 0, 0, rng.uniform(-0.02, 0.02)])
            self.reqs.append((ref, B, init, RNG_L, 2 + k % 3))
        self._alone = None

    def make_server(self, budget=8 << 30, slots=64):
        from paper_1709_06948_gb300 import align
        s = align.align_server_create(budget, slots)
        ids = [align.align_server_add_reference(s, A, spec.origin, spec.res_m, spec.dims, spec.feature,
                                                spec.count_levels, spec.var_levels) for A, spec in self.refs]
        return s, ids

    def standalone(self):
        """align_search_ex of every request on its own grid."""
        if self._alone is None:
            from paper_1709_06948_gb300 import align
            grids = []
            for A, spec in self.refs:
                L = lib_grid(spec)
                align.align_set_reference(L, A)
                grids.append(L)
            self._alone = []
            for ref, B, init, rng, levels in self.reqs:
                T, mi, _ = align.align_search(grids[ref], B, init, rng, levels=levels, counts=COUNTS)
                self._alone.append((T, mi))
        return self._alone


@pytest.fixture(scope="module")
def world():
    return World()


def _submit(align, s, ids, req):
    ref, B, init, rng, levels = req
    return align.align_submit(s, ids[ref], B, init, rng, levels=levels, counts=COUNTS)


def test_each_request_alone_matches_search(world):
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server()
    for req, (T, mi) in zip(world.reqs, world.standalone()):
        r = align.align_wait(s, _submit(align, s, ids, req), 60000)
        assert r["status"] == 0
        assert r["T"].tolist() == T.tolist() and r["mi"] == mi
    st = align.align_server_stats(s)
    assert st["max_active"] == 1 and st["done"] == len(world.reqs)
    s.close()


def test_tiny_request_matches_oracle(world):
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server()
    r = align.align_wait(s, _submit(align, s, ids, world.reqs[0]), 60000)
    G = oracle_grid(world.tiny.grid)
    symA, boxA = G.reference(world.tiny.xyzA)
    To, mio, _ = G.search(symA, boxA, world.tiny.xyzB, np.zeros(6), RNG_T, counts=COUNTS, levels=3, nthreads=NT)
    assert r["T"].tolist() == To.tolist() and abs(r["mi"] - mio) <= 1e-5
    s.close()


def test_mix_runs_concurrently_and_results_unchanged(world):
    """All requests submitted at once: several run at the same time (their intervals from
    admission to completion overlap) and each result is bit-identical to the request run
    alone."""
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server()
    tickets = [_submit(align, s, ids, req) for req in world.reqs]
    res = [align.align_wait(s, t, 120000) for t in tickets]
    st = align.align_server_stats(s)
    for r, (T, mi) in zip(res, world.standalone()):
        assert r["status"] == 0
        assert r["T"].tolist() == T.tolist() and r["mi"] == mi
    total_levels = sum(req[4] for req in world.reqs)
    assert st["max_active"] > 1 and st["steps"] == total_levels
    overlaps = sum(1 for a in res for b in res if a is not b and a["t_start"] < b["t_done"] and b["t_start"] < a["t_done"])
    assert overlaps > 0
    assert st["admitted"] == len(world.reqs) and st["queued"] == 0
    s.close()


def test_staggered_arrivals_join_running_batches(world):
    """Requests arriving while others run are admitted between steps."""
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server()
    tickets = []
    for req in world.reqs:
        tickets.append(_submit(align, s, ids, req))
        time.sleep(0.002)
    res = [align.align_wait(s, t, 120000) for t in tickets]
    for r, (T, mi) in zip(res, world.standalone()):
        assert r["T"].tolist() == T.tolist() and r["mi"] == mi
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    s.close()


def test_memory_budget_limits_admission(world):
    from paper_1709_06948_gb300 import align
    probe, ids = world.make_server(slots=1)
    base = align.align_server_stats(probe)["bytes_held"]  # the references
    probe.close()

    # room for the references and the largest of three requests, not for two of them (a
    # request's bytes as the server estimates them: what its slot holds after running it alone)
    def est(req):
        p, pid = world.make_server(slots=1)
        align.align_wait(p, _submit(align, p, pid, req), 60000)
        held = align.align_server_stats(p)["bytes_held"] - base
        p.close()
        return held
    sizes = sorted(est(r) for r in world.reqs[1:4])
    assert sizes[0] + sizes[1] > sizes[2]
    s, ids = world.make_server(budget=base + sizes[2], slots=64)
    tickets = [_submit(align, s, ids, req) for req in world.reqs[1:4]]
    res = [align.align_wait(s, t, 120000) for t in tickets]
    st = align.align_server_stats(s)
    assert st["max_active"] == 1
    for r, (T, mi) in zip(res, world.standalone()[1:4]):
        assert r["T"].tolist() == T.tolist() and r["mi"] == mi
    big = np.zeros((2_000_000, 3), np.float32)
    with pytest.raises(align.AlignError) as e:
        align.align_submit(s, ids[2], big, np.zeros(6), RNG_L, levels=1, counts=COUNTS)
    assert e.value.status == align.ALIGN_E_OOM
    s.close()


def test_slot_limit(world):
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server(slots=2)
    tickets = [_submit(align, s, ids, req) for req in world.reqs]
    res = [align.align_wait(s, t, 120000) for t in tickets]
    assert align.align_server_stats(s)["max_active"] <= 2
    for r, (T, mi) in zip(res, world.standalone()):
        assert r["T"].tolist() == T.tolist()
    s.close()


def test_poll_and_errors(world):
    from paper_1709_06948_gb300 import align
    s, ids = world.make_server()
    t = _submit(align, s, ids, world.reqs[1])
    r = None
    for _ in range(20000):
        r = align.align_poll(s, t)
        if r is not None:
            break
        time.sleep(0.001)
    assert r is not None and r["status"] == 0
    with pytest.raises(align.AlignError):
        align.align_poll(s, t)  # delivered once
    t0 = align.align_submit(s, ids[0], world.tiny.xyzB, np.ones(6), RNG_T, levels=0, counts=COUNTS)
    r0 = align.align_wait(s, t0, 1000)
    assert r0["T"].tolist() == [1.0] * 6
    with pytest.raises(align.AlignError) as e:
        align.align_submit(s, 99, world.tiny.xyzB, np.zeros(6), RNG_T, levels=1)
    assert e.value.status == align.ALIGN_E_INVALID
    s.close()

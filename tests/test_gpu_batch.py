"""Many pairs in one launch sequence (align_eval_batch: one packing launch, an eval launch per
pair, one composition and one argmax launch; capturable as one CUDA graph) against the
oracle and against align_eval_mi on each pair alone: grids of different resolutions,
features and symbol counts in one batch; empty inputs; graph capture and replay; every
kernel shape with one and two poses per CTA; the tuner; device-resident inputs and outputs.

Bar: each pair's MI within 1e-5 nats of the oracle's FP64 MI and its argmax equal (or
within the FP32 band); bit-identical MI and argmax to the same pair evaluated alone."""
import math

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import check_argmax, lib_grid, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()


class Case:
    def __init__(self, xyzA, xyzB, spec, etas):
        from paper_1709_06948_gb300 import align
        self.spec, self.xyzA, self.xyzB, self.etas = spec, xyzA, xyzB, etas
        self.L = lib_grid(spec)
        align.align_set_reference(self.L, xyzA)
        self._oracle = None

    def oracle_mi(self):
        if self._oracle is None:
            G = oracle_grid(self.spec)
            symA, boxA = G.reference(self.xyzA)
            mo, _, _ = G.eval_mi(symA, boxA, self.xyzB, G.round_pose(self.etas), nthreads=NT)
            self._oracle = mo
        return self._oracle


@pytest.fixture(scope="module")
def cases():
    rng = np.random.default_rng(51)
    out = []
    t = scangen.tiny_pair()
    out.append(Case(t.xyzA, t.xyzB, t.grid, scangen.tiny_poses()[::3]))
    t2 = scangen.tiny_pair(seed=scangen.SEED_BASE + 52, n=3000)
    out.append(Case(t2.xyzA, t2.xyzB, t2.grid, scangen.tiny_poses()[::7]))
    lp = scangen.lidar_pair(seed=scangen.SEED_BASE + 53, n_beams=32)
    for res in (1.0, 0.5):
        spec = scangen.lidar_grid(res)
        B = scangen.subsample(lp.xyzB, 30000 if res == 1.0 else 45000, rng)
        etas = scangen.lidar_poses(center=lp.T, half_width=(1.0, 1.0, 0.1, 0.01, 0.01, 0.05))[::29]
        out.append(Case(lp.xyzA, B, spec, etas))
    joint = scangen.GridSpec(origin=(-40.0, -40.0, -1.0), res_m=0.5, dims=(160, 160, 16), feature=2,
                             count_levels=7, var_levels=8)
    out.append(Case(lp.xyzA, lp.xyzB[:20000], joint, scangen.lidar_poses(center=lp.T)[::97]))
    return out


def _pairs(cases):
    return [(c.L, c.xyzB, c.etas) for c in cases]


def test_batch_matches_oracle_and_single(cases):
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    res = align.align_eval_batch(b, _pairs(cases))
    for c, (mi, am) in zip(cases, res):
        mo = c.oracle_mi()
        assert mi.shape == (len(c.etas),)
        assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
        check_argmax(am, mo, mi)
        mi1, am1, _ = align.align_eval_mi(c.L, c.xyzB, eta6=c.etas)
        assert np.array_equal(mi, mi1) and am == am1
    st = align.align_batch_stats(b)
    # one batch launch: pack, compose, argmax, and an eval + redo kernel per pair
    assert st["launches"] == 1 and st["kernel_launches"] == 3 + 2 * len(cases)


def test_every_shape_same_result(cases):
    """Every kernel shape, one pose or two poses per CTA: identical results."""
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    align.align_batch_set_poses_per_cta(b, 1)
    ref = align.align_eval_batch(b, _pairs(cases))
    assert align.align_batch_stats(b)["poses_per_cta"] == 1
    for shape in range(3):
        for ppc in (1, 2):
            align.align_batch_set_shape(b, shape)
            align.align_batch_set_poses_per_cta(b, ppc)
            res = align.align_eval_batch(b, _pairs(cases))
            st = align.align_batch_stats(b)
            # pairs need pre-rotated tiles, which one of these pairs' pose sets rules out
            assert st["shape"] == shape and st["poses_per_cta"] in ((1,) if ppc == 1 else (1, 2))
            for (mi0, am0), (mi, am) in zip(ref, res):
                assert np.array_equal(mi0, mi) and am0 == am


def test_pose_pairs_in_a_batch():
    """Lattice pose sets (rotations repeat): with two poses per CTA every pair's lattice is
    evaluated as pose pairs; results equal one pose per CTA, align_eval_mi alone, and the
    oracle on a sample."""
    from paper_1709_06948_gb300 import align
    cases = []
    for k, res in enumerate((0.5, 1.0, 0.5)):
        lp = scangen.lidar_pair(seed=scangen.SEED_BASE + 80 + k, n_beams=32)
        spec = scangen.lidar_grid(res)
        etas = scangen.pose_grid(lp.T, (0.8, 0.8, 0.1, 0.01, 0.01, 0.04), (8, 4, 2, 1, 1, 2))
        cases.append(Case(lp.xyzA, lp.xyzB, spec, etas))
    b = align.align_batch_create()
    align.align_batch_set_poses_per_cta(b, 2)
    res2 = align.align_eval_batch(b, _pairs(cases))
    assert align.align_batch_stats(b)["poses_per_cta"] == 2
    align.align_batch_set_poses_per_cta(b, 1)
    res1 = align.align_eval_batch(b, _pairs(cases))
    assert align.align_batch_stats(b)["poses_per_cta"] == 1
    for c, (mi2, am2), (mi1, am1) in zip(cases, res2, res1):
        assert np.array_equal(mi2, mi1) and am2 == am1
        mi0, am0, _ = align.align_eval_mi(c.L, c.xyzB, eta6=c.etas)
        assert np.array_equal(mi2, mi0) and am2 == am0
        mo = c.oracle_mi()
        assert np.max(np.abs(mi2.astype(np.float64) - mo)) <= mi_tolerance()
        check_argmax(am2, mo, mi2)


def test_key_partitions_in_a_batch():
    """Pairs on a 0.25 m grid whose single poses need key partitions: after the grid has
    learned them, the batch sweeps B once per pose and queues the later partitions' runs
    (spill queues, as align_eval_mi does); with the queues switched off on the grid it sweeps
    B once per partition; with two poses per CTA it sweeps pose pairs, queued as well.  All
    batches, align_eval_mi alone and the oracle on a sample agree (MI and argmax
    bit-identical between the library's paths)."""
    from paper_1709_06948_gb300 import align
    pair = scangen.lidar_pair()
    spec = scangen.lidar_grid(0.25)
    etas = scangen.lidar_poses()[::8]
    c = Case(pair.xyzA, pair.xyzB, spec, etas)
    small = Case(pair.xyzA, scangen.subsample(pair.xyzB, 20000, np.random.default_rng(84)), spec, etas[::4])
    for _ in range(2):  # the grid learns its partitions (and that pose pairs need more)
        align.align_eval_mi(c.L, c.xyzB, eta6=c.etas)
    assert align.align_eval_stats(c.L)["passes"] >= 2
    b = align.align_batch_create()
    align.align_batch_set_shape(b, 0)  # the shape whose partitions the grid learned
    align.align_batch_set_poses_per_cta(b, 1)
    res_q = align.align_eval_batch(b, _pairs([c, small]))
    align.align_set_spill(c.L, False)
    res_p = align.align_eval_batch(b, _pairs([c, small]))
    align.align_set_spill(c.L, True)
    # pose pairs (their own partitions, queued as well) give the same results
    align.align_batch_set_poses_per_cta(b, 2)
    res_2 = align.align_eval_batch(b, _pairs([c, small]))
    assert align.align_batch_stats(b)["poses_per_cta"] == 2
    for cc, (mi_q, am_q), (mi_p, am_p), (mi_2, am_2) in zip((c, small), res_q, res_p, res_2):
        assert np.array_equal(mi_q, mi_p) and am_q == am_p
        assert np.array_equal(mi_q, mi_2) and am_q == am_2
        mi0, am0, _ = align.align_eval_mi(cc.L, cc.xyzB, eta6=cc.etas)
        assert np.array_equal(mi_q, mi0) and am_q == am0
    G = oracle_grid(spec)
    symA, boxA = G.reference(c.xyzA)
    sample = np.unique(np.concatenate([[res_q[0][1]], np.arange(0, len(etas), 16)]))
    mo, _, _ = G.eval_mi(symA, boxA, c.xyzB, G.round_pose(etas[sample]), nthreads=NT)
    assert np.max(np.abs(res_q[0][0][sample].astype(np.float64) - mo)) <= mi_tolerance()


def test_graph_replay(cases):
    """Same shape, new poses: the graph is captured once and replayed; results equal the
    non-graph launch."""
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    g = align.align_batch_create()
    shifted = []
    for k in range(3):
        pairs = [(c.L, c.xyzB, c.etas + np.array([0.05 * k, -0.03 * k, 0, 0, 0, 0.002 * k])) for c in cases]
        r_graph = align.align_eval_batch(g, pairs, graph=True)
        r_plain = align.align_eval_batch(b, pairs)
        for (mi0, am0), (mi, am) in zip(r_plain, r_graph):
            assert np.array_equal(mi0, mi) and am0 == am
        shifted.append(r_graph)
    st = align.align_batch_stats(g)
    assert st["graph_captures"] == 1 and st["graph_replays"] == 2


def test_tuner_picks_a_shape_and_caches(cases, tmp_path, monkeypatch):
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    ref = align.align_eval_batch(b, _pairs(cases))
    res = align.align_eval_batch(b, _pairs(cases), tune=True)
    st = align.align_batch_stats(b)
    # every kernel shape x poses per CTA candidate timed once, then cached per batch class
    assert st["tuner_trials"] == 6 and 0 <= st["shape"] < 3 and st["poses_per_cta"] in (1, 2)
    res2 = align.align_eval_batch(b, _pairs(cases), tune=True)
    assert align.align_batch_stats(b)["tuner_trials"] == 6  # cached
    for (mi0, am0), (mi1, am1), (mi2, am2) in zip(ref, res, res2):
        assert np.array_equal(mi0, mi1) and np.array_equal(mi0, mi2) and am0 == am1 == am2


def test_device_inputs_outputs(cases):
    import torch
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    ref = align.align_eval_batch(b, _pairs(cases))
    pairs, outs = [], []
    for c in cases:
        poses = torch.from_numpy(align.align_round_poses(c.spec.origin, c.etas)).cuda()
        pairs.append((c.L, torch.from_numpy(c.xyzB).cuda(), None, poses))
        outs.append((torch.empty(len(c.etas), device="cuda"), torch.empty(1, dtype=torch.int64, device="cuda")))
    align.align_eval_batch(b, pairs, out=outs)
    torch.cuda.synchronize()
    for (mi0, am0), (mi_t, am_t) in zip(ref, outs):
        assert np.array_equal(mi0, mi_t.cpu().numpy()) and am0 == int(am_t.item())


def test_empty_pairs_in_a_batch(cases):
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    c = cases[0]
    pairs = [(c.L, c.xyzB, np.zeros((0, 6))), (c.L, np.zeros((0, 3), np.float32), c.etas), (c.L, c.xyzB, c.etas)]
    res = align.align_eval_batch(b, pairs)
    assert res[0][0].shape == (0,) and res[0][1] == -1
    assert np.all(res[1][0] == 0.0) and res[1][1] == 0
    mi1, am1, _ = align.align_eval_mi(c.L, c.xyzB, eta6=c.etas)
    assert np.array_equal(res[2][0], mi1) and res[2][1] == am1
    assert align.align_eval_batch(b, []) == []


def test_batch_errors(cases):
    from paper_1709_06948_gb300 import align
    b = align.align_batch_create()
    c = cases[0]
    L = lib_grid(c.spec)  # no reference
    with pytest.raises(align.AlignError) as e:
        align.align_eval_batch(b, [(L, c.xyzB, c.etas)])
    assert e.value.status == align.ALIGN_E_NOREF
    bad = c.etas.copy()
    bad[0, 0] = math.nan
    with pytest.raises(align.AlignError) as e:
        align.align_eval_batch(b, [(c.L, c.xyzB, bad)])
    assert e.value.status == align.ALIGN_E_INVALID

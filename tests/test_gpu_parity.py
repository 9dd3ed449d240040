"""GPU path vs the CPU oracle on the same seeded inputs, through the C ABI.

Bar: voxel sums, symbols, boxes, joint histograms bit-exact; MI within 1e-5 nats of the
oracle's FP64 MI; the argmax equal (or, on an FP32 near-tie, within the band).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import check_argmax, lib_grid, lowest_argmax, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()


class Setup:
    def __init__(self, pair):
        from paper_1709_06948_gb300 import align
        self.pair = pair
        self.G = oracle_grid(pair.grid)
        self.symA, self.boxA = self.G.reference(pair.xyzA)
        self.L = lib_grid(pair.grid)
        align.align_set_reference(self.L, pair.xyzA)


@pytest.fixture(scope="module")
def tiny():
    return Setup(scangen.tiny_pair())


@pytest.fixture(scope="module")
def lidar():
    return Setup(scangen.lidar_pair())


def _eval_both(S, etas, with_hist=True, sample=None):
    from paper_1709_06948_gb300 import align
    mi, am, hist = align.align_eval_mi(S.L, S.pair.xyzB, eta6=etas, with_hist=with_hist)
    poses = S.G.round_pose(etas)
    mo, ho, _ = S.G.eval_mi(S.symA, S.boxA, S.pair.xyzB, poses, nthreads=NT, with_hist=with_hist)
    return mi, am, hist, mo, ho


@pytest.mark.parametrize("which", ["tiny", "lidar"])
def test_reference_parity(which, request):
    from paper_1709_06948_gb300 import align
    S = request.getfixturevalue(which)
    sym, box = align.align_get_reference(S.L)
    assert np.array_equal(sym, S.symA)
    assert box.tolist() == S.boxA.tolist()


@pytest.mark.parametrize("which", ["tiny", "lidar"])
def test_accumulate_parity(which, request):
    from paper_1709_06948_gb300 import align
    S = request.getfixturevalue(which)
    etas = [S.pair.T, np.zeros(6), np.array([0.7, -1.3, 0.05, 0.01, -0.02, 0.09])]
    for eta in etas:
        pose = S.G.round_pose(eta)[0]
        acc, box = align.align_accumulate(S.L, S.pair.xyzB, pose)
        cnt, s1, s2, obox, _ = S.G.accumulate(S.pair.xyzB, pose)
        assert np.array_equal(acc[:, 0], cnt)
        assert np.array_equal(acc[:, 1], s1)
        assert np.array_equal(acc[:, 2], s2)
        assert box.tolist() == obox.tolist()


def test_tiny_all_poses(tiny):
    etas = scangen.tiny_poses()
    mi, am, hist, mo, ho = _eval_both(tiny, etas)
    assert np.array_equal(hist, ho)
    assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
    check_argmax(am, mo, mi)


def test_lidar_full_batch(lidar):
    """The benchmark's launch: 4,096 poses on the 120k-point pair; every pose's joint
    histogram is compared bit for bit and every MI within the tolerance."""
    from paper_1709_06948_gb300 import align
    etas = scangen.lidar_poses(center=np.zeros(6))
    mi, am, hist = align.align_eval_mi(lidar.L, lidar.pair.xyzB, eta6=etas, with_hist=True)
    poses = lidar.G.round_pose(etas)
    mo, ho, _ = lidar.G.eval_mi(lidar.symA, lidar.boxA, lidar.pair.xyzB, poses, nthreads=NT, with_hist=True)
    bad = np.flatnonzero([not np.array_equal(hist[i], ho[i]) for i in range(len(etas))])
    assert bad.size == 0, f"histograms differ at poses {bad[:10].tolist()}"
    assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
    check_argmax(am, mo, mi)
    # FP64 MI recomputed from the GPU's histograms is the oracle's MI exactly
    for i in range(0, 4096, 128):
        assert oracle.mi_from_hist(hist[i]) == pytest.approx(mo[i], abs=1e-12)


def test_lidar_truth_lattice(lidar):
    etas = scangen.lidar_poses(center=lidar.pair.T, half_width=(0.5, 0.5, 0.1, 0.01, 0.01, 0.03))[::7]
    mi, am, hist, mo, ho = _eval_both(lidar, etas)
    assert np.array_equal(hist, ho)
    assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
    check_argmax(am, mo, mi)


def test_eta_and_poses12_agree(tiny):
    from paper_1709_06948_gb300 import align
    etas = scangen.tiny_poses()[::5]
    a = align.align_eval_mi(tiny.L, tiny.pair.xyzB, eta6=etas, with_hist=True)
    b = align.align_eval_mi(tiny.L, tiny.pair.xyzB, poses12=tiny.G.round_pose(etas), with_hist=True)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])


def test_device_inputs_outputs(tiny):
    import torch
    from paper_1709_06948_gb300 import align
    etas = scangen.tiny_poses()
    host = align.align_eval_mi(tiny.L, tiny.pair.xyzB, eta6=etas, with_hist=True)
    xyz = torch.from_numpy(tiny.pair.xyzB).cuda()
    poses = torch.from_numpy(tiny.G.round_pose(etas)).cuda()
    P = etas.shape[0]
    mi = torch.empty(P, dtype=torch.float32, device="cuda")
    am = torch.empty(1, dtype=torch.int64, device="cuda")
    hist = torch.empty((P, tiny.L.K, tiny.L.K), dtype=torch.int32, device="cuda")
    align.align_eval_mi(tiny.L, xyz, poses12=poses, out=(mi, am, hist))
    torch.cuda.synchronize()
    assert np.array_equal(mi.cpu().numpy(), host[0])
    assert int(am.item()) == host[1]
    assert np.array_equal(hist.cpu().numpy().view(np.uint32), host[2])


def test_repeat_is_deterministic(lidar):
    from paper_1709_06948_gb300 import align
    etas = scangen.lidar_poses()[::3]
    a = align.align_eval_mi(lidar.L, lidar.pair.xyzB, eta6=etas, with_hist=True)
    b = align.align_eval_mi(lidar.L, lidar.pair.xyzB, eta6=etas, with_hist=True)
    assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])


def test_permuting_poses_permutes_outputs(tiny):
    from paper_1709_06948_gb300 import align
    etas = scangen.tiny_poses()
    perm = np.random.default_rng(2).permutation(len(etas))
    a = align.align_eval_mi(tiny.L, tiny.pair.xyzB, eta6=etas, with_hist=True)
    b = align.align_eval_mi(tiny.L, tiny.pair.xyzB, eta6=etas[perm], with_hist=True)
    assert np.array_equal(a[0][perm], b[0]) and np.array_equal(a[2][perm], b[2])


def test_hand_fixture_on_gpu():
    from paper_1709_06948_gb300 import align
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_4x4x2.json")) as f:
        hand = json.load(f)
    g = hand["grid"]
    for mode in ("zvar", "count"):
        if mode == "zvar":
            L = align.align_create_grid(g["origin"], g["res_m"], g["dims"], align.ALIGN_FEAT_ZVAR,
                                        var_levels=hand["zvar"]["var_levels"], var_thresh=hand["zvar"]["var_thresh"])
        else:
            L = align.align_create_grid(g["origin"], g["res_m"], g["dims"], align.ALIGN_FEAT_COUNT,
                                        count_levels=hand["count"]["count_levels"])
        align.align_set_reference(L, hand["xyzA"])
        sym, box = align.align_get_reference(L)
        assert {int(v): int(sym[v]) for v in np.nonzero(sym)[0]} == {int(k): v for k, v in hand[mode]["symA"].items()}
        assert box.tolist() == hand["boxA"]
        mi, am, hist = align.align_eval_mi(L, hand["xyzB"], eta6=[hand["eta_B"]], with_hist=True)
        assert hist[0].tolist() == hand[mode]["hist"]
        acc, bbox = align.align_accumulate(L, hand["xyzB"], align.align_round_poses(g["origin"], [hand["eta_B"]])[0])
        occ = {int(v): acc[v].tolist() for v in np.nonzero(acc[:, 0])[0]}
        assert occ == {int(k): v for k, v in hand["sumsB"].items()}
        assert bbox.tolist() == hand["boxB"]
        exp = oracle.mi_from_hist(np.array(hand[mode]["hist"]))
        assert abs(mi[0] - exp) <= mi_tolerance()


@pytest.mark.parametrize("res,feature", [(0.5, 1), (1.0, 1), (1.0, 0)])
def test_pose_pairs_match_single_pose_kernel(res, feature):
    """A lattice given as host poses is evaluated two poses per sweep (poses that share their
    rotation, t_y and t_z); the same poses given as device poses go through the single-pose
    kernel.  Histograms and MI must agree bit for bit, for each table layout (three value
    words at 1 m z-variance, the packed two-word layout at 0.5 m, the count-only layout),
    and a sample must match the oracle."""
    import torch
    from paper_1709_06948_gb300 import align
    pair = scangen.lidar_pair(seed=scangen.SEED_BASE + 71, n_beams=32)
    spec = scangen.lidar_grid(res)
    over = dict(feature=feature, count_levels=7, var_levels=15 if feature == 1 else 1)
    L = lib_grid(spec, **over)
    align.align_set_reference(L, pair.xyzA)
    single_slots = align.align_eval_stats(L)["table_slots"]
    etas = scangen.pose_grid(pair.T, (0.8, 0.8, 0.1, 0.01, 0.01, 0.04), (8, 4, 2, 1, 1, 2))
    mi_p, am_p, h_p = align.align_eval_mi(L, pair.xyzB, eta6=etas, with_hist=True)
    assert align.align_eval_stats(L)["table_slots"] != single_slots  # the pair kernel ran
    poses = align.align_round_poses(spec.origin, etas)
    P = len(etas)
    mi_d = torch.empty(P, device="cuda")
    am_d = torch.empty(1, dtype=torch.int64, device="cuda")
    h_d = torch.empty((P, L.K, L.K), dtype=torch.int32, device="cuda")
    align.align_eval_mi(L, torch.from_numpy(pair.xyzB).cuda(), poses12=torch.from_numpy(poses).cuda(),
                        out=(mi_d, am_d, h_d))
    torch.cuda.synchronize()
    assert np.array_equal(h_p, h_d.cpu().numpy().view(np.uint32))
    assert np.array_equal(mi_p, mi_d.cpu().numpy()) and am_p == int(am_d.item())
    G = oracle_grid(spec, **over)
    symA, boxA = G.reference(pair.xyzA)
    sample = np.arange(0, P, 5)
    mo, ho, _ = G.eval_mi(symA, boxA, pair.xyzB, poses[sample], nthreads=NT, with_hist=True)
    assert np.array_equal(h_p[sample], ho)
    assert np.max(np.abs(mi_p[sample].astype(np.float64) - mo)) <= mi_tolerance()


def test_every_sweep_kind_agrees_on_a_fine_grid():
    """The 120k-point LiDAR pair on a 0.25 m grid (320x320x32, z-variance), 4,096 lattice
    poses swept each way the library has (one pose per CTA and pose pairs, each with its key
    partitions' runs queued after one sweep of B, with queues of 64 runs that overflow and
    send the poses to the exact path, or with one sweep per partition; one pose per 2-CTA
    cluster with its table split between two shared memories; the automatic choice),
    each on a fresh grid: MI, argmax and every histogram are identical across the kinds, and
    a sample holding the argmax and every exact-path pose matches the oracle."""
    from paper_1709_06948_gb300 import align
    pair = scangen.lidar_pair()
    spec = scangen.lidar_grid(0.25)
    etas = scangen.lidar_poses()
    P = len(etas)
    runs, must = [], set()
    for kind, spill, queue_runs in ((0, True, 0), (0, True, 64), (0, False, 0), (1, True, 0), (1, True, 64),
                                    (1, False, 0), (2, True, 0), (-1, True, 0)):
        L = lib_grid(spec)
        align.align_set_reference(L, pair.xyzA)
        align.align_set_sweep(L, kind)
        align.align_set_spill(L, spill, queue_runs)
        for i in range(2):  # the second launch starts from the partitions the first learned
            mi, am, hist = align.align_eval_mi(L, pair.xyzB, eta6=etas, with_hist=True)
            st = align.align_eval_stats(L)
            if kind >= 0:
                assert st["sweep"] == kind, (kind, st)
            redo = align.align_eval_redo_poses(L)
            if queue_runs and i == 1:  # the queues overflowed: the exact path took the poses
                assert len(redo) > P // 2, len(redo)
            else:
                must.update(redo.tolist())
            runs.append((kind, spill, mi, am, hist))
        assert am == lowest_argmax(mi)
        must.add(am)
        L.close()
    _, _, mi0, am0, h0 = runs[0]
    for kind, spill, mi, am, hist in runs:
        assert np.array_equal(mi, mi0) and am == am0 and np.array_equal(hist, h0), (kind, spill)
    rng = np.random.default_rng(83)
    must = np.array(sorted(must), dtype=np.int64)
    rest = np.setdiff1d(np.arange(P), must)
    sample = np.sort(np.concatenate([must, rng.choice(rest, max(0, 96 - len(must)), replace=False)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(pair.xyzA)
    poses = align.align_round_poses(spec.origin, etas)
    mo, ho, _ = G.eval_mi(symA, boxA, pair.xyzB, poses[sample], nthreads=NT, with_hist=True)
    assert np.array_equal(h0[sample], ho)
    assert np.max(np.abs(mi0[sample].astype(np.float64) - mo)) <= mi_tolerance()


def test_spill_queues_with_raw_tiles():
    """Poses whose rotations do not repeat (random, as a Nelder-Mead simplex gives) use raw
    tiles that the kernel rotates itself; on the 0.25 m grid they need key partitions.  With
    the spill queues and with one sweep of B per partition the results are identical, and a
    sample matches the oracle."""
    from paper_1709_06948_gb300 import align
    pair = scangen.lidar_pair()
    spec = scangen.lidar_grid(0.25)
    rng = np.random.default_rng(86)
    etas = np.concatenate([rng.uniform(-2, 2, (600, 2)), rng.uniform(-0.2, 0.2, (600, 1)),
                           rng.uniform(-0.02, 0.02, (600, 2)), rng.uniform(-0.1, 0.1, (600, 1))], 1)
    res = []
    for spill in (True, False):
        L = lib_grid(spec)
        align.align_set_reference(L, pair.xyzA)
        align.align_set_sweep(L, 0)
        align.align_set_spill(L, spill)
        align.align_eval_mi(L, pair.xyzB, eta6=etas)  # learns the partitions
        res.append(align.align_eval_mi(L, pair.xyzB, eta6=etas, with_hist=True))
        assert align.align_eval_stats(L)["passes"] >= 2
        L.close()
    (mi, am, hist), (mi_p, am_p, hist_p) = res
    assert np.array_equal(mi, mi_p) and am == am_p and np.array_equal(hist, hist_p)
    assert am == lowest_argmax(mi)
    sample = np.unique(np.concatenate([[am], np.arange(0, len(etas), 40)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(pair.xyzA)
    poses = align.align_round_poses(spec.origin, etas[sample])
    mo, ho, _ = G.eval_mi(symA, boxA, pair.xyzB, poses, nthreads=NT, with_hist=True)
    assert np.array_equal(hist[sample], ho)
    assert np.max(np.abs(mi[sample].astype(np.float64) - mo)) <= mi_tolerance()

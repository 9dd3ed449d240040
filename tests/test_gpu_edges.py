"""Edge cases and the kernel's rare paths, each checked against the oracle on the GPU:
empty and ragged inputs, batches around the CTA count, everything outside the grid,
key partitioning (more occupied voxels than one shared-memory table holds) and the
64-bit side sums (more points in one voxel than 32-bit sums allow)."""
import math

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import check_argmax, lib_grid, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()


def _compare(spec, xyzA, xyzB, etas, **grid_over):
    from paper_1709_06948_gb300 import align
    G = oracle_grid(spec, **grid_over)
    L = lib_grid(spec, **grid_over)
    symA, boxA = G.reference(xyzA)
    align.align_set_reference(L, xyzA)
    sym, box = align.align_get_reference(L)
    assert np.array_equal(sym, symA) and box.tolist() == boxA.tolist()
    mi, am, hist = align.align_eval_mi(L, xyzB, eta6=etas, with_hist=True)
    mo, ho, _ = G.eval_mi(symA, boxA, xyzB, G.round_pose(etas), nthreads=NT, with_hist=True)
    assert np.array_equal(hist, ho)
    assert np.max(np.abs(mi.astype(np.float64) - mo)) <= mi_tolerance()
    if len(etas):
        check_argmax(am, mo, mi)
    return mi, am, align.align_eval_stats(L)


@pytest.fixture(scope="module")
def tiny():
    return scangen.tiny_pair()


def test_empty_b(tiny):
    mi, am, _ = _compare(tiny.grid, tiny.xyzA, np.zeros((0, 3), np.float32), scangen.tiny_poses()[:40])
    assert np.all(mi == 0.0) and am == 0


def test_empty_a(tiny):
    mi, am, _ = _compare(tiny.grid, np.zeros((0, 3), np.float32), tiny.xyzB, scangen.tiny_poses()[:40])
    assert np.all(mi == 0.0) and am == 0


def test_b_outside_grid(tiny):
    far = tiny.xyzB + np.float32(500.0)
    mi, am, _ = _compare(tiny.grid, tiny.xyzA, far, scangen.tiny_poses()[:33])
    assert np.all(mi == 0.0)


def test_poses_moving_b_out(tiny):
    etas = np.zeros((20, 6))
    etas[:, 0] = np.linspace(-80, 80, 20)  # most of these leave no overlap
    _compare(tiny.grid, tiny.xyzA, tiny.xyzB, etas)


def test_single_point(tiny):
    _compare(tiny.grid, tiny.xyzA, tiny.xyzB[:1], scangen.tiny_poses()[:17])
    _compare(tiny.grid, tiny.xyzA[:1], tiny.xyzB, scangen.tiny_poses()[:17])


@pytest.mark.parametrize("n", [1023, 1024, 1025, 3001])
def test_ragged_point_counts(tiny, n):
    xyz = np.concatenate([tiny.xyzB, tiny.xyzB])[:n]
    _compare(tiny.grid, tiny.xyzA, xyz, scangen.tiny_poses()[::9])


@pytest.mark.parametrize("P", [1, 2, 151, 152, 153, 305])
def test_batch_sizes(tiny, P):
    _compare(tiny.grid, tiny.xyzA, tiny.xyzB, scangen.tiny_poses()[:P])


def test_zero_poses(tiny):
    from paper_1709_06948_gb300 import align
    L = lib_grid(tiny.grid)
    align.align_set_reference(L, tiny.xyzA)
    mi, am, hist = align.align_eval_mi(L, tiny.xyzB, eta6=np.zeros((0, 6)))
    assert mi.shape == (0,) and am == -1


def test_no_reference_is_an_error(tiny):
    from paper_1709_06948_gb300 import align
    L = lib_grid(tiny.grid)
    with pytest.raises(align.AlignError) as e:
        align.align_eval_mi(L, tiny.xyzB, eta6=np.zeros((1, 6)))
    assert e.value.status == align.ALIGN_E_NOREF


def test_key_partitioning_many_voxels():
    """~60k occupied 0.25 m voxels per pose: more than one table holds, so the kernel
    splits the keys into partitions; results must not change."""
    rng = np.random.default_rng(31)
    spec = scangen.GridSpec(origin=(-20.0, -20.0, -1.0), res_m=0.25, dims=(160, 160, 32), feature=1, var_levels=15)
    xyzA = np.stack([rng.uniform(-19, 19, 60000), rng.uniform(-19, 19, 60000), rng.uniform(-0.9, 6.9, 60000)], 1)
    xyzB = xyzA + rng.normal(0, 0.05, xyzA.shape)
    etas = np.zeros((9, 6))
    etas[:, 0] = np.linspace(-0.4, 0.4, 9)
    mi, am, stats = _compare(spec, xyzA.astype(np.float32), xyzB.astype(np.float32), etas)
    assert stats["passes"] > 1
    assert am == 4


def test_wide_sums_dense_voxel():
    """25,000 points in one 0.5 m voxel exceed the 32-bit per-voxel sums; the kernel moves
    the excess to 64-bit side sums.  Sums and symbols must stay exact."""
    from paper_1709_06948_gb300 import align
    rng = np.random.default_rng(37)
    spec = scangen.lidar_grid(0.5)
    dense = np.stack([rng.uniform(1.01, 1.49, 25000), rng.uniform(2.01, 2.49, 25000), rng.uniform(0.01, 0.49, 25000)], 1)
    rest = np.stack([rng.uniform(-30, 30, 5000), rng.uniform(-30, 30, 5000), rng.uniform(-0.5, 5, 5000)], 1)
    xyz = np.concatenate([dense, rest]).astype(np.float32)
    etas = np.zeros((5, 6))
    etas[:, 1] = np.linspace(-0.1, 0.1, 5)
    mi, am, stats = _compare(spec, xyz, xyz, etas)
    assert stats["wide_voxels"] >= 1
    G = oracle_grid(spec)
    L = lib_grid(spec)
    align.align_set_reference(L, xyz)
    pose = G.round_pose(np.zeros(6))[0]
    acc, box = align.align_accumulate(L, xyz, pose)
    cnt, s1, s2, obox, _ = G.accumulate(xyz, pose)
    assert np.array_equal(acc[:, 0], cnt) and np.array_equal(acc[:, 1], s1) and np.array_equal(acc[:, 2], s2)
    assert cnt.max() >= 25000


def test_joint_feature_and_count_feature_lidar():
    pair = scangen.lidar_pair(seed=scangen.SEED_BASE + 40, n_beams=32)
    etas = scangen.lidar_poses(center=pair.T, half_width=(1.0, 1.0, 0.1, 0.01, 0.01, 0.05))[::64]
    spec_joint = scangen.GridSpec(origin=(-40.0, -40.0, -1.0), res_m=0.5, dims=(160, 160, 16), feature=2,
                                  count_levels=7, var_levels=8)
    _compare(spec_joint, pair.xyzA, pair.xyzB, etas)
    spec_count = scangen.GridSpec(origin=(-40.0, -40.0, -1.0), res_m=1.0, dims=(80, 80, 8), feature=0, count_levels=7)
    _compare(spec_count, pair.xyzA, pair.xyzB, etas)


def test_custom_thresholds():
    pair = scangen.tiny_pair(seed=scangen.SEED_BASE + 41)
    spec = scangen.GridSpec(origin=(-20.0, -20.0, -1.0), res_m=1.0, dims=(40, 40, 8), feature=1, var_levels=5)
    _compare(spec, pair.xyzA, pair.xyzB, scangen.tiny_poses()[::11], var_thresh=[10, 100, 1000, 100000])
    spec = scangen.GridSpec(origin=(-20.0, -20.0, -1.0), res_m=1.0, dims=(40, 40, 8), feature=0, count_levels=4)
    _compare(spec, pair.xyzA, pair.xyzB, scangen.tiny_poses()[::11], count_thresh=[3, 3, 50])


def test_large_angles(tiny):
    rng = np.random.default_rng(43)
    etas = np.concatenate([rng.uniform(-3, 3, (64, 3)), rng.uniform(-math.pi, math.pi, (64, 3))], 1)
    _compare(tiny.grid, tiny.xyzA, tiny.xyzB, etas)


def test_non_finite_points_are_dropped(tiny):
    """NaN / inf coordinates fall outside the grid under every pose (both load paths)."""
    xyz = tiny.xyzB.copy()
    xyz[::7, 0] = np.nan
    xyz[1::11, 1] = np.inf
    xyz[2::13, 2] = -np.inf
    etas = scangen.tiny_poses()[::5]
    _compare(tiny.grid, tiny.xyzA, xyz, etas)            # host poses: pre-rotated copies
    import torch
    from paper_1709_06948_gb300 import align
    G = oracle_grid(tiny.grid)
    L = lib_grid(tiny.grid)
    symA, boxA = G.reference(tiny.xyzA)
    align.align_set_reference(L, tiny.xyzA)
    poses = G.round_pose(etas)
    P = len(etas)
    mi = torch.empty(P, device="cuda")
    am = torch.empty(1, dtype=torch.int64, device="cuda")
    hist = torch.empty((P, L.K, L.K), dtype=torch.int32, device="cuda")
    align.align_eval_mi(L, torch.from_numpy(xyz).cuda(), poses12=torch.from_numpy(poses).cuda(), out=(mi, am, hist))
    torch.cuda.synchronize()
    _, ho, _ = G.eval_mi(symA, boxA, xyz, poses, with_hist=True)
    assert np.array_equal(hist.cpu().numpy().view(np.uint32), ho)  # device poses: in-kernel rotation


def test_non_finite_pose_rejected(tiny):
    from paper_1709_06948_gb300 import align
    L = lib_grid(tiny.grid)
    align.align_set_reference(L, tiny.xyzA)
    etas = np.zeros((3, 6))
    etas[1, 0] = np.inf
    with pytest.raises(align.AlignError) as e:
        align.align_eval_mi(L, tiny.xyzB, eta6=etas)
    assert e.value.status == align.ALIGN_E_INVALID


def test_exact_path_does_not_escalate_partitions():
    """Poses finished on the exact path (wide sums) many times over: a voxel of 70,000 points,
    past the per-voxel limit of the packed layout (which the first launch uses) and of the
    three-word layout (which the grid takes after it).  The layout changes once; the
    partition count the next launches start with stays where the data put it (no growth per
    launch), and the results never change."""
    from paper_1709_06948_gb300 import align
    rng = np.random.default_rng(38)
    spec = scangen.lidar_grid(0.5)
    n = 70000
    dense = np.stack([rng.uniform(1.01, 1.49, n), rng.uniform(2.01, 2.49, n), rng.uniform(0.01, 0.49, n)], 1)
    xyz = dense.astype(np.float32)
    L = lib_grid(spec)
    align.align_set_reference(L, xyz)
    etas = np.zeros((3, 6))
    first, _, _ = align.align_eval_mi(L, xyz, eta6=etas)
    slots_packed = align.align_eval_stats(L)["table_slots"]
    for _ in range(20):
        mi, _, _ = align.align_eval_mi(L, xyz, eta6=etas)
        assert np.array_equal(mi, first)
    st = align.align_eval_stats(L)
    assert st["table_slots"] < slots_packed  # the three-word layout (fewer, larger slots)
    assert st["wide_voxels"] >= 1 and st["passes"] <= 2


@pytest.mark.parametrize("res,n_dense", [(0.5, 900), (0.5, 1500), (0.5, 2100), (0.25, 1100), (1.0, 3000),
                                         (1.0, 4500)])
def test_dense_voxel_near_table_limits(res, n_dense):
    """One voxel holding about as many points as the table's per-voxel sums allow: below,
    at and above the bound of the packed layout (fine grids) and of the three-word layout
    (coarse grids).  Voxels past a bound go to the exact path; results stay exact."""
    from paper_1709_06948_gb300 import align
    rng = np.random.default_rng(41 + n_dense)
    spec = scangen.lidar_grid(res)
    lo = np.array([1.0, 2.0, 0.0]) + 0.01 * res
    dense = lo + rng.uniform(0.0, 0.98 * res, (n_dense, 3))
    rest = np.stack([rng.uniform(-30, 30, 8000), rng.uniform(-30, 30, 8000), rng.uniform(-0.5, 5, 8000)], 1)
    xyz = np.concatenate([dense, rest]).astype(np.float32)
    etas = np.zeros((7, 6))
    etas[:, 0] = np.linspace(-0.3 * res, 0.3 * res, 7)
    _compare(spec, xyz, xyz, etas)
    G = oracle_grid(spec)
    L = lib_grid(spec)
    align.align_set_reference(L, xyz)
    pose = G.round_pose(np.zeros(6))[0]
    acc, box = align.align_accumulate(L, xyz, pose)
    cnt, s1, s2, obox, _ = G.accumulate(xyz, pose)
    assert np.array_equal(acc[:, 0], cnt) and np.array_equal(acc[:, 1], s1) and np.array_equal(acc[:, 2], s2)
    assert cnt.max() >= n_dense

"""The large workload (128-beam scans of ~260k points, 400x400x40 grid at 0.2 m = 6.4M
voxels, joint count x z-variance feature with 57 symbols, key-partitioned tables) against
the oracle: the whole 32,768-pose lattice is evaluated in one launch, as the benchmark
does, and 1,024 of its poses are compared element by element (histograms bit-exact, MI
within 1e-5 nats).  The compared set always holds the launch's argmax and every pose that
the exact path finished, besides a seeded random sample."""
import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, lowest_argmax, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()
N_COMPARED = 1024


@pytest.fixture(scope="module")
def large():
    return scangen.large_pair()


def test_large_lattice_matches_oracle(large):
    import torch
    from paper_1709_06948_gb300 import align
    spec = large.grid
    L = lib_grid(spec)
    align.align_set_reference(L, large.xyzA)
    etas = scangen.large_poses()
    P = len(etas)
    poses = align.align_round_poses(spec.origin, etas)
    mi = torch.empty(P, device="cuda")
    am = torch.empty(1, dtype=torch.int64, device="cuda")
    hist = torch.empty((P, L.K, L.K), dtype=torch.int32, device="cuda")
    B = torch.from_numpy(large.xyzB).cuda()
    align.align_eval_mi(L, B, poses12=torch.from_numpy(poses).cuda(), out=(mi, am, hist))
    torch.cuda.synchronize()
    redo = align.align_eval_redo_poses(L)  # poses the exact path finished in this launch
    mi_h = mi.cpu().numpy()
    am_h = int(am.item())
    assert am_h == lowest_argmax(mi_h)
    align.align_eval_mi(L, large.xyzB, eta6=etas[:304])  # a synchronising call collects the counters
    assert align.align_eval_stats(L)["passes"] > 1  # the tables were partitioned
    rng = np.random.default_rng(81)
    must = np.unique(np.concatenate([[am_h], redo]))
    rest = np.setdiff1d(np.arange(P), must)
    sample = np.sort(np.concatenate([must, rng.choice(rest, max(0, N_COMPARED - len(must)), replace=False)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(large.xyzA)
    mo, ho, _ = G.eval_mi(symA, boxA, large.xyzB, poses[sample], nthreads=NT, with_hist=True)
    hist_s = hist[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint32)
    bad = [int(sample[i]) for i in range(len(sample)) if not np.array_equal(hist_s[i], ho[i])]
    assert not bad, f"histograms differ at poses {bad[:10]}"
    assert np.max(np.abs(mi_h[sample].astype(np.float64) - mo)) <= mi_tolerance()
    # the oracle's maximum over the compared poses is the GPU's argmax (within the FP32 band)
    o = int(sample[oracle.argmax(mo)])
    assert o == am_h or abs(mo[np.searchsorted(sample, am_h)] - mo.max()) <= 2e-5


def test_large_every_sweep_kind_agrees(large):
    """The same 4,096 large-grid poses evaluated repeatedly on one grid: the library first
    tries pose pairs, learns that their table needs more key partitions and evaluates single
    poses, then pose pairs again (with spill queues, twice the single-pose partitions pay);
    then the grid is set to one pose per 2-CTA cluster (a table split between two CTAs' shared
    memories, starting from half the single-pose partitions).
    Every call's MI and histograms are identical, and a sample (with each call's argmax and
    exact-path poses) matches the oracle."""
    from paper_1709_06948_gb300 import align
    spec = large.grid
    L = lib_grid(spec)
    align.align_set_reference(L, large.xyzA)
    etas = scangen.large_poses()[::8]
    P = len(etas)
    kinds, runs, must = [], [], set()
    for i in range(5):
        if i == 3:
            align.align_set_sweep(L, 2)
        mi, am, hist = align.align_eval_mi(L, large.xyzB, eta6=etas, with_hist=True)
        st = align.align_eval_stats(L)
        kinds.append((st["sweep"], st["passes"]))
        runs.append((mi, am, hist))
        must.update(align.align_eval_redo_poses(L).tolist())
        must.add(am)
    assert kinds[0][0] == 1 and kinds[1][0] == 0 and kinds[3][0] == 2, kinds
    assert kinds[3][1] < kinds[1][1], kinds  # the cluster's table needs fewer partitions
    for mi, am, hist in runs[1:]:
        assert np.array_equal(mi, runs[0][0]) and am == runs[0][1] and np.array_equal(hist, runs[0][2])
    rng = np.random.default_rng(82)
    must = np.array(sorted(must), dtype=np.int64)
    rest = np.setdiff1d(np.arange(P), must)
    sample = np.sort(np.concatenate([must, rng.choice(rest, max(0, 256 - len(must)), replace=False)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(large.xyzA)
    poses = align.align_round_poses(spec.origin, etas)
    mo, ho, _ = G.eval_mi(symA, boxA, large.xyzB, poses[sample], nthreads=NT, with_hist=True)
    assert np.array_equal(runs[0][2][sample], ho)
    assert np.max(np.abs(runs[0][0][sample].astype(np.float64) - mo)) <= mi_tolerance()


@pytest.mark.parametrize("layout", ["count", "three_words"])
def test_spill_queues_every_table_layout(large, layout):
    """Key partitions with B swept once and its runs queued per partition, for the table
    layouts the LiDAR and large-grid tests do not partition: the count feature (one value
    word) on the 0.2 m large grid, and the z-variance feature on a 0.6 m grid, whose packed
    word would hold too few points per voxel (three value words), with B subsampled to 60k
    points.  After the grid has learned its partitions, MI, argmax and histograms equal those
    of one sweep of B per partition, no pose needs the exact path, and a sample matches the
    oracle."""
    from paper_1709_06948_gb300 import align
    if layout == "count":
        spec = scangen.GridSpec(origin=large.grid.origin, res_m=0.2, dims=(400, 400, 40), feature=0,
                                count_levels=7, var_levels=1)
        B = large.xyzB
    else:
        spec = scangen.GridSpec(origin=(-120.0, -120.0, -5.0), res_m=0.6, dims=(400, 400, 33), feature=1,
                                count_levels=1, var_levels=15)
        B = scangen.subsample(large.xyzB, 60000, np.random.default_rng(85))
    etas = scangen.large_poses()[::64]
    res = []
    for spill in (True, False):
        L = lib_grid(spec)
        align.align_set_reference(L, large.xyzA)
        align.align_set_sweep(L, 0)
        align.align_set_spill(L, spill)
        align.align_eval_mi(L, B, eta6=etas)  # learns the partitions
        res.append(align.align_eval_mi(L, B, eta6=etas, with_hist=True))
        assert align.align_eval_stats(L)["passes"] >= 2
        assert len(align.align_eval_redo_poses(L)) == 0
        L.close()
    (mi, am, hist), (mi_p, am_p, hist_p) = res
    assert np.array_equal(mi, mi_p) and am == am_p and np.array_equal(hist, hist_p)
    assert am == lowest_argmax(mi)
    sample = np.unique(np.concatenate([[am], np.arange(0, len(etas), 16)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(large.xyzA)
    poses = align.align_round_poses(spec.origin, etas[sample])
    mo, ho, _ = G.eval_mi(symA, boxA, B, poses, nthreads=NT, with_hist=True)
    assert np.array_equal(hist[sample], ho)
    assert np.max(np.abs(mi[sample].astype(np.float64) - mo)) <= mi_tolerance()


@pytest.mark.parametrize("res", [1.0, 0.5])
def test_dense_scan_keeps_the_fast_path(large, res):
    """The 128-beam large scan on coarse z-variance grids (240 m square): voxels near the
    sensor hold thousands of points, past the packed layout's per-voxel limit at 0.5 m and
    past the uncentred three-word limit at 1 m.  The three-word layout sums z offsets from the
    voxel's middle (a quarter of the squares), and a grid whose packed-layout poses went to the
    exact path takes that layout from its next launch on (where its first poses may still
    overflow the smaller tables until the partitions of single poses and pose pairs are
    learned): by the fifth launch no more than 2% of the poses need the exact path, every
    launch gives the same results, and a sample matches the oracle."""
    from paper_1709_06948_gb300 import align
    n = int(round(240 / res))
    spec = scangen.GridSpec(origin=(-120.0, -120.0, -5.0), res_m=res, dims=(n, n, int(round(20 / res))), feature=1,
                            count_levels=1, var_levels=15)
    L = lib_grid(spec)
    align.align_set_reference(L, large.xyzA)
    etas = scangen.large_poses()[::64]
    runs, exact = [], []
    for _ in range(5):
        runs.append(align.align_eval_mi(L, large.xyzB, eta6=etas, with_hist=True))
        exact.append(len(align.align_eval_redo_poses(L)))
    assert exact[-1] <= len(etas) // 50, exact
    for mi, am, hist in runs[1:]:
        assert np.array_equal(mi, runs[0][0]) and am == runs[0][1] and np.array_equal(hist, runs[0][2])
    mi, am, hist = runs[-1]
    assert am == lowest_argmax(mi)
    sample = np.unique(np.concatenate([[am], np.arange(0, len(etas), 32)]))
    G = oracle_grid(spec)
    symA, boxA = G.reference(large.xyzA)
    poses = align.align_round_poses(spec.origin, etas[sample])
    mo, ho, _ = G.eval_mi(symA, boxA, large.xyzB, poses, nthreads=NT, with_hist=True)
    assert np.array_equal(hist[sample], ho)
    assert np.max(np.abs(mi[sample].astype(np.float64) - mo)) <= mi_tolerance()

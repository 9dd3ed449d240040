"""The large workload (128-beam scans of ~260k points, 400x400x40 grid at 0.2 m = 6.4M
voxels, joint count x z-variance feature with 57 symbols, key-partitioned tables) against
the oracle on sampled poses of its 32,768-pose lattice: histograms bit-exact, MI within
1e-5 nats.  The launch evaluates the whole lattice as the benchmark does."""
import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import lib_grid, mi_tolerance, oracle_grid

pytestmark = pytest.mark.gpu
NT = oracle.host_cores()


@pytest.fixture(scope="module")
def large():
    return scangen.large_pair()


def test_large_lattice_sampled_poses_match_oracle(large):
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
    align.align_eval_mi(L, torch.from_numpy(large.xyzB).cuda(), poses12=torch.from_numpy(poses).cuda(),
                        out=(mi, am, hist))
    torch.cuda.synchronize()
    align.align_eval_mi(L, large.xyzB, eta6=etas[:304])  # a synchronising call collects the counters
    assert align.align_eval_stats(L)["passes"] > 1  # the tables were partitioned
    G = oracle_grid(spec)
    symA, boxA = G.reference(large.xyzA)
    rng = np.random.default_rng(81)
    sample = np.sort(rng.choice(P, 6, replace=False))
    mo, ho, _ = G.eval_mi(symA, boxA, large.xyzB, poses[sample], nthreads=NT, with_hist=True)
    assert np.array_equal(hist[torch.from_numpy(sample).cuda()].cpu().numpy().view(np.uint32), ho)
    assert np.max(np.abs(mi.cpu().numpy()[sample].astype(np.float64) - mo)) <= mi_tolerance()

"""Pins of the CPU oracle against what the paper and plain mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a hand-derived
worked example, closed forms, exact rational arithmetic, an independent numpy route,
or a property the definitions imply.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import scangen
from tests.helpers import oracle_grid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_4x4x2.json")


def _ent(counts):
    """Plain entropy (nats) of a list of counts, written out for the closed forms below."""
    N = float(sum(counts))
    return -sum((c / N) * math.log(c / N) for c in counts if c > 0)


@pytest.fixture(scope="module")
def hand():
    with open(GOLDEN) as f:
        return json.load(f)


def _hand_grid(hand, mode):
    g = hand["grid"]
    if mode == "zvar":
        return oracle.Grid(g["origin"], g["res_m"], g["dims"], oracle.FEAT_ZVAR, var_levels=hand["zvar"]["var_levels"],
                           var_thresh=hand["zvar"]["var_thresh"])
    return oracle.Grid(g["origin"], g["res_m"], g["dims"], oracle.FEAT_COUNT, count_levels=hand["count"]["count_levels"])


# ---------------------------------------------------------------------------------------
# Hand-derived worked example (Sec. III-A, Algorithm 1, Eqs. 2-5)
# ---------------------------------------------------------------------------------------
def test_hand_keys_and_dz(hand):
    G = _hand_grid(hand, "zvar")
    ident = G.round_pose(np.zeros(6))[0]
    kA, dA = G.point_keys(ident, hand["xyzA"])
    assert kA.tolist() == hand["keysA"]
    assert dA.tolist() == hand["dzA"]
    pB = G.round_pose(hand["eta_B"])[0]
    kB, dB = G.point_keys(pB, hand["xyzB"])
    assert kB.tolist() == hand["keysB"]
    assert dB.tolist() == hand["dzB"]


def test_hand_sums_and_boxes(hand):
    G = _hand_grid(hand, "zvar")
    for side, key_sums, key_box, eta in (("xyzA", "sumsA", "boxA", np.zeros(6)), ("xyzB", "sumsB", "boxB", hand["eta_B"])):
        cnt, s1, s2, box, inside = G.accumulate(hand[side], G.round_pose(eta)[0])
        exp = {int(k): v for k, v in hand[key_sums].items()}
        occ = {int(v): [int(cnt[v]), int(s1[v]), int(s2[v])] for v in np.nonzero(cnt)[0]}
        assert occ == exp
        assert box.tolist() == hand[key_box]
        assert inside == sum(v[0] for v in exp.values())


@pytest.mark.parametrize("mode", ["zvar", "count"])
def test_hand_symbols_hist_mi(hand, mode):
    G = _hand_grid(hand, mode)
    symA, boxA = G.reference(hand["xyzA"])
    expA = {int(k): v for k, v in hand[mode]["symA"].items()}
    assert {int(v): int(symA[v]) for v in np.nonzero(symA)[0]} == expA
    assert boxA.tolist() == hand["boxA"]
    h, N, box = G.joint_hist(symA, boxA, hand["xyzB"], G.round_pose(hand["eta_B"])[0])
    assert N == hand["n_overlap"]
    assert h.tolist() == hand[mode]["hist"]
    mi = oracle.mi_from_hist(h)
    if mode == "zvar":
        expect = 2 * _ent([27, 3, 1, 1]) - _ent([27, 2, 1, 1, 1])
        assert abs(expect - 0.522204) < 5e-6  # the hand value written in the fixture
    else:
        expect = 2 * _ent([27, 3, 2]) - _ent([27, 2, 1, 1, 1])
    assert abs(mi - expect) < 1e-12


# ---------------------------------------------------------------------------------------
# Eqs. 2-5: closed forms and invariants
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (1000, 1), (7, 93)])
def test_mi_diagonal_2x2_is_binary_entropy(a, b):
    q = a / (a + b)
    hb = -q * math.log(q) - (1 - q) * math.log(1 - q)
    assert abs(oracle.mi_from_hist([[a, 0], [0, b]]) - hb) < 1e-12


@pytest.mark.parametrize("K", [2, 3, 8, 16])
def test_mi_uniform_diagonal_is_log_k(K):
    assert abs(oracle.mi_from_hist(np.eye(K, dtype=np.uint64) * 11) - math.log(K)) < 1e-12


def test_mi_outer_product_is_zero():
    rng = np.random.default_rng(5)
    for _ in range(20):
        K = int(rng.integers(2, 17))
        r = rng.integers(0, 50, K)
        c = rng.integers(0, 50, K)
        r[0] += 1
        c[0] += 1
        assert abs(oracle.mi_from_hist(np.outer(r, c))) < 1e-12


def test_mi_symmetric_bounds_and_permutation():
    rng = np.random.default_rng(7)
    for _ in range(50):
        K = int(rng.integers(2, 17))
        h = rng.integers(0, 30, (K, K)) * (rng.uniform(size=(K, K)) < 0.4)
        h[0, 0] += 1
        mi = oracle.mi_from_hist(h)
        hx, hy, hxy = oracle.entropies(h)
        assert abs(mi - oracle.mi_from_hist(h.T)) < 1e-12  # swapping the roles of A and B
        assert -1e-12 <= mi <= min(hx, hy) + 1e-12
        assert min(hx, hy) <= math.log(K) + 1e-12
        perm = rng.permutation(K)
        assert abs(mi - oracle.mi_from_hist(h[perm][:, perm])) < 1e-12  # symbol relabelling
        # against the plain entropy of the count lists
        assert abs(hx - _ent(h.sum(1).tolist())) < 1e-12
        assert abs(hxy - _ent(h.reshape(-1).tolist())) < 1e-12


def test_mi_empty_overlap_is_zero():
    assert oracle.mi_from_hist(np.zeros((4, 4), dtype=np.uint64), N=0) == 0.0


# ---------------------------------------------------------------------------------------
# Feature levels: integer comparison vs exact rational variance
# ---------------------------------------------------------------------------------------
def test_variance_level_matches_rational_variance():
    rng = np.random.default_rng(11)
    G = oracle.Grid((0, 0, 0), 0.5, (4, 4, 4), oracle.FEAT_ZVAR, var_levels=15)
    _, vt = G.thresholds()
    assert vt.tolist() == [250000 >> (16 - j) for j in range(14)]  # 3 ... 31250 mm^2
    for _ in range(400):
        n = int(rng.integers(1, 60))
        dz = rng.integers(-1, 502, n)
        if rng.uniform() < 0.3:
            dz[:] = dz[0]  # zero variance
        mean = Fraction(int(dz.sum()), n)
        var = sum((Fraction(int(d)) - mean) ** 2 for d in dz) / n  # two-pass, exact
        level = sum(1 for t in vt if var >= t)
        s1, s2 = int(dz.sum()), int((dz.astype(np.int64) ** 2).sum())
        assert G.symbol(n, s1, s2) == 1 + level


def test_count_level_is_floor_log2_capped():
    G = oracle.Grid((0, 0, 0), 1.0, (4, 4, 4), oracle.FEAT_COUNT, count_levels=7)
    assert G.symbol(0, 0, 0) == 0
    for n in range(1, 300):
        assert G.symbol(n, 0, 0) == min(7, 1 + int(math.floor(math.log2(n))))


def test_joint_symbol_layout():
    G = oracle.Grid((0, 0, 0), 0.2, (4, 4, 4), oracle.FEAT_COUNT_ZVAR, count_levels=7, var_levels=8)
    assert G.K == 57
    # one point: count level 0, variance 0 -> level 0 -> symbol 1
    assert G.symbol(1, 50, 2500) == 1
    # 4 points at the two z faces: count level 2, variance res^2/4 -> top variance level 7
    assert G.symbol(4, 400, 2 * 200 * 200) == 1 + 2 * 8 + 7


# ---------------------------------------------------------------------------------------
# Pose rounding (FP64 R = Rz Ry Rx rounded once; t' = t - origin)
# ---------------------------------------------------------------------------------------
def test_round_pose_matches_matrix_product():
    rng = np.random.default_rng(3)
    G = oracle.Grid((-40.0, -40.0, -1.0), 0.5, (160, 160, 16))
    for _ in range(200):
        eta = np.concatenate([rng.uniform(-5, 5, 3), rng.uniform(-math.pi, math.pi, 3)])
        p = G.round_pose(eta)[0]
        R = scangen.rot_zyx(eta)  # independent route: numpy product of the three rotations
        assert np.max(np.abs(p[:9].astype(np.float64) - R.reshape(-1))) < 1.5e-7
        assert np.allclose(p[9:], eta[:3] - np.array([-40.0, -40.0, -1.0]), atol=1e-5)


def test_round_pose_axes():
    G = oracle.Grid((0, 0, 0), 1.0, (4, 4, 4))
    Rz = G.round_pose([0, 0, 0, 0, 0, math.pi / 2])[0][:9].reshape(3, 3)
    assert np.allclose(Rz @ [1, 0, 0], [0, 1, 0], atol=1e-7)
    Rx = G.round_pose([0, 0, 0, math.pi / 2, 0, 0])[0][:9].reshape(3, 3)
    assert np.allclose(Rx @ [0, 1, 0], [0, 0, 1], atol=1e-7)
    Ry = G.round_pose([0, 0, 0, 0, math.pi / 2, 0])[0][:9].reshape(3, 3)
    assert np.allclose(Ry @ [0, 0, 1], [1, 0, 0], atol=1e-7)
    # order: x rotation applied first, z last
    R = G.round_pose([0, 0, 0, math.pi / 2, 0, math.pi / 2])[0][:9].reshape(3, 3)
    assert np.allclose(R @ [0, 1, 0], [0, 0, 1], atol=1e-7)      # Rx sends y to z, Rz keeps z
    assert np.allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-7)      # Rx keeps x, Rz sends x to y


# ---------------------------------------------------------------------------------------
# Voxel-point map: brute force in FP64 on points away from cell faces
# ---------------------------------------------------------------------------------------
def test_point_keys_bruteforce_fp64():
    rng = np.random.default_rng(17)
    spec = scangen.lidar_grid(0.5)
    G = oracle_grid(spec)
    X, Y, Z = spec.dims
    checked = 0
    for _ in range(6):
        eta = np.concatenate([rng.uniform(-2, 2, 2), rng.uniform(-0.3, 0.3, 1), rng.uniform(-0.1, 0.1, 3)])
        pose = G.round_pose(eta)[0]
        pts = np.stack([rng.uniform(-45, 45, 600), rng.uniform(-45, 45, 600), rng.uniform(-1.5, 7.5, 600)], 1)
        pts = pts.astype(np.float32)
        keys, dz = G.point_keys(pose, pts)
        R = pose[:9].astype(np.float64).reshape(3, 3)
        g = pts.astype(np.float64) @ R.T + pose[9:].astype(np.float64)
        f = g / 0.5
        k = np.floor(f)
        inside = np.all((k >= 0) & (k < [X, Y, Z]), 1)
        frac = f - k
        safe = np.all((frac > 1e-3) & (frac < 1 - 1e-3), 1)
        zmm = g[:, 2] * 1000.0
        safe &= np.abs(zmm - np.floor(zmm) - 0.5) > 1e-2
        exp_key = np.where(inside, (k[:, 2] * Y + k[:, 1]) * X + k[:, 0], -1).astype(np.int64)
        exp_dz = np.rint(zmm).astype(np.int64) - (k[:, 2] * 500).astype(np.int64)
        assert np.array_equal(keys[safe], exp_key[safe])
        sel = safe & inside
        assert np.array_equal(dz[sel], exp_dz[sel])
        checked += int(sel.sum())
    assert checked > 1000


# ---------------------------------------------------------------------------------------
# Two routes to the joint histogram: the oracle's dense box scan vs a sparse composition
# with per-symbol prefix sums written here in numpy
# ---------------------------------------------------------------------------------------
def _sparse_hist(G, symA, boxA, cnt, s1, s2):
    X, Y, Z = G.dims
    K = G.K
    occ = np.nonzero(cnt)[0]
    h = np.zeros((K, K), dtype=np.int64)
    if occ.size == 0:
        return h, 0
    kx, ky, kz = occ % X, (occ // X) % Y, occ // (X * Y)
    boxB = [kx.min(), ky.min(), kz.min(), kx.max(), ky.max(), kz.max()]
    lo = [max(boxA[i], boxB[i]) for i in range(3)]
    hi = [min(boxA[3 + i], boxB[3 + i]) for i in range(3)]
    if any(lo[i] > hi[i] for i in range(3)):
        return h, 0
    N = int(np.prod([hi[i] - lo[i] + 1 for i in range(3)]))
    vol = symA.reshape(Z, Y, X)
    cntA = np.zeros(K, dtype=np.int64)
    for a in range(1, K):
        sat = np.zeros((Z + 1, Y + 1, X + 1), dtype=np.int64)
        sat[1:, 1:, 1:] = np.cumsum(np.cumsum(np.cumsum(vol == a, 0), 1), 2)
        x0, y0, z0, x1, y1, z1 = lo[0], lo[1], lo[2], hi[0] + 1, hi[1] + 1, hi[2] + 1
        cntA[a] = (sat[z1, y1, x1] - sat[z1, y1, x0] - sat[z1, y0, x1] - sat[z0, y1, x1] + sat[z1, y0, x0]
                   + sat[z0, y1, x0] + sat[z0, y0, x1] - sat[z0, y0, x0])
    cntA[0] = N - cntA[1:].sum()
    inb = (kx >= lo[0]) & (kx <= hi[0]) & (ky >= lo[1]) & (ky <= hi[1]) & (kz >= lo[2]) & (kz <= hi[2])
    for v in occ[inb]:
        h[symA[v], G.symbol(cnt[v], s1[v], s2[v])] += 1
    h[:, 0] = cntA - h[:, 1:].sum(1)
    return h, N


@pytest.mark.parametrize("which", ["tiny", "lidar"])
def test_two_routes_agree(which, lidar_pair_small):
    if which == "tiny":
        pair = scangen.tiny_pair()
        etas = scangen.tiny_poses()[::97]
    else:
        pair = lidar_pair_small
        etas = scangen.lidar_poses()[::701]
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    for eta in etas:
        pose = G.round_pose(eta)[0]
        h, N, _ = G.joint_hist(symA, boxA, pair.xyzB, pose)
        cnt, s1, s2, _, _ = G.accumulate(pair.xyzB, pose)
        h2, N2 = _sparse_hist(G, symA, boxA, cnt, s1, s2)
        assert N == N2
        assert np.array_equal(h.astype(np.int64), h2)


@pytest.fixture(scope="module")
def lidar_pair_small():
    # a lighter LiDAR-shaped pair (16 beams) for CPU-time budget
    return scangen.lidar_pair(seed=scangen.SEED_BASE + 20, n_beams=16)


# ---------------------------------------------------------------------------------------
# Method-level properties
# ---------------------------------------------------------------------------------------
def test_self_alignment_mi_equals_entropy_of_a():
    pair = scangen.tiny_pair()
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    ident = G.round_pose(np.zeros(6))[0]
    h, N, box = G.joint_hist(symA, boxA, pair.xyzA, ident)
    assert box.tolist() == boxA.tolist()
    assert np.count_nonzero(h - np.diag(np.diag(h))) == 0  # joint histogram is diagonal
    hx = _ent(np.diag(h).tolist())
    assert abs(oracle.mi_from_hist(h) - hx) < 1e-12


def test_recovery_on_lattice_tiny():
    s = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])
    sign = np.array([1, -1, 0, 0, 1, -1])
    T = sign * s
    pair = scangen.tiny_pair(T=T)
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    etas = scangen.tiny_poses()
    mi, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(etas), nthreads=oracle.host_cores())
    best = oracle.argmax(mi)
    assert np.allclose(etas[best], T, atol=1e-12)


def test_mi_peaks_at_truth_lidar(lidar_pair_small):
    """Sec. III-A / Fig. 3: at the true pose the feature maps agree best (MI is highest
    along a sweep of t_x and of the heading through the truth)."""
    pair = lidar_pair_small
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    T = pair.T
    for axis, step in ((0, 0.5), (5, math.radians(2.0))):
        etas = np.repeat(T[None], 9, 0)
        etas[:, axis] += step * np.arange(-4, 5)
        mi, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(etas), nthreads=oracle.host_cores())
        assert abs(int(np.argmax(mi)) - 4) <= 1


def test_lattice_order_and_values():
    c = np.array([1.0, -2.0, 0.5, 0.01, -0.02, 0.3])
    r = np.array([2.0, 2.0, 0.25, 0.017, 0.017, 0.087])
    counts = (8, 8, 2, 2, 2, 8)
    L = oracle.lattice(c, r, counts)
    assert L.shape == (4096, 6)
    assert np.allclose(L.min(0), c - r) and np.allclose(L.max(0), c + r)
    # rotation axes outermost, tz fastest
    assert L[0, 2] != L[1, 2] and L[0, 0] == L[1, 0]
    assert np.all(L[:512, 3] == L[0, 3])
    # single-sample axes sit at the centre; three samples are centre -/0/+ range
    L3 = oracle.lattice(c, r, (3, 1, 1, 1, 1, 1))
    assert np.allclose(L3[:, 0], [c[0] - r[0], c[0], c[0] + r[0]]) and np.all(L3[:, 1:] == c[1:])


def test_argmax_ties_go_to_the_lowest_index():
    """Eq. 1 with the tie rule of the C ABI: of several equal maxima the first one wins.
    MI is piecewise constant in the pose, so exact ties are common on a lattice."""
    assert oracle.argmax([0.1, 0.5, 0.2, 0.5, 0.5]) == 1
    assert oracle.argmax([0.3, 0.3, 0.3]) == 0
    assert oracle.argmax([-1.0, -0.5, -0.5]) == 1
    assert oracle.argmax([0.0] * 7 + [1e-300]) == 7
    assert oracle.argmax(np.repeat([0.2, 0.7, 0.7, 0.1], 5)) == 5
    assert oracle.argmax([2.0]) == 0
    assert oracle.argmax(np.zeros(0)) == -1


def test_search_schedule_hand_computed():
    """The lattice search level by level: the lattice around the current centre with the
    current ranges, centre <- its best sample (lowest index on ties), ranges halved.  The
    per-level lattices are written out here with hand-computed offsets (three samples per
    searched axis: -r, 0, +r with r = 1, 0.5, 0.25 m in x and y, 0.08, 0.04, 0.02 rad in yaw)."""
    T = np.array([0.35, -0.6, 0.0, 0.0, 0.0, math.radians(3.0)])
    pair = scangen.tiny_pair(T=T)
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    nt = oracle.host_cores()
    offs_t = [[-1.0, 0.0, 1.0], [-0.5, 0.0, 0.5], [-0.25, 0.0, 0.25]]
    offs_yaw = [[-0.08, 0.0, 0.08], [-0.04, 0.0, 0.04], [-0.02, 0.0, 0.02]]
    c = np.zeros(6)
    centres, bests = [], []
    for lvl in range(3):
        # pose order: rotation samples outermost (only yaw varies here), then tx, then ty
        etas = np.array([[c[0] + offs_t[lvl][ix], c[1] + offs_t[lvl][iy], c[2], c[3], c[4],
                          c[5] + offs_yaw[lvl][iz]]
                         for iz in range(3) for ix in range(3) for iy in range(3)])
        mi, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(etas), nthreads=nt)
        b = int(np.flatnonzero(mi == mi.max())[0])
        bests.append(b)
        c = etas[b].copy()
        centres.append(c)
    Tout, mi_out, lb = G.search(symA, boxA, pair.xyzB, np.zeros(6), np.array([1.0, 1.0, 0.0, 0.0, 0.0, 0.08]),
                                counts=(3, 3, 1, 1, 1, 3), levels=3, nthreads=nt)
    assert lb.tolist() == bests
    assert Tout.tolist() == centres[-1].tolist()
    assert len({tuple(x) for x in centres}) > 1  # the centre moved: the schedule was exercised
    mo, _, _ = G.eval_mi(symA, boxA, pair.xyzB, G.round_pose(centres[-1][None]), nthreads=1)
    assert mi_out == mo[0]


def test_search_recovers_tiny_within_final_step():
    T = np.array([0.35, -0.6, 0.1, math.radians(1.0), math.radians(-1.5), math.radians(3.0)])
    pair = scangen.tiny_pair(T=T)
    G = oracle_grid(pair.grid)
    symA, boxA = G.reference(pair.xyzA)
    rng = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])
    levels = 5
    Tout, mi, lb = G.search(symA, boxA, pair.xyzB, np.zeros(6), rng, counts=(3, 3, 3, 3, 3, 3), levels=levels,
                            nthreads=oracle.host_cores())
    final_step = rng / 2 ** (levels - 1)
    # translation recovered to within a voxel-scale step; heading within two final steps
    assert np.all(np.abs(Tout[:2] - T[:2]) <= 0.3)
    assert abs(Tout[5] - T[5]) <= 2 * final_step[5] + math.radians(1.0)
    assert mi > 0


def _quad(w, c, v):
    s = 0.0  # same operation order as the oracle's test objective
    for i in range(6):
        s += float(w[i]) * (float(v[i]) - float(c[i])) * (float(v[i]) - float(c[i]))
    return s


def test_nelder_mead_matches_scipy_on_quadratics():
    """The oracle's Nelder-Mead (Algorithm 1's optimiser) equals SciPy's implementation of
    the same method (standard coefficients, given initial simplex) step for step on
    quadratic objectives without ties (SciPy's maxiter counts the initial simplex)."""
    optimize = pytest.importorskip("scipy.optimize")
    step = np.array([8, 8, 1, 0.1, 0.1, 0.8])
    for seed in range(4):
        rng = np.random.default_rng(seed)
        w = rng.uniform(0.3, 3, 6)
        c = rng.uniform(-1, 1, 6) * np.array([2, 2, 0.3, 0.05, 0.05, 0.3])
        x0 = rng.uniform(-1, 1, 6) * np.array([3, 3, 0.3, 0.05, 0.05, 0.2])
        sim = np.array([x0] + [x0 + np.eye(6)[i] * step[i] for i in range(6)])
        for it in (1, 7, 25, 60):
            x, f, n = oracle.nm_quadratic(w, c, x0, step, it)
            r = optimize.minimize(lambda v: _quad(w, c, v), x0, method="Nelder-Mead",
                                  options=dict(initial_simplex=sim, maxiter=it + 1, xatol=0, fatol=0,
                                               maxfev=100000))
            assert n == it
            assert np.array_equal(x, r.x) and f == r.fun


def test_nelder_mead_converges_and_stops_on_ftol():
    w = np.ones(6)
    c = np.array([0.5, -0.25, 0.1, 0.02, -0.01, 0.2])
    x, f, n = oracle.nm_quadratic(w, c, np.zeros(6), np.array([1, 1, 1, 0.1, 0.1, 0.1]), 2000, ftol=1e-14)
    assert n < 2000 and f < 1e-10 and np.max(np.abs(x - c)) < 1e-4

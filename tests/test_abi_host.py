"""The C-ABI library loads, exports every symbol include/*.h declares, and its host-only
logic agrees with the oracle (no GPU needed)."""
import glob
import math
import os
import re

import numpy as np
import pytest

import oracle
import scangen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(align_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1709_06948_gb300 import align
    lib = align.load()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert declared == set(align.EXPORTS)
    # nm view of the .so: every declared name is an exported text symbol
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", align.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (align_\w+)", out))
    assert declared <= exported


def test_round_poses_bit_exact_with_oracle():
    from paper_1709_06948_gb300 import align
    rng = np.random.default_rng(23)
    origin = (-40.0, -40.0, -1.0)
    G = oracle.Grid(origin, 0.5, (160, 160, 16))
    eta = np.concatenate([rng.uniform(-10, 10, (500, 3)), rng.uniform(-math.pi, math.pi, (500, 3))], 1)
    eta[:50, 3:] = 0.0
    eta[50:60, 3:] = math.pi / 2
    mine = align.align_round_poses(origin, eta)
    ref = G.round_pose(eta)
    assert mine.view(np.uint32).tolist() == ref.view(np.uint32).tolist()


def test_lattice_poses_bit_exact_with_oracle():
    """The search's lattice goes through the same rounding; pin the shared convention on a
    lattice the search would build."""
    from paper_1709_06948_gb300 import align
    L = oracle.lattice([0.3, -0.2, 0.0, 0.0, 0.0, 0.1], [2, 2, 0.25, 0.017, 0.017, 0.087], (8, 8, 2, 2, 2, 8))
    origin = (-40.0, -40.0, -1.0)
    assert (align.align_round_poses(origin, L).view(np.uint32) ==
            oracle.Grid(origin, 0.5, (160, 160, 16)).round_pose(L).view(np.uint32)).all()


def test_no_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1709_06948_gb300 import align
    with pytest.raises(align.AlignError) as e:
        align.align_create_grid((0, 0, 0), 1.0, (4, 4, 4), align.ALIGN_FEAT_COUNT)
    assert e.value.status == align.ALIGN_E_CUDA


@pytest.mark.parametrize("bad", [
    dict(res_m=0.0), dict(res_m=0.0004), dict(res_m=0.3333), dict(dims=(0, 4, 4)), dict(dims=(1 << 21, 4, 4)),
    dict(feature=5), dict(var_levels=0), dict(var_levels=64), dict(feature=2, count_levels=8, var_levels=8),
    dict(var_thresh=[5, 3] + [0] * 12),
    dict(dims=(8, 8, 2098)),  # 2,098 layers of 0.5 m: z above 2^20 mm, beyond the exact z-offset bound
])
def test_invalid_grid_rejected_before_gpu(bad):
    from paper_1709_06948_gb300 import align
    kw = dict(origin=(0, 0, 0), res_m=0.5, dims=(8, 8, 8), feature=1, count_levels=7, var_levels=15)
    kw.update(bad)
    with pytest.raises(align.AlignError) as e:
        align.align_create_grid(**kw)
    assert e.value.status == align.ALIGN_E_INVALID


def test_scangen_shapes():
    p = scangen.tiny_pair()
    assert p.xyzA.shape == (8000, 3) and p.xyzB.shape == (8000, 3) and p.xyzA.dtype == np.float32
    assert np.all(np.hypot(p.xyzA[:, 0], p.xyzA[:, 1]) <= 20.0 + 1e-4)
    assert np.linalg.norm(p.T[:3]) <= 1.0 and np.all(np.abs(p.T[3:]) <= math.radians(5))
    assert scangen.tiny_poses().shape == (729, 6)
    assert scangen.lidar_poses().shape == (4096, 6)

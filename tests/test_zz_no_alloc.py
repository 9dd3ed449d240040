"""align_reference_noalloc: A's feature map and bbox computed without any device
allocation by the library (for callers whose device memory belongs to another
allocator, or who may not allocate inside their loop).  Its output must equal what
align_set_reference + align_get_reference give, call after call, although every call
shares one fixed working area.  Collected last so that a failure here does not stop an
-x run before the other tests."""
import numpy as np
import pytest

import scangen
from tests.helpers import lib_grid

pytestmark = pytest.mark.gpu


def _existing(spec, xyz):
    from paper_1709_06948_gb300 import align
    L = lib_grid(spec)
    align.align_set_reference(L, xyz)
    sym, box = align.align_get_reference(L)
    L.close()
    return sym, box


def _noalloc(spec, xyz):
    import torch
    from paper_1709_06948_gb300 import align
    X, Y, Z = spec.dims
    sym = torch.full((X * Y * Z,), 0xAB, dtype=torch.uint8, device="cuda")   # poison: must be overwritten
    box = torch.full((6,), 12345, dtype=torch.int32, device="cuda")
    desc = dict(origin=spec.origin, res_m=spec.res_m, dims=spec.dims, feature=spec.feature,
                count_levels=spec.count_levels, var_levels=spec.var_levels)
    align.align_reference_noalloc(desc, torch.from_numpy(np.ascontiguousarray(xyz, np.float32)).cuda(), sym, box)
    torch.cuda.synchronize()
    return sym.cpu().numpy(), box.cpu().numpy()


def test_noalloc_matches_set_reference_on_consecutive_calls():
    lidar = scangen.lidar_pair(seed=scangen.SEED_BASE + 60, n_beams=16)   # 160 x 160 x 16, z-variance
    tiny = scangen.tiny_pair(seed=scangen.SEED_BASE + 61)                 # 40 x 40 x 8, point count
    calls = [(lidar.grid, lidar.xyzA), (tiny.grid, tiny.xyzA), (lidar.grid, lidar.xyzB)]
    for spec, xyz in calls:  # consecutive calls: each must clear what the previous one left
        sym_ref, box_ref = _existing(spec, xyz)
        sym, box = _noalloc(spec, xyz)
        assert np.array_equal(sym, sym_ref)
        assert box.tolist() == box_ref.tolist()
        assert (sym > 0).sum() > 100


def test_noalloc_allocates_nothing():
    """After one warm-up call (which looks up the working area's address), further calls leave
    the device's free memory unchanged: nothing is allocated on the caller's behalf."""
    import torch
    from paper_1709_06948_gb300 import align
    tiny = scangen.tiny_pair(seed=scangen.SEED_BASE + 62)
    spec = tiny.grid
    X, Y, Z = spec.dims
    desc = dict(origin=spec.origin, res_m=spec.res_m, dims=spec.dims, feature=spec.feature,
                count_levels=spec.count_levels, var_levels=spec.var_levels)
    xyz = torch.from_numpy(np.ascontiguousarray(tiny.xyzA, np.float32)).cuda()
    sym = torch.empty(X * Y * Z, dtype=torch.uint8, device="cuda")
    box = torch.empty(6, dtype=torch.int32, device="cuda")
    align.align_reference_noalloc(desc, xyz, sym, box)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        align.align_reference_noalloc(desc, xyz, sym, box)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    sym_ref, box_ref = _existing(spec, tiny.xyzA)
    assert np.array_equal(sym.cpu().numpy(), sym_ref) and box.cpu().numpy().tolist() == box_ref.tolist()


def test_noalloc_checks_its_buffers():
    import torch
    from paper_1709_06948_gb300 import align
    tiny = scangen.tiny_pair(seed=scangen.SEED_BASE + 63)
    spec = tiny.grid
    X, Y, Z = spec.dims
    desc = dict(origin=spec.origin, res_m=spec.res_m, dims=spec.dims, feature=spec.feature,
                count_levels=spec.count_levels, var_levels=spec.var_levels)
    xyz = torch.from_numpy(np.ascontiguousarray(tiny.xyzA, np.float32)).cuda()
    box = torch.empty(6, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):  # symA shorter than the grid
        align.align_reference_noalloc(desc, xyz, torch.empty(X * Y * Z - 1, dtype=torch.uint8, device="cuda"), box)
    with pytest.raises(ValueError):  # wrong dtype of the points
        align.align_reference_noalloc(desc, xyz.double(), torch.empty(X * Y * Z, dtype=torch.uint8, device="cuda"),
                                      box)
    with pytest.raises(ValueError):  # box of 5 entries
        align.align_reference_noalloc(desc, xyz, torch.empty(X * Y * Z, dtype=torch.uint8, device="cuda"),
                                      box[:5])


def test_noalloc_rejects_grids_beyond_its_working_area():
    import torch
    from paper_1709_06948_gb300 import align
    desc = dict(origin=(-40.0, -40.0, -1.0), res_m=0.25, dims=(320, 320, 32), feature=1, count_levels=7,
                var_levels=15)
    sym = torch.zeros(320 * 320 * 32, dtype=torch.uint8, device="cuda")
    box = torch.zeros(6, dtype=torch.int32, device="cuda")
    xyz = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(align.AlignError) as e:
        align.align_reference_noalloc(desc, xyz, sym, box)
    assert e.value.status == align.ALIGN_E_INVALID
    assert "2^19" in str(e.value)

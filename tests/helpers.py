"""Test helpers: build matching grids for the oracle and the library from one GridSpec."""
from __future__ import annotations

import numpy as np

import oracle


def oracle_grid(spec, **over):
    kw = dict(origin=spec.origin, res_m=spec.res_m, dims=spec.dims, feature=spec.feature,
              count_levels=spec.count_levels, var_levels=spec.var_levels)
    kw.update(over)
    return oracle.Grid(**kw)


def lib_grid(spec, **over):
    from paper_1709_06948_gb300 import align
    kw = dict(origin=spec.origin, res_m=spec.res_m, dims=spec.dims, feature=spec.feature,
              count_levels=spec.count_levels, var_levels=spec.var_levels)
    kw.update(over)
    return align.align_create_grid(**kw)


def mi_tolerance() -> float:
    """|MI_gpu - MI_oracle| bound in nats (FP32 entropies of exact histograms vs FP64)."""
    return 1e-5


def lowest_argmax(mi) -> int:
    """Index of the largest value, the lowest one on ties (Eq. 1's rule), or -1 if empty."""
    mi = np.asarray(mi)
    return int(np.flatnonzero(mi == mi.max())[0]) if mi.size else -1


def check_argmax(gpu_idx: int, mi_oracle: np.ndarray, mi_gpu: np.ndarray, tie_band: float = 2e-5):
    """The GPU's argmax is exactly the lowest-index maximum of its own FP32 MI array, and it is
    the oracle's argmax unless the two poses lie within the FP32-versus-FP64 band."""
    assert gpu_idx == lowest_argmax(mi_gpu), (gpu_idx, lowest_argmax(mi_gpu))
    o = int(oracle.argmax(mi_oracle))
    if gpu_idx == o:
        return True
    assert abs(mi_oracle[gpu_idx] - mi_oracle[o]) <= tie_band, (gpu_idx, o, mi_oracle[gpu_idx], mi_oracle[o])
    return False

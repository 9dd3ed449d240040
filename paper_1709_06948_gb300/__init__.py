"""GB300 (sm_103a) library for the voxelized-feature mutual-information scan-alignment
cost of arXiv 1709.06948: pose-batched MI evaluation, argmax and lattice search.

The compute path is the C ABI in include/align.h (hand-written CUDA kernels under
csrc/); ``align`` is its Python binding.
"""
from . import align  # noqa: F401
from .align import (ALIGN_FEAT_COUNT, ALIGN_FEAT_COUNT_ZVAR, ALIGN_FEAT_ZVAR, AlignError,  # noqa: F401
                    align_accumulate, align_create_grid, align_destroy_grid, align_eval_mi, align_eval_stats,
                    align_get_reference, align_last_error, align_round_poses, align_search, align_set_reference)

__all__ = ["align"]

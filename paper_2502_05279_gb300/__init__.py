"""GB300-native black-box multigrid (BoxMG) for 2D 5-/9-point stencils.

The solver lives in the CUDA library libbmg.so (C ABI declared in
include/bmg.h; libbmg_debug.so with device bounds checks when BMG_LIB=debug);
this package only marshals torch tensors into that ABI.
There is no CPU fallback: importing the binding fails when the library is
missing or cannot load.
"""
from ._lib import (  # noqa: F401
    BMG_BF16_IR, BMG_EBOUNDS, BMG_EINVAL, BMG_ENOMEM, BMG_ESINGULAR, BMG_FP32_IR, BMG_FP64, BMG_PERIODIC_X,
    BMG_PERIODIC_Y, Batch, BmgError, Hierarchy, coarse_factor, coarse_solve, debug_build, debug_shrink, debug_take,
    dendy_interp,
    interp_correct, learned_interp, fill_uniform, lib, library_path, measure_fp64_rate, Mlp, mlp_features, rap, relax,
    relax_line,
    resid_restrict, residual, TILE_SWEEP,
)

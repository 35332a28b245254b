"""GB300-native local multiple traces formulation (MTF) for time-harmonic
Maxwell transmission problems (arXiv 2502.10907).

The compute path is the C-ABI library ``libmtf`` (hand-written CUDA for
sm_103a, declared in ``include/mtf.h``); this package is its Python binding
(``_lib``: one function per entry point) plus thin handle wrappers
(``api``).  PyTorch is used for device memory and streams only.
"""
from . import _lib
from ._lib import (MtfError, load, mtf_default_options, mtf_mesh_create, mtf_mesh_info,
                   mtf_mesh_pair_counts, mtf_mesh_destroy, mtf_assemble, mtf_get_block, mtf_matvec,
                   mtf_rhs, mtf_solve, mtf_precond_apply, mtf_farfield, mtf_system_destroy, MTF_PREC_FP64,
                   MTF_PREC_MIXED, MTF_PRECOND_NONE, MTF_PRECOND_OSRC)

__all__ = ["MtfError", "load", "mtf_default_options", "mtf_mesh_create", "mtf_mesh_info",
           "mtf_mesh_pair_counts", "mtf_mesh_destroy", "mtf_assemble", "mtf_get_block", "mtf_matvec",
           "mtf_rhs", "mtf_solve", "mtf_precond_apply", "mtf_farfield", "mtf_system_destroy", "MTF_PREC_FP64",
           "MTF_PREC_MIXED", "MTF_PRECOND_NONE", "MTF_PRECOND_OSRC"]

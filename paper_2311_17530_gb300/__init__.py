"""GB300-native optimal multiple sequence alignment by dynamic programming.

The compute path is libmsadp (C-ABI in include/msadp.h, CUDA kernels for
sm_103a in csrc/); this package holds its build script and a ctypes binding.
"""
from .msadp import (MSA_EBADHANDLE, MSA_ECUDA, MSA_EINVAL, MSA_ENOMEM, MSA_ETIMEOUT, MSA_ETOOBIG,
                    MSA_OK, MSA_PENDING, MsaError, Plan, library, msa_align, msa_cancel, msa_config,
                    msa_drain, msa_poll, msa_set_stream, msa_submit, msa_tile_shape, msa_wait_any,
                    msa_wave_sizes, msa_autotune, msa_set_tile_edge, msa_get_tile_edge,
                    msa_set_line_segment, msa_get_line_segment, msa_near_optimal,
                    msa_align_pruned, msa_tile_bounds)

__all__ = ["MSA_EBADHANDLE", "MSA_ECUDA", "MSA_EINVAL", "MSA_ENOMEM", "MSA_ETIMEOUT", "MSA_ETOOBIG",
           "MSA_OK", "MSA_PENDING", "MsaError", "Plan", "library", "msa_align", "msa_cancel",
           "msa_config", "msa_drain", "msa_poll", "msa_set_stream", "msa_submit", "msa_tile_shape",
           "msa_wait_any", "msa_wave_sizes", "msa_autotune", "msa_set_tile_edge", "msa_get_tile_edge",
           "msa_set_line_segment", "msa_get_line_segment", "msa_near_optimal",
           "msa_align_pruned", "msa_tile_bounds"]

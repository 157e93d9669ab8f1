"""GB300 (sm_103a) stencil sweeps recast as banded matrix products.

The compute path is the CUDA library ``libmms.so`` (``csrc/``, C ABI in
``include/mms.h``); this package is its thin Python binding plus the
autograd wrapper of the wave propagator, the tile autotuner and the z-slab
decomposition across ranks (``distributed``).  Importing
the package does not load the library; the first call does, and fails
loudly if the library has not been built.
"""
from ._lib import (BOX, BOX2D, PATHS, STAR, STAR2D, MMSError, apply, grad_divide_m, apply_dense, apply_f64, apply_host, auto_path, check_device,
                   default_variant,
                   dot_f64, field_geometry, grad_to_velocity, load, model_from_velocity,
                   num_variants, padded_empty, padded_empty2d, pitches, set_variant, sum_f64, tc_pipeline_config,
                   to_padded_device, to_padded_device2d,
                   version, vti_model, vti_step, wave_adjoint, wave_adjoint_lap, wave_adjoint_scaled, wave_desc, wave_forward, wave_step,
                   wave_step_lap, wave_step_to,
                   aniso_num_variants, aniso_set_variant, tti_model, tti_step)
from .build import build

__all__ = ["BOX", "BOX2D", "PATHS", "STAR", "STAR2D", "MMSError", "apply", "grad_divide_m", "apply_dense", "apply_f64", "apply_host", "auto_path", "build",
           "check_device",
           "default_variant", "dot_f64", "field_geometry", "grad_to_velocity", "load",
           "model_from_velocity", "num_variants", "padded_empty", "padded_empty2d", "pitches", "set_variant", "sum_f64",
           "tc_pipeline_config",
           "to_padded_device", "to_padded_device2d", "version", "wave_adjoint", "wave_desc", "wave_forward", "wave_step",
           "wave_step_to", "wave_step_lap", "wave_adjoint_lap", "wave_adjoint_scaled", "vti_model", "vti_step", "aniso_num_variants", "aniso_set_variant",
           "tti_model", "tti_step"]

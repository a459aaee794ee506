"""GB300-native CTIS reconstruction: the shift-invariant projector pair and the
EM iteration of White, Bell and Haygood, as sm_103a CUDA kernels behind a C ABI
(include/ctis.h, libctis.so). This package is the thin Python binding."""
from ._native import (CTIS_BF16, CTIS_BOUNDARY_CLIP, CTIS_BOUNDARY_REJECT, CTIS_BOUNDARY_WRAP,
                      CTIS_F32, CTIS_SOLVER_EM, CTIS_SOLVER_SART, CTIS_SOLVER_SMART, EXPORTED,
                      LIB_PATH, NSTATS, STAT_NAMES, CtisError,
                      Plan, fma_peak, load, reconstruct_batched, shard_wavelengths,
                      slice_psf, tables_inspect)

__all__ = ["Plan", "CtisError", "load", "LIB_PATH", "EXPORTED", "NSTATS", "STAT_NAMES",
           "CTIS_F32", "CTIS_BF16", "CTIS_BOUNDARY_REJECT", "CTIS_BOUNDARY_CLIP",
           "CTIS_BOUNDARY_WRAP", "CTIS_SOLVER_EM", "CTIS_SOLVER_SART", "CTIS_SOLVER_SMART",
           "reconstruct_batched", "tables_inspect", "fma_peak", "shard_wavelengths",
           "slice_psf"]

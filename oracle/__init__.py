"""FP64 CPU oracle (test infrastructure only; never imported by the GPU path)."""
from .ctis_oracle import *  # noqa: F401,F403
from .ctis_oracle import (Geometry, Taps, BlockH, OutOfBounds, check_bounds, merge_psf,
                          index_map, build_H, ratio, em_update, stats, mlem, em_step,
                          forward_at, adjoint_at, dense_H, fft_forward, fft_adjoint,
                          psf_value_grad, poisson_nll, with_values, unrolled_nll,
                          row_sums, sart_step, smart_step, solve)

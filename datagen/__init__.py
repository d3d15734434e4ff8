"""Seeded synthetic float32 fields that stand in for the paper's datasets.

The SDRB fields the paper evaluates on (Hurricane, CESM-ATM, SCALE-LETKF,
Miranda; Table 3) and the RTM data are not available, so every workload here is
synthetic, with the shapes of Table 3 and of the benchmark configurations. This
module holds no compression arithmetic: it only draws numbers. Both the oracle
tests and the GPU tests/benchmark take their inputs from it.
"""
from .fields import (sines_1d, grf, lat_bands_2d, field_set_batched, small_cases,
                     GRF_SHAPES, REL_BOUNDS)

__all__ = ["sines_1d", "grf", "lat_bands_2d", "field_set_batched", "small_cases",
           "GRF_SHAPES", "REL_BOUNDS"]

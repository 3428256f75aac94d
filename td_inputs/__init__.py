"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This package builds decoding problems and samples shots. It contains none of the
decoder's arithmetic (no tensor contraction, no truncation): only the problem
statement of Sec. 2.4 -- a detector error model (H, p, l) with space-time
coordinates for its detectors -- and a counter-based random source for shots.
"""
from .codes import (DEM, GenProblem, point_sector_3d, loop_sector_3d, rotated_phenomenological,
                    repetition_phenomenological, five_qubit_code, log_uniform_rates)
from .sampler import splitmix64, uniform53, sample_shots

__all__ = ["DEM", "GenProblem", "point_sector_3d", "loop_sector_3d", "rotated_phenomenological", "repetition_phenomenological",
           "five_qubit_code", "log_uniform_rates", "splitmix64", "uniform53", "sample_shots"]

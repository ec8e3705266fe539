"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This package holds input generation only (right-hand sides, problem-size draws, request
streams, coefficient masks of test problems); none of the Chebyshev-Jacobi arithmetic lives
here.
"""
from .rhs import (grid_h, manufactured_rhs, manufactured_solution, smooth_random_modes,
                  smooth_random_rhs, splitmix64_stream, gaussian_stream, uniform_stream,
                  paper_problem)
from .streams import batch_problems, request_stream, log_uniform_int
from . import masks

__all__ = ["grid_h", "manufactured_rhs", "manufactured_solution", "smooth_random_modes",
           "smooth_random_rhs", "splitmix64_stream", "gaussian_stream", "uniform_stream",
           "batch_problems", "request_stream", "log_uniform_int", "paper_problem", "masks"]

"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

Holds scene rendering, trajectories and correspondence sampling only; none of the
pose solver's arithmetic lives here.
"""
from .configs import (Problem, cfg1, cfg2, cfg3, cfg4_global, cfg5, chunk_problem, global_problem, large_global_problem,  # noqa: F401
                      chunk_batch, seed_for)
from . import scene  # noqa: F401

"""Seeded synthetic inputs for the BoxMG solver: random numbers, coefficient
fields, right-hand sides and the 5-/9-point stencils assembled from them.

This package holds no step of the multigrid method itself.  Both the CUDA path
(through its Python binding, the tests and bench.py) and the CPU oracle (through
the tests) receive the arrays it produces; neither side computes its inputs.
"""
from .gen import *  # noqa: F401,F403

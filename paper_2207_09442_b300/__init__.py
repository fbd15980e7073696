"""Batched differentiable nonlinear least squares (GN/LM + implicit backward) for B300 (sm_103a).

Only the seeded workload generator is imported eagerly; the CUDA library binding is loaded on
first use of :mod:`paper_2207_09442_b300.dnls` and fails loudly if ``libdnls.so`` is missing.
"""
from . import synth  # noqa: F401

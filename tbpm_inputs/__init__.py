"""Seeded synthetic inputs for TBPM workloads.

Shared by the CUDA library's tests and benchmark and by the CPU oracle's
tests.  It only generates lattices, bond lists and random draws; it holds
none of the propagation method's arithmetic.
"""
from . import lattice, rng, workloads  # noqa: F401

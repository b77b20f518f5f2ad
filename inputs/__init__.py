"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This package only draws random numbers and fixes the shapes of the five
workloads (double integrator, one random n=10 system, 64 ragged random systems,
a 100-mass spring chain, and the warm-start training/test sets).  It holds
none of the method's arithmetic: no matrix exponential, no quadrature, no
solver.  Both the CUDA path and the CPU oracle consume what it returns.
"""
from .workloads import *  # noqa: F401,F403

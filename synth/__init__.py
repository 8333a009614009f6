"""Seeded synthetic inputs (geometry and random draws) shared by the oracle and the CUDA path."""
from .workloads import Cluster, batch64, pd13_small, pd13_uniform65, pd2_dimer, pd55_graded129, pd561_graded385, potential_energy  # noqa: F401

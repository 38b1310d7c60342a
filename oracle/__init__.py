"""CPU oracle for the Q4C integration path -- test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline (and its
reference arm) may import this package.  It wraps the plain C oracle in
q4c_oracle.c through ctypes; it shares no code with the CUDA library and
takes its inputs from workloads/.
"""
from .oracle import (  # noqa: F401
    build, lib, OracleBasis, gauss_legendre, radial_shells, cutoff, tabulate, spline_eval,
    ylm_spherical, solid_harmonic, K_lm, becke_weight, partition_weight, PARTITIONS, grid, grid_near, centres,
    Pattern,
)

"""Seeded inputs shared by the oracle, the tests and the benchmark.

This module holds data and random numbers only, none of the method's
arithmetic:

* ``DVM_TABLES``: the discrete velocity models exactly as the paper prints
  them (one representative velocity per symmetry group, the group size, the
  group weight and the lattice speed c), Appendix A and Appendix B tables.
  Expanding a group into its velocities, projecting 3D sets onto the (x, z)
  plane and every check of the tables are done separately by the oracle and
  by the library.
* ``rho_field``: the seeded density perturbation of the channel runs.
* ``batch_workload`` / ``serving_workload``: seeded lists of channel solves.
"""
from .tables import DVM_TABLES, TEXTBOOK_TABLES
from .fields import rho_field, kn_sweep, batch_workload, serving_workload

__all__ = ["DVM_TABLES", "TEXTBOOK_TABLES", "rho_field", "kn_sweep",
           "batch_workload", "serving_workload"]

"""CPU FP64 oracle of the nested-grid multigrid Poisson solver.

TEST INFRASTRUCTURE ONLY: imported by the tests, the package smoke check and
the benchmark's CPU-baseline/reference arm, never by the product path.
"""

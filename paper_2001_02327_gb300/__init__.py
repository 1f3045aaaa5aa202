"""GB300 (sm_103a) nested-grid multigrid Poisson solver.

``paper_2001_02327_gb300.mg`` is the ctypes binding of the C ABI in
``include/mg.h`` (libmg.so, built by ``paper_2001_02327_gb300.build``);
``paper_2001_02327_gb300.inputs`` generates seeded synthetic workloads.
Importing the package loads nothing; importing ``mg`` loads libmg.so and
raises if it has not been built.
"""

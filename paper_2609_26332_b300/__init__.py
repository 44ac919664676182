"""B300-native coupled phase-field / surfactant / flow lattice Boltzmann solver.

The hot path is hand-written CUDA for sm_103a behind a C ABI (``include/surflbm.h``);
``binding`` marshals arguments to it.  Importing this package loads nothing native:
``from paper_2609_26332_b300 import binding`` does, and fails loudly if the library
is missing.
"""

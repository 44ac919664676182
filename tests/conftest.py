"""Shared pytest configuration.

Markers: ``gpu`` tests need a CUDA device and call the C-ABI library; everything
else runs on the CPU (oracle pins, host logic, library load/export checks).
"""
import os
import sys

# one BLAS thread per process: the oracle works on small arrays and the suite runs
# its slow pins in parallel worker processes
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled sm_103a library")
    config.addinivalue_line("markers", "slow: long oracle relaxation (still CPU-only)")

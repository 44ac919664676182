"""FP64 CPU oracle for the coupled phase-field / surfactant / flow lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports, calls or links
anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg of ``bench.py`` use it.  It shares no code with the CUDA path: the two meet only
through the seeded input generators in ``paper_2609_26332_b300.inputs`` (which hold
none of the method's arithmetic).

The oracle is the algorithm written out step by step in numpy float64 from the
paper (Huang, Chai, Liu, Huang, "A thermodynamically consistent and conservative
phase-field model for surfactant contact line dynamics with solid adsorption"):

* ``params``   - parameter derivation (Sec. 2.1, Sec. 3, Sec. 4 dimensionless groups)
* ``lattice``  - D2Q9 velocities, weights, the natural-moment MRT basis (Sec. 3)
* ``lbm``      - the three coupled MRT lattice Boltzmann equations (Sec. 3)
* ``analysis`` - contact angle, zero-level-set area, free energy (Sec. 4)
* ``warmstart`` - the warm-start network (convolutions, adjoints, loss) in float64
* ``mms``      - manufactured-solution convergence harness of the scalar equations (Sec. 4.1)
* ``lattice3d``, ``lbm3d`` - the same scheme in three dimensions on D3Q19 (Sec. 2.3 states
  the model for d = 2, 3), single relaxation time, x and z periodic, y walls

Pins (tests that tie it to something other than itself) live in
``tests/test_oracle_*.py``.  Parts without such a pin are marked "parity unpinned"
in their docstrings.
"""

from .params import OracleParams, Wall, derive
from .lbm import Oracle
from .lbm3d import Oracle3D

__all__ = ["OracleParams", "Wall", "derive", "Oracle", "Oracle3D"]

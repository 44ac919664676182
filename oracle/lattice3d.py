"""D3Q19 lattice constants of the oracle's three-dimensional extension.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Sec. 2.3 states the model for d = 2, 3;
Sec. 3 writes the lattice Boltzmann scheme for a DdQq lattice.

Velocity ordering: rest, the six axis links (+x, -x, +y, -y, +z, -z), then the twelve
edge diagonals in the xy, xz and yz planes.  Weights 1/3, 1/18, 1/36; c_s^2 = 1/3.
"""

import numpy as np

_V = [(0, 0, 0),
      (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0),
      (1, 0, 1), (-1, 0, 1), (-1, 0, -1), (1, 0, -1),
      (0, 1, 1), (0, -1, 1), (0, -1, -1), (0, 1, -1)]
CX = np.array([v[0] for v in _V], dtype=np.int64)
CY = np.array([v[1] for v in _V], dtype=np.int64)
CZ = np.array([v[2] for v in _V], dtype=np.int64)
Q = 19
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12, dtype=np.float64)
CS2 = 1.0 / 3.0


def _index(v):
    return _V.index(v)


# opposite direction, and the direction with the y component reversed (specular
# reflection at a y-wall)
OPP = np.array([_index((-a, -b, -c)) for (a, b, c) in _V], dtype=np.int64)
MIRY = np.array([_index((a, -b, c)) for (a, b, c) in _V], dtype=np.int64)

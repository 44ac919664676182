"""D2Q9 lattice constants and the MRT transform used by the oracle (Sec. 3).

The paper does not print the transformation matrix M.  The oracle uses the
natural (raw) moment basis ordered to match the relaxation matrix
S = diag(s0, s1, s1, s2, s2, s2, s3, s3, s4) of Sec. 3:

    [1, cx, cy, cx^2, cx*cy, cy^2, cx^2*cy, cx*cy^2, cx^2*cy^2]

With all rates equal, M^-1 S M = s I whatever M is, so the choice only matters for
runs with distinct rates.
"""

import numpy as np

# velocity ordering: rest, four axis links, four diagonals
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.int64)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.int64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)
# direction with the y component reversed (specular reflection at a y-wall)
MIRY = np.array([0, 1, 4, 3, 2, 8, 7, 6, 5], dtype=np.int64)
CS2 = 1.0 / 3.0
Q = 9


def moment_matrix():
    """Rows are the natural moments evaluated on the nine velocities."""
    cx = CX.astype(np.float64)
    cy = CY.astype(np.float64)
    rows = [np.ones(Q), cx, cy, cx * cx, cx * cy, cy * cy, cx * cx * cy, cx * cy * cy, cx * cx * cy * cy]
    return np.array(rows, dtype=np.float64)


def rate_vector(s0, s1, s2, s3, s4):
    """Diagonal of S in the order of ``moment_matrix`` (Sec. 3, relaxation matrices)."""
    return np.array([s0, s1, s1, s2, s2, s2, s3, s3, s4], dtype=np.float64)

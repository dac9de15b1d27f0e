"""Oracle: direct solution of [M + S] p = s (Section 3.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper factorises the impedance matrix with a sparse direct solver in
single precision.  The oracle solves the same assembled system exactly in
complex128: banded LU (scipy.linalg.solve_banded -> LAPACK gbsv) for grids up
to ~36^3, dense LU (numpy.linalg.solve) for tiny grids.  The point source of
Section 3.1 (s = delta(x - x_s)) is a grid-node delta of amplitude 1/h^3.

Optional "mass-spread" source (a reading, not the paper's stated source): the
delta is distributed over the 27 nodes with the consistent-mass weights of the
source row (wm1 centre, wm2 faces, wm3 edges, wm4 corners).  With the plain
delta every phase-exact weight set has far-field amplitude 1/(1 - (kh)^2/12)
along the axes (26 % high at G = 4, since X = 1 - cos(a) on an axis for any
ws); the spread source cancels that factor to leading order, which is the
accuracy level of the paper's Table 2 (0.024 for G4 at G = 4).

Pins (tests/test_oracle_solve.py): banded == dense to 1e-12 on small grids
and ||s - A p|| / ||s|| <= 1e-12; the homogeneous solution approaches the
analytic Green's function and improves when the PML thickens.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def point_sources(shape, h, nodes, amps=None, mass_w7=None):
    """Right-hand sides (R, nz, ny, nx) complex128, one RHS per entry of
    ``nodes`` = [(ix, iy, iz)]: amp/h^3 at the node, or, when ``mass_w7`` (one
    7-weight row per source, the weights of the source row) is given, amp/h^3
    times the mass weight of each of the 27 surrounding nodes inside the grid."""
    nz, ny, nx = shape
    s = np.zeros((len(nodes), nz, ny, nx), dtype=np.complex128)
    for r, (ix, iy, iz) in enumerate(nodes):
        a = 1.0 if amps is None else amps[r]
        if mass_w7 is None:
            s[r, iz, iy, ix] = a / h ** 3
            continue
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    k, j, i = iz + dz, iy + dy, ix + dx
                    if 0 <= k < nz and 0 <= j < ny and 0 <= i < nx:
                        s[r, k, j, i] += a * mass_w7[r][3 + abs(dx) + abs(dy) + abs(dz)] / h ** 3
    return s


def bandwidth(shape):
    nz, ny, nx = shape
    return nx * ny + nx + 1


def solve_banded(A, b):
    """Solve A x = b with A's band (kl = ku = n_x n_y + n_x + 1) by LAPACK
    banded LU.  b: (N,) or (N, R)."""
    N = A.shape[0]
    Ad = A.tocoo()
    k = int(np.max(np.abs(Ad.col - Ad.row)))
    ab = np.zeros((2 * k + 1, N), dtype=np.complex128)
    ab[k + Ad.row - Ad.col, Ad.col] = Ad.data
    return sla.solve_banded((k, k), ab, b, check_finite=False)


def solve_dense(A, b):
    return np.linalg.solve(A.toarray(), b)


def relative_residual(A, x, b):
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))

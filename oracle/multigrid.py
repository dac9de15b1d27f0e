"""Oracle: textbook multigrid pieces of the complex-shifted-Laplacian (CSL)
preconditioner.  NOT IN THE PAPER (the paper uses a direct solver); these are
the plain definitions the GPU preconditioner is built from, so that each GPU
kernel can be checked on its own.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Vertex-centred coarsening: coarse node I sits on fine node 2I, so an axis of
  n fine nodes has (n + 1) // 2 coarse nodes.  Values beyond the grid are 0.
* Trilinear prolongation P: fine node i takes the coarse value at i/2 when i is
  even, the mean of its two coarse neighbours when odd (per axis, tensorised).
* Full-weighting restriction R = P^T / 8: weights 1/8 (centre), 1/16 (faces),
  1/32 (edges), 1/64 (corners) on the 27 fine nodes around 2I.
* Damped Jacobi: x <- x + omega_J D^{-1} (b - A x), D = diag(A).
* Coarse velocity by injection v_c[I] = v[2I]; the coarse operator is the same
  27-point row (``operator.row_coefficients``) at spacing 2h with the fine
  level's physical PML profile, the same shift, and 1/G clamped to the table.

Pins (tests/test_oracle_multigrid.py): P reproduces trilinear functions
exactly at interior fine nodes; R == P^T / 8 as matrices; the Jacobi
iteration's fixed point is A^{-1} b.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def coarse_shape(shape):
    return tuple((n + 1) // 2 for n in shape)


def _prolong_1d(n_fine):
    n_c = (n_fine + 1) // 2
    P = sp.lil_matrix((n_fine, n_c))
    for i in range(n_fine):
        if i % 2 == 0:
            P[i, i // 2] = 1.0
        else:
            P[i, i // 2] = 0.5
            if i // 2 + 1 < n_c:
                P[i, i // 2 + 1] = 0.5
    return P.tocsr()


def prolongation_matrix(shape):
    """P as a sparse matrix (fine N x coarse N), lexicographic x fastest."""
    nz, ny, nx = shape
    return sp.kron(sp.kron(_prolong_1d(nz), _prolong_1d(ny)), _prolong_1d(nx)).tocsr()


def restriction_matrix(shape):
    return (prolongation_matrix(shape).T / 8.0).tocsr()


def prolong(e_c, fine_shape):
    """e_c: (R, nzc, nyc, nxc) -> (R, nz, ny, nx)."""
    P = prolongation_matrix(fine_shape)
    R = e_c.shape[0]
    return (P @ e_c.reshape(R, -1).T).T.reshape((R,) + tuple(fine_shape))


def restrict(r_f):
    """r_f: (R, nz, ny, nx) -> (R, nzc, nyc, nxc)."""
    shape = r_f.shape[1:]
    Rm = restriction_matrix(shape)
    R = r_f.shape[0]
    return (Rm @ r_f.reshape(R, -1).T).T.reshape((R,) + coarse_shape(shape))


def inject_velocity(v):
    return np.ascontiguousarray(v[::2, ::2, ::2])


def jacobi_sweep(A, x, b, omega_j):
    """One damped-Jacobi sweep on (R, N) arrays."""
    d = A.diagonal()
    r = b - (A @ x.T).T
    return x + omega_j * r / d[None, :]

"""Oracle: rows of the impedance matrix [M + S] (Section 2.1, Eqs. 3-8).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Discrete problem (Eq. 3): [M + S] p = s on an n_x x n_y x n_z grid, unknowns
ordered lexicographically with x fastest (row r = ix + n_x (iy + n_y iz)),
constant density b = 1 (Section 3.1), kappa = v^2, exp(-i omega t).  Points
outside the grid are zero (Dirichlet behind the PML); stencil entries that
would reach them are dropped.

Stiffness (Eq. 4: S = ws1 S1 + ws2/3 sum S2,i + ws3/4 sum S3,i).  The paper
names two equivalent constructions (rotated-coordinate staggered grids, or
the "average-derivative" mixed stencil of Min et al. 2000 / Chen 2012); the
explicit rotated-frame PML handling is not in the text.  Reading used here:

    S p = sum_{d in x,y,z}  T_d [ delta_d p ]

* delta_d is the stretched second difference along d (see ``pml``):
  delta_x p(i) = [ (p(i+1)-p(i))/xi(i+1/2) - (p(i)-p(i-1))/xi(i-1/2) ] / (xi(i) h^2)
* T_d averages over the 3x3 plane transverse to d with the row's weights:
  centre t0 = ws1 + 2 ws2/3 + ws3/2, each of the 4 in-plane face neighbours
  t1 = ws2/12, each of the 4 in-plane corners t2 = ws3/8.

In the interior (xi = 1) this gives the class coefficients
  c0 = -6 t0/h^2, c_face = (t0 - ws2/3)/h^2, c_edge = (ws2/6 - ws3/4)/h^2,
  c_corner = 3 ws3/(8 h^2),
which equal ws1 x (7-point) + ws2 x (the average of the three rotated 11-point
stencils) + ws3 x (the average of the four diagonal stencils): their
plane-wave symbol is -(2/h^2) X with X the radicand of Eq. vtilde.

Mass: second form of Eq. 8 (kappa at the collocation point; its second sum
must run over 12 points): (omega^2/v_0^2) [wm1 p0 + wm2 sum_6 faces +
wm3 sum_12 edges + wm4 sum_8 corners], per-point weights (see ``weights``).
For the complex-shifted Laplacian used by the GPU preconditioner omega^2 is
replaced by (1 + i beta) omega^2 (beta = 0 is the paper's operator).

Weights per row (GA stencil, Section 3.1): interpolated in the table at the
row's own 1/G = f h / v.  GAm (Section 3.1): the row's weights are the mean
of the weights of the 27 stencil points, each looked up at its own 1/G.
Reading: the mean runs over the stencil points inside the grid (at a grid
edge the missing points carry no velocity).

Mass, first form of Eq. 8 (``mass_form=1``): each of the 27 points enters
with its own 1/kappa, i.e. the coefficient of neighbour j is
(omega^2 / v_j^2) w_class(j) instead of (omega^2 / v_0^2) w_class(j).

Heterogeneous density and attenuation (Eq. 2, Eqs. 1.1-1.4; the paper's
benchmarks keep b = 1 and no attenuation, Section 3.1): with buoyancy b = 1/rho
each stretched second difference becomes the conservative form
  [b(i+1/2)(p(i+1)-p(i))/xi(i+1/2) - b(i-1/2)(p(i)-p(i-1))/xi(i-1/2)] / (xi(i) h^2)
on its own stencil line, b at a half node the mean of its two nodes (b at the
node where the other lies outside the grid); the mass omega^2/kappa becomes
omega^2 b / c*^2 with the complex velocity c* = v (1 - i/(2Q)), so plane waves
decay as exp(-Im(k) r) for exp(-i omega t).  The weights stay those of the
real G = v / (f h).  Pins (tests/test_oracle_medium.py): b = 1 and 1/Q = 0
give the operator above; a constant b scales A; the 7-point weights give the
textbook variable-coefficient Laplacian D^T diag(b_half) D assembled from
difference matrices; an attenuated homogeneous solve decays at the rate of
the complex wavenumber.

Pins of the variants (tests/test_oracle_operator_variants.py): on a constant
model both reduce to the GA / second-form operator; with weights that do not
depend on the row (the non-adaptive G4 / Gm stencils) and no PML, the first
mass form is the transpose of the second (M1 = W diag(m) = (diag(m) W)^T
with W symmetric); a pure-Python loop over rows and stencil points on tiny
grids gives the same rows (GAm averages, class stencils of Eq. 4); with a
table linear in 1/G and 1/G quadratic along x, u0 + c x^2, GAm's row at
column x equals the Eq. 4 classes at the closed-form mean u0 + c (x^2 + 2/3).

Pins (tests/test_oracle_operator.py): interior symbol == m J - 2X/h^2 on a
periodic box (Eq. vtilde, independent formulas); stiffness annihilates
constants and linear fields and maps x^2+y^2+z^2 to 6; ws=(1,0,0), wm=(1,0,0,0)
gives the Kronecker-sum 7-point Laplacian with PML (scipy.sparse.kron); a
homogeneous model with any weights equals a Kronecker assembly of
delta_d (x) T_d; every row of a heterogeneous model equals the row of the
homogeneous model with that row's velocity.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import pml as _pml
from . import weights as _w

OFFSETS = tuple(itertools.product((-1, 0, 1), repeat=3))   # (dk, dj, di)


def axis_coefficients(prof, n, h, omega):
    """Per-node coefficients of delta_d towards i+1 (up) and i-1 (dn)."""
    xi_i, xi_h = _pml.xi_nodes(prof, n, h, omega)
    up = 1.0 / (xi_i * xi_h[1:] * h * h)
    dn = 1.0 / (xi_i * xi_h[:-1] * h * h)
    return up, dn


def profiles_for(shape, h, npml, v_ref, r_coef):
    """Physical profiles (x, y, z) for a grid of shape (nz, ny, nx) with
    npml = (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi) nodes."""
    nz, ny, nx = shape
    return (_pml.Profile1D.from_grid(nx, h, npml[0], npml[1], v_ref, r_coef),
            _pml.Profile1D.from_grid(ny, h, npml[2], npml[3], v_ref, r_coef),
            _pml.Profile1D.from_grid(nz, h, npml[4], npml[5], v_ref, r_coef))


def _neighbour(v, ix, iy, iz, si, sj, sk):
    """Velocity of stencil point (si, sj, sk) of each row and whether it lies
    inside the grid (outside: the row's own velocity, never used)."""
    nz, ny, nx = v.shape
    jx, jy, jz = ix + si, iy + sj, iz + sk
    ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
    vj = v[np.where(ok, jz, iz), np.where(ok, jy, iy), np.where(ok, jx, ix)].astype(np.float64)
    return vj, ok


def _field_at(a, jx, jy, jz):
    """a at (jx, jy, jz) with the indices clamped into the grid."""
    nz, ny, nx = a.shape
    return a[np.clip(jz, 0, nz - 1), np.clip(jy, 0, ny - 1), np.clip(jx, 0, nx - 1)].astype(np.float64)


def _half_buoyancy(b, px, py, pz, d, s):
    """b at the half node between point p and its neighbour p + s e_d (Eq. 2
    with heterogeneous buoyancy).  Reading: the arithmetic mean of the two
    nodes; where the neighbour lies outside the grid, b at p."""
    nz, ny, nx = b.shape
    q = [px, py, pz]
    q[d] = q[d] + s
    inside = (q[0] >= 0) & (q[0] < nx) & (q[1] >= 0) & (q[1] < ny) & (q[2] >= 0) & (q[2] < nz)
    bp = _field_at(b, px, py, pz)
    return np.where(inside, 0.5 * (bp + _field_at(b, q[0], q[1], q[2])), bp)


def row_coefficients(v, h, f, profiles, table, inv_g_nodes, rows=None, beta=0.0, weights="GA",
                     mass_form=2, buoyancy=None, inv_q=None):
    """27 complex coefficients for the requested rows.

    v: float array (nz, ny, nx); rows: flat row indices (None = all rows);
    weights: "GA" (the row's own G) or "GAm" (mean over the stencil points);
    mass_form: 2 (kappa at the collocation point) or 1 (kappa at each point);
    buoyancy: b = 1/rho per node (None: 1, the paper's benchmarks);
    inv_q: 1/Q per node (None: 0, no attenuation).
    Returns coef of shape (len(rows), 27) in OFFSETS order (dk, dj, di) and the
    validity mask (neighbour inside the grid)."""
    if weights not in ("GA", "GAm") or mass_form not in (1, 2):
        raise ValueError("weights must be GA or GAm, mass_form 1 or 2")
    nz, ny, nx = v.shape
    omega = 2.0 * np.pi * f
    if rows is None:
        rows = np.arange(nx * ny * nz)
    rows = np.asarray(rows, dtype=np.int64)
    ix = rows % nx
    iy = (rows // nx) % ny
    iz = rows // (nx * ny)
    v0 = v.reshape(-1)[rows].astype(np.float64)

    if weights == "GA":
        w = _w.lookup(table, inv_g_nodes, f * h / v0)
    else:
        acc = np.zeros((rows.size, 7))
        cnt = np.zeros(rows.size)
        for sk, sj, si in OFFSETS:
            vj, ok = _neighbour(v, ix, iy, iz, si, sj, sk)
            acc += np.where(ok[:, None], _w.lookup(table, inv_g_nodes, f * h / vj), 0.0)
            cnt += ok
        w = acc / cnt[:, None]
    ws1, ws2, ws3, wm1, wm2, wm3, wm4 = (w[:, k] for k in range(7))
    tw = (ws1 + 2.0 * ws2 / 3.0 + 0.5 * ws3, ws2 / 12.0, ws3 / 8.0)   # T_d weights
    mu = (wm1, wm2, wm3, wm4)                                        # mass per class

    def mass_at(jx, jy, jz, vj):
        # omega^2 / kappa* with kappa* = rho c*^2, c* = v (1 - i/(2Q)) (decay
        # for exp(-i omega t)); (1 + i beta) for the shifted operator
        mj = (1.0 + 1j * beta) * omega ** 2 / vj ** 2
        if buoyancy is not None:
            mj = mj * _field_at(buoyancy, jx, jy, jz)
        if inv_q is not None:
            mj = mj / (1.0 - 0.5j * _field_at(inv_q, jx, jy, jz)) ** 2
        return mj

    m = mass_at(ix, iy, iz, v0)

    ux, dx = axis_coefficients(profiles[0], nx, h, omega)
    uy, dy = axis_coefficients(profiles[1], ny, h, omega)
    uz, dz = axis_coefficients(profiles[2], nz, h, omega)

    def second(up, dn, i, s):
        if s == 1:
            return up[i]
        if s == -1:
            return dn[i]
        return -(up[i] + dn[i])

    coef = np.zeros((rows.size, 27), dtype=np.complex128)
    valid = np.zeros((rows.size, 27), dtype=bool)
    def second_b(up, dn, i, s, d, line):
        # the same along axis d on the stencil line through point `line`
        # (buoyancy at the line's half nodes)
        bp = _half_buoyancy(buoyancy, *line, d, +1)
        bm = _half_buoyancy(buoyancy, *line, d, -1)
        if s == 1:
            return up[i] * bp
        if s == -1:
            return dn[i] * bm
        return -(up[i] * bp + dn[i] * bm)

    for k, (sk, sj, si) in enumerate(OFFSETS):
        mk = m
        if mass_form == 1:
            vj, _ = _neighbour(v, ix, iy, iz, si, sj, sk)
            mk = mass_at(ix + si, iy + sj, iz + sk, vj)
        if buoyancy is None:
            sx, sy, sz = second(ux, dx, ix, si), second(uy, dy, iy, sj), second(uz, dz, iz, sk)
        else:
            sx = second_b(ux, dx, ix, si, 0, (ix, iy + sj, iz + sk))
            sy = second_b(uy, dy, iy, sj, 1, (ix + si, iy, iz + sk))
            sz = second_b(uz, dz, iz, sk, 2, (ix + si, iy + sj, iz))
        c = (tw[abs(sj) + abs(sk)] * sx + tw[abs(si) + abs(sk)] * sy + tw[abs(si) + abs(sj)] * sz
             + mk * mu[abs(si) + abs(sj) + abs(sk)])
        coef[:, k] = c
        valid[:, k] = ((ix + si >= 0) & (ix + si < nx) & (iy + sj >= 0) & (iy + sj < ny)
                       & (iz + sk >= 0) & (iz + sk < nz))
    return coef, valid


def assemble_csr(v, h, f, profiles, table, inv_g_nodes, beta=0.0, weights="GA", mass_form=2,
                 buoyancy=None, inv_q=None):
    """The impedance matrix as scipy CSR (complex128), 27 entries per row
    (fewer at the grid edges)."""
    nz, ny, nx = v.shape
    N = nx * ny * nz
    rows = np.arange(N)
    coef, valid = row_coefficients(v, h, f, profiles, table, inv_g_nodes, rows, beta, weights, mass_form,
                                   buoyancy, inv_q)
    cols = np.empty((N, 27), dtype=np.int64)
    for k, (sk, sj, si) in enumerate(OFFSETS):
        cols[:, k] = rows + si + nx * (sj + ny * sk)
    r = np.repeat(rows, 27).reshape(N, 27)
    A = sp.csr_matrix((coef[valid], (r[valid], cols[valid])), shape=(N, N))
    A.sort_indices()
    return A


def apply_rows(v, h, f, profiles, table, inv_g_nodes, x, rows, beta=0.0, weights="GA", mass_form=2,
               buoyancy=None, inv_q=None):
    """(A x) at the requested rows only, x of shape (R, nz, ny, nx); returns
    (R, len(rows)).  Used to check full-size GPU applies on sampled outputs."""
    nz, ny, nx = v.shape
    coef, valid = row_coefficients(v, h, f, profiles, table, inv_g_nodes, rows, beta, weights, mass_form,
                                   buoyancy, inv_q)
    rows = np.asarray(rows, dtype=np.int64)
    ix = rows % nx
    iy = (rows // nx) % ny
    iz = rows // (nx * ny)
    xf = x.reshape(x.shape[0], -1)
    out = np.zeros((x.shape[0], rows.size), dtype=np.complex128)
    for k, (sk, sj, si) in enumerate(OFFSETS):
        ok = valid[:, k]
        col = (ix + si) + nx * ((iy + sj) + ny * (iz + sk))
        col = np.where(ok, col, 0)
        out += np.where(ok, coef[:, k], 0.0)[None, :] * xf[:, col]
    return out


def interior_class_coefficients(w7, h, omega, v, beta=0.0):
    """(c0, c_face, c_edge, c_corner) of an interior row (xi = 1) written out
    from the class decomposition of Eq. 4: ws1 x 7-point, ws2 x mean of the
    three 11-point stencils, ws3 x mean of the four diagonal stencils, plus the
    mass of Eq. 8 -- an independent route to the same numbers as
    ``row_coefficients`` away from the PML."""
    ws1, ws2, ws3, wm1, wm2, wm3, wm4 = w7
    m = (1.0 + 1j * beta) * omega ** 2 / v ** 2
    # class stencils (centre, face, edge, corner) times h^2
    s1 = (-6.0, 1.0, 0.0, 0.0)
    s2 = (-4.0, 1.0 / 3.0, 1.0 / 6.0, 0.0)
    s3 = (-3.0, 0.5, -0.25, 3.0 / 8.0)
    mass = (wm1, wm2, wm3, wm4)
    return tuple((ws1 * s1[k] + ws2 * s2[k] + ws3 * s3[k]) / h ** 2 + m * mass[k] for k in range(4))

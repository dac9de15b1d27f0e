"""Pins of the oracle's impedance-matrix rows (Section 2.1, Eqs. 3-8).

The row is checked against: the plane-wave symbol of Eq. vtilde (independent
formulas), consistency of the stiffness on polynomials, the textbook 7-point
Laplacian with stretched coordinates assembled by scipy.sparse.kron, a
Kronecker assembly of the transverse-averaged form for homogeneous models, the
class decomposition of Eq. 4, and the continuous PML operator on a smooth
function (calculus, O(h^2)).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import operator as O
from oracle import pml as P
from oracle import weights as W


def _const_table(w7, n=5):
    nodes = np.linspace(0.0, 0.4, n)
    return nodes, np.tile(np.asarray(w7, dtype=np.float64), (n, 1))


def _no_pml(shape, h):
    return O.profiles_for(shape, h, (0,) * 6, 1500.0, 1e-3)


W_GENERIC = np.array([0.3, 0.5, 0.2, 0.55, 0.04, 0.012, 0.0])
W_GENERIC[6] = (1 - W_GENERIC[3] - 6 * W_GENERIC[4] - 12 * W_GENERIC[5]) / 8


def _interior_rows(shape, margin=1):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(margin, nz - margin), np.arange(margin, ny - margin),
                          np.arange(margin, nx - margin), indexing="ij")
    return (i + nx * (j + ny * k)).ravel()


@pytest.mark.parametrize("theta,phi,inv_g", [(0.3, 0.2, 0.17), (1.1, 0.6, 0.31), (0.0, 0.0, 0.05)])
def test_interior_symbol_matches_eq_vtilde(theta, phi, inv_g):
    # A plane wave exp(i k.x) is an eigenfunction of the interior stencil with
    # eigenvalue m J - (2/h^2) X, X and J from Eq. vtilde.
    shape, h, f, v = (7, 8, 9), 10.0, 12.0, 1800.0
    inv_g_nodes, table = _const_table(W_GENERIC)
    vel = np.full(shape, v, dtype=np.float32)
    kh = 2 * np.pi * inv_g
    d = np.array([np.cos(phi) * np.cos(theta), np.cos(phi) * np.sin(theta), np.sin(phi)])
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    p = np.exp(1j * kh * (d[0] * x + d[1] * y + d[2] * z))[None]
    rows = _interior_rows(shape)
    Ap = O.apply_rows(vel, h, f, _no_pml(shape, h), table, inv_g_nodes, p, rows)[0]
    omega = 2 * np.pi * f
    X = W.stiffness_X(inv_g, theta, phi, W_GENERIC)
    J = W.mass_J(inv_g, theta, phi, W_GENERIC)
    lam = omega ** 2 / v ** 2 * J - 2.0 * X / h ** 2
    assert np.allclose(Ap, lam * p.reshape(-1)[rows], rtol=1e-12, atol=1e-15)


def test_stiffness_consistency_on_polynomials():
    # With zero mass weights the row is S alone: S 1 = 0, S x = 0, and
    # S (x^2 + y^2 + z^2) = 6 (in grid units, divided by h^2 -> times h^2 here).
    shape, h = (6, 7, 8), 3.0
    w7 = W_GENERIC.copy()
    w7[3:] = 0.0
    nodes, table = _const_table(w7)
    vel = np.full(shape, 2000.0, dtype=np.float32)
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float) for n in shape), indexing="ij")
    rows = _interior_rows(shape)
    for field, expect in ((np.ones(shape), 0.0), (x + 2 * y - z, 0.0),
                          (x ** 2 + y ** 2 + z ** 2, 6.0 / h ** 2)):
        out = O.apply_rows(vel, h, 7.0, _no_pml(shape, h), table, nodes, field[None], rows)[0]
        assert np.allclose(out, expect, atol=1e-12)


def test_seven_point_with_pml_is_kronecker_sum():
    # ws = (1,0,0), wm = (1,0,0,0): the row is the 7-point stretched Laplacian
    # plus lumped mass; assemble it independently as a Kronecker sum of the
    # 1-D operators (scipy.sparse.kron) and compare every entry.
    shape, h, f = (7, 6, 9), 20.0, 6.0
    npml = (2, 3, 1, 2, 3, 2)
    nodes, table = _const_table([1, 0, 0, 1, 0, 0, 0])
    rng = np.random.default_rng(0)
    vel = rng.uniform(1500, 3000, size=shape).astype(np.float32)
    prof = O.profiles_for(shape, h, npml, 3000.0, 1e-3)
    A = O.assemble_csr(vel, h, f, prof, table, nodes)
    omega = 2 * np.pi * f
    nz, ny, nx = shape
    D = []
    for ax, n in enumerate((nx, ny, nz)):
        xi_i, xi_h = P.xi_nodes(prof[ax], n, h, omega)
        D.append(sp.csr_matrix(P.second_difference_1d(n, h, xi_i, xi_h)))
    I = [sp.identity(n) for n in (nx, ny, nz)]
    K = (sp.kron(sp.kron(I[2], I[1]), D[0]) + sp.kron(sp.kron(I[2], D[1]), I[0])
         + sp.kron(sp.kron(D[2], I[1]), I[0]))
    K = K + sp.diags(omega ** 2 / vel.reshape(-1).astype(float) ** 2)
    assert abs(A - K).max() < 1e-14 * abs(K).max()


def test_homogeneous_rows_equal_kronecker_form():
    # Homogeneous model, generic weights, PML on: S = sum_d delta_d (x) T_d and
    # M = sum over classes of wm_c (sum of shifts), each built with sparse kron.
    shape, h, f, v = (6, 7, 5), 15.0, 8.0, 2100.0
    npml = (2, 1, 2, 2, 1, 2)
    nodes, table = _const_table(W_GENERIC)
    vel = np.full(shape, v, dtype=np.float32)
    prof = O.profiles_for(shape, h, npml, 2500.0, 1e-3)
    A = O.assemble_csr(vel, h, f, prof, table, nodes)
    omega = 2 * np.pi * f
    nz, ny, nx = shape
    ws1, ws2, ws3, wm1, wm2, wm3, wm4 = W_GENERIC
    t0, t1, t2 = ws1 + 2 * ws2 / 3 + ws3 / 2, ws2 / 12, ws3 / 8

    def shift_sum(n):       # ones on the two off-diagonals
        return sp.diags([np.ones(n - 1), np.ones(n - 1)], [-1, 1])

    def T2(na, nb):         # transverse 3x3 average on a (b slower, a faster) plane
        Ia, Ib = sp.identity(na), sp.identity(nb)
        Ea, Eb = shift_sum(na), shift_sum(nb)
        return t0 * sp.kron(Ib, Ia) + t1 * (sp.kron(Eb, Ia) + sp.kron(Ib, Ea)) + t2 * sp.kron(Eb, Ea)

    D = []
    for ax, n in enumerate((nx, ny, nz)):
        xi_i, xi_h = P.xi_nodes(prof[ax], n, h, omega)
        D.append(sp.csr_matrix(P.second_difference_1d(n, h, xi_i, xi_h)))
    Ix, Iy, Iz = (sp.identity(n) for n in (nx, ny, nz))
    Ex, Ey, Ez = (shift_sum(n) for n in (nx, ny, nz))
    # x-term: T over (z, y) kron D_x ; y-term: T over (z, x) with D_y in the middle
    Sx = sp.kron(T2(ny, nz), D[0])
    Sy = (t0 * sp.kron(sp.kron(Iz, D[1]), Ix) + t1 * (sp.kron(sp.kron(Ez, D[1]), Ix)
          + sp.kron(sp.kron(Iz, D[1]), Ex)) + t2 * sp.kron(sp.kron(Ez, D[1]), Ex))
    Sz = sp.kron(D[2], T2(nx, ny))
    # mass: class c counts the nonzero offsets; expand products of (I + E)
    M = sp.csr_matrix((nx * ny * nz, nx * ny * nz))
    mu = (wm1, wm2, wm3, wm4)
    for az, Mz in ((0, Iz), (1, Ez)):
        for ay, My in ((0, Iy), (1, Ey)):
            for ax_, Mx in ((0, Ix), (1, Ex)):
                M = M + mu[az + ay + ax_] * sp.kron(sp.kron(Mz, My), Mx)
    K = Sx + Sy + Sz + (omega ** 2 / v ** 2) * M
    assert abs(A - K).max() < 1e-13 * abs(K).max()


def test_heterogeneous_row_equals_homogeneous_row_at_its_velocity():
    # GA stencil: row i uses only v_i (weights at its own G and kappa_0 = v_i^2).
    shape, h, f = (6, 6, 7), 25.0, 9.0
    npml = (2,) * 6
    nodes, table = W.fit_table(d_inv_g=0.02)
    rng = np.random.default_rng(5)
    vel = rng.uniform(1500, 4000, size=shape).astype(np.float32)
    prof = O.profiles_for(shape, h, npml, 4000.0, 1e-3)
    rows = rng.choice(vel.size, size=12, replace=False)
    coef, valid = O.row_coefficients(vel, h, f, prof, table, nodes, rows)
    for k, r in enumerate(rows):
        vh = np.full(shape, vel.reshape(-1)[r], dtype=np.float32)
        ch, vh_ok = O.row_coefficients(vh, h, f, prof, table, nodes, [r])
        assert np.array_equal(valid[k], vh_ok[0])
        assert np.allclose(coef[k], ch[0], rtol=1e-14, atol=0)


def test_interior_class_decomposition():
    # Away from the PML every row has the cubic-symmetric class form; its four
    # numbers from Eq. 4's class decomposition equal the assembled ones.
    shape, h, f = (7, 7, 7), 25.0, 9.0
    nodes, table = W.fit_table(d_inv_g=0.02)
    rng = np.random.default_rng(11)
    vel = rng.uniform(1500, 4000, size=shape).astype(np.float32)
    rows = _interior_rows(shape, 2)
    coef, _ = O.row_coefficients(vel, h, f, _no_pml(shape, h), table, nodes, rows, beta=0.5)
    omega = 2 * np.pi * f
    for k, r in enumerate(rows):
        v = float(vel.reshape(-1)[r])
        w7 = W.lookup(table, nodes, f * h / v)
        c = O.interior_class_coefficients(w7, h, omega, v, beta=0.5)
        cls = np.array([abs(a) + abs(b) + abs(cc) for a, b, cc in O.OFFSETS])
        for q in range(4):
            assert np.allclose(coef[k, cls == q], c[q], rtol=1e-13)


def test_stretched_second_difference_converges_to_continuous_operator():
    # (1/xi) d/dx ((1/xi) dp/dx) for p = sin(kx) on a layer with quadratic gamma:
    # compare against the derivative computed by calculus; error falls like h^2.
    errs = []
    for n in (41, 81, 161):
        L = 1000.0
        h = L / (n - 1)
        omega, g0 = 2 * np.pi * 3.0, 40.0
        prof = P.Profile1D(x_lo=0.0, x_hi=0.0, len_lo=0.0, len_hi=L, g0_lo=0.0, g0_hi=g0)
        xi_i, xi_h = P.xi_nodes(prof, n, h, omega)
        D = P.second_difference_1d(n, h, xi_i, xi_h)
        x = np.arange(n) * h
        k = 2 * np.pi / 400.0
        p = np.sin(k * x)
        xi = 1 + 1j * g0 * (x / L) ** 2 / omega
        dxi = 1j * g0 * 2 * x / L ** 2 / omega
        exact = (-(dxi / xi ** 3) * k * np.cos(k * x) - k ** 2 * np.sin(k * x) / xi ** 2)
        inner = slice(n // 4, n - 2)
        errs.append(np.max(np.abs((D @ p)[inner] - exact[inner])))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_pml_profile_reading():
    prof = P.Profile1D.from_grid(20, 25.0, 4, 4, 1500.0, 1e-3)
    g = prof.gamma(np.arange(20) * 25.0)
    assert np.all(g[4:16] == 0) and g[0] > g[1] > g[2] > g[3] > 0
    L = 4 * 25.0
    assert np.isclose(g[0], 3 * 1500.0 / (2 * L) * np.log(1e3))
    assert np.allclose(g[::-1], g)

"""Pins of the oracle's operator variants (Section 3.1 GAm weights; first
consistent-mass form of Eq. 8), independent of the oracle's own vectorised
assembly: special cases that reduce to the pinned GA / second-form operator,
the transpose identity between the two mass forms, and a pure-Python loop
over rows and stencil points on tiny grids."""
import itertools

import numpy as np
import pytest

from oracle import operator as O
from oracle import weights as W


@pytest.fixture(scope="module")
def table():
    return W.fit_table()


def _model(shape, seed, lo=1500.0, hi=3500.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)


def test_variants_reduce_to_ga_on_a_constant_model(table):
    nodes, T = table
    v = np.full((7, 6, 8), 2100.0, np.float32)
    prof = O.profiles_for(v.shape, 25.0, (2, 2, 1, 2, 2, 1), 2100.0, 1e-3)
    ref, valid = O.row_coefficients(v, 25.0, 7.0, prof, T, nodes, beta=0.4)
    for weights, mass_form in (("GAm", 2), ("GA", 1), ("GAm", 1)):
        c, ok = O.row_coefficients(v, 25.0, 7.0, prof, T, nodes, beta=0.4, weights=weights,
                                   mass_form=mass_form)
        assert np.array_equal(ok, valid)
        np.testing.assert_allclose(c[valid], ref[valid], rtol=1e-13, atol=0)


def test_first_mass_form_is_the_transpose_of_the_second_with_fixed_weights(table):
    # With weights that do not depend on the row (non-adaptive G4) and no PML,
    # S and W are symmetric constant-coefficient stencils, so
    # S + W diag(m) = (S + diag(m) W)^T.
    nodes, _ = table
    g4 = np.tile(W.expand_weights(W.fit_joint([0.25])[None, :])[0], (len(nodes), 1))
    v = _model((6, 7, 5), 3)
    prof = O.profiles_for(v.shape, 20.0, (0,) * 6, 3500.0, 1e-3)
    A2 = O.assemble_csr(v, 20.0, 6.0, prof, g4, nodes)
    A1 = O.assemble_csr(v, 20.0, 6.0, prof, g4, nodes, mass_form=1)
    scale = abs(A2).max()
    assert abs(A1 - A2.T).max() <= 1e-13 * scale
    assert abs(A1 - A2).max() > 1e-3 * scale          # the forms do differ here
    # with the PML the stiffness is no longer symmetric, but the difference of
    # the two forms is still the mass commutator W diag(m) - diag(m) W
    prof = O.profiles_for(v.shape, 20.0, (1,) * 6, 3500.0, 1e-3)
    D = (O.assemble_csr(v, 20.0, 6.0, prof, g4, nodes, mass_form=1)
         - O.assemble_csr(v, 20.0, 6.0, prof, g4, nodes))
    assert abs(D + D.T).max() <= 1e-13 * scale        # antisymmetric


def _brute_rows(v, h, f, table, weights, mass_form, beta):
    """Rows of the operator without PML by loops: the weights (the row's own,
    or the mean over the in-grid stencil points), the class stencils of Eq. 4
    via ``interior_class_coefficients`` and the mass of either form."""
    nodes, T = table
    nz, ny, nx = v.shape
    omega = 2.0 * np.pi * f
    out = {}
    for iz, iy, ix in itertools.product(range(nz), range(ny), range(nx)):
        pts = []
        for sk, sj, si in itertools.product((-1, 0, 1), repeat=3):
            jx, jy, jz = ix + si, iy + sj, iz + sk
            if 0 <= jx < nx and 0 <= jy < ny and 0 <= jz < nz:
                pts.append(((sk, sj, si), float(v[jz, jy, jx])))
        v0 = float(v[iz, iy, ix])
        if weights == "GA":
            w7 = W.lookup(T, nodes, f * h / v0)
        else:
            w7 = sum(W.lookup(T, nodes, f * h / vj) for _, vj in pts) / len(pts)
        stiff = O.interior_class_coefficients(np.concatenate([w7[:3], np.zeros(4)]), h, omega, v0)
        for off, vj in pts:
            cls = sum(abs(o) for o in off)
            vm = vj if mass_form == 1 else v0
            out[(ix + nx * (iy + ny * iz), off)] = stiff[cls] + (1 + 1j * beta) * omega ** 2 / vm ** 2 * w7[3 + cls]
    return out


@pytest.mark.parametrize("weights,mass_form", [("GAm", 2), ("GA", 1), ("GAm", 1)])
def test_variant_rows_match_a_loop_over_stencil_points(table, weights, mass_form):
    nodes, T = table
    v = _model((3, 5, 4), 11)
    prof = O.profiles_for(v.shape, 25.0, (0,) * 6, 3500.0, 1e-3)
    coef, valid = O.row_coefficients(v, 25.0, 9.0, prof, T, nodes, beta=0.3, weights=weights,
                                     mass_form=mass_form)
    ref = _brute_rows(v, 25.0, 9.0, table, weights, mass_form, 0.3)
    n = 0
    for (row, off), c in ref.items():
        k = O.OFFSETS.index(off)
        assert valid[row, k]
        assert abs(coef[row, k] - c) <= 1e-12 * abs(c) + 1e-15
        n += 1
    assert n == valid.sum()


def test_unknown_variant_is_refused(table):
    nodes, T = table
    v = np.full((3, 3, 3), 1500.0, np.float32)
    prof = O.profiles_for(v.shape, 25.0, (0,) * 6, 1500.0, 1e-3)
    with pytest.raises(ValueError):
        O.row_coefficients(v, 25.0, 5.0, prof, T, nodes, weights="G4")
    with pytest.raises(ValueError):
        O.row_coefficients(v, 25.0, 5.0, prof, T, nodes, mass_form=3)


def test_gam_weights_are_the_table_at_the_stencil_mean_of_a_quadratic_inverse_g():
    # With a table linear in 1/G the interpolation is exact, so GAm's weights at
    # a row are the table at the mean of 1/G over its 27 stencil points.  For
    # 1/G quadratic along x, u = u0 + c x^2, that mean at column x is
    # u0 + c (x^2 + 2/3), since each of the offsets -1, 0, 1 carries 9 of the 27
    # points.  A 7-point mean (2/7), a mean without the corners or without the
    # row itself, or a divisor other than 27 each miss it by about 1e-3 of the
    # coefficients.  The row's classes then follow from Eq. 4 through
    # interior_class_coefficients (no PML, so every row is an interior row).
    nodes = np.linspace(0.0, 0.4, 41)
    a = np.array([0.7, 0.2, 0.1, 0.5, 0.05, 0.02, 0.01])
    b = np.array([-0.8, 0.5, 0.3, 0.4, -0.1, 0.05, 0.02])
    T = a[None, :] + b[None, :] * nodes[:, None]
    f, h, beta = 5.0, 25.0, 0.3
    nz, ny, nx = 5, 5, 9
    u0, c = 0.12, 0.004
    xc = np.arange(nx) - 4.0
    u = u0 + c * xc ** 2
    v = np.broadcast_to((f * h / u)[None, None, :], (nz, ny, nx)).astype(np.float64)
    prof = O.profiles_for(v.shape, h, (0,) * 6, float(v.max()), 1e-3)
    rows = [ix + nx * (iy + ny * iz) for iz in range(1, nz - 1) for iy in range(1, ny - 1)
            for ix in range(1, nx - 1)]
    coef, ok = O.row_coefficients(v, h, f, prof, T, nodes, rows=rows, weights="GAm", beta=beta)
    assert ok.all()
    cls = np.array([abs(s[0]) + abs(s[1]) + abs(s[2]) for s in O.OFFSETS])
    for r, row in enumerate(rows):
        ix = row % nx
        w7 = a + b * (u0 + c * (xc[ix] ** 2 + 2.0 / 3.0))
        want = np.array(O.interior_class_coefficients(w7, h, 2.0 * np.pi * f, f * h / u[ix], beta=beta))
        np.testing.assert_allclose(coef[r], want[cls], rtol=1e-12, atol=0)
    # the same rows with GA use the row's own 1/G and differ at this size
    ga, _ = O.row_coefficients(v, h, f, prof, T, nodes, rows=rows, weights="GA", beta=beta)
    assert np.max(np.abs(ga - coef)) > 1e-4 * np.max(np.abs(coef))

"""Pins of the oracle's heterogeneous-density and attenuation operator (Eq. 2
with buoyancy b = 1/rho; complex velocity c* = v (1 - i/(2Q))), independent of
the oracle's own assembly loop: the reductions to the constant-density
operator, the scaling by a constant b, the textbook variable-coefficient
7-point Laplacian assembled from difference matrices (scipy.sparse), and the
decay rate of an attenuated wave solved by banded LU."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import operator as O
from oracle import solve as S
from oracle import weights as W


@pytest.fixture(scope="module")
def table():
    return W.fit_table()


def _model(shape, seed, lo, hi):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(np.float32)


def test_unit_buoyancy_and_no_attenuation_reduce_to_the_operator(table):
    nodes, T = table
    v = _model((6, 7, 9), 1, 1500.0, 3500.0)
    prof = O.profiles_for(v.shape, 25.0, (2, 1, 2, 2, 1, 2), 3500.0, 1e-3)
    ref, valid = O.row_coefficients(v, 25.0, 7.0, prof, T, nodes, beta=0.3)
    c, ok = O.row_coefficients(v, 25.0, 7.0, prof, T, nodes, beta=0.3, buoyancy=np.ones_like(v),
                               inv_q=np.zeros_like(v))
    assert np.array_equal(ok, valid)
    np.testing.assert_allclose(c[valid], ref[valid], rtol=1e-14, atol=0)


@pytest.mark.parametrize("mass_form", [2, 1])
def test_constant_buoyancy_scales_the_operator(table, mass_form):
    # b constant: div(b grad p) + omega^2 b / v^2 p = b (laplacian p + omega^2/v^2 p)
    nodes, T = table
    v = _model((5, 8, 7), 2, 1500.0, 3000.0)
    prof = O.profiles_for(v.shape, 20.0, (2,) * 6, 3000.0, 1e-3)
    ref, valid = O.row_coefficients(v, 20.0, 8.0, prof, T, nodes, mass_form=mass_form)
    c, _ = O.row_coefficients(v, 20.0, 8.0, prof, T, nodes, mass_form=mass_form,
                              buoyancy=np.full_like(v, 0.375))
    np.testing.assert_allclose(c[valid], 0.375 * ref[valid], rtol=1e-13, atol=0)


def _face_buoyancy(b, axis):
    """b on the n+1 faces along `axis` (0 = x): interior faces the mean of
    their two nodes, the two boundary faces the boundary node's b."""
    a = np.moveaxis(b.astype(np.float64), 2 - axis, -1)
    f = np.concatenate([a[..., :1], 0.5 * (a[..., 1:] + a[..., :-1]), a[..., -1:]], axis=-1)
    return np.moveaxis(f, -1, 2 - axis)


def test_seven_point_weights_give_the_conservative_laplacian(table):
    # ws = (1, 0, 0), wm = (1, 0, 0, 0), no PML: the row is
    #   sum_d [b(i+1/2)(p(i+1)-p(i)) - b(i-1/2)(p(i)-p(i-1))] / h^2 + omega^2 b/v^2 p,
    # i.e. -sum_d D_d^T diag(b_faces) D_d / h^2 + diag(omega^2 b / v^2) with D_d
    # the node-to-face difference matrices (zero outside the grid).
    nodes, _ = table
    T7 = np.tile([1.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0], (len(nodes), 1))
    nz, ny, nx = shape = (5, 6, 7)
    v = _model(shape, 3, 1500.0, 3000.0)
    b = _model(shape, 4, 0.3, 1.0)
    h, f = 20.0, 6.0
    prof = O.profiles_for(shape, h, (0,) * 6, 3000.0, 1e-3)
    A = O.assemble_csr(v, h, f, prof, T7, nodes, buoyancy=b)

    def d1(n):                       # (n+1) x n: faces -1|0 ... n-1|n
        return sp.diags([np.ones(n), -np.ones(n)], [0, -1], shape=(n + 1, n))

    I = sp.identity
    D = [sp.kron(I(nz), sp.kron(I(ny), d1(nx))),
         sp.kron(I(nz), sp.kron(d1(ny), I(nx))),
         sp.kron(d1(nz), sp.kron(I(ny), I(nx)))]
    L = sum(-(Dd.T @ sp.diags(_face_buoyancy(b, ax).reshape(-1)) @ Dd) for ax, Dd in enumerate(D)) / h ** 2
    omega = 2 * np.pi * f
    ref = L + sp.diags((omega ** 2 * b.astype(np.float64) / v.astype(np.float64) ** 2).reshape(-1))
    assert abs(A - ref).max() <= 1e-12 * abs(ref).max()


def test_attenuation_decays_at_the_complex_wavenumber(table):
    # homogeneous medium, constant Q: |p(r)| r falls off as exp(-Im(k*) r),
    # k* = omega / c*, c* = v (1 - i/(2Q)); without attenuation it stays flat
    nodes, T = table
    n, h, v0, f, npml = 31, 25.0, 1500.0, 7.5, 6      # G = 8
    v = np.full((n, n, n), v0, np.float32)
    prof = O.profiles_for(v.shape, h, (npml,) * 6, v0, 1e-3)
    c = n // 2
    s = S.point_sources(v.shape, h, [(c, c, c)])[0].reshape(-1)
    omega = 2 * np.pi * f
    r1, r2 = 3, 8                                     # nodes from the source along the axes
    rates = {}
    for q in (None, 25.0):
        iq = None if q is None else np.full_like(v, 1.0 / q)
        A = O.assemble_csr(v, h, f, prof, T, nodes, inv_q=iq)
        p = S.solve_banded(A, s).reshape(v.shape)
        amp = lambda r: np.mean([abs(p[c, c, c + r]), abs(p[c, c + r, c]), abs(p[c + r, c, c]),
                                 abs(p[c, c, c - r]), abs(p[c, c - r, c]), abs(p[c - r, c, c])]) * r
        rates[q] = np.log(amp(r1) / amp(r2)) / ((r2 - r1) * h)
    im_k = omega / v0 * (0.5 / 25.0) / (1 + 0.25 / 25.0 ** 2)
    assert abs(rates[None]) < 0.1 * im_k                 # lossless: flat (to the PML / grid error)
    assert abs((rates[25.0] - rates[None]) - im_k) < 0.05 * im_k

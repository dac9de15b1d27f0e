"""Pins of the textbook multigrid pieces (not in the paper)."""
import numpy as np
import scipy.sparse as sp

from oracle import multigrid as MG


def test_prolongation_exact_on_trilinear_functions():
    shape = (9, 7, 11)          # odd: coarse nodes on both ends
    cz, cy, cx = MG.coarse_shape(shape)
    Z, Y, X = np.meshgrid(np.arange(cz) * 2.0, np.arange(cy) * 2.0, np.arange(cx) * 2.0, indexing="ij")
    f = lambda x, y, z: 1 + 2 * x - y + 0.5 * z + 0.25 * x * y - z * x + 0.1 * x * y * z
    fine = MG.prolong(f(X, Y, Z)[None], shape)[0]
    z, y, x = np.meshgrid(*(np.arange(n, dtype=float) for n in shape), indexing="ij")
    assert np.allclose(fine, f(x, y, z), atol=1e-12)


def test_restriction_is_scaled_transpose_and_weights():
    shape = (5, 6, 7)
    R = MG.restriction_matrix(shape)
    P = MG.prolongation_matrix(shape)
    assert abs(R - P.T / 8).max() == 0
    # an interior coarse node sees 1/8, 1/16, 1/32, 1/64 on 1, 6, 12, 8 fine nodes
    nz, ny, nx = shape
    cz, cy, cx = MG.coarse_shape(shape)
    I = 1 + cx * (1 + cy * 1)
    row = R.getrow(I).toarray().ravel()
    vals = np.sort(row[row > 0])
    assert np.allclose(np.unique(vals), [1 / 64, 1 / 32, 1 / 16, 1 / 8])
    assert np.isclose(row.sum(), 1.0)


def test_jacobi_fixed_point():
    rng = np.random.default_rng(0)
    n = 30
    A = sp.diags([rng.uniform(4, 5, n) + 1j, -np.ones(n - 1), -np.ones(n - 1)], [0, 1, -1]).tocsr()
    b = rng.normal(size=(2, n)) + 0j
    x = np.linalg.solve(A.toarray(), b.T).T
    assert np.allclose(MG.jacobi_sweep(A, x, b, 0.7), x, atol=1e-13)
    y = np.zeros_like(b)
    for _ in range(200):
        y = MG.jacobi_sweep(A, y, b, 0.8)
    assert np.allclose(y, x, atol=1e-10)


def _two_grid_rate(npml, cap=None, n=17, f=5.0, beta=1.0, nu=2, om=0.6):
    # asymptotic error reduction of damped-Jacobi two-grid cycles with an exact
    # Galerkin coarse solve on the shifted operator (oracle pieces only)
    import scipy.sparse.linalg as spl
    from oracle import operator as O
    from oracle import pml as PM
    from oracle import weights as W
    from paper_2108_08730_gb300 import synth
    nodes, T = W.fit_table(d_inv_g=0.01)
    wl = synth.linear_gradient(n=n, npml=npml, f=f)
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    if cap is not None:
        w = 2 * np.pi * f
        prof = tuple(PM.Profile1D(p.x_lo, p.x_hi, p.len_lo, p.len_hi, min(p.g0_lo, cap * w),
                                  min(p.g0_hi, cap * w)) for p in prof)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes, beta=beta).tocsr()
    P = MG.prolongation_matrix(wl.shape)
    R = MG.restriction_matrix(wl.shape)
    lu = spl.splu((R @ A @ P).tocsc())
    d = A.diagonal()
    rng = np.random.default_rng(0)
    e = rng.normal(size=A.shape[0]) + 1j * rng.normal(size=A.shape[0])
    rate = 0.0
    for _ in range(10):
        r = A @ e
        x = om * r / d
        for _ in range(nu - 1):
            x = x + om * (r - A @ x) / d
        x = x + P @ lu.solve(R @ (r - A @ x))
        for _ in range(nu):
            x = x + om * (r - A @ x) / d
        e2 = e - x
        rate = np.linalg.norm(e2) / np.linalg.norm(e)
        e = e2
    return rate


def test_pml_stretching_breaks_jacobi_two_grid_and_cap_restores_it():
    # The reason the preconditioner caps its PML damping (gamma/omega <= 1):
    # without a PML the two-grid cycle contracts; with the full PML
    # (gamma/omega ~ 5 at the outer edge) it diverges; with the cap it contracts.
    assert _two_grid_rate(npml=0) < 0.5
    assert _two_grid_rate(npml=4) > 1.0
    assert _two_grid_rate(npml=4, cap=1.0) < 0.8

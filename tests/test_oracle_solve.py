"""Pins of the oracle's direct solves (Section 3.1-3.3).

Banded LU is checked against dense LU and by its residual (brute force on
tiny grids); the solution of the assembled system is checked against the
analytic Green's functions, including the closed-form far-field amplitude of
the grid-delta source derived from the stencil's symbol."""
import numpy as np
import pytest

from oracle import analytic as AN
from oracle import metrics as M
from oracle import operator as O
from oracle import solve as S
from oracle import weights as W
from paper_2108_08730_gb300 import synth


@pytest.fixture(scope="module")
def table():
    return W.fit_table()


@pytest.mark.parametrize("shape", [(5, 6, 7), (8, 8, 8)])
def test_banded_equals_dense(shape, table):
    nodes, T = table
    v = synth.random_velocity(shape, 11, 1500, 3000)
    prof = O.profiles_for(shape, 25.0, (2, 2, 1, 2, 2, 1), 3000.0, 1e-3)
    A = O.assemble_csr(v, 25.0, 8.0, prof, T, nodes)
    b = synth.random_field(shape, 2, 3).reshape(2, -1).T
    xb = S.solve_banded(A, b)
    xd = S.solve_dense(A, b)
    assert np.max(np.abs(xb - xd)) <= 1e-12 * np.max(np.abs(xd))
    for r in range(2):
        assert S.relative_residual(A, xb[:, r], b[:, r]) <= 1e-12


def _homog_solution(table, n, npml, f, spread, h=25.0):
    nodes, T = table
    wl = synth.homogeneous(n=n, npml=npml, f=f, h=h)
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    mw = [W.lookup(T, nodes, f * h / 1500.0)] if spread else None
    s = S.point_sources(wl.shape, wl.h, wl.sources, mass_w7=mw)
    p = S.solve_banded(A, s.reshape(-1)).reshape(wl.shape)
    c = wl.sources[0]
    ratios = []
    for d in (3, 4, 5):
        for (dx, dy, dz) in ((d, 0, 0), (0, d, 0), (d, d, 0), (d, d, d)):
            r = h * np.sqrt(dx * dx + dy * dy + dz * dz)
            ratios.append(p[c[2] + dz, c[1] + dy, c[0] + dx] / AN.green_homog(r, 0, 0, (0, 0, 0), 1500.0, f))
    return p, np.array(ratios), wl


@pytest.mark.parametrize("f", [5.0, 10.0])
def test_delta_source_far_field_amplitude(table, f):
    # Along the axes X = 1 - cos(a) for any ws, so a phase-exact stencil has
    # symbol slope -2k (1 - (kh)^2/12) on the characteristic surface and the
    # grid-delta source radiates with amplitude 1/(1 - (kh)^2/12) (10 % at G=6).
    _, ratios, wl = _homog_solution(table, 26, 7, f, spread=False)
    kh2 = (2 * np.pi * f * wl.h / 1500.0) ** 2
    expect = 1.0 / (1.0 - kh2 / 12.0)
    assert np.all(np.abs(ratios - expect) < 0.01 * expect), (ratios, expect)


@pytest.mark.parametrize("f", [5.0, 10.0])
def test_mass_spread_source_matches_analytic(table, f):
    # The mass-spread source cancels that factor: the discrete wavefield is the
    # analytic -exp(ikr)/(4 pi r) to <1 % at r = 3..5 h for G = 6 and 12.
    _, ratios, _ = _homog_solution(table, 26, 7, f, spread=True)
    assert np.all(np.abs(ratios - 1.0) < 0.01), ratios


def test_pml_absorbs(table):
    # Thin PML reflects more: the interior error against the analytic solution
    # (mass-spread source, G = 12) grows when npml drops from 7 to 1.
    errs = []
    for npml in (7, 1):
        _, ratios, _ = _homog_solution(table, 26, npml, 5.0, spread=True)
        errs.append(np.max(np.abs(ratios - 1.0)))
    assert errs[0] < 0.01 and errs[1] > 3 * errs[0], errs


def test_gradient_model_matches_analytic(table):
    # v = v0 + alpha z on a 24^3 grid (h = 20 m, f = 5 Hz, G = 15..18): the
    # mass-spread solution follows the analytic gradient-medium field.
    nodes, T = table
    n, h, f, npml = 24, 20.0, 5.0, 6
    wl = synth.linear_gradient(n=n, h=h, f=f, npml=npml)
    wl.sources[0] = (12, 12, 9)
    prof = O.profiles_for(wl.shape, h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, h, f, prof, T, nodes)
    c = wl.sources[0]
    mw = [W.lookup(T, nodes, f * h / float(wl.v[c[2], c[1], c[0]]))]
    s = S.point_sources(wl.shape, h, wl.sources, mass_w7=mw)
    p = S.solve_banded(A, s.reshape(-1)).reshape(wl.shape)
    z, y, x = np.meshgrid(*(np.arange(k) * h for k in wl.shape), indexing="ij")
    src = (c[0] * h, c[1] * h, c[2] * h)
    r = np.sqrt((x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2)
    inner = np.zeros(wl.shape, bool)
    inner[npml:n - npml, npml:n - npml, npml:n - npml] = True
    mask = inner & (r >= 3 * h)
    ga = AN.green_gradient(x[mask], y[mask], z[mask], src, wl.meta["v0"], wl.meta["alpha"], f)
    assert M.rel_l2(p[mask], ga) < 0.02

"""GPU parity of the operator variants (Section 3.1 GAm weights, first
consistent-mass form of Eq. 8; hx_set_operator_form) against the oracle.

Same elementwise bound as the GA operator tests: |y_gpu - y_ref| <= tol *
sum_k |a_ik| |x_k|, tol = 1e-12 (FP64) and 2e-5 (FP32).  Row coefficients and
the assembled CSR to 1e-13 of the row scale.  Solves with a variant operator
(the preconditioner stays GA / second form) reach the oracle's relative
residual bound 1e-10 of the mixed-precision refinement.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operator as O
from oracle import solve as S
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth

TOL = {64: 1e-12, 32: 2e-5}
VARIANTS = [("GAm", 2), ("GA", 1), ("GAm", 1)]


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture
def ctx(otable):
    c = B.Context(0)
    c.set_table(otable[1], 0.001)
    yield c
    c.close()


# (shape (nz, ny, nx), h, f, npml, vmin, vmax): several tiles, ragged edges
CASES = [((13, 11, 37), 25.0, 6.0, (3, 2, 2, 3, 2, 3), 1500.0, 4500.0),
         ((7, 9, 8), 20.0, 9.0, (0,) * 6, 1800.0, 3000.0)]


def _bound_check(A, x, y_gpu, tol):
    Aabs = abs(A)
    for r in range(x.shape[0]):
        ref = A @ x[r].reshape(-1)
        bound = Aabs @ np.abs(x[r].reshape(-1))
        err = np.abs(y_gpu[r].reshape(-1) - ref)
        assert np.max(err / (bound + 1e-300)) <= tol


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"{v[0]}-m{v[1]}")
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_variant_apply_and_sweeps_match_oracle(ctx, otable, variant, prec, case):
    shape, h, f, npml, vmin, vmax = CASES[case]
    nodes, T = otable
    weights, mass_form = variant
    v = synth.random_velocity(shape, 300 + case, vmin, vmax)
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    beta = 0.5
    A = O.assemble_csr(v, h, f, prof, T, nodes, beta=beta, weights=weights, mass_form=mass_form)
    ctx.set_operator_form(weights, mass_form)
    g = B.make_grid(shape, h, f, npml, vmax)
    dt = torch.complex128 if prec == 64 else torch.complex64
    vd = torch.from_numpy(v).cuda()
    xd = torch.from_numpy(synth.random_field(shape, 3, 40 + case)).to(dt).cuda()
    bd = torch.from_numpy(synth.random_field(shape, 3, 50 + case)).to(dt).cuda()
    yd = torch.empty_like(xd)
    ctx.apply(g, vd, xd, yd, shift_beta=beta)
    torch.cuda.synchronize()
    x = xd.cpu().numpy().astype(np.complex128)
    b = bd.cpu().numpy().astype(np.complex128)
    _bound_check(A, x, yd.cpu().numpy().astype(np.complex128), TOL[prec])
    # residual and damped-Jacobi sweeps of the same operator
    ctx.sweep(g, vd, "residual", xd, bd, yd, shift_beta=beta)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.complex128).reshape(3, -1)
    for r in range(3):
        # the subtraction from b rounds at |b| as well
        ref = b[r].reshape(-1) - A @ x[r].reshape(-1)
        scale = abs(A) @ np.abs(x[r].reshape(-1)) + np.abs(b[r].reshape(-1))
        assert np.max(np.abs(got[r] - ref) / scale) <= TOL[prec]
    om = 0.6
    ctx.sweep(g, vd, "jacobi", xd, bd, yd, shift_beta=beta, omega=om)
    torch.cuda.synchronize()
    d = A.diagonal()
    got = yd.cpu().numpy().astype(np.complex128).reshape(3, -1)
    for r in range(3):
        ref = x[r].reshape(-1) + om * (b[r].reshape(-1) - A @ x[r].reshape(-1)) / d
        scale = np.abs(x[r].reshape(-1)) + om * (np.abs(b[r].reshape(-1)) + abs(A) @ np.abs(x[r].reshape(-1))) / np.abs(d)
        assert np.max(np.abs(got[r] - ref) / scale) <= 4 * TOL[prec]


@pytest.mark.parametrize("variant", VARIANTS, ids=lambda v: f"{v[0]}-m{v[1]}")
def test_variant_rows_and_csr_match_oracle(ctx, otable, variant):
    shape, h, f, npml, vmin, vmax = CASES[0]
    nodes, T = otable
    weights, mass_form = variant
    v = synth.random_velocity(shape, 310, vmin, vmax)
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    ref, valid = O.row_coefficients(v, h, f, prof, T, nodes, beta=0.25, weights=weights, mass_form=mass_form)
    ctx.set_operator_form(weights, mass_form)
    g = B.make_grid(shape, h, f, npml, vmax)
    vd = torch.from_numpy(v).cuda()
    coef = torch.empty(v.size * 27 * 2, dtype=torch.float64, device="cuda")
    ctx.row_coefficients(g, vd, coef, shift_beta=0.25)
    got = coef.cpu().numpy().view(np.complex128).reshape(-1, 27)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(np.where(valid, got - ref, got)) / scale) < 1e-13
    A = O.assemble_csr(v, h, f, prof, T, nodes, weights=weights, mass_form=mass_form)
    for fn in (ctx.assemble_csr, ctx.assemble_csr_noalloc):
        rowptr, col, val = fn(g, vd)
        assert np.array_equal(rowptr, A.indptr) and np.array_equal(col, A.indices)
        assert np.max(np.abs(val - A.data)) < 1e-13 * np.max(np.abs(A.data))


@pytest.mark.parametrize("variant", [("GAm", 2), ("GAm", 1)], ids=lambda v: f"{v[0]}-m{v[1]}")
def test_solve_with_a_variant_operator(ctx, otable, variant):
    # the Krylov operator and the FP64 residual use the variant; the
    # multigrid preconditioner stays GA / second form
    nodes, T = otable
    weights, mass_form = variant
    wl = synth.homogeneous(n=26, npml=5)
    wl.v = synth.random_velocity(wl.shape, 320, 1500.0, 2600.0)
    wl.v_ref = 2600.0
    ctx.set_operator_form(weights, mass_form)
    src = [(13, 12, 14, 0, 1.0), (9, 15, 10, 1, 1j)]
    out = torch.zeros((2,) + wl.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), src, 2, out)
    assert rep["status"] == 0
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes, weights=weights, mass_form=mass_form)
    s = S.point_sources(wl.shape, wl.h, [q[:3] for q in src], amps=[q[4] for q in src])
    p = out.cpu().numpy()
    for k in range(2):
        assert S.relative_residual(A, p[k].reshape(-1), s[k].reshape(-1)) <= 1e-10
    # the GA operator's solution is a different field
    A_ga = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    assert S.relative_residual(A_ga, p[0].reshape(-1), s[0].reshape(-1)) > 1e-6


def test_variant_settings_and_refusals(ctx, otable):
    with pytest.raises(B.HxError) as e:
        ctx.set_operator_form("G4", 2)
    assert e.value.code == -1
    with pytest.raises(B.HxError):
        ctx.set_operator_form("GA", 3)
    shape = (8, 9, 10)
    v = synth.random_velocity(shape, 330, 1500.0, 3000.0)
    g = B.make_grid(shape, 25.0, 6.0, (2,) * 6, 3000.0)
    vd = torch.from_numpy(v).cuda()
    x = torch.from_numpy(synth.random_field(shape, 1, 60)).to(torch.complex64).cuda()
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    ctx.apply(g, vd, x, y0)
    ctx.set_operator_form("GAm", 1)
    with pytest.raises(B.HxError) as e:           # the persistent batched kernel is GA only
        ctx.apply_batched([(g, vd, x, y1)])
    assert e.value.code == -7
    ctx.set_operator_form("GA", 2)                  # back to the z-marching kernel
    ctx.apply(g, vd, x, y1)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)

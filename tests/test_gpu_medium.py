"""GPU parity of the heterogeneous-density / attenuation operator
(hx_set_medium; Eq. 2 with buoyancy b = 1/rho, complex velocity
c* = v (1 - i/(2Q))) against the oracle.

Bounds as in test_gpu_operator_variants.py: apply and sweeps elementwise
against tol * (sum_k |a_ik| |x_k| (+ |b|)), tol = 1e-12 (FP64) / 2e-5 (FP32);
row coefficients and CSR to 1e-13 of the row scale; solves to the relative
residual 1e-10 of the oracle's assembled matrix.
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
SHAPE, H, F, NPML = (11, 13, 35), 25.0, 6.0, (3, 2, 2, 3, 2, 3)


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture
def ctx(otable):
    c = B.Context(0)
    c.set_table(otable[1], 0.001)
    yield c
    c.close()


def _medium(shape, seed):
    rng = np.random.default_rng(seed)
    v = synth.random_velocity(shape, seed, 1500.0, 4000.0)
    b = rng.uniform(0.35, 1.0, size=shape).astype(np.float32)        # 1 / (1000..2900 kg/m^3), scaled
    iq = rng.uniform(0.0, 0.05, size=shape).astype(np.float32)       # Q >= 20
    return v, b, iq


MEDIA = [("b", True, False), ("Q", False, True), ("bQ", True, True)]


@pytest.mark.parametrize("medium", MEDIA, ids=lambda m: m[0])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("mass_form", [2, 1])
def test_medium_apply_and_sweeps_match_oracle(ctx, otable, medium, prec, mass_form):
    nodes, T = otable
    _, use_b, use_q = medium
    v, b, iq = _medium(SHAPE, 400)
    bb, qq = (b if use_b else None), (iq if use_q else None)
    prof = O.profiles_for(SHAPE, H, NPML, float(v.max()), 1e-3)
    beta = 0.5
    A = O.assemble_csr(v, H, F, prof, T, nodes, beta=beta, mass_form=mass_form, buoyancy=bb, inv_q=qq)
    ctx.set_operator_form("GA", mass_form)
    ctx.set_medium(torch.from_numpy(b).cuda() if use_b else None, torch.from_numpy(iq).cuda() if use_q else None)
    g = B.make_grid(SHAPE, H, F, NPML, float(v.max()))
    dt = torch.complex128 if prec == 64 else torch.complex64
    vd = torch.from_numpy(v).cuda()
    xd = torch.from_numpy(synth.random_field(SHAPE, 2, 41)).to(dt).cuda()
    bd = torch.from_numpy(synth.random_field(SHAPE, 2, 42)).to(dt).cuda()
    yd = torch.empty_like(xd)
    x = xd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    rhs = bd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    Aabs = abs(A)
    ctx.apply(g, vd, xd, yd, shift_beta=beta)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    for r in range(2):
        assert np.max(np.abs(got[r] - A @ x[r]) / (Aabs @ np.abs(x[r]))) <= TOL[prec]
    ctx.sweep(g, vd, "residual", xd, bd, yd, shift_beta=beta)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    for r in range(2):
        scale = Aabs @ np.abs(x[r]) + np.abs(rhs[r])
        assert np.max(np.abs(got[r] - (rhs[r] - A @ x[r])) / scale) <= TOL[prec]
    ctx.sweep(g, vd, "jacobi", xd, bd, yd, shift_beta=beta, omega=0.6)
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    d = A.diagonal()
    for r in range(2):
        ref = x[r] + 0.6 * (rhs[r] - A @ x[r]) / d
        scale = np.abs(x[r]) + 0.6 * (np.abs(rhs[r]) + Aabs @ np.abs(x[r])) / np.abs(d)
        assert np.max(np.abs(got[r] - ref) / scale) <= 4 * TOL[prec]


@pytest.mark.parametrize("weights", ["GA", "GAm"])
def test_medium_rows_and_csr_match_oracle(ctx, otable, weights):
    nodes, T = otable
    v, b, iq = _medium(SHAPE, 410)
    prof = O.profiles_for(SHAPE, H, NPML, float(v.max()), 1e-3)
    ref, valid = O.row_coefficients(v, H, F, prof, T, nodes, beta=0.25, weights=weights, buoyancy=b, inv_q=iq)
    ctx.set_operator_form(weights, 2)
    bt, qt = torch.from_numpy(b).cuda(), torch.from_numpy(iq).cuda()
    ctx.set_medium(bt, qt)
    g = B.make_grid(SHAPE, H, F, NPML, float(v.max()))
    vd = torch.from_numpy(v).cuda()
    coef = torch.empty(v.size * 27 * 2, dtype=torch.float64, device="cuda")
    ctx.row_coefficients(g, vd, coef, shift_beta=0.25)
    got = coef.cpu().numpy().view(np.complex128).reshape(-1, 27)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(np.where(valid, got - ref, got)) / scale) < 1e-13
    A = O.assemble_csr(v, H, F, prof, T, nodes, weights=weights, buoyancy=b, inv_q=iq)
    for fn in (ctx.assemble_csr, ctx.assemble_csr_noalloc):
        rowptr, col, val = fn(g, vd)
        assert np.array_equal(rowptr, A.indptr) and np.array_equal(col, A.indices)
        assert np.max(np.abs(val - A.data)) < 1e-13 * np.max(np.abs(A.data))


def test_solve_in_a_heterogeneous_medium(ctx, otable):
    # density and attenuation in the Krylov operator and the FP64 residual;
    # the multigrid preconditioner keeps b = 1 and no Q
    nodes, T = otable
    wl = synth.homogeneous(n=26, npml=5)
    v, b, iq = _medium(wl.shape, 420)
    v = np.clip(v, 1500.0, 2600.0).astype(np.float32)
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, 2600.0, wl.r_coef)
    g = B.make_grid(wl.shape, wl.h, wl.f, wl.npml, 2600.0)
    ctx.set_medium(torch.from_numpy(b).cuda(), torch.from_numpy(iq).cuda())
    src = [(13, 12, 14, 0, 1.0), (9, 15, 10, 1, 1j)]
    out = torch.zeros((2,) + wl.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(g, torch.from_numpy(v).cuda(), src, 2, out)
    assert rep["status"] == 0
    A = O.assemble_csr(v, wl.h, wl.f, prof, T, nodes, buoyancy=b, inv_q=iq)
    s = S.point_sources(wl.shape, wl.h, [q[:3] for q in src], amps=[q[4] for q in src])
    p = out.cpu().numpy()
    for k in range(2):
        assert S.relative_residual(A, p[k].reshape(-1), s[k].reshape(-1)) <= 1e-10
    # and a medium-free operator would not fit this field
    A0 = O.assemble_csr(v, wl.h, wl.f, prof, T, nodes)
    assert S.relative_residual(A0, p[0].reshape(-1), s[0].reshape(-1)) > 1e-6


def test_medium_refusals_and_reset(ctx, otable):
    shape = (8, 9, 10)
    v = synth.random_velocity(shape, 430, 1500.0, 3000.0)
    g = B.make_grid(shape, 25.0, 6.0, (2,) * 6, 3000.0)
    vd = torch.from_numpy(v).cuda()
    x = torch.from_numpy(synth.random_field(shape, 1, 61)).to(torch.complex64).cuda()
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    ctx.apply(g, vd, x, y0)
    ctx.set_medium(torch.ones(shape, dtype=torch.float32, device="cuda"), None)
    with pytest.raises(B.HxError) as e:              # the persistent batched kernel has no medium
        ctx.apply_batched([(g, vd, x, y1)])
    assert e.value.code == -7
    ctx.set_medium(None, None)                        # back to b = 1, the z-marching kernel
    ctx.apply(g, vd, x, y1)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)

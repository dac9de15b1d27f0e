"""GPU parity of every launch configuration of the complex64 operator kernel
and of the residual / damped-Jacobi sweeps (Eq. 3 rows, Eqs. 4-8, GA weights)
against the oracle's assembled matrix, through the C ABI.

Tolerances (elementwise, against the natural bound of the 27-term complex
dot product, as in test_gpu_operator.py): FP32 2e-5, FP64 1e-12.
  residual  y = b - A x:            |y - y_ref| <= tol (|b| + |A||x|)
  Jacobi    y = x + w D^-1 (b - A x): |y - y_ref| <= tol (|x| + |w/D| (|b| + |A||x|))
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operator as O
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth

TOL = {64: 1e-12, 32: 2e-5}

# (shape (nz,ny,nx), h, f, npml, vmin, vmax): several x/y tiles, ragged tails,
# several z-chunks, PML on some faces only
CASES = [
    ((23, 19, 70), 25.0, 6.0, (3, 4, 2, 5, 4, 3), 1500.0, 4500.0),
    ((9, 9, 9), 20.0, 10.0, (2, 2, 2, 2, 2, 2), 1500.0, 3000.0),
    ((5, 33, 40), 30.0, 5.0, (0, 0, 0, 0, 0, 0), 2000.0, 5000.0),
    ((31, 37, 35), 25.0, 5.0, (6, 5, 4, 6, 5, 6), 1500.0, 4500.0),
]


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture(scope="module")
def ctx(otable):
    c = B.Context(0)
    c.set_table(otable[1], 0.001)
    yield c
    c.close()


_A = {}


def _problem(case, beta, otable):
    key = (case, beta)
    if key not in _A:
        shape, h, f, npml, vmin, vmax = CASES[case]
        nodes, T = otable
        v = synth.random_velocity(shape, 200 + case, vmin, vmax)
        prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
        A = O.assemble_csr(v, h, f, prof, T, nodes, beta=beta)
        _A[key] = (v, A, B.make_grid(shape, h, f, npml, vmax))
    return _A[key]


def test_config_table():
    cfgs = B.kernel_configs()
    assert len(cfgs) >= 3
    assert all(r >= 1 and k >= 1 for r, k in cfgs)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("cfg", range(3))
@pytest.mark.parametrize("nrhs", [1, 3, 6])
def test_apply32_every_config(ctx, otable, case, cfg, nrhs):
    beta = 0.5 if (case + cfg + nrhs) % 2 else 0.0
    v, A, g = _problem(case, beta, otable)
    x = synth.random_field(v.shape, nrhs, 31 + case + cfg)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    yd = torch.full_like(xd, complex(np.nan, np.nan))
    ctx.set_kernel_config(cfg)
    try:
        ctx.apply(g, torch.from_numpy(v).cuda(), xd, yd, shift_beta=beta)
        torch.cuda.synchronize()
    finally:
        ctx.set_kernel_config(-1)
    xr = xd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    y = yd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    ref = (A @ xr.T).T
    bound = (abs(A) @ np.abs(xr).T).T
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - ref) / bound) <= TOL[32]


def _sweep_ref(A, kind, x, b, omega):
    Ax = (A @ x.T).T
    bound = (abs(A) @ np.abs(x).T).T + (np.abs(b) if b is not None else 0)
    r = (b if b is not None else 0) - Ax
    if kind == "residual":
        return r, bound
    d = A.diagonal()[None, :]
    return x + omega * r / d, np.abs(x) + np.abs(omega / d) * bound


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["residual", "jacobi"])
@pytest.mark.parametrize("cfg", [-1, 0, 2])
def test_sweeps_match_oracle(ctx, otable, case, prec, kind, cfg):
    if prec == 64 and cfg != -1:
        pytest.skip("configurations select complex64 kernels only")
    beta = 0.5
    nrhs = 3
    v, A, g = _problem(case, beta, otable)
    dt = torch.complex64 if prec == 32 else torch.complex128
    x = synth.random_field(v.shape, nrhs, 41 + case)
    bb = synth.random_field(v.shape, nrhs, 51 + case)
    xd = torch.from_numpy(x).to(dt).cuda()
    bd = torch.from_numpy(bb).to(dt).cuda()
    yd = torch.full_like(xd, complex(np.nan, np.nan))
    omega = 0.6
    ctx.set_kernel_config(cfg)
    try:
        ctx.sweep(g, torch.from_numpy(v).cuda(), kind, xd, bd, yd, shift_beta=beta, omega=omega)
        torch.cuda.synchronize()
    finally:
        ctx.set_kernel_config(-1)
    xr = xd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    br = bd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    ref, bound = _sweep_ref(A, kind, xr, br, omega)
    y = yd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    assert np.max(np.abs(y - ref) / bound) <= TOL[prec]


def test_residual_without_b(ctx, otable):
    v, A, g = _problem(0, 0.5, otable)
    x = synth.random_field(v.shape, 2, 61)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    yd = torch.empty_like(xd)
    ctx.sweep(g, torch.from_numpy(v).cuda(), "residual", xd, None, yd, shift_beta=0.5)
    torch.cuda.synchronize()
    xr = xd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    ref, bound = _sweep_ref(A, "residual", xr, None, 0.0)
    y = yd.cpu().numpy().astype(np.complex128).reshape(2, -1)
    assert np.max(np.abs(y - ref) / bound) <= TOL[32]


def test_autotune_records_a_valid_choice(ctx, otable):
    v, A, g = _problem(3, 0.0, otable)
    vd = torch.from_numpy(v).cuda()
    best, ms = ctx.autotune(g, vd, 4, ncalls=2)
    assert 0 <= best < len(B.kernel_configs())
    assert all(t > 0 for t in ms) and ms[best] == min(ms)
    # the tuned configuration is used by later applies of that size and still matches
    x = synth.random_field(v.shape, 4, 71)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    yd = torch.empty_like(xd)
    ctx.apply(g, vd, xd, yd)
    torch.cuda.synchronize()
    xr = xd.cpu().numpy().astype(np.complex128).reshape(4, -1)
    ref = (A @ xr.T).T
    bound = (abs(A) @ np.abs(xr).T).T
    assert np.max(np.abs(yd.cpu().numpy().reshape(4, -1) - ref) / bound) <= TOL[32]


def test_sweep_and_config_errors(ctx):
    g = B.make_grid((8, 8, 8), 25.0, 5.0, (2,) * 6, 1500.0)
    v = torch.full((8, 8, 8), 1500.0, device="cuda")
    x = torch.zeros((1, 8, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(B.HxError):
        ctx.sweep(g, v, "jacobi", x, None, torch.empty_like(x))        # Jacobi needs b
    with pytest.raises(B.HxError):
        ctx.sweep(g, v, "residual", x, x, x)                           # aliasing
    with pytest.raises(B.HxError):
        ctx.set_kernel_config(99)


@pytest.mark.parametrize("cfg", range(3))
def test_apply32_long_z_reuses_the_ring(ctx, otable, cfg):
    # Enough tiles x RHS blocks that every configuration marches through many
    # z-planes per CTA, so each shared-memory ring slot is refilled several
    # times (odd nx, odd plane size: the parity offset of a slot alternates
    # with z); the x-boundary columns read the zero halo after every refill.
    shape, h, f, npml = (40, 64, 161), 25.0, 5.0, (5, 6, 4, 5, 6, 5)
    nrhs = 8
    key = ("long", cfg)
    if key not in _A:
        nodes, T = otable
        v = synth.random_velocity(shape, 300, 1500.0, 4500.0)
        prof = O.profiles_for(shape, h, npml, 4500.0, 1e-3)
        _A[key] = (v, O.assemble_csr(v, h, f, prof, T, nodes, beta=0.5), B.make_grid(shape, h, f, npml, 4500.0))
    v, A, g = _A[key]
    x = synth.random_field(shape, nrhs, 81 + cfg)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    yd = torch.full_like(xd, complex(np.nan, np.nan))
    ctx.set_kernel_config(cfg)
    try:
        ctx.apply(g, torch.from_numpy(v).cuda(), xd, yd, shift_beta=0.5)
        torch.cuda.synchronize()
    finally:
        ctx.set_kernel_config(-1)
    xr = xd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    y = yd.cpu().numpy().astype(np.complex128).reshape(nrhs, -1)
    ref = (A @ xr.T).T
    bound = (abs(A) @ np.abs(xr).T).T
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - ref) / bound) <= TOL[32]


def _batch_problems(otable):
    # uneven sizes, PML on some faces, different nrhs; each with its oracle matrix
    specs = [((23, 19, 70), (3, 4, 2, 5, 4, 3), 4), ((9, 9, 9), (2,) * 6, 1), ((31, 37, 35), (6, 5, 4, 6, 5, 6), 3),
             ((40, 64, 161), (5, 6, 4, 5, 6, 5), 2), ((5, 33, 40), (0,) * 6, 5)]
    out = []
    nodes, T = otable
    for k, (shape, npml, nrhs) in enumerate(specs):
        key = ("batch", k)
        if key not in _A:
            v = synth.random_velocity(shape, 400 + k, 1500.0, 4500.0)
            prof = O.profiles_for(shape, 25.0, npml, 4500.0, 1e-3)
            _A[key] = (v, O.assemble_csr(v, 25.0, 5.0, prof, T, nodes, beta=0.5),
                       B.make_grid(shape, 25.0, 5.0, npml, 4500.0))
        v, A, g = _A[key]
        x = torch.from_numpy(synth.random_field(shape, nrhs, 90 + k)).to(torch.complex64).cuda()
        out.append((g, torch.from_numpy(v).cuda(), x, A))
    return out


@pytest.mark.parametrize("cfg", [-1, 0, 1, 2])
def test_apply_batched_equals_single_applies(ctx, otable, cfg):
    probs = _batch_problems(otable)
    ys = [torch.full_like(x, complex(np.nan, np.nan)) for _, _, x, _ in probs]
    ctx.set_kernel_config(cfg)
    try:
        ctx.apply_batched([(g, v, x, y) for (g, v, x, _), y in zip(probs, ys)], shift_beta=0.5)
        torch.cuda.synchronize()
        singles = []
        for g, v, x, _ in probs:
            y1 = torch.empty_like(x)
            if cfg >= 0:
                ctx.apply(g, v, x, y1, shift_beta=0.5)       # same configuration: identical arithmetic
            singles.append(y1)
        torch.cuda.synchronize()
    finally:
        ctx.set_kernel_config(-1)
    for (g, v, x, A), y, y1 in zip(probs, ys, singles):
        yy = y.cpu().numpy().astype(np.complex128).reshape(x.shape[0], -1)
        xr = x.cpu().numpy().astype(np.complex128).reshape(x.shape[0], -1)
        ref = (A @ xr.T).T
        bound = (abs(A) @ np.abs(xr).T).T
        assert np.all(np.isfinite(yy))
        assert np.max(np.abs(yy - ref) / bound) <= TOL[32]
        if cfg >= 0 and g.nx % 2 == 1:
            # odd nx: hx_apply_operator runs the same cp.async kernel (even nx takes
            # the TMA kernel, which rounds in another order; checked against the oracle above)
            assert torch.equal(y, y1)


def test_apply_batched_replays_in_a_cuda_graph(ctx, otable):
    probs = _batch_problems(otable)
    ys = [torch.zeros_like(x) for _, _, x, _ in probs]
    items = [(g, v, x, y) for (g, v, x, _), y in zip(probs, ys)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.apply_batched(items, shift_beta=0.5, stream=s.cuda_stream)     # sizes the plan buffers
    torch.cuda.synchronize()
    want = [y.clone() for y in ys]
    for y in ys:
        y.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ctx.apply_batched(items, shift_beta=0.5, stream=s.cuda_stream)
    for _ in range(2):
        for y in ys:
            y.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for y, w in zip(ys, want):
            assert torch.equal(y, w)


def test_operator_table_role_changes_only_the_operator(ctx, otable):
    # hx_set_table_ex(..., HX_TABLE_OPERATOR): applies use the new table
    nodes, T = otable
    v, A, g = _problem(3, 0.0, otable)
    w7 = B.fit_joint_weights([0.25])
    fixed = B.fixed_table(w7, len(nodes))
    c = B.Context(0, table=T)
    c.set_table(fixed, role="operator")
    shape, h, f, npml, vmin, vmax = CASES[3]
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    Af = O.assemble_csr(v, h, f, prof, fixed, nodes)
    x = synth.random_field(shape, 1, 123)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    c.apply(g, torch.from_numpy(v).cuda(), xd, yd)
    torch.cuda.synchronize()
    xr = x.reshape(1, -1)
    ref = (Af @ xr.T).T
    bound = (abs(Af) @ np.abs(xr).T).T
    assert np.max(np.abs(yd.cpu().numpy().reshape(1, -1) - ref) / bound) <= TOL[64]
    c.close()

"""GPU parity of the matrix-free operator against the oracle (Eqs. 3-8).

All GPU calls go through the C ABI (paper_2108_08730_gb300.binding).  Both
sides use the oracle's weight table (installed with hx_set_table), so the
comparison isolates the row formation and the apply.  Tolerances, elementwise
against the natural bound of a 27-term complex dot product:
    |y_gpu - y_ref| <= tol * sum_k |a_ik| |x_k|
with tol = 1e-12 for the FP64 path and 2e-5 for the FP32 path (FP32 table,
coefficients and accumulation: a few ulps of 6e-8 times the cancellation in
the class coefficients).
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


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture(scope="module")
def ctx(otable):
    c = B.Context(0)
    c.set_table(otable[1], 0.001)
    yield c
    c.close()


def _cases():
    # (shape (nz,ny,nx), h, f, npml, vmin, vmax) -- several tiles + ragged tails
    return [
        ((23, 19, 70), 25.0, 6.0, (3, 4, 2, 5, 4, 3), 1500.0, 4500.0),
        ((9, 9, 9), 20.0, 10.0, (2, 2, 2, 2, 2, 2), 1500.0, 3000.0),
        ((5, 33, 40), 30.0, 5.0, (0, 0, 0, 0, 0, 0), 2000.0, 5000.0),
        ((20, 20, 20), 25.0, 10.0, (4, 4, 4, 4, 4, 4), 1500.0, 1500.0),
    ]


def _bound_check(A, x, y_gpu, tol):
    Aabs = abs(A)
    for r in range(x.shape[0]):
        ref = A @ x[r].reshape(-1)
        bound = Aabs @ np.abs(x[r].reshape(-1))
        err = np.abs(y_gpu[r].reshape(-1) - ref)
        worst = np.max(err / (bound + 1e-300))
        assert worst <= tol, (r, worst)


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nrhs", [1, 5])
@pytest.mark.parametrize("beta", [0.0, 0.5])
@pytest.mark.parametrize("direct", [False, True], ids=["tiled", "direct"])
def test_apply_matches_oracle_csr(ctx, otable, case, prec, nrhs, beta, direct):
    shape, h, f, npml, vmin, vmax = _cases()[case]
    nodes, T = otable
    v = synth.random_velocity(shape, 100 + case, vmin, vmax) if vmin < vmax else \
        np.full(shape, vmin, dtype=np.float32)
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    A = O.assemble_csr(v, h, f, prof, T, nodes, beta=beta)
    x = synth.random_field(shape, nrhs, 7 + case)
    dt = torch.complex128 if prec == 64 else torch.complex64
    g = B.make_grid(shape, h, f, npml, vmax)
    vd = torch.from_numpy(v).cuda()
    xd = torch.from_numpy(x).to(dt).cuda()
    yd = torch.empty_like(xd)
    ctx.apply(g, vd, xd, yd, shift_beta=beta, direct=direct)
    torch.cuda.synchronize()
    xr = xd.cpu().numpy().astype(np.complex128)     # the values the GPU saw
    _bound_check(A, xr, yd.cpu().numpy().astype(np.complex128), TOL[prec])


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_row_coefficients_match_oracle(ctx, otable, beta):
    shape, h, f, npml, vmin, vmax = _cases()[0]
    nodes, T = otable
    v = synth.random_velocity(shape, 100, vmin, vmax)
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    ref, valid = O.row_coefficients(v, h, f, prof, T, nodes, beta=beta)
    g = B.make_grid(shape, h, f, npml, vmax)
    coef = torch.empty(v.size * 27 * 2, dtype=torch.float64, device="cuda")
    ctx.row_coefficients(g, torch.from_numpy(v).cuda(), coef, shift_beta=beta)
    got = coef.cpu().numpy().view(np.complex128).reshape(-1, 27)
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    assert np.max(np.abs(np.where(valid, got - ref, got)) / scale) < 1e-13


def test_assemble_csr_matches_oracle(ctx, otable):
    shape, h, f, npml, vmin, vmax = _cases()[1]
    nodes, T = otable
    v = synth.random_velocity(shape, 101, vmin, vmax)
    prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
    A = O.assemble_csr(v, h, f, prof, T, nodes)
    g = B.make_grid(shape, h, f, npml, vmax)
    rowptr, col, val = ctx.assemble_csr(g, torch.from_numpy(v).cuda())
    assert np.array_equal(rowptr, A.indptr) and np.array_equal(col, A.indices)
    assert np.max(np.abs(val - A.data)) < 1e-13 * np.max(np.abs(A.data))


@pytest.mark.parametrize("name,nrhs", [("tectonic", 16), ("sharp_contrast", 8)])
def test_apply_full_size_sampled_rows(ctx, otable, name, nrhs):
    # Full-size models in the bench's launch configuration; outputs checked on
    # 3000 sampled rows (half of them in the PML) one by one by the oracle.
    nodes, T = otable
    wl = synth.CONFIGS[name]()
    g = B.grid_of(wl)
    shape = wl.shape
    N = wl.n_points
    gen = torch.Generator(device="cuda").manual_seed(123)
    xd = torch.complex(torch.rand((nrhs,) + shape, generator=gen, device="cuda") - 0.5,
                       torch.rand((nrhs,) + shape, generator=gen, device="cuda") - 0.5)
    yd = torch.empty_like(xd)
    vd = torch.from_numpy(wl.v).cuda()
    ctx.apply(g, vd, xd, yd)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    nz, ny, nx = shape
    k = rng.integers(0, nz, 3000)
    j = rng.integers(0, ny, 3000)
    i = rng.integers(0, nx, 3000)
    i[:1500] = rng.choice(np.r_[0:wl.npml[0], nx - wl.npml[1]:nx], 1500)
    rows = i + nx * (j + ny * k)
    # gather the 27-neighbourhoods of the sampled rows
    offs = np.array([si + nx * (sj + ny * sk) for sk, sj, si in O.OFFSETS])
    nb = np.clip(rows[:, None] + offs[None, :], 0, N - 1)
    uniq, inv = np.unique(nb, return_inverse=True)
    xs = xd.reshape(nrhs, -1)[:, torch.from_numpy(uniq).cuda()].cpu().numpy().astype(np.complex128)
    xnb = xs[:, inv.reshape(nb.shape)]                     # (nrhs, 3000, 27)
    prof = O.profiles_for(shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    coef, valid = O.row_coefficients(wl.v, wl.h, wl.f, prof, T, nodes, rows)
    c = np.where(valid, coef, 0.0)[None]
    ref = np.sum(c * xnb, axis=2)
    bound = np.sum(np.abs(c) * np.abs(xnb), axis=2)
    got = yd.reshape(nrhs, -1)[:, torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref) / bound) <= TOL[32]


def test_apply_rejects_bad_arguments(ctx):
    g = B.make_grid((8, 8, 8), 25.0, 5.0, (4, 0, 0, 0, 0, 0), 1500.0)   # npml >= n/2
    v = torch.full((8, 8, 8), 1500.0, device="cuda")
    x = torch.zeros((1, 8, 8, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(B.HxError) as e:
        ctx.apply(g, v, x, torch.empty_like(x))
    assert e.value.code == -1
    g = B.make_grid((8, 8, 8), 25.0, 5.0, (2,) * 6, 1500.0)
    with pytest.raises(B.HxError):
        ctx.apply(g, v, x, x)                                           # aliasing

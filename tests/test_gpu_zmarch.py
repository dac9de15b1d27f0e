"""GPU parity of the TMA z-marching complex64 kernel (hx_zmarch.cu) against
the oracle's assembled matrix (Eq. 3 rows, Eqs. 4-8, GA weights), through the
C ABI (hx_stencil_pitched with padded rows, hx_apply_operator /
hx_stencil_sweep on even-nx grids).

Cases cover: every launch configuration (rows per CTA x RHS per CTA); y = A x,
the residual with and without b, and the damped-Jacobi sweep; the shifted and
the plain operator; RHS counts that leave a partial RHS block; padded row
pitches (odd nx in an even pitch, and wider pitches) whose padding holds NaN
and must be neither read nor written; PML frames of uneven widths per face,
a grid without PML (no frame rows), and a tall narrow grid whose launch
splits z into many chunks (halo planes at every chunk boundary).

Tolerances (elementwise against the bound of the 27-term dot product, as in
test_gpu_kernels32.py): FP32 2e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import operator as O
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth

TOL = 2e-5
ZM_FIRST = 3          # configuration ids of the TMA kernel: 3 .. count - 1

# (shape (nz, ny, nx), h, f, npml, vmin, vmax)
CASES = [
    ((23, 19, 70), 25.0, 6.0, (3, 4, 2, 5, 4, 3), 1500.0, 4500.0),     # even nx, uneven PML
    ((17, 21, 45), 25.0, 5.0, (5, 2, 3, 4, 2, 6), 1500.0, 4000.0),     # odd nx: padded pitch
    ((5, 33, 40), 30.0, 5.0, (0, 0, 0, 0, 0, 0), 2000.0, 5000.0),      # no PML: no frame rows
    ((120, 9, 33), 25.0, 6.0, (2, 3, 1, 1, 7, 5), 1500.0, 3500.0),     # tall and narrow: many z-chunks
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
        v = synth.random_velocity(shape, 300 + case, vmin, vmax)
        prof = O.profiles_for(shape, h, npml, vmax, 1e-3)
        A = O.assemble_csr(v, h, f, prof, T, nodes, beta=beta)
        _A[key] = (v, A, B.make_grid(shape, h, f, npml, vmax))
    return _A[key]


def _padded(field, pitch, fill):
    """(R, nz, ny, nx) complex -> (R, nz, ny, pitch) complex64 CUDA tensor,
    padding columns set to `fill`."""
    R, nz, ny, nx = field.shape
    out = np.full((R, nz, ny, pitch), fill, dtype=np.complex64)
    out[..., :nx] = field
    return torch.from_numpy(out).cuda()


def _reference(A, kind, x, b, omega):
    Ax = (A @ x.T).T
    bound = (abs(A) @ np.abs(x).T).T + (np.abs(b) if b is not None else 0)
    if kind == "apply":
        return Ax, (abs(A) @ np.abs(x).T).T
    r = (b if b is not None else 0) - Ax
    if kind == "residual":
        return r, bound
    d = A.diagonal()[None, :]
    return x + omega * r / d, np.abs(x) + np.abs(omega / d) * bound


def _run(ctx, otable, case, cfg, kind, nrhs, beta, with_b=True, extra_pitch=None):
    v, A, g = _problem(case, beta, otable)
    nz, ny, nx = v.shape
    pitch = extra_pitch if extra_pitch is not None else (nx + (nx & 1))
    x = synth.random_field(v.shape, nrhs, 71 + case + 3 * cfg)
    bb = synth.random_field(v.shape, nrhs, 81 + case) if (kind != "apply" and with_b) else None
    nan = complex(np.nan, np.nan)
    xd = _padded(x, pitch, nan)
    bd = _padded(bb, pitch, nan) if bb is not None else None
    yd = torch.full((nrhs, nz, ny, pitch), nan, dtype=torch.complex64, device="cuda")
    omega = 0.6
    ctx.set_kernel_config(cfg)
    try:
        ctx.stencil_pitched(g, torch.from_numpy(v).cuda(), kind, xd, bd, yd, pitch, shift_beta=beta, omega=omega)
        torch.cuda.synchronize()
    finally:
        ctx.set_kernel_config(-1)
    yh = yd.cpu().numpy()
    # padding untouched (still NaN), every grid value written (finite)
    if pitch > nx:
        assert np.all(np.isnan(yh[..., nx:].real))
    y = yh[..., :nx].astype(np.complex128).reshape(nrhs, -1)
    assert np.all(np.isfinite(y))
    xr = xd.cpu().numpy()[..., :nx].astype(np.complex128).reshape(nrhs, -1)
    br = bd.cpu().numpy()[..., :nx].astype(np.complex128).reshape(nrhs, -1) if bd is not None else None
    ref, bound = _reference(A, kind, xr, br, omega)
    return np.max(np.abs(y - ref) / bound)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("cfg", range(ZM_FIRST, ZM_FIRST + 6))
@pytest.mark.parametrize("kind", ["apply", "residual", "jacobi"])
def test_every_config_and_mode(ctx, otable, case, cfg, kind):
    nrhs = (1, 3, 5, 9)[(case + cfg) % 4]                  # partial RHS blocks included
    beta = 0.0 if (kind == "apply" and case % 2 == 0) else 0.5
    assert _run(ctx, otable, case, cfg, kind, nrhs, beta) <= TOL


@pytest.mark.parametrize("cfg", [ZM_FIRST, ZM_FIRST + 3])
def test_residual_without_b_and_wide_pitch(ctx, otable, cfg):
    assert _run(ctx, otable, 1, cfg, "residual", 4, 0.5, with_b=False, extra_pitch=52) <= TOL
    assert _run(ctx, otable, 0, cfg, "apply", 2, 0.0, extra_pitch=74) <= TOL


def test_even_nx_public_calls_use_the_tma_kernel(ctx, otable):
    # hx_apply_operator with even nx takes the same kernel (pitch = nx)
    v, A, g = _problem(0, 0.0, otable)
    x = synth.random_field(v.shape, 3, 91)
    xd = torch.from_numpy(x).to(torch.complex64).cuda()
    yd = torch.full_like(xd, complex(np.nan, np.nan))
    ctx.apply(g, torch.from_numpy(v).cuda(), xd, yd)
    torch.cuda.synchronize()
    xr = xd.cpu().numpy().astype(np.complex128).reshape(3, -1)
    ref, bound = _reference(A, "apply", xr, None, 0.0)
    y = yd.cpu().numpy().astype(np.complex128).reshape(3, -1)
    assert np.max(np.abs(y - ref) / bound) <= TOL


def test_pitched_argument_errors(ctx, otable):
    v, A, g = _problem(1, 0.0, otable)
    nz, ny, nx = v.shape
    xd = torch.zeros((1, nz, ny, nx + 2), dtype=torch.complex64, device="cuda")
    yd = torch.zeros_like(xd)
    vd = torch.from_numpy(v).cuda()
    for bad_pitch in (nx - 1, nx + 2):                   # below nx; odd and != nx
        with pytest.raises(B.HxError) as e:
            ctx.stencil_pitched(g, vd, "apply", xd, None, yd, bad_pitch)
        assert e.value.code == -1

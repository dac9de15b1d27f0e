"""Solve parity on the two large batched workloads (synthetic stand-ins for the
paper's heterogeneous models of Sections 3.4-3.5, shaped as in Table 1):

* sharp contrast 201 x 201 x 101, h = 25 m, f = 4 Hz, 8 of its 64 lattice
  sources as right-hand sides (G 15 -> 45, 5 multigrid levels);
* tectonic 401 x 401 x 187, h = 25 m, f = 5 Hz, 2 of its 16 sources
  (30 M unknowns per RHS, the multi-wave launches of the z-marching kernel).

The library's own weight table (hx_build_weight_table) is used on both sides:
the GPU solves with it, and the oracle forms its rows from the same table
(oracle.operator.apply_rows), so the check covers the table the library
serves with and the GPU's operator, Krylov, multigrid and refinement.

Check per RHS, on the CPU with the oracle's row formula: the FP64 residual
r = s - A x of the GPU wavefield on every source row and on a strided sample
of about 10^5 rows.  The source rows carry all of s; the strided sample,
scaled by sqrt(N / rows), estimates the full residual norm.  Both must be
<= 1e-10 ||s|| (the solve runs to 1e-11).  At the sharp-contrast size the
mixed-precision wavefield of one RHS is also compared with the plain FP64 GPU
solve (relative L2 <= 1e-6, the stated target of the mixed form).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import metrics as M
from oracle import operator as O
from oracle import solve as S
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth


@pytest.fixture(scope="module")
def libtable():
    return B.build_weight_table()


@pytest.fixture(scope="module")
def ctx(libtable):
    c = B.Context(0, table=libtable[1])
    yield c
    c.close()


def _subset(wl, k):
    """k of the workload's sources spread over its lattice, renumbered 0..k-1."""
    src = B.sources_of(wl)
    pick = np.linspace(0, len(src) - 1, k).round().astype(int)
    return [(s[0], s[1], s[2], j, s[4]) for j, s in enumerate(src[i] for i in pick)]


def _sampled_residuals(wl, table, x, sources, stride):
    nodes, T = table
    N = wl.n_points
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    nz, ny, nx = wl.shape
    src_rows = np.array([ix + nx * (iy + ny * iz) for ix, iy, iz, _, _ in sources], dtype=np.int64)
    strided = np.setdiff1d(np.arange(stride // 2, N, stride, dtype=np.int64), src_rows)
    rows = np.concatenate([src_rows, strided])
    Ax = O.apply_rows(wl.v, wl.h, wl.f, prof, T, nodes, x, rows)
    R = x.shape[0]
    s = np.zeros((R, rows.size), dtype=np.complex128)
    s_norm = np.zeros(R)
    for j, (ix, iy, iz, r, amp) in enumerate(sources):
        val = S.point_sources(wl.shape, wl.h, [(ix, iy, iz)], amps=[amp])[0][iz, iy, ix]
        s[r, j] += val
        s_norm[r] = np.sqrt(s_norm[r] ** 2 + abs(val) ** 2)
    res = s - Ax
    ns = src_rows.size
    at_sources = np.array([np.max(np.abs(res[r, :ns])) for r in range(R)]) / s_norm
    estimate = np.sqrt(N / strided.size) * np.linalg.norm(res[:, ns:], axis=1) / s_norm
    return at_sources, estimate


def _solve(ctx, wl, sources, **kw):
    R = max(s[3] for s in sources) + 1
    out = torch.zeros((R,) + wl.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), sources, R, out, **kw)
    assert rep["status"] == 0, rep
    return out, rep


@pytest.mark.parametrize("name,k,stride", [("sharp_contrast", 8, 41), ("tectonic", 2, 301)])
def test_batched_solve_oracle_residual(ctx, libtable, name, k, stride):
    wl = synth.CONFIGS[name]()
    src = _subset(wl, k)
    out, rep = _solve(ctx, wl, src, tol=1e-11, time_limit_s=240.0)
    at_src, est = _sampled_residuals(wl, libtable, out.cpu().numpy(), src, stride)
    print(f"{name} {k} RHS: {rep['inner_iters']} iterations, {rep['outer_iters']} refinements, "
          f"{rep['solve_ms'] / 1e3:.1f} s; oracle residual at sources {at_src.max():.2e}, "
          f"sampled estimate {est.max():.2e}, library {rep['rel_residual']:.2e}")
    assert np.all(at_src <= 1e-10) and np.all(est <= 1e-10)


def test_sharp_contrast_mixed_matches_fp64(ctx):
    wl = synth.sharp_contrast()
    src = _subset(wl, 1)
    xm, _ = _solve(ctx, wl, src, tol=1e-11, time_limit_s=240.0)
    x64, rep64 = _solve(ctx, wl, src, mode=B.SOLVE_FP64, tol=1e-11, max_iter=20000, time_limit_s=400.0)
    err = M.rel_l2(xm.cpu().numpy(), x64.cpu().numpy())
    print(f"sharp contrast, 1 RHS: mixed vs FP64 {err:.2e} (FP64 {rep64['inner_iters']} iterations, "
          f"{rep64['solve_ms'] / 1e3:.1f} s)")
    assert err <= 1e-6

"""GPU solve parity against the oracle (Eq. 3 solved for point sources).

All GPU work goes through the C ABI (hx_solve).  References:
  * small grids: the oracle's banded LU of its own CSR assembly (complex128);
  * the full linear-gradient workload (101^3): the oracle's CSR residual
    ||s - A x|| / ||s|| of the GPU wavefield, computed on the CPU, and the
    mixed-precision result against the plain FP64 GPU solve.
Tolerance: relative L2 error <= 1e-6 (the stated target of the mixed form);
residual bounds as in the solve options.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import metrics as M
from oracle import operator as O
from oracle import solve as S
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B
from paper_2108_08730_gb300 import synth


@pytest.fixture(scope="module")
def otable():
    return W.fit_table()


@pytest.fixture(scope="module")
def ctx(otable):
    c = B.Context(0, table=otable[1])
    yield c
    c.close()


def _oracle_solution(wl, otable, sources, spread=False):
    nodes, T = otable
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    R = max(s[3] for s in sources) + 1
    rhs = np.zeros((R,) + wl.shape, dtype=np.complex128)
    for ix, iy, iz, r, amp in sources:
        mw = None
        if spread:
            mw = [W.lookup(T, nodes, wl.f * wl.h / float(wl.v[iz, iy, ix]))]
        rhs[r] += S.point_sources(wl.shape, wl.h, [(ix, iy, iz)], amps=[amp], mass_w7=mw)[0]
    x = S.solve_banded(A, rhs.reshape(R, -1).T).T.reshape(rhs.shape)
    return x, A, rhs


def _gpu_solve(ctx, wl, sources, **kw):
    R = max(s[3] for s in sources) + 1
    out = torch.zeros((R,) + wl.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), sources, R, out, **kw)
    return out.cpu().numpy(), rep


@pytest.mark.parametrize("mode", [B.SOLVE_MIXED, B.SOLVE_FP64])
def test_homogeneous_matches_banded_lu(ctx, otable, mode):
    wl = synth.homogeneous()                         # 20^3, 4-node PML, G = 6
    src = B.sources_of(wl)
    ref, _, _ = _oracle_solution(wl, otable, src)
    got, rep = _gpu_solve(ctx, wl, src, mode=mode, tol=1e-12)
    assert rep["rel_residual"] <= 1e-12
    assert M.rel_l2(got, ref) <= 1e-6


def test_spread_source_and_multi_rhs_match_banded_lu(ctx, otable):
    # 3 RHS on a heterogeneous 18x16x20 grid; RHS 1 has two sources; spread
    # (consistent-mass) sources, one next to the grid edge.
    wl = synth.homogeneous(n=18)
    wl.v = synth.random_velocity((20, 16, 18), 21, 1500.0, 2500.0)
    wl.v_ref = 2500.0
    wl.npml = (3, 3, 2, 4, 3, 3)
    src = [(9, 8, 10, 0, 1.0), (4, 5, 6, 1, 0.5 - 1j), (12, 10, 14, 1, 2.0), (1, 14, 3, 2, 1j)]
    ref, _, _ = _oracle_solution(wl, otable, src, spread=True)
    got, rep = _gpu_solve(ctx, wl, src, tol=1e-12, source_spread=1)
    assert M.rel_l2(got, ref) <= 1e-6
    for r in range(3):
        assert M.rel_l2(got[r], ref[r]) <= 1e-6


def test_gradient_fp64_and_mixed_against_oracle_residual(ctx, otable):
    # Full-size linear-gradient workload: the oracle checks the GPU wavefields
    # through its own CSR residual; mixed vs FP64 within 1e-6.
    wl = synth.linear_gradient()
    src = B.sources_of(wl)
    x64, rep64 = _gpu_solve(ctx, wl, src, mode=B.SOLVE_FP64, tol=1e-11, max_iter=20000)
    xm, repm = _gpu_solve(ctx, wl, src, mode=B.SOLVE_MIXED, tol=1e-11)
    nodes, T = otable
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    s = S.point_sources(wl.shape, wl.h, wl.sources).reshape(-1)
    assert S.relative_residual(A, x64.reshape(-1), s) <= 1e-10
    assert S.relative_residual(A, xm.reshape(-1), s) <= 1e-10
    assert M.rel_l2(xm, x64) <= 1e-6


def test_batch_invariance(ctx, otable):
    # Each RHS solved alone equals the same RHS solved in a batch of four
    # (per-RHS recurrences and deterministic per-RHS reductions).
    wl = synth.homogeneous(n=24, npml=5)
    wl.v = synth.random_velocity(wl.shape, 33, 1500.0, 2200.0)
    wl.v_ref = 2200.0
    src = [(12, 12, 12, 0, 1.0), (8, 15, 10, 1, 1.0), (16, 9, 7, 2, 1j), (10, 10, 17, 3, 2.0)]
    batch, _ = _gpu_solve(ctx, wl, src, tol=1e-12)
    for k in range(4):
        ix, iy, iz, _, amp = src[k]
        alone, _ = _gpu_solve(ctx, wl, [(ix, iy, iz, 0, amp)], tol=1e-12)
        assert M.rel_l2(alone[0], batch[k]) <= 1e-9


@pytest.mark.parametrize("opts", [{"bicg_kappa": 0.7}, {"bicg_kappa": 0.5}, {"coarse_velocity": 1}])
def test_solver_options_reach_the_oracle_residual(ctx, otable, opts):
    # The omega safeguard and the averaged coarse velocity change only the
    # iterates: on a small sharp-contrast model (bodies and lens) the wavefield
    # must meet the oracle's FP64 CSR residual and agree with the default solve.
    wl = synth.sharp_contrast(40, 36, 32, 25.0, 7.0, 5, seed=79, n_src_side=2)   # 44 % at 4500, 52 % lens
    src = B.sources_of(wl)
    ref, _ = _gpu_solve(ctx, wl, src, tol=1e-11)
    got, rep = _gpu_solve(ctx, wl, src, tol=1e-11, **opts)
    assert rep["status"] == 0
    nodes, T = otable
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, wl.v_ref, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    for r, (ix, iy, iz) in enumerate(wl.sources):
        s = S.point_sources(wl.shape, wl.h, [(ix, iy, iz)]).reshape(-1)
        assert S.relative_residual(A, got[r].reshape(-1), s) <= 1e-10
    assert M.rel_l2(got, ref) <= 1e-6


def test_solve_argument_errors(ctx):
    wl = synth.homogeneous()
    g = B.grid_of(wl)
    v = torch.from_numpy(wl.v).cuda()
    out = torch.zeros((1,) + wl.shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(B.HxError) as e:
        ctx.solve(g, v, [(25, 1, 1, 0, 1.0)], 1, out)            # source outside the grid
    assert e.value.code == -1
    vbad = v.clone()
    vbad[3, 4, 5] = -1.0
    with pytest.raises(B.HxError) as e:
        ctx.solve(g, vbad, B.sources_of(wl), 1, out)              # negative velocity
    assert e.value.code == -1
    vslow = torch.full_like(v, 50.0)                              # G < 2.5
    with pytest.raises(B.HxError) as e:
        ctx.solve(g, vslow, B.sources_of(wl), 1, out)
    assert e.value.code == -1
    for bad in ({"bicg_kappa": 1.0}, {"bicg_kappa": -0.1}, {"coarse_velocity": 2}):
        with pytest.raises(B.HxError) as e:
            ctx.solve(g, v, B.sources_of(wl), 1, out, **bad)
        assert e.value.code == -1
    c2 = B.Context(0)                                             # no table yet
    with pytest.raises(B.HxError) as e:
        c2.solve(g, v, B.sources_of(wl), 1, out)
    assert e.value.code == -7
    c2.close()


def test_not_converged_reports_best_iterate(ctx):
    wl = synth.homogeneous()
    out = torch.zeros((1,) + wl.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), B.sources_of(wl), 1, out,
                    check=False, max_iter=2, max_outer=1, tol=1e-14)
    assert rep["status"] == -3
    assert 0 < rep["rel_residual"] < 1
    assert torch.isfinite(torch.view_as_real(out)).all()


def test_profiler_counts_fine_level_kernels(ctx):
    wl = synth.homogeneous()
    out = torch.zeros((1,) + wl.shape, dtype=torch.complex128, device="cuda")
    ctx.profile(True)
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), B.sources_of(wl), 1, out)
    p = ctx.profile_read()
    ctx.profile(False)
    # two fine-level applies per BiCGStab iteration
    assert p["apply32"][0] == 2 * rep["inner_iters"]
    assert p["apply32"][1] > 0 and p["apply32"][2] == p["apply32"][0] * (16 * wl.n_points + 4 * wl.n_points)
    assert p["all"][0] > p["apply32"][0] + p["smooth32"][0]


def test_time_limit_stops_a_solve_with_its_best_iterate(ctx):
    # hx_solve_opts.time_limit_s: a deadline checked where the host
    # synchronises; an unreachable tolerance makes the solve run into it
    wl = synth.linear_gradient(n=61, npml=8)
    out = torch.zeros((1,) + wl.shape, dtype=torch.complex128, device="cuda")
    import time
    t0 = time.perf_counter()
    rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), B.sources_of(wl), 1, out,
                    check=False, tol=1e-30, max_outer=1000, time_limit_s=0.5)
    el = time.perf_counter() - t0
    assert rep["status"] == -3                                   # HX_ERR_NOT_CONVERGED
    assert el < 10.0
    assert 0 < rep["rel_residual"] < 1e-6                        # the refinement did progress
    assert torch.isfinite(torch.view_as_real(out)).all()


def test_autotune_option_records_a_configuration(ctx):
    # hx_solve tunes the complex64 kernel once per (grid size, nrhs) above
    # 2^20 point*RHS; the solve converges the same either way
    wl = synth.linear_gradient(n=64, npml=8)
    g = B.grid_of(wl)
    vd = torch.from_numpy(wl.v).cuda()
    src = [(s[0], s[1], s[2], r, 1.0) for r, s in enumerate([wl.sources[0]] * 4)]
    outs = []
    for tune in (0, 1):
        out = torch.zeros((4,) + wl.shape, dtype=torch.complex128, device="cuda")
        rep = ctx.solve(g, vd, src, 4, out, autotune=tune)
        assert rep["status"] == 0
        outs.append(out)
    assert torch.linalg.vector_norm(outs[0] - outs[1]) <= 1e-6 * torch.linalg.vector_norm(outs[0])


_PDL_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2])
from oracle import weights as W
from paper_2108_08730_gb300 import binding as B, synth
wl = synth.homogeneous(n=28, npml=5)
wl.v = synth.random_velocity(wl.shape, 41, 1500.0, 2400.0)
wl.v_ref = 2400.0
ctx = B.Context(0, table=W.fit_table()[1])
out = torch.zeros((2,) + wl.shape, dtype=torch.complex128, device="cuda")
src = [(14, 13, 12, 0, 1.0), (9, 17, 15, 1, 1j)]
rep = ctx.solve(B.grid_of(wl), torch.from_numpy(wl.v).cuda(), src, 2, out, check=False)
assert rep["status"] == 0, rep
np.save(sys.argv[1], out.cpu().numpy())
"""


def test_dependent_launch_does_not_change_results(tmp_path):
    # Every solver kernel is launched with programmatic dependent launch
    # (HX_PDL, default on) and waits for its predecessor before touching
    # memory; the wavefield must be bit-identical with the attribute off.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = {}
    for flag in ("0", "1"):
        f = tmp_path / f"pdl{flag}.npy"
        env = dict(os.environ, HX_PDL=flag)
        subprocess.run([sys.executable, "-c", _PDL_CHILD, str(f), root], env=env, check=True, timeout=600)
        res[flag] = np.load(f)
    assert np.array_equal(res["0"], res["1"])

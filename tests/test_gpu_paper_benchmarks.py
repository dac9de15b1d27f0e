"""The paper's first two benchmarks at their full size (Sections 3.2-3.3,
Table 1): a 10 km x 20 km x 10 km medium at h = 50 m with a 16-node PML on
every face (233 x 433 x 233 = 23.5 M unknowns), the source at (5 km, 2 km,
5 km), scored with the paper's l1 measure (Eq. eqerror) against the
continuous solutions.

* homogeneous: v = 1500 m/s;
* linear: v rising from 1500 m/s at the start of the 20 km axis to 8500 m/s at
  its end (gradient 0.35 1/s), G from G_min to 5.7 G_min.

Both models run at the paper's frequency, 7.5 Hz (G_min = 4), and at 5.45 Hz
(G_min = 5.5, where the paper places G4's largest dispersion error).  The long
axis is this grid's z axis, along which the oracle's gradient solution
varies.  Samples: the interior outside 3 nodes around the source; the source
is spread over its 27 nodes with the row's consistent-mass weights, which
cancels the 1/(1 - (kh)^2/12) far-field amplitude bias of a grid delta (as in
test_gpu_accuracy.py).  Stencils: GA and Gm (G4 does not converge with this
solver, see test_gpu_accuracy.py), and in the linear model GA with the first
mass form of Eq. 8 (the paper does not say which form its tables use).
Asserted: every solve converges and GA is more accurate than Gm; the errors
are printed.

A few seconds of GPU time per solve and about 4 GB of host memory per model.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import analytic as AN
from paper_2108_08730_gb300 import binding as B

H, NPML = 50.0, 16
NX, NY, NZ = 201 + 2 * NPML, 201 + 2 * NPML, 401 + 2 * NPML   # long axis = z
V0, ALPHA = 1500.0, 0.35
SRC = (NPML + 100, NPML + 100, NPML + 40)                       # (5, 5, 2) km


@pytest.fixture(scope="module")
def tables():
    nodes, ga = B.build_weight_table()
    gm = B.fixed_table(B.fit_joint_weights([0.25, 1 / 6, 1 / 8, 0.1]), len(nodes))
    return {"GA": ga, "Gm": gm}


def _score(p, exact):
    """Paper l1 (oracle.metrics.paper_l1, summed slab by slab to bound host
    memory) over the interior minus 3 nodes around the source."""
    x = (np.arange(NX) - NPML) * H
    y = (np.arange(NY) - NPML) * H
    sx, sy, sz = ((c - NPML) * H for c in SRC)
    num_re = num_im = den_re = den_im = 0.0
    X, Y = np.meshgrid(x[NPML:NX - NPML], y[NPML:NY - NPML], indexing="xy")
    for k in range(NPML, NZ - NPML):
        z = (k - NPML) * H
        dist = np.sqrt((X - sx) ** 2 + (Y - sy) ** 2 + (z - sz) ** 2)
        ok = dist > 3 * H
        ref = exact(X, Y, np.full_like(X, z))
        u = p[k, NPML:NY - NPML, NPML:NX - NPML]
        w, d, r = dist[ok], (ref - u)[ok], ref[ok]
        num_re += np.sum(np.abs(w * d.real))
        num_im += np.sum(np.abs(w * d.imag))
        den_re += np.sum(np.abs(w * r.real))
        den_im += np.sum(np.abs(w * r.imag))
    return float(num_re / den_re + num_im / den_im)


def _solve(tables, name, v, F):
    ctx = B.Context(0, table=tables["GA"])
    if name == "GA-m1":
        ctx.set_operator_form("GA", 1)
    elif name != "GA":
        ctx.set_table(tables[name], role="operator")
    g = B.make_grid(v.shape, H, F, (NPML,) * 6, float(v.max()))
    p = torch.zeros((1,) + v.shape, dtype=torch.complex128, device="cuda")
    rep = ctx.solve(g, torch.from_numpy(v).cuda(), [(SRC[0], SRC[1], SRC[2], 0, 1.0)], 1, p, tol=1e-9,
                    source_spread=1, max_iter=20000, time_limit_s=120.0, check=False)
    out = p[0].cpu().numpy()
    ctx.close()
    return rep, out


@pytest.mark.parametrize("g_min", [5.5, 4.0])                  # 4: the paper's 7.5 Hz
@pytest.mark.parametrize("model", ["homogeneous", "linear"])
def test_full_size_benchmark(tables, model, g_min):
    F = V0 / (g_min * H)
    if model == "homogeneous":
        v = np.full((NZ, NY, NX), V0, np.float32)
        exact = lambda x, y, z: AN.green_homog(x, y, z, [(c - NPML) * H for c in SRC], V0, F)
    else:
        vz = V0 + ALPHA * (np.arange(NZ) - NPML) * H               # 1500 at the first interior plane
        v = np.broadcast_to(vz[:, None, None], (NZ, NY, NX)).astype(np.float32).copy()
        exact = lambda x, y, z: AN.green_gradient(x, y, z, [(c - NPML) * H for c in SRC], V0, ALPHA, F)
    err = {}
    for name in ("GA", "Gm") + (("GA-m1",) if model == "linear" else ()):
        rep, p = _solve(tables, name, v, F)
        assert rep["status"] == 0, (model, name, rep)
        err[name] = _score(p, exact)
        print(f"{model} {NX}x{NY}x{NZ} f={F:.3f} Hz: {name} l1 {err[name]:.4f}, "
              f"{rep['inner_iters']} iterations, {rep['solve_ms'] / 1e3:.1f} s")
    assert err["GA"] < err["Gm"]

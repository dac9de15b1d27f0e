"""Seeded synthetic inputs: velocity models, source layouts, random fields.

This module holds none of the method's arithmetic; it only draws inputs.  It
is the one piece shared by the CUDA library's callers (tests, bench, serving)
and the CPU oracle's callers.  All draws use numpy's PCG64 with an explicit
seed; models are float32 arrays v[nz][ny][nx] in m/s, z downward from grid
plane 0, h in metres.

The paper's heterogeneous benchmarks (SEG/EAGE overthrust and salt,
GO_3D_OBS, Table 1) are not available; ``sharp_contrast`` and ``tectonic``
stand in for them with the same kind of structure and value ranges.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    v: np.ndarray                 # float32 (nz, ny, nx)
    h: float
    f: float
    npml: tuple                   # (x_lo, x_hi, y_lo, y_hi, z_lo, z_hi)
    sources: list                 # [(ix, iy, iz)], one RHS each
    v_ref: float                  # PML reference speed (model maximum)
    r_coef: float = 1e-3
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.v.shape

    @property
    def n_points(self):
        return int(self.v.size)

    @property
    def nrhs(self):
        return len(self.sources)


def _pml6(n):
    return (n, n, n, n, n, n)


def homogeneous(n=20, h=25.0, f=10.0, v0=1500.0, npml=4):
    """Benchmark-1 analogue: constant 1500 m/s, source at the centre node."""
    v = np.full((n, n, n), v0, dtype=np.float32)
    c = n // 2
    return Workload("homogeneous", v, h, f, _pml6(npml), [(c, c, c)], float(v0))


def linear_gradient(n=101, h=20.0, f=5.0, v0=1500.0, alpha=0.7, npml=10):
    """Benchmark-2 analogue: v(z) = v0 + alpha z, z = iz h from plane 0; one
    source near the surface at (n/2, n/2, npml + 3)."""
    z = np.arange(n, dtype=np.float64) * h
    vz = v0 + alpha * z
    v = np.broadcast_to(vz[:, None, None], (n, n, n)).astype(np.float32).copy()
    return Workload("linear_gradient", v, h, f, _pml6(npml), [(n // 2, n // 2, npml + 3)],
                    float(vz.max()), meta={"v0": v0, "alpha": alpha})


def _surface_lattice(nx, ny, npml, k, depth):
    xs = np.linspace(npml + 2, nx - npml - 3, k).round().astype(int)
    ys = np.linspace(npml + 2, ny - npml - 3, k).round().astype(int)
    return [(int(x), int(y), int(depth)) for y in ys for x in xs]


def sharp_contrast(nx=201, ny=201, nz=101, h=25.0, f=4.0, npml=10, seed=3001, n_src_side=8):
    """Salt-like stand-in: seeded 1-D gradient 1500->4500 m/s (end value
    jittered +-10 %, clipped), three random rotated ellipsoids at 4500 m/s and
    one 1500 m/s lens; 8x8 sources on a lattice at depth npml + 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = np.arange(nz) * h
    y = np.arange(ny) * h
    x = np.arange(nx) * h
    zmax = z[-1]
    vbot = 4500.0 * (1.0 + rng.uniform(-0.1, 0.1))
    vz = np.clip(1500.0 + (vbot - 1500.0) * z / zmax, 1500.0, 4500.0)
    v = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).astype(np.float64).copy()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    for body in range(4):
        c = np.array([rng.uniform(0.2, 0.8) * x[-1], rng.uniform(0.2, 0.8) * y[-1],
                      rng.uniform(0.3, 0.8) * zmax])
        ax = rng.uniform(250.0, 1250.0, size=3)
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        d = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1) @ q
        inside = np.sum((d / ax) ** 2, axis=-1) <= 1.0
        v[inside] = 4500.0 if body < 3 else 1500.0
    src = _surface_lattice(nx, ny, npml, n_src_side, npml + 2)
    return Workload("sharp_contrast", v.astype(np.float32), h, f, _pml6(npml), src,
                    float(v.max()), meta={"seed": seed})


def tectonic(nx=401, ny=401, nz=187, h=25.0, f=5.0, npml=10, seed=4001, n_src_side=4):
    """Overthrust-like stand-in: 12 seeded layers (sorted speeds in
    1800..6000 m/s) whose interfaces are folded by sinusoids (amplitude 200 m,
    wavelengths U(2,5) km in x and y) and offset by two planar faults with 300 m
    throw; 4x4 sources at depth npml + 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    z = np.arange(nz) * h
    speeds = np.sort(rng.uniform(1800.0, 6000.0, size=12))
    speeds[0], speeds[-1] = 1800.0, 6000.0
    depths = np.sort(rng.uniform(0.05, 0.95, size=11)) * z[-1]
    lx, ly = rng.uniform(2000.0, 5000.0, size=2)
    px, py = rng.uniform(0, 2 * np.pi, size=2)
    Y, X = np.meshgrid(y, x, indexing="ij")
    fold = 200.0 * np.sin(2 * np.pi * X / lx + px) * np.sin(2 * np.pi * Y / ly + py)
    throw = np.zeros_like(fold)
    for _ in range(2):
        nrm = rng.normal(size=2)
        nrm /= np.linalg.norm(nrm)
        off = rng.uniform(0.3, 0.7) * np.array([x[-1], y[-1]])
        side = (X - off[0]) * nrm[0] + (Y - off[1]) * nrm[1] > 0
        throw += np.where(side, 300.0, 0.0)
    shift = fold + throw                                  # (ny, nx) interface offset
    zz = z[:, None, None] - shift[None, :, :]             # depth in unfolded frame
    layer = np.searchsorted(depths, zz)                   # 0..11
    v = speeds[layer].astype(np.float32)
    src = _surface_lattice(nx, ny, npml, n_src_side, npml + 2)
    return Workload("tectonic", v, h, f, _pml6(npml), src, float(v.max()), meta={"seed": seed})


def serving_request(seed, side_lo=64, side_hi=256, h=25.0, f_lo=2.0, f_hi=10.0, npml=8,
                    max_sources=32):
    """One serving request: a model family (uniform over the four above) on a
    subvolume with log-uniform sides, f ~ U(f_lo, f_hi), 1..max_sources
    sources."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nx, ny, nz = np.exp(rng.uniform(np.log(side_lo), np.log(side_hi), size=3)).astype(int)
    f = float(rng.uniform(f_lo, f_hi))
    nsrc = int(rng.integers(1, max_sources + 1))
    fam = int(rng.integers(0, 4))
    sub = int(rng.integers(0, 2 ** 31 - 1))
    if fam == 0:
        v = np.full((nz, ny, nx), 1500.0 + 1000.0 * rng.uniform(), dtype=np.float32)
    elif fam == 1:
        vz = 1500.0 + 0.7 * np.arange(nz) * h
        v = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).astype(np.float32).copy()
    elif fam == 2:
        v = sharp_contrast(nx, ny, nz, h, f, npml, seed=sub, n_src_side=1).v
    else:
        v = tectonic(nx, ny, nz, h, f, npml, seed=sub, n_src_side=1).v
    xs = rng.integers(npml + 1, nx - npml - 1, size=nsrc)
    ys = rng.integers(npml + 1, ny - npml - 1, size=nsrc)
    src = [(int(a), int(b), npml + 2) for a, b in zip(xs, ys)]
    return Workload(f"serve_{seed}", v, h, f, _pml6(npml), src, float(v.max()),
                    meta={"family": fam, "seed": seed})


def random_field(shape, nrhs, seed, dtype=np.complex128):
    """Uniform(-1,1) + i Uniform(-1,1) field of shape (nrhs,) + shape."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.uniform(-1.0, 1.0, size=(nrhs,) + tuple(shape))
    b = rng.uniform(-1.0, 1.0, size=(nrhs,) + tuple(shape))
    return (a + 1j * b).astype(dtype)


def random_velocity(shape, seed, vmin=1500.0, vmax=4500.0):
    """Piecewise-smooth random model for operator tests (float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(vmin, vmax, size=shape).astype(np.float32)


CONFIGS = {
    "homogeneous": homogeneous,
    "linear_gradient": linear_gradient,
    "sharp_contrast": sharp_contrast,
    "tectonic": tectonic,
}

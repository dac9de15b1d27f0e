"""Pins of the analytic Green's functions (Section 3.2-3.3 references).

Both must satisfy laplacian p + (omega/v)^2 p = 0 away from the source; the
check uses a 10th-order finite-difference Laplacian on a small patch, which is
independent of the closed forms."""
import numpy as np
import pytest

from oracle import analytic as AN

# 10th-order central second-derivative weights (offsets 0..5)
C10 = np.array([-5269 / 1800, 5 / 3, -5 / 21, 5 / 126, -5 / 1008, 1 / 3150])


def _lap(fun, x, y, z, d):
    out = 3 * C10[0] * fun(x, y, z)
    for k in range(1, 6):
        for e in ((d * k, 0, 0), (0, d * k, 0), (0, 0, d * k)):
            out = out + C10[k] * (fun(x + e[0], y + e[1], z + e[2]) + fun(x - e[0], y - e[1], z - e[2]))
    return out / d ** 2


def test_homogeneous_green_satisfies_helmholtz():
    f, v = 10.0, 1500.0
    src = (0.0, 0.0, 0.0)
    k = 2 * np.pi * f / v
    rng = np.random.default_rng(1)
    pts = rng.uniform(200, 600, size=(20, 3)) * rng.choice([-1, 1], size=(20, 3))
    fun = lambda x, y, z: AN.green_homog(x, y, z, src, v, f)
    for x, y, z in pts:
        res = _lap(fun, x, y, z, 2.0) + k ** 2 * fun(x, y, z)
        assert abs(res) < 1e-7 * k ** 2 * abs(fun(x, y, z))


@pytest.mark.parametrize("alpha", [0.7, 0.35])
def test_gradient_green_satisfies_helmholtz(alpha):
    f, v0 = 5.0, 1500.0
    src = (1000.0, 1000.0, 260.0)
    omega = 2 * np.pi * f
    rng = np.random.default_rng(2)
    pts = np.c_[rng.uniform(0, 2000, 20), rng.uniform(0, 2000, 20), rng.uniform(0, 2000, 20)]
    fun = lambda x, y, z: AN.green_gradient(x, y, z, src, v0, alpha, f)
    for x, y, z in pts:
        if np.linalg.norm(np.array([x, y, z]) - src) < 100:
            continue
        vz = v0 + alpha * z
        res = _lap(fun, x, y, z, 2.0) + (omega / vz) ** 2 * fun(x, y, z)
        assert abs(res) < 1e-6 * (omega / vz) ** 2 * abs(fun(x, y, z))


def test_gradient_reduces_to_homogeneous():
    f, v0 = 5.0, 1500.0
    src = (0.0, 0.0, 300.0)
    x, y, z = 250.0, -120.0, 500.0
    a = AN.green_gradient(x, y, z, src, v0, 1e-6, f)
    b = AN.green_homog(x, y, z, src, v0 + 1e-6 * 0.5 * (300 + 500), f)
    assert abs(a - b) < 1e-6 * abs(b)


def test_unit_source_strength():
    # -4 pi r p -> 1 as r -> 0 for both (unit point source).
    for fun in (lambda r: AN.green_homog(r, 0, 0, (0, 0, 0), 1500.0, 5.0),
                lambda r: AN.green_gradient(r, 0, 300.0, (0, 0, 300.0), 1500.0, 0.7, 5.0)):
        r = 1e-4
        assert abs(-4 * np.pi * r * fun(r) - 1) < 1e-5

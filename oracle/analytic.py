"""Oracle: analytic references of the first two benchmarks (Sections 3.2-3.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The discrete system approximates  laplacian p + (omega^2/v^2) p = delta(x-x_s)
(Eq. 2 with b = 1 and a unit point source), so with exp(-i omega t) and an
outgoing wave p = -G where G solves laplacian G + k^2 G = -delta.

* Homogeneous medium: G = exp(i k r) / (4 pi r), k = omega / v.
* Constant-gradient medium v = v0 + alpha z (the paper cites Kuvshinov &
  Mulder 2006 without the formula).  With zt = z + v0/alpha (so v = alpha zt),
  nu = sqrt(omega^2/alpha^2 - 1/4) and the hyperbolic distance
  cosh(sigma) = 1 + |x - x_s|^2 / (2 zt zt_s):
      G = exp(i nu sigma) / (4 pi sqrt(zt zt_s) sinh(sigma)).
  It tends to the homogeneous G as alpha -> 0.

Pins (tests/test_oracle_analytic.py): both satisfy the PDE away from the
source to the truncation error of a 10th-order finite-difference Laplacian;
the gradient formula reduces to the homogeneous one for small alpha; the
1/(4 pi r) singularity has unit strength.
"""
from __future__ import annotations

import numpy as np


def green_homog(x, y, z, src, v, f):
    """-exp(i k r)/(4 pi r): the continuous solution p for a unit source."""
    k = 2.0 * np.pi * f / v
    r = np.sqrt((x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2)
    return -np.exp(1j * k * r) / (4.0 * np.pi * r)


def green_gradient(x, y, z, src, v0, alpha, f):
    """Continuous p for v(z) = v0 + alpha z (z measured from the same origin
    as src[2]); unit source.  Returns -G (see module header)."""
    omega = 2.0 * np.pi * f
    zt = z + v0 / alpha
    zs = src[2] + v0 / alpha
    r = np.sqrt((x - src[0]) ** 2 + (y - src[1]) ** 2 + (z - src[2]) ** 2)
    # cosh(sigma) = 1 + r^2/(2 zt zs)  <=>  sinh(sigma/2) = r / (2 sqrt(zt zs));
    # the second form keeps full precision when r^2 << zt zs.
    sigma = 2.0 * np.arcsinh(r / (2.0 * np.sqrt(zt * zs)))
    nu = np.sqrt(omega ** 2 / alpha ** 2 - 0.25)
    G = np.exp(1j * nu * sigma) / (4.0 * np.pi * np.sqrt(zt * zs) * np.sinh(sigma))
    return -G

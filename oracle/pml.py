"""Oracle: PML complex stretching (Section 2.1, Eqs. 1.1-1.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper stretches each coordinate by xi_d = 1 + i gamma_d / omega with the
time convention exp(-i omega t) and defers gamma_d to Operto et al. 2007,
Appendix A, which is not in the text.  Reading used here (and by the library):

* PML nodes are part of the grid: npml_lo nodes at the low end and npml_hi at
  the high end of each axis (n nodes, spacing h).  The inner PML faces sit at
  x_lo = npml_lo*h and x_hi = (n - 1 - npml_hi)*h.
* gamma(x) = gamma0 * (d / L)^2 where d >= 0 is the distance from the inner
  face into the layer (0 inside the physical domain) and L = npml*h.
* gamma0 = 3 v_ref / (2 L) * ln(1 / R) with v_ref the reference speed
  (normally the model's maximum) and R the target reflection coefficient.
* The profile is a function of position, so it can be evaluated at integer
  nodes i*H and half nodes (i+1/2)*H of any spacing H (a coarse multigrid level
  uses the fine level's physical profile).

Pin: with a 7-point stencil the stretched operator is the Kronecker sum of the
1-D operators built here (tests/test_oracle_operator.py, against a
scipy.sparse.kron assembly); that the PML absorbs is checked against the
analytic Green's function (tests/test_oracle_solve.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Profile1D:
    """Physical PML profile of one axis."""
    x_lo: float       # inner face of the low layer (m)
    x_hi: float       # inner face of the high layer (m)
    len_lo: float     # thickness of the low layer (m); 0 = no layer
    len_hi: float
    g0_lo: float      # gamma0 of each layer (1/s)
    g0_hi: float

    @staticmethod
    def from_grid(n, h, npml_lo, npml_hi, v_ref, r_coef):
        def g0(npml):
            return 0.0 if npml <= 0 else 3.0 * v_ref / (2.0 * npml * h) * np.log(1.0 / r_coef)
        return Profile1D(npml_lo * h, (n - 1 - npml_hi) * h, npml_lo * h, npml_hi * h,
                         g0(npml_lo), g0(npml_hi))

    def gamma(self, x):
        x = np.asarray(x, dtype=np.float64)
        gam = np.zeros_like(x)
        if self.len_lo > 0:
            d = np.maximum(self.x_lo - x, 0.0)
            gam = gam + self.g0_lo * (d / self.len_lo) ** 2
        if self.len_hi > 0:
            d = np.maximum(x - self.x_hi, 0.0)
            gam = gam + self.g0_hi * (d / self.len_hi) ** 2
        return gam


def xi_nodes(prof: Profile1D, n, h, omega):
    """xi at the n integer nodes i*h and at the n+1 half nodes (k - 1/2)*h,
    k = 0..n (so entry i is the half node below node i, entry i+1 above)."""
    x_int = np.arange(n) * h
    x_half = (np.arange(n + 1) - 0.5) * h
    return 1.0 + 1j * prof.gamma(x_int) / omega, 1.0 + 1j * prof.gamma(x_half) / omega


def second_difference_1d(n, h, xi_int, xi_half):
    """1-D stretched second difference (1/xi) d/dx (1/xi) d/dx with Dirichlet
    zero outside the grid, as a dense (n, n) complex matrix:
    row i = [ (p_{i+1}-p_i)/xi_{i+1/2} - (p_i-p_{i-1})/xi_{i-1/2} ] / (xi_i h^2)."""
    D = np.zeros((n, n), dtype=np.complex128)
    for i in range(n):
        up = 1.0 / (xi_int[i] * xi_half[i + 1] * h * h)   # towards i+1
        dn = 1.0 / (xi_int[i] * xi_half[i] * h * h)       # towards i-1
        D[i, i] = -(up + dn)
        if i + 1 < n:
            D[i, i + 1] = up
        if i - 1 >= 0:
            D[i, i - 1] = dn
    return D

"""Oracle: error measures.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``rel_l2``: ||a - b||_2 / ||b||_2, the parity measure between wavefields.
* ``paper_l1``: Eq. eqerror, |W Re(u_ref - u)|_1 / |W Re(u_ref)|_1 plus the
  same for the imaginary part, W a linear gain with distance from the source.
  The paper does not say which samples enter the sum nor the gain's origin;
  reading: all supplied samples, W = distance to the source in metres.
  No worked example in the paper; pinned by properties of the definition
  (tests/test_oracle_metrics.py): a field scaled by (1 - eps) scores 2 eps,
  real and imaginary parts are scored apart, W matters up to a factor.
"""
from __future__ import annotations

import numpy as np


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def paper_l1(u_ref, u, dist):
    W = np.asarray(dist, dtype=np.float64)
    d = np.asarray(u_ref) - np.asarray(u)
    re = np.sum(np.abs(W * d.real)) / np.sum(np.abs(W * np.real(u_ref)))
    im = np.sum(np.abs(W * d.imag)) / np.sum(np.abs(W * np.imag(u_ref)))
    return float(re + im)

"""Pins of the oracle's error measures (Eq. eqerror of Section 3.1 and the
relative L2 parity measure) by properties that hold for any wavefield:
a wavefield scaled by (1 - eps) has paper error 2 eps (eps on the real part
plus eps on the imaginary part); the real and imaginary parts are scored
separately, so a 90-degree phase error is not a small error; the gain W
matters only up to a positive factor; identical fields score 0."""
import numpy as np

from oracle import metrics as M


def _field(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n), rng.uniform(1.0, 50.0, n)


def test_scaled_field_has_error_two_eps():
    u, w = _field(1000, 1)
    for eps in (1e-3, 0.1, 0.5):
        assert abs(M.paper_l1(u, (1 - eps) * u, w) - 2 * eps) < 1e-12


def test_real_and_imaginary_parts_scored_separately():
    u, w = _field(1000, 2)
    # an error only in the imaginary part counts only through the second term
    v = u.real + 1j * (1.1 * u.imag)
    assert abs(M.paper_l1(u, v, w) - 0.1) < 1e-12
    # i u swaps the parts: a large error though |i u| = |u| everywhere
    assert M.paper_l1(u, 1j * u, w) > 1.0


def test_gain_matters_up_to_a_factor_and_zero_for_equal_fields():
    u, w = _field(500, 3)
    v = u + 0.05 * _field(500, 4)[0]
    assert abs(M.paper_l1(u, v, w) - M.paper_l1(u, v, 7.5 * w)) < 1e-12
    assert M.paper_l1(u, v, w) != M.paper_l1(u, v, w ** 2)       # the weights do enter
    assert M.paper_l1(u, u, w) == 0.0


def test_relative_l2():
    u, _ = _field(300, 5)
    assert abs(M.rel_l2(1.25 * u, u) - 0.25) < 1e-12
    assert M.rel_l2(u, u) == 0.0

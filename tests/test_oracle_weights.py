"""Pins of the oracle's dispersion analysis and weight table (Section 2.2).

Each test checks the oracle against something other than itself: the
independent dispersion formula (Eq. vtilde), closed-form limits, linear-algebra
facts, a library least-squares routine, and statements of the paper's text.
"""
import numpy as np
import pytest

from oracle import weights as W


def _rand_w5(rng):
    return rng.uniform(-1.0, 1.0, size=5)


@pytest.mark.parametrize("inv_g", [0.02, 0.1, 0.25, 0.4])
def test_linear_form_matches_dispersion_identity(inv_g):
    # Eq. linear_basic is Eq. vtilde rearranged: H w - g == X - K J for ANY
    # weights (K = 2 pi^2 / G^2).  A dropped term or wrong sign in H or g
    # breaks this identity for random w.
    rng = np.random.default_rng(7)
    th, ph = W.angle_grid()
    H, g = W.linear_form(inv_g, th, ph)
    K = 2 * np.pi ** 2 * inv_g ** 2
    for _ in range(5):
        w5 = _rand_w5(rng)
        w7 = W.expand_weights(w5)
        lhs = H @ w5 - g
        rhs = W.stiffness_X(inv_g, th, ph, w7) - K * W.mass_J(inv_g, th, ph, w7)
        assert np.max(np.abs(lhs - rhs)) < 1e-13 * max(1.0, np.max(np.abs(rhs)))


def test_printed_H2_breaks_identity():
    # The paper's printed H2 lacks the constant 1/2; with it the identity fails
    # by O(0.1-0.7), which is why the derived H2 is used.
    th, ph = W.angle_grid()
    A, B, C = W.abc_functions(0.25, th, ph)
    H, g = W.linear_form(0.25, th, ph)
    printed = 0.5 * (3 * A - 5 * B / 3 + C / 3)
    assert np.allclose(H[:, 1] - printed, 0.5)


def test_phase_velocity_limit_is_one():
    # Any consistent weights give a second-order accurate stencil: v~ -> 1 as
    # G -> infinity, with error O(1/G^2).
    rng = np.random.default_rng(3)
    th, ph = W.angle_grid()
    w7 = W.expand_weights(np.array([0.4, 0.3, 0.5, 0.05, 0.02]) + 0.01 * rng.normal(size=5))
    e1 = np.max(np.abs(W.phase_velocity(1e-2, th, ph, w7) - 1))
    e2 = np.max(np.abs(W.phase_velocity(5e-3, th, ph, w7) - 1))
    assert e1 < 1e-2 and 3.5 < e1 / e2 < 4.5


def test_seven_point_lumped_dispersion_is_textbook():
    # ws = (1,0,0), lumped mass: v~^2 = (3 - C) G^2 / (2 pi^2), the classic
    # 7-point result sum_d 4 sin^2(k_d h/2) / (k h)^2.
    th, ph = W.angle_grid()
    w7 = np.array([1.0, 0, 0, 1.0, 0, 0, 0])
    inv_g = 0.2
    kh = 2 * np.pi * inv_g
    kd = kh * np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)])
    textbook = np.sqrt(np.sum(4 * np.sin(kd / 2) ** 2, axis=0)) / kh
    assert np.allclose(W.phase_velocity(inv_g, th, ph, w7), textbook, rtol=1e-13)


@pytest.mark.parametrize("inv_g", [0.05, 0.25, 0.4])
def test_per_g_matrix_has_rank_three(inv_g):
    # All five H_l vanish at (A,B,C) = (1,3,3): they lie in a 3-D subspace of
    # span{1, A, B, C}, so H^(i) has numerical rank 3 and Eq. OPFD alone
    # leaves a 2-D family of minimisers -- the reason for the Tikhonov term.
    H, _ = W.block(inv_g)
    s = np.linalg.svd(H, compute_uv=False)
    assert s[2] / s[0] > 1e-8
    assert s[3] / s[0] < 1e-13


@pytest.fixture(scope="module")
def table():
    return W.fit_table()


def test_table_constraints_exact(table):
    inv_g, T = table
    assert T.shape == (401, 7)
    assert np.allclose(inv_g[[0, 1, -1]], [0.0, 0.001, 0.4])
    assert np.max(np.abs(T[:, :3].sum(1) - 1)) < 1e-14
    assert np.max(np.abs(T[:, 3] + 6 * T[:, 4] + 12 * T[:, 5] + 8 * T[:, 6] - 1)) < 1e-14


def test_table_dispersion_equals_fit_prediction(table):
    # The error v~ - 1 of Eq. vtilde with the fitted weights is exactly what the
    # fit's residual predicts: v~^2 - 1 = (H w - g) / (K J).
    inv_g, T = table
    th, ph = W.angle_grid()
    for i in (10, 100, 250, 400):
        H, g = W.linear_form(inv_g[i], th, ph)
        w5 = T[i, [0, 1, 3, 4, 5]]
        K = 2 * np.pi ** 2 * inv_g[i] ** 2
        pred = np.sqrt(1 + (H @ w5 - g) / (K * W.mass_J(inv_g[i], th, ph, T[i])))
        vt = W.phase_velocity(inv_g[i], th, ph, T[i])
        assert np.max(np.abs(pred - vt)) < 1e-9


def test_table_reaches_per_g_optimum(table):
    # Smoothing costs almost nothing: at every tabulated G >= 2.5 (1/G >= 0.01)
    # the adaptive weights' worst phase-velocity error is within 1e-6 of, or
    # 5 % above, the per-G least-squares optimum (numpy lstsq, Eq. OPFD).
    inv_g, T = table
    th, ph = W.angle_grid()
    for i in range(10, 401, 13):
        w_opt, _ = W.fit_per_g(inv_g[i])
        e_opt = np.max(np.abs(W.phase_velocity(inv_g[i], th, ph, W.expand_weights(w_opt)) - 1))
        e_tab = np.max(np.abs(W.phase_velocity(inv_g[i], th, ph, T[i]) - 1))
        assert e_tab <= max(1.05 * e_opt, e_opt + 1e-6), (i, e_tab, e_opt)


def test_lambda_to_zero_converges_to_per_g_optimum():
    # As lam -> 0 each node's misfit ||H^(i) w^(i) - g^(i)|| decreases
    # monotonically to the per-G lstsq optimum (at least like sqrt(lam), the
    # rate where that optimum is ~0).  Coarse table for speed.
    kw = dict(inv_g_max=0.4, d_inv_g=0.02)
    gaps = []
    for lam in (1e-1, 1e-3, 1e-5, 1e-7, 1e-9):
        inv_g, T = W.fit_table(lam=lam, **kw)
        gap = 0.0
        for i in range(1, len(inv_g)):
            H, g = W.block(inv_g[i])
            r_tab = np.linalg.norm(H @ T[i, [0, 1, 3, 4, 5]] - g)
            r_opt = W.fit_per_g(inv_g[i])[1]
            assert r_tab >= r_opt * (1 - 1e-9) - 1e-15
            gap += r_tab - r_opt
        gaps.append(gap)
    assert all(a > b for a, b in zip(gaps, gaps[1:])), gaps
    assert gaps[-1] < 1e-4 * gaps[0]


def test_g4_error_peaks_near_5_5():
    # Section 2.2: weights fitted at G = 4 alone are accurate at G = 4 and
    # reach their largest error near G = 5.5.
    th, ph = W.angle_grid()
    w7 = W.expand_weights(W.fit_joint([0.25]))
    Gs = np.linspace(3.0, 30.0, 541)
    err = np.array([np.max(np.abs(W.phase_velocity(1 / G, th, ph, w7) - 1)) for G in Gs])
    assert np.max(np.abs(W.phase_velocity(0.25, th, ph, w7) - 1)) < 1e-4
    G_peak = Gs[np.argmax(np.where(Gs > 4.2, err, 0))]
    assert 5.0 <= G_peak <= 6.5, G_peak


def test_gm_is_an_average_compromise():
    # Section 2.2: the joint fit for G = 4, 6, 8, 10 lowers the errors over that
    # range in an average sense but its error at G = 4 is higher than G4's.
    th, ph = W.angle_grid()
    g4 = W.expand_weights(W.fit_joint([0.25]))
    gm = W.expand_weights(W.fit_joint([1 / 4, 1 / 6, 1 / 8, 1 / 10]))
    Gs = np.linspace(4.0, 10.0, 61)

    def err(w7):
        return np.array([np.max(np.abs(W.phase_velocity(1 / G, th, ph, w7) - 1)) for G in Gs])

    e4, em = err(g4), err(gm)
    assert em.mean() < e4.mean()
    assert em[0] > e4[0]


def test_lookup_interpolates_linearly(table):
    inv_g, T = table
    mid = W.lookup(T, inv_g, 0.2505)
    assert np.allclose(mid, 0.5 * (T[250] + T[251]), rtol=0, atol=1e-15)
    assert np.allclose(W.lookup(T, inv_g, 0.9), T[-1])


def test_adaptive_weights_beat_fixed_ones_at_every_g(table):
    # Section 2.2 / the paper's central claim: weights picked by the local G
    # keep the phase-velocity error at every G below that of the fixed G4 and
    # Gm weights (max over the propagation angles, G from 4 to 30)
    inv_g, T = table
    th, ph = W.angle_grid()
    g4 = W.expand_weights(W.fit_joint([0.25]))
    gm = W.expand_weights(W.fit_joint([1 / 4, 1 / 6, 1 / 8, 1 / 10]))

    def err(w7, G):
        return np.max(np.abs(W.phase_velocity(1 / G, th, ph, w7) - 1))

    for G in np.linspace(4.0, 30.0, 105):
        ga = err(W.lookup(T, inv_g, 1 / G), G)
        assert ga <= err(g4, G) and ga <= err(gm, G), G
        assert ga < 1e-4

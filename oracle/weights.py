"""Oracle: dispersion analysis and the weight table (Section 2.2 of the paper).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Notation follows the paper.  A plane wave of unit direction
(cos(phi)cos(theta), cos(phi)sin(theta), sin(phi)) sampled with G grid points
per wavelength has per-axis phase increments a, b, c = 2*pi*(direction)/G.
With those, Eq. vtilde defines

    A = cos a cos b cos c,   B = cos a cos b + cos a cos c + cos b cos c,
    C = cos a + cos b + cos c,
    X = ws1 (3 - C) + ws2/3 (6 - C - B) + 2 ws3/4 (3 - 3A + B - C),
    J = wm1 + 2 wm2 C + 4 wm3 B + 8 wm4 A,
    v~ = G / (sqrt(2 J) pi) * sqrt(X).

Weights are stored as the 7-vector [ws1, ws2, ws3, wm1, wm2, wm3, wm4] with
PER-POINT mass weights (wm1 centre, wm2 each face, wm3 each edge, wm4 each
corner) so that ws1 + ws2 + ws3 = 1 and wm1 + 6 wm2 + 12 wm3 + 8 wm4 = 1.
The paper's J uses per-point weights while its Eq. 7 divides class weights by
6/12/8; both describe the same family (class weight = count x point weight).
The paper indexes the mass weights 0..3 in Eq. 7 and 1..4 in Fig. 4; here the
centre is wm1.

Eq. linear_basic: eliminating ws3 and wm4 and requiring v~ = 1 gives
sum_l H_l w_l = g for w = [ws1, ws2, wm1, wm2, wm3].  The printed H2 lacks a
constant term; deriving it from Eq. vtilde gives H2 = (1 + 3A - 5B/3 + C/3)/2
(the only choice for which H w - g == X - K J holds identically and H2
vanishes as G -> infinity like every other H_l).  K = 2 pi^2 / G^2.

Pins (tests/test_oracle_weights.py): the identity H w - g == X - K J for
random w (checks H, g against the independent Eq. vtilde); v~ -> 1 as G -> inf;
numerical rank 3 of the per-G matrix (all H_l vanish at A=1, B=3, C=3);
constraint sums; lam -> 0 convergence of the per-node misfit to the per-G
least-squares optimum (a library lstsq); the G4 error peak near G = 5.5
(Section 2.2 text); the paper's angle grid (Fig. 2 caption).
"""
from __future__ import annotations

import numpy as np

# Fig. 2 caption: dip and azimuth from 0 to 45 degrees in 10-degree steps.
# Reading: the end point 45 is included, giving {0,10,20,30,40,45}.
DEFAULT_ANGLES_DEG = (0.0, 10.0, 20.0, 30.0, 40.0, 45.0)
# Fig. 2 caption: 1/G from 0 to 0.4 with step 0.001.
DEFAULT_INV_G_MAX = 0.4
DEFAULT_D_INV_G = 0.001
# Tikhonov weight (the paper does not print it).  Reading: 1e-6, chosen once on
# this oracle as the largest value that keeps every tabulated G >= 2.5 within 5 %
# (or 1e-6) of the per-G optimum dispersion error while the stacked system's
# condition number stays near 2.5e7; the L-curve is flat because the
# irreducible misfit at large 1/G dominates the global norm.
DEFAULT_LAMBDA = 1e-6


def angle_grid(theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG):
    """All (theta, phi) pairs in radians, theta varying fastest within phi
    (the row order of H^(i) in Section 2.2: j over theta, then k over phi)."""
    th = np.deg2rad(np.asarray(theta_deg, dtype=np.float64))
    ph = np.deg2rad(np.asarray(phi_deg, dtype=np.float64))
    PH, TH = np.meshgrid(ph, th, indexing="ij")
    return TH.ravel(), PH.ravel()


def abc_functions(inv_g, theta, phi):
    """A, B, C of Eq. vtilde for 1/G = inv_g and angles in radians."""
    a = 2.0 * np.pi * np.cos(phi) * np.cos(theta) * inv_g
    b = 2.0 * np.pi * np.cos(phi) * np.sin(theta) * inv_g
    c = 2.0 * np.pi * np.sin(phi) * inv_g
    ca, cb, cc = np.cos(a), np.cos(b), np.cos(c)
    A = ca * cb * cc
    B = ca * cb + ca * cc + cb * cc
    C = ca + cb + cc
    return A, B, C


def expand_weights(w5):
    """[ws1, ws2, wm1, wm2, wm3] -> [ws1, ws2, ws3, wm1, wm2, wm3, wm4] using
    ws1+ws2+ws3 = 1 (Eq. eqsws) and wm1+6wm2+12wm3+8wm4 = 1 (Eq. eqswm in
    per-point form)."""
    w5 = np.asarray(w5, dtype=np.float64)
    ws1, ws2, wm1, wm2, wm3 = (w5[..., k] for k in range(5))
    ws3 = 1.0 - ws1 - ws2
    wm4 = (1.0 - wm1 - 6.0 * wm2 - 12.0 * wm3) / 8.0
    return np.stack([ws1, ws2, ws3, wm1, wm2, wm3, wm4], axis=-1)


def stiffness_X(inv_g, theta, phi, w7):
    """Radicand X of Eq. vtilde (the stiffness symbol times -h^2/2)."""
    A, B, C = abc_functions(inv_g, theta, phi)
    ws1, ws2, ws3 = w7[0], w7[1], w7[2]
    return ws1 * (3.0 - C) + ws2 / 3.0 * (6.0 - C - B) + 2.0 * ws3 / 4.0 * (3.0 - 3.0 * A + B - C)


def mass_J(inv_g, theta, phi, w7):
    """J of Eq. vtilde (the consistent-mass symbol)."""
    A, B, C = abc_functions(inv_g, theta, phi)
    wm1, wm2, wm3, wm4 = w7[3], w7[4], w7[5], w7[6]
    return wm1 + 2.0 * wm2 * C + 4.0 * wm3 * B + 8.0 * wm4 * A


def phase_velocity(inv_g, theta, phi, w7):
    """Normalised numerical phase velocity v~ of Eq. vtilde, written as
    G/(sqrt(2J) pi) sqrt(X) with G = 1/inv_g (inv_g > 0)."""
    X = stiffness_X(inv_g, theta, phi, w7)
    J = mass_J(inv_g, theta, phi, w7)
    return np.sqrt(X) / (np.sqrt(2.0 * J) * np.pi * inv_g)


def linear_form(inv_g, theta, phi):
    """H (..., 5) and g (...) of Eq. linear_basic, H2 as derived (see header)."""
    A, B, C = abc_functions(inv_g, theta, phi)
    K = 2.0 * np.pi ** 2 * inv_g ** 2
    H1 = 0.5 * (3.0 + 3.0 * A - B - C)
    H2 = 0.5 * (1.0 + 3.0 * A - 5.0 / 3.0 * B + 1.0 / 3.0 * C)
    H3 = K * (A - 1.0)
    H4 = K * (6.0 * A - 2.0 * C)
    H5 = K * (12.0 * A - 4.0 * B)
    g = 0.5 * ((4.0 * np.pi ** 2 * inv_g ** 2 + 3.0) * A - B + C - 3.0)
    return np.stack([H1, H2, H3, H4, H5], axis=-1), g


def block(inv_g, theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG):
    """H^(i), g^(i) of Eq. OPFD for one tabulated 1/G."""
    th, ph = angle_grid(theta_deg, phi_deg)
    return linear_form(inv_g, th, ph)


def fit_per_g(inv_g, theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG):
    """Eq. OPFD for one G by numpy's lstsq (minimum-norm: H^(i) has rank 3, so
    the minimiser is a 2-D affine family; the minimal residual is unique).
    Returns (w5, residual norm)."""
    H, g = block(inv_g, theta_deg, phi_deg)
    w = np.linalg.lstsq(H, g, rcond=None)[0]
    return w, float(np.linalg.norm(H @ w - g))


def fit_joint(inv_g_list, theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG):
    """Eq. eq_cost: one weight vector for several G at once (the non-adaptive
    G4 stencil for [1/4], Gm for [1/4, 1/6, 1/8, 1/10])."""
    Hs, gs = zip(*(block(ig, theta_deg, phi_deg) for ig in inv_g_list))
    H = np.vstack(Hs)
    g = np.concatenate(gs)
    return np.linalg.lstsq(H, g, rcond=None)[0]


def table_system(inv_g_max=DEFAULT_INV_G_MAX, d_inv_g=DEFAULT_D_INV_G,
                 theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG):
    """Dense block-diagonal H, stacked g and L = D P of the regularised problem.

    Unknown ordering is the paper's: w = [w^(1); ...; w^(N_G)], each w^(i) the
    5 free weights.  P reorders to series-major; D is the first-order forward
    difference along the tabulated 1/G for each of the 5 series (no wrap, free
    ends -- the paper's "appropriate boundary conditions" is unspecified).
    """
    n_g = int(round(inv_g_max / d_inv_g)) + 1
    inv_g = np.arange(n_g, dtype=np.float64) * d_inv_g
    th, ph = angle_grid(theta_deg, phi_deg)
    n_dir = th.size
    H = np.zeros((n_dir * n_g, 5 * n_g))
    g = np.zeros(n_dir * n_g)
    for i, ig in enumerate(inv_g):
        Hi, gi = linear_form(ig, th, ph)
        H[n_dir * i:n_dir * (i + 1), 5 * i:5 * i + 5] = Hi
        g[n_dir * i:n_dir * (i + 1)] = gi
    # P: series-major permutation, (P w)[l*n_g + i] = w[5 i + l]
    P = np.zeros((5 * n_g, 5 * n_g))
    for l in range(5):
        for i in range(n_g):
            P[l * n_g + i, 5 * i + l] = 1.0
    d1 = np.zeros((n_g - 1, n_g))
    d1[np.arange(n_g - 1), np.arange(n_g - 1)] = -1.0
    d1[np.arange(n_g - 1), np.arange(1, n_g)] = 1.0
    D = np.kron(np.eye(5), d1)
    return inv_g, H, g, D @ P


def fit_table(inv_g_max=DEFAULT_INV_G_MAX, d_inv_g=DEFAULT_D_INV_G,
              theta_deg=DEFAULT_ANGLES_DEG, phi_deg=DEFAULT_ANGLES_DEG,
              lam=DEFAULT_LAMBDA):
    """minimise ||H w - g||^2 + lam ||L w||^2 (Section 2.2), solved as the
    stacked least-squares problem [H; sqrt(lam) L] w = [g; 0] with numpy's
    SVD-based lstsq (no normal equations).  Returns (inv_g nodes, table
    [n_g, 7] as [ws1, ws2, ws3, wm1, wm2, wm3, wm4])."""
    inv_g, H, g, L = table_system(inv_g_max, d_inv_g, theta_deg, phi_deg)
    M = np.vstack([H, np.sqrt(lam) * L])
    rhs = np.concatenate([g, np.zeros(L.shape[0])])
    w = np.linalg.lstsq(M, rhs, rcond=None)[0]
    return inv_g, expand_weights(w.reshape(-1, 5))


def lookup(table, inv_g_nodes, inv_g):
    """Linear interpolation of the table at 1/G (the per-row weight selection of
    the GA stencil, Section 3.1), clamped to the tabulated range."""
    d = inv_g_nodes[1] - inv_g_nodes[0]
    u = np.clip(np.asarray(inv_g, dtype=np.float64) / d, 0.0, len(inv_g_nodes) - 1)
    i0 = np.minimum(np.floor(u).astype(np.int64), len(inv_g_nodes) - 2)
    t = (u - i0)[..., None]
    return (1.0 - t) * table[i0] + t * table[i0 + 1]

"""Closed-form steady profiles used to pin the oracle.  TEST INFRASTRUCTURE ONLY.

- Hartmann flow between plates with equal wall conductance ratio c (Sec. VIII.A,
  the Chang & Lundgren profiles u*(xi), B_x*(xi) with U_ref = a^2 F/(rho nu),
  B_ref = a^2 F mu_m (sigma/(rho nu))^(1/2), Ha = B0 a (sigma/(rho nu))^(1/2)).
- the same body-force flow with lower/upper ratios c_l, c_u (derived in hartmann_walls_constants
  the way App. C treats the shear-driven case).
- Hartmann-Couette flow with lower/upper ratios c_l, c_u, top wall moving at U_w
  (App. C, Eqs. 1DMHDmovingwallfinalsolution and 1DMHDmovingwallintconstants;
  u* = u/U_w, B* = B_x/(U_w (rho nu sigma)^(1/2) mu_m)).

The constants K1, K2 of App. C are written with s = c_u Ha, l = c_l Ha, t = tanh Ha,
which is the same algebra as the phi = c_l/c_u form but finite at c_u = 0.
c = +inf is taken as the limit of each expression.

Lattice units as in the oracle: rho = mu_m = 1, sigma = 1/eta,
nu = (tau_f - 1/2)/3, eta = (tau_m - 1/2)/3.
"""
import math

import numpy as np


def _cosh_ratio(ha, xi):
    """cosh(Ha xi)/cosh(Ha), evaluated without overflow for large Ha."""
    ax = np.abs(xi)
    return np.exp(ha * (ax - 1.0)) * (1.0 + np.exp(-2.0 * ha * ax)) / (1.0 + math.exp(-2.0 * ha))


def _sinh_over_cosh(ha, xi):
    """sinh(Ha xi)/cosh(Ha)."""
    ax = np.abs(xi)
    return np.sign(xi) * np.exp(ha * (ax - 1.0)) * (1.0 - np.exp(-2.0 * ha * ax)) / (1.0 + math.exp(-2.0 * ha))


def _sinh_ratio(ha, xi):
    """sinh(Ha xi)/sinh(Ha)."""
    ax = np.abs(xi)
    return np.sign(xi) * np.exp(ha * (ax - 1.0)) * (1.0 - np.exp(-2.0 * ha * ax)) / (1.0 - math.exp(-2.0 * ha))


def _cosh_over_sinh(ha, xi):
    """cosh(Ha xi)/sinh(Ha)."""
    ax = np.abs(xi)
    return np.exp(ha * (ax - 1.0)) * (1.0 + np.exp(-2.0 * ha * ax)) / (1.0 - math.exp(-2.0 * ha))


def _hartmann_factor(ha, c):
    """(c + 1)/(Ha c + tanh Ha); tends to 1/Ha as c -> inf."""
    if math.isinf(c):
        return 1.0 / ha
    return (c + 1.0) / (ha * c + math.tanh(ha))


def hartmann_u_star(xi, ha, c):
    """Normalised velocity u/U_ref of body-force Hartmann flow (Sec. VIII.A)."""
    xi = np.asarray(xi, dtype=np.float64)
    return (1.0 / ha) * _hartmann_factor(ha, c) * (1.0 - _cosh_ratio(ha, xi))


def hartmann_b_star(xi, ha, c):
    """Normalised induced field B_x/B_ref of body-force Hartmann flow (Sec. VIII.A)."""
    xi = np.asarray(xi, dtype=np.float64)
    return -xi / ha + (1.0 / ha) * _hartmann_factor(ha, c) * _sinh_over_cosh(ha, xi)


def hartmann_walls_constants(ha, c_l, c_u):
    """P, D of body-force Hartmann flow with lower/upper wall conductance ratios c_l, c_u.

    Derived here the way App. C treats the shear-driven case: integrating B*'' + Ha u*' = 0 once
    gives B*' + Ha u* = K, so u*'' - Ha^2 u* = -(1 + Ha K) and, with u*(+-1) = 0,
        u* = P (1 - cosh(Ha xi)/cosh Ha),   B* = -xi/Ha + P sinh(Ha xi)/cosh Ha + D,
    P = (1 + Ha K)/Ha^2.  The Shercliff conditions -B*' + B*/c_l = 0 at xi = -1 and
    B*' + B*/c_u = 0 at xi = +1, multiplied by c, read
        P (Ha c_u + t) + D = (1 + c_u)/Ha,   -P (Ha c_l + t) + D = -(1 + c_l)/Ha,   t = tanh Ha,
    whence P = (2 + c_l + c_u)/(Ha (Ha (c_l + c_u) + 2 t)) and D = (1 + c_u)/Ha - P (Ha c_u + t),
    which expands to D = (c_l - c_u)(Ha - t)/(Ha (Ha (c_l + c_u) + 2 t)) (no cancellation of large
    terms when a ratio is large).  c = inf reduces its condition to B*' = 0: P = 1/Ha^2 and
    D = -+(Ha - t)/Ha^2 for c_u or c_l infinite; with both walls perfectly conducting D is taken as
    0, the symmetric limit (D is then fixed by the initial state, not by the walls).  c_l = c_u
    gives D = 0 and P = (c + 1)/(Ha (Ha c + t)), the equal-walls profile."""
    t = math.tanh(ha)
    if math.isinf(c_l) and math.isinf(c_u):
        return 1.0 / (ha * ha), 0.0
    if math.isinf(c_u):
        return 1.0 / (ha * ha), -(ha - t) / (ha * ha)
    if math.isinf(c_l):
        return 1.0 / (ha * ha), (ha - t) / (ha * ha)
    den = ha * (ha * (c_l + c_u) + 2.0 * t)
    return (2.0 + c_l + c_u) / den, (c_l - c_u) * (ha - t) / den


def hartmann_walls_u_star(xi, ha, c_l, c_u):
    """u/U_ref of body-force Hartmann flow with conductance ratios c_l (xi = -1) and c_u (xi = +1)."""
    xi = np.asarray(xi, dtype=np.float64)
    p, _ = hartmann_walls_constants(ha, c_l, c_u)
    return p * (1.0 - _cosh_ratio(ha, xi))


def hartmann_walls_b_star(xi, ha, c_l, c_u):
    """B_x/B_ref of body-force Hartmann flow with conductance ratios c_l (xi = -1) and c_u (xi = +1)."""
    xi = np.asarray(xi, dtype=np.float64)
    p, d = hartmann_walls_constants(ha, c_l, c_u)
    return -xi / ha + p * _sinh_over_cosh(ha, xi) + d


def couette_constants(ha, c_l, c_u):
    """K1, K2 of App. C (Eq. 1DMHDmovingwallintconstants), in the s, l form."""
    t = math.tanh(ha)
    s = c_u * ha
    l = c_l * ha
    if math.isinf(c_u) and math.isinf(c_l):
        raise ValueError("no steady state with both walls perfectly conducting")
    if math.isinf(c_u):
        # divide numerator and denominator by s and let s -> inf
        return 1.0, 0.5 * (t + 1.0 / t) + l
    if math.isinf(c_l):
        return 0.0, 0.5 * (t + 1.0 / t) + s
    den = 2.0 * t + s + l
    k1 = (t + s) / den
    k2 = (1.0 + 0.5 * (s + l) * (t + 1.0 / t) + s * l) / den
    return k1, k2


def couette_u_star(xi, ha, c_l, c_u):
    """Normalised velocity u/U_w of Hartmann-Couette flow (Eq. 1DMHDmovingwallfinalsolution)."""
    xi = np.asarray(xi, dtype=np.float64)
    k1, _ = couette_constants(ha, c_l, c_u)
    return k1 + (0.5 - k1) * _cosh_ratio(ha, xi) + 0.5 * _sinh_ratio(ha, xi)


def couette_b_star(xi, ha, c_l, c_u):
    """Normalised induced field of Hartmann-Couette flow (Eq. 1DMHDmovingwallfinalsolution)."""
    xi = np.asarray(xi, dtype=np.float64)
    k1, k2 = couette_constants(ha, c_l, c_u)
    return k2 - (0.5 - k1) * _sinh_over_cosh(ha, xi) - 0.5 * _cosh_over_sinh(ha, xi)


def lattice_scales(tau_f, tau_m):
    """nu, eta in lattice units (Sec. IV, Sec. V)."""
    return (tau_f - 0.5) / 3.0, (tau_m - 0.5) / 3.0


def b0_from_ha(ha, a, tau_f, tau_m):
    """Applied field giving Hartmann number Ha on half-width a: B0 = Ha sqrt(nu eta)/a."""
    nu, eta = lattice_scales(tau_f, tau_m)
    return ha * math.sqrt(nu * eta) / a


def force_for_centre_speed(u_c, ha, c, a, tau_f):
    """Body force giving centreline speed u_c in the analytic Hartmann profile."""
    nu = (tau_f - 0.5) / 3.0
    return u_c * nu / (a * a * float(hartmann_u_star(0.0, ha, c)))


def hartmann_profiles(y, a, ha, c, fx, tau_f, tau_m):
    """Dimensional (lattice-unit) u_x(y), B_x(y) of body-force Hartmann flow."""
    nu, eta = lattice_scales(tau_f, tau_m)
    u_ref = a * a * fx / nu
    b_ref = a * a * fx / math.sqrt(nu * eta)
    xi = np.asarray(y, dtype=np.float64) / a
    return u_ref * hartmann_u_star(xi, ha, c), b_ref * hartmann_b_star(xi, ha, c)


def hartmann_walls_profiles(y, a, ha, c_l, c_u, fx, tau_f, tau_m):
    """Dimensional u_x(y), B_x(y) of body-force Hartmann flow with conductance ratios c_l, c_u."""
    nu, eta = lattice_scales(tau_f, tau_m)
    u_ref = a * a * fx / nu
    b_ref = a * a * fx / math.sqrt(nu * eta)
    xi = np.asarray(y, dtype=np.float64) / a
    return u_ref * hartmann_walls_u_star(xi, ha, c_l, c_u), b_ref * hartmann_walls_b_star(xi, ha, c_l, c_u)


def couette_profiles(y, a, ha, c_l, c_u, u_w, tau_f, tau_m):
    """Dimensional u_x(y), B_x(y) of Hartmann-Couette flow (top wall at U_w)."""
    nu, eta = lattice_scales(tau_f, tau_m)
    xi = np.asarray(y, dtype=np.float64) / a
    return u_w * couette_u_star(xi, ha, c_l, c_u), u_w * math.sqrt(nu / eta) * couette_b_star(xi, ha, c_l, c_u)


def rel_l2(computed, analytic):
    """RMS error over the nodes across the channel (Sec. VIII.A) divided by max|analytic|."""
    computed = np.asarray(computed, dtype=np.float64)
    analytic = np.asarray(analytic, dtype=np.float64)
    rms = math.sqrt(float(np.mean((computed - analytic) ** 2)))
    scale = float(np.max(np.abs(analytic)))
    return rms / scale if scale > 0 else rms

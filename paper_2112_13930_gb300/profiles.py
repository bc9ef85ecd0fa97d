"""Closed-form steady profiles for the accuracy gate of solved channels (product side).

Body-force Hartmann flow between plates of equal wall conductance ratio c (Chang & Lundgren, as
quoted in Sec. VIII.A), the same flow with a different ratio on each plate (solved like App. C's
shear-driven case), and Hartmann-Couette flow with lower/upper ratios c_l, c_u and the top plate
at U_w (App. C, Eqs. 1DMHDmovingwallfinalsolution / 1DMHDmovingwallintconstants).  Written with
exponentials of Ha (|xi| - 1), which stay finite for any Ha, and with the App. C constants in the
form that is finite at c_u = 0 (numerator and denominator multiplied by c_u).

Lattice units: rho = mu_m = 1, nu = (tau_f - 1/2)/3, eta = (tau_m - 1/2)/3, sigma = 1/eta,
Ha = B0 a / sqrt(nu eta).
"""
import math

import numpy as np


def node_y(ny, closure):
    """Wall-normal coordinates of the rows: link-based walls half-way outside rows 0 and ny-1
    (a = ny/2), moment-based walls on those rows (a = (ny-1)/2)."""
    if closure in ("link", 0):
        a = ny / 2.0
        return a, np.arange(ny) + 0.5 - a
    a = (ny - 1) / 2.0
    return a, np.arange(ny) - a


def _ch(ha, xi):
    """cosh(Ha xi)/cosh(Ha)."""
    e = np.exp(ha * (np.abs(xi) - 1.0))
    return e * (1.0 + np.exp(-2.0 * ha * np.abs(xi))) / (1.0 + math.exp(-2.0 * ha))


def _sh(ha, xi):
    """sinh(Ha xi)/cosh(Ha)."""
    e = np.exp(ha * (np.abs(xi) - 1.0))
    return np.sign(xi) * e * (1.0 - np.exp(-2.0 * ha * np.abs(xi))) / (1.0 + math.exp(-2.0 * ha))


def hartmann(y, a, ha, c, fx, tau_f, tau_m):
    """u_x(y), B_x(y) of body-force Hartmann flow; c may be math.inf."""
    nu, eta = (tau_f - 0.5) / 3.0, (tau_m - 0.5) / 3.0
    xi = np.asarray(y, dtype=np.float64) / a
    k = 1.0 / ha if math.isinf(c) else (c + 1.0) / (ha * c + math.tanh(ha))
    u_ref = a * a * fx / nu
    b_ref = a * a * fx / math.sqrt(nu * eta)
    u = u_ref * (k / ha) * (1.0 - _ch(ha, xi))
    b = b_ref * (-xi / ha + (k / ha) * _sh(ha, xi))
    return u, b


def hartmann_force(u_c, ha, c, a, tau_f):
    """Body force that gives centreline speed u_c."""
    nu = (tau_f - 0.5) / 3.0
    k = 1.0 / ha if math.isinf(c) else (c + 1.0) / (ha * c + math.tanh(ha))
    return u_c * nu / (a * a * (k / ha) * (1.0 - 1.0 / math.cosh(ha)))


def _walls_pd(ha, c_l, c_u):
    """Amplitude P of u/U_ref and offset D of B_x/B_ref for body-force Hartmann flow with the
    lower/upper conductance ratios c_l, c_u: the Shercliff conditions at both plates fix
    P = (2 + c_l + c_u)/(Ha (Ha (c_l + c_u) + 2 tanh Ha)), D = (c_l - c_u)(Ha - tanh Ha)/(same)."""
    t = math.tanh(ha)
    if math.isinf(c_l) or math.isinf(c_u):
        if math.isinf(c_l) and math.isinf(c_u):
            return 1.0 / ha ** 2, 0.0
        sign = 1.0 if math.isinf(c_l) else -1.0
        return 1.0 / ha ** 2, sign * (ha - t) / ha ** 2
    den = ha * (ha * (c_l + c_u) + 2.0 * t)
    return (2.0 + c_l + c_u) / den, (c_l - c_u) * (ha - t) / den


def hartmann_walls(y, a, ha, c_l, c_u, fx, tau_f, tau_m):
    """u_x(y), B_x(y) of body-force Hartmann flow with conductance ratio c_l on the lower plate and
    c_u on the upper one (either may be math.inf)."""
    nu, eta = (tau_f - 0.5) / 3.0, (tau_m - 0.5) / 3.0
    xi = np.asarray(y, dtype=np.float64) / a
    pa, d = _walls_pd(ha, c_l, c_u)
    u = (a * a * fx / nu) * pa * (1.0 - _ch(ha, xi))
    b = (a * a * fx / math.sqrt(nu * eta)) * (-xi / ha + pa * _sh(ha, xi) + d)
    return u, b


def hartmann_walls_force(u_c, ha, c_l, c_u, a, tau_f):
    """Body force that gives centreline speed u_c with conductance ratios c_l, c_u."""
    nu = (tau_f - 0.5) / 3.0
    pa, _ = _walls_pd(ha, c_l, c_u)
    return u_c * nu / (a * a * pa * (1.0 - 1.0 / math.cosh(ha)))


def couette(y, a, ha, c_l, c_u, u_w, tau_f, tau_m):
    """u_x(y), B_x(y) of Hartmann-Couette flow with the top plate at U_w (c_l, c_u may be inf,
    not both)."""
    nu, eta = (tau_f - 0.5) / 3.0, (tau_m - 0.5) / 3.0
    xi = np.asarray(y, dtype=np.float64) / a
    t = math.tanh(ha)
    if math.isinf(c_u) and math.isinf(c_l):
        raise ValueError("both plates perfectly conducting: no steady state")
    if math.isinf(c_u):
        k1, k2 = 1.0, 0.5 * (t + 1.0 / t) + c_l * ha
    elif math.isinf(c_l):
        k1, k2 = 0.0, 0.5 * (t + 1.0 / t) + c_u * ha
    else:
        s, l = c_u * ha, c_l * ha
        d = 2.0 * t + s + l
        k1 = (t + s) / d
        k2 = (1.0 + 0.5 * (s + l) * (t + 1.0 / t) + s * l) / d
    shs = _sh(ha, xi) / t          # sinh(Ha xi)/sinh(Ha)
    chs = _ch(ha, xi) / t          # cosh(Ha xi)/sinh(Ha)
    u = k1 + (0.5 - k1) * _ch(ha, xi) + 0.5 * shs
    b = k2 - (0.5 - k1) * _sh(ha, xi) - 0.5 * chs
    return u_w * u, u_w * math.sqrt(nu / eta) * b


def rel_l2(computed, exact):
    """RMS error over the channel's nodes divided by max|exact| (the paper's L2 norm, made
    relative to the profile scale)."""
    computed = np.asarray(computed, dtype=np.float64)
    exact = np.asarray(exact, dtype=np.float64)
    s = float(np.max(np.abs(exact)))
    r = math.sqrt(float(np.mean((computed - exact) ** 2)))
    return r / s if s > 0 else r

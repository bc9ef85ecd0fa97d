"""Pins of the closed-form profiles in oracle/analytic.py against the mathematics.

Each closed form is checked against the boundary-value problem it solves (finite
differences of the profile, not its formula), against textbook special cases, and
against the paper's own intermediate linear system of App. C.
"""
import math

import numpy as np
import pytest

from oracle import analytic as an


def _d1(fn, x, h=1e-4):
    return (fn(x + h) - fn(x - h)) / (2 * h)


def _d2(fn, x, h=1e-4):
    return (fn(x + h) - 2 * fn(x) + fn(x - h)) / (h * h)


HARTMANN_CASES = [(ha, c) for ha in (1.0, 5.0, 20.0) for c in (0.0, 0.1, 0.5, 1.0, 1e4, math.inf)]


@pytest.mark.parametrize("ha,c", HARTMANN_CASES)
def test_hartmann_solves_bvp(ha, c):
    """u*'' + Ha B*' + 1 = 0 and B*'' + Ha u*' = 0 (Sec. II reduced to 1D with body force),
    u* = 0 at the plates, Shercliff condition of Eq. ShercliffBCforHartmannFlow at xi = -1, +1."""
    u = lambda x: an.hartmann_u_star(x, ha, c)
    b = lambda x: an.hartmann_b_star(x, ha, c)
    h = 1e-4 if ha < 10 else 2e-5
    xi = np.linspace(-0.98, 0.98, 41)
    scale_u = float(np.max(np.abs(u(np.linspace(-1, 1, 201)))))
    r1 = _d2(u, xi, h) + ha * _d1(b, xi, h) + 1.0
    r2 = _d2(b, xi, h) + ha * _d1(u, xi, h)
    assert np.max(np.abs(r1)) < 1e-3 * max(1.0, ha * ha * scale_u)
    assert np.max(np.abs(r2)) < 1e-3 * max(1.0, ha * ha * scale_u)
    assert abs(u(-1.0)) < 1e-12 and abs(u(1.0)) < 1e-12
    hh = 1e-6
    db_lo = (b(-1.0 + hh) - b(-1.0)) / hh
    db_hi = (b(1.0) - b(1.0 - hh)) / hh
    tol = 1e-4 * max(1.0, ha)
    if math.isinf(c):
        assert abs(db_lo) < tol and abs(db_hi) < tol
    else:
        # -c B' + B = 0 at xi = -1 and c B' + B = 0 at xi = +1 (condition times c)
        assert abs(-c * db_lo + b(-1.0)) < tol * max(1.0, c)
        assert abs(c * db_hi + b(1.0)) < tol * max(1.0, c)


WALLS_CASES = [(ha, cl, cu) for ha in (1.0, 5.0, 20.0)
               for cl, cu in ((0.0, 0.5), (0.1, 2.0), (1e4, 0.0), (math.inf, 0.3), (0.5, math.inf))]


@pytest.mark.parametrize("ha,cl,cu", WALLS_CASES)
def test_hartmann_walls_solves_bvp(ha, cl, cu):
    """Body force with different conductance ratios on the two plates: the same ODEs, u* = 0 at
    the plates, and the Shercliff condition with c_l at xi = -1 and c_u at xi = +1."""
    u = lambda x: an.hartmann_walls_u_star(x, ha, cl, cu)
    b = lambda x: an.hartmann_walls_b_star(x, ha, cl, cu)
    h = 1e-4 if ha < 10 else 2e-5
    xi = np.linspace(-0.98, 0.98, 41)
    scale = max(1.0, ha * ha * float(np.max(np.abs(u(np.linspace(-1, 1, 201))))))
    assert np.max(np.abs(_d2(u, xi, h) + ha * _d1(b, xi, h) + 1.0)) < 1e-3 * scale
    assert np.max(np.abs(_d2(b, xi, h) + ha * _d1(u, xi, h))) < 1e-3 * scale
    assert abs(u(-1.0)) < 1e-12 and abs(u(1.0)) < 1e-12
    hh = 1e-6
    db_lo = (b(-1.0 + hh) - b(-1.0)) / hh
    db_hi = (b(1.0) - b(1.0 - hh)) / hh
    tol = 1e-4 * max(1.0, ha)
    if math.isinf(cl):
        assert abs(db_lo) < tol
    else:
        assert abs(-cl * db_lo + b(-1.0)) < tol * max(1.0, cl)
    if math.isinf(cu):
        assert abs(db_hi) < tol
    else:
        assert abs(cu * db_hi + b(1.0)) < tol * max(1.0, cu)


@pytest.mark.parametrize("ha,c", HARTMANN_CASES)
def test_hartmann_walls_equal_ratios_is_equal_walls_profile(ha, c):
    xi = np.linspace(-1, 1, 41)
    assert np.allclose(an.hartmann_walls_u_star(xi, ha, c, c), an.hartmann_u_star(xi, ha, c), rtol=1e-12, atol=1e-15)
    assert np.allclose(an.hartmann_walls_b_star(xi, ha, c, c), an.hartmann_b_star(xi, ha, c), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("ha,cl,cu", WALLS_CASES)
def test_hartmann_walls_mirror(ha, cl, cu):
    """Swapping the plates mirrors the flow: u*(xi) unchanged, B* odd under xi -> -xi."""
    xi = np.linspace(-1, 1, 41)
    assert np.allclose(an.hartmann_walls_u_star(xi, ha, cu, cl), an.hartmann_walls_u_star(-xi, ha, cl, cu), atol=1e-14)
    assert np.allclose(an.hartmann_walls_b_star(xi, ha, cu, cl), -an.hartmann_walls_b_star(-xi, ha, cl, cu),
                       atol=1e-13)


@pytest.mark.parametrize("ha", [0.5, 3.0, 10.0, 40.0])
def test_hartmann_insulating_is_textbook(ha):
    """c = 0: the classical Hartmann (1937) profiles u* = (cosh Ha - cosh Ha xi)/(Ha sinh Ha),
    B* = sinh(Ha xi)/(Ha sinh Ha) - xi/Ha."""
    xi = np.linspace(-1, 1, 101)
    u_tb = (np.cosh(ha) - np.cosh(ha * xi)) / (ha * np.sinh(ha))
    b_tb = np.sinh(ha * xi) / (ha * np.sinh(ha)) - xi / ha
    np.testing.assert_allclose(an.hartmann_u_star(xi, ha, 0.0), u_tb, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(an.hartmann_b_star(xi, ha, 0.0), b_tb, rtol=1e-12, atol=1e-14)


def test_hartmann_small_ha_is_poiseuille():
    """Ha -> 0: u* -> (1 - xi^2)/2 (plane Poiseuille flow) for any c."""
    xi = np.linspace(-1, 1, 51)
    for c in (0.0, 1.0):
        np.testing.assert_allclose(an.hartmann_u_star(xi, 1e-4, c), 0.5 * (1 - xi ** 2), atol=1e-7)


def test_hartmann_velocity_decreases_with_c():
    """Higher wall conductance gives smaller velocity at fixed Ha (Sec. VIII.A)."""
    xi = np.linspace(-0.99, 0.99, 21)
    prev = an.hartmann_u_star(xi, 5.0, 0.0)
    for c in (0.1, 0.5, 1.0, 1e4):
        cur = an.hartmann_u_star(xi, 5.0, c)
        assert np.all(cur < prev)
        prev = cur


COUETTE_CASES = [(ha, cl, cu) for ha in (1.0, 5.0, 20.0)
                 for (cu, cl) in ((0.0, 0.0), (0.5, 0.5), (0.0, 0.5), (0.1, 0.0), (1.0, 0.0), (1e4, 0.0),
                                  (math.inf, 0.0), (2.0, 0.3), (0.3, math.inf))]


@pytest.mark.parametrize("ha,cl,cu", COUETTE_CASES)
def test_couette_solves_bvp(ha, cl, cu):
    """App. C: u*'' + Ha B*' = 0, B*'' + Ha u*' = 0 (Eq. 1DMHDsystemnondim), u*(-1) = 0,
    u*(1) = 1, -B*' + B*/c_l = 0 at -1 and B*' + B*/c_u = 0 at +1 (Eq. 1DMHDBCs)."""
    u = lambda x: an.couette_u_star(x, ha, cl, cu)
    b = lambda x: an.couette_b_star(x, ha, cl, cu)
    h = 1e-4 if ha < 10 else 2e-5
    xi = np.linspace(-0.98, 0.98, 41)
    r1 = _d2(u, xi, h) + ha * _d1(b, xi, h)
    r2 = _d2(b, xi, h) + ha * _d1(u, xi, h)
    assert np.max(np.abs(r1)) < 1e-3 * max(1.0, ha * ha)
    assert np.max(np.abs(r2)) < 1e-3 * max(1.0, ha * ha)
    assert abs(u(-1.0)) < 1e-12 and abs(u(1.0) - 1.0) < 1e-12
    hh = 1e-6
    db_lo = (b(-1.0 + hh) - b(-1.0)) / hh
    db_hi = (b(1.0) - b(1.0 - hh)) / hh
    tol = 1e-4 * max(1.0, ha)
    if math.isinf(cl):
        assert abs(db_lo) < tol
    else:
        assert abs(-cl * db_lo + b(-1.0)) < tol * max(1.0, cl)
    if math.isinf(cu):
        assert abs(db_hi) < tol
    else:
        assert abs(cu * db_hi + b(1.0)) < tol * max(1.0, cu)


@pytest.mark.parametrize("ha,cl,cu", [(5.0, 0.0, 0.0), (5.0, 0.5, 0.5), (20.0, 0.5, 0.0), (3.0, 0.3, 2.0),
                                      (5.0, 0.0, 1e4)])
def test_couette_constants_from_paper_linear_system(ha, cl, cu):
    """K1 = p + p', K2 = p - p' solve the 2x2 system of App. C (Eqs. constraintsystemtforconstants,
    coefficientsexpressions).  The upper-wall row is +lambda_2 (p+p') + (p-p') = gamma_2: that sign
    is what the printed solution (Eq. pprimesumdiffexpression) solves, and what substituting
    Eq. 1DMHDsolutionmovingwallhyprbolfunc2 into the upper Shercliff condition gives."""
    t = math.tanh(ha)
    lam1 = cl * ha + t
    lam2 = cu * ha + t
    g1 = 0.5 * (1.0 / t - t)
    g2 = 0.5 * (1.0 / t + t) + cu * ha
    x, y = np.linalg.solve(np.array([[-lam1, 1.0], [lam2, 1.0]]), np.array([g1, g2]))
    k1, k2 = an.couette_constants(ha, cl, cu)
    assert k1 == pytest.approx(x, rel=1e-12, abs=1e-14)
    assert k2 == pytest.approx(y, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("ha,c", [(5.0, 0.0), (5.0, 0.5), (20.0, 0.1), (2.0, 10.0)])
def test_couette_equal_walls_special_case(ha, c):
    """phi = 1 (Eq. 1DMHDmovingwallfinalsolutionsplcase): u* = (1 + sinh(Ha xi)/sinh Ha)/2,
    independent of c (Sec. VIII.B), and the printed B* with K2 for equal walls."""
    xi = np.linspace(-1, 1, 81)
    u_sp = 0.5 * (1.0 + np.sinh(ha * xi) / np.sinh(ha))
    t = math.tanh(ha)
    s = c * ha
    b_sp = (1.0 + s * (t + 1.0 / t) + s * s) / (2.0 * (t + s)) - 0.5 * np.cosh(ha * xi) / np.sinh(ha)
    np.testing.assert_allclose(an.couette_u_star(xi, ha, c, c), u_sp, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(an.couette_b_star(xi, ha, c, c), b_sp, rtol=1e-12, atol=1e-13)


def test_couette_insulating_special_case():
    """c_l = c_u = 0 (Eq. 1DMHDmovingwallfinalsolutionsplinsulcase): B* = (1 - cosh(Ha xi)/cosh Ha)/(2 tanh Ha)."""
    ha = 5.0
    xi = np.linspace(-1, 1, 81)
    b_sp = (1.0 - np.cosh(ha * xi) / np.cosh(ha)) / (2.0 * math.tanh(ha))
    np.testing.assert_allclose(an.couette_b_star(xi, ha, 0.0, 0.0), b_sp, rtol=1e-12, atol=1e-14)


def test_couette_small_ha_is_linear_shear():
    """Ha -> 0 with insulating walls: plane Couette flow u* = (1 + xi)/2."""
    xi = np.linspace(-1, 1, 41)
    np.testing.assert_allclose(an.couette_u_star(xi, 1e-4, 0.0, 0.0), 0.5 * (1 + xi), atol=1e-7)


def test_couette_contrast_changes_velocity():
    """A contrast c_l != c_u changes u* (Sec. VIII.B); equal walls do not."""
    xi = np.linspace(-0.9, 0.9, 19)
    u00 = an.couette_u_star(xi, 5.0, 0.0, 0.0)
    u55 = an.couette_u_star(xi, 5.0, 0.5, 0.5)
    u05 = an.couette_u_star(xi, 5.0, 0.5, 0.0)
    np.testing.assert_allclose(u00, u55, rtol=1e-12)
    assert np.max(np.abs(u05 - u00)) > 1e-2


def test_lattice_parameters_of_hartmann_channel():
    """4 x 65 link-based channel, tau = 0.8, Ha = 10, c = 0.1: a = 32.5, B0 = Ha sqrt(nu eta)/a,
    theta = c a/(tau_m - 1/2) = 10.8333 (Eq. weightingfactor)."""
    a = 65 / 2
    b0 = an.b0_from_ha(10.0, a, 0.8, 0.8)
    assert b0 == pytest.approx(10.0 * 0.1 / 32.5, rel=1e-14)
    assert 0.1 * a / (0.8 - 0.5) == pytest.approx(10.833333333333334, rel=1e-14)
    fx = an.force_for_centre_speed(0.01, 10.0, 0.1, a, 0.8)
    u, _ = an.hartmann_profiles(np.array([0.0]), a, 10.0, 0.1, fx, 0.8, 0.8)
    assert u[0] == pytest.approx(0.01, rel=1e-13)

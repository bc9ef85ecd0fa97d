"""Pins of the oracle's wall closures that do not rely on the upper wall alone.

1. Mirror symmetry.  The D2Q9/D2Q5 scheme is equivariant under the reflection y -> -y combined with
   B_x -> -B_x (B_y, u_x unchanged, u_y -> -u_y): the lattice maps onto itself (directions 2<->4,
   5<->8, 6<->7), g^eq and the Maxwell stress map onto their mirror images, and so does the Lorentz
   force.  A channel whose bottom plate moves, with the conductance ratios of the two plates swapped,
   must therefore evolve as the exact mirror image of the channel whose top plate moves -- the
   reflection symmetry of the 1D equations of App. C (nu u'' + B0 B' + F = 0, eta B'' + B0 u' = 0 are
   invariant under u(y) -> u(-y), B(y) -> -B(-y)).  The upper-plate closures are pinned by the closed
   forms of App. C; this carries the pin over to the lower plate: its moving-wall g term of
   Eq. movingwalllinkbasedclosure, its Ladd term (App. B.1) and the moment-based lower-wall forms
   (App. B.2) must be the mirror of the upper ones, to rounding.
2. The closed form of App. C with the roles of the plates swapped (bottom plate moving).
3. Decoupled closure check: with u frozen at 0 and B0 = 0 the induction equation is plain diffusion,
   dB_x/dt = eta d^2B_x/dy^2, with the Shercliff (Robin) conditions B + c a dB/dn = 0 on each plate
   (Eq. ShercliffBClocalcoordinate).  Its slowest mode cos(k y + psi) decays at the rate eta k^2, with
   k the smallest positive root of the textbook Robin eigenvalue condition (k tan(ka) = 1/(c a) for
   equal plates; cos modes for c = 0, Neumann for c = inf).  Both closures must reproduce that rate to
   second order in the grid spacing.
4. Planted one-token mutants of the lower-plate moving-wall terms fail pins 1 and 2.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from oracle import analytic as an

MIR9 = [0, 1, 4, 3, 2, 8, 7, 6, 5]
MIR5 = [0, 1, 4, 3, 2]
W5 = np.array([1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6])


def _mirror_state(f, g):
    """Populations of the reflected lattice: rows reversed, directions mirrored, g_x negated."""
    fm = f[MIR9][:, ::-1, :]
    gm = np.empty_like(g)
    gm[0] = -g[0][MIR5][:, ::-1, :]
    gm[1] = g[1][MIR5][:, ::-1, :]
    return fm, gm


# (closure, c of the moving plate, c of the plate at rest, body force, coupling)
MIRROR_CASES = [
    (oracle.LINK, 0.0, 0.0, 0.0, 0),
    (oracle.LINK, 0.4, 2.5, 0.0, 0),
    (oracle.LINK, math.inf, 0.0, 0.0, 0),
    (oracle.LINK, 0.7, math.inf, 3e-6, 0),
    (oracle.LINK, 0.3, 1.2, 2e-6, 1),
    (oracle.MOMENT, 0.0, 0.0, 0.0, 0),
    (oracle.MOMENT, 0.4, 2.5, 0.0, 0),
    (oracle.MOMENT, math.inf, 0.0, 0.0, 0),
    (oracle.MOMENT, 0.7, math.inf, 3e-6, 0),
    (oracle.MOMENT, 0.3, 1.2, 2e-6, 1),
]


def _pair(closure, c_move, c_rest, fx, coupling, lib=None, nx=3, ny=17, steps=400, u_w=0.04):
    """Top plate moving (reference) and bottom plate moving with the ratios swapped."""
    runs = []
    for bottom_moves in (False, True):
        o = oracle.Oracle(nx, ny, 0.7, 0.85, 0.03, fx, closure, coupling=coupling, seed=11, perturb_amp=0.0)
        if bottom_moves:
            o.set_walls(c_move, c_rest, u_w, 0.0)
        else:
            o.set_walls(c_rest, c_move, 0.0, u_w)
        if lib is None:
            o.step(steps)
        else:
            P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            assert lib.orc_run(ctypes.byref(o.p), P(o.f), P(o.g), steps) == 0
        runs.append(o)
    return runs


@pytest.mark.parametrize("closure,c_move,c_rest,fx,coupling", MIRROR_CASES)
def test_lower_moving_wall_is_mirror_of_upper(closure, c_move, c_rest, fx, coupling):
    top, bot = _pair(closure, c_move, c_rest, fx, coupling)
    fm, gm = _mirror_state(top.f, top.g)
    # equal to rounding: the mirrored directions are summed in a different order
    np.testing.assert_allclose(bot.f, fm, rtol=0, atol=1e-14)
    np.testing.assert_allclose(bot.g, gm, rtol=0, atol=1e-15)
    # and the induced field is genuinely present, so the g_x comparison means something
    assert np.max(np.abs(top.moments()[3])) > 1e-7
    mt, mb = top.moments(), bot.moments()
    np.testing.assert_allclose(mb[1], mt[1][::-1], rtol=0, atol=1e-14)
    np.testing.assert_allclose(mb[3], -mt[3][::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("closure", [oracle.LINK, oracle.MOMENT])
@pytest.mark.parametrize("ha,c_move,c_rest", [(5.0, 0.5, 0.0), (10.0, 1e4, 0.0), (5.0, 0.3, 2.0)])
def test_lower_moving_wall_couette_closed_form(closure, ha, c_move, c_rest):
    """Bottom plate at +U_w, top at rest: the App. C solution reflected, u(y) = U u*(-xi) and
    B_x(y) = -U sqrt(nu/eta) B*(-xi), with c_l, c_u of the reflected problem = (c_top, c_bot)."""
    ny, u_w = 65, 0.05
    a = ny / 2 if closure == oracle.LINK else (ny - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    o = oracle.Oracle(3, ny, 0.8, 0.8, b0, 0.0, closure, c_move, c_rest, u_w, 0.0)
    r = o.run_to_steady(1e-9, 200, 400_000)
    assert r < 1e-9
    u, b = o.profiles()
    ua, ba = an.couette_profiles(-o.y(), a, ha, c_rest, c_move, u_w, 0.8, 0.8)
    tol = 5e-3 if ha <= 10 else 1e-2
    assert an.rel_l2(u, ua) < tol
    assert an.rel_l2(b, -ba) < tol


# ---- decoupled closure check: Robin eigenvalue decay of B_x with u frozen ----

def _robin_rows(k, a, c_bot, c_top):
    """Rows of the 2x2 system for phi = A cos(ky) + B sin(ky) with phi + c_t a phi' = 0 at y = a and
    phi - c_b a phi' = 0 at y = -a (the outward normal is -y there); c = inf keeps phi' = 0."""
    s, co = math.sin(k * a), math.cos(k * a)
    top = [-k * s, k * co] if math.isinf(c_top) else [co - c_top * a * k * s, s + c_top * a * k * co]
    bot = [-k * s, -k * co] if math.isinf(c_bot) else [co - c_bot * a * k * s, -(s + c_bot * a * k * co)]
    return np.array([top, bot])


def robin_mode(a, c_bot, c_top):
    """Smallest positive k with a nontrivial mode, and the mode's (A, B)."""
    det = lambda k: float(np.linalg.det(_robin_rows(k, a, c_bot, c_top)))
    ks = np.linspace(1e-6 / a, 2.0 * math.pi / a, 4001)
    d = [det(k) for k in ks]
    for i in range(len(ks) - 1):
        if d[i] * d[i + 1] < 0:
            k = brentq(det, ks[i], ks[i + 1], xtol=1e-15, rtol=1e-15)
            _, _, vt = np.linalg.svd(_robin_rows(k, a, c_bot, c_top))
            return k, vt[-1]
    raise AssertionError("no root")


def test_robin_mode_textbook_limits():
    """The eigenvalue solver itself: c = 0 gives cos(ka) = 0, c = inf on both plates the first odd
    Neumann mode (k = pi/(2a)), (0, inf) gives k = pi/(4a); equal finite c solves k tan(ka) = 1/(ca)."""
    a = 10.0
    assert robin_mode(a, 0.0, 0.0)[0] == pytest.approx(math.pi / (2 * a), rel=1e-12)
    assert robin_mode(a, math.inf, math.inf)[0] == pytest.approx(math.pi / (2 * a), rel=1e-12)
    assert robin_mode(a, 0.0, math.inf)[0] == pytest.approx(math.pi / (4 * a), rel=1e-12)
    k = robin_mode(a, 0.3, 0.3)[0]
    assert k * math.tan(k * a) == pytest.approx(1.0 / (0.3 * a), rel=1e-10)


def robin_decay_error(closure, c_bot, c_top, ny, tau_m=0.8, lib=None):
    """Relative error of the measured decay rate of the slowest Robin mode against eta k^2."""
    o = oracle.Oracle(1, ny, 0.8, tau_m, 0.0, 0.0, closure, c_bot, c_top, freeze_u=True)
    a, y, eta = o.a, o.y(), (tau_m - 0.5) / 3.0
    k, (A, B) = robin_mode(a, c_bot, c_top)
    phi = A * np.cos(k * y) + B * np.sin(k * y)
    phi /= np.max(np.abs(phi))
    o.g[0] = W5[:, None, None] * (1e-3 * phi)[None, :, None]
    o.g[1] = 0.0
    T = a * a / eta
    n1, n2 = int(0.2 * T), int(0.6 * T)
    amps = []
    for n in (n1, n2 - n1):
        if lib is None:
            o.step(n)
        else:
            P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            assert lib.orc_run(ctypes.byref(o.p), P(o.f), P(o.g), n) == 0
        amps.append(float(o.moments()[3][:, 0] @ phi))
    rate = -math.log(amps[1] / amps[0]) / (n2 - n1)
    return rate / (eta * k * k) - 1.0


ROBIN_CASES = [(0.0, 0.0), (0.3, 0.3), (math.inf, math.inf), (0.0, math.inf), (0.05, 2.0), (math.inf, 0.1)]


@pytest.mark.parametrize("closure", [oracle.LINK, oracle.MOMENT])
@pytest.mark.parametrize("c_bot,c_top", ROBIN_CASES)
def test_robin_decay_rate_second_order(closure, c_bot, c_top):
    e33 = robin_decay_error(closure, c_bot, c_top, 33)
    e65 = robin_decay_error(closure, c_bot, c_top, 65)
    assert abs(e65) < 2e-4, e65
    order = math.log(abs(e33 / e65)) / math.log(64.0 / 32.0 if closure == oracle.MOMENT else 65.0 / 33.0)
    assert 1.8 < order < 2.2, order


# ---- planted mutants of the lower plate ----

SRC = os.path.join(os.path.dirname(oracle.__file__), "lks_oracle.c")

LOWER_MUTANTS = {
    "link_ladd_lower_sign": ("double uw = (EY9[a] > 0) ? p->u_bot : p->u_top;",
                             "double uw = (EY9[a] > 0) ? -p->u_bot : p->u_top;"),
    "link_g_moving_lower_sign": ("double uw = bottom ? p->u_bot : p->u_top;\n                        double r",
                                 "double uw = bottom ? -p->u_bot : p->u_top;\n                        double r"),
    "moment_g_moving_lower_sign_inf": ("g[0][2] = g[0][4] - B0 * uw;", "g[0][2] = g[0][4] + B0 * uw;"),
    "moment_f_lower_momentum_sign": ("f[5] = 0.5 * (P + rho * uw - hfx) - (f[1] + f[8]);",
                                     "f[5] = 0.5 * (P - rho * uw - hfx) - (f[1] + f[8]);"),
}


def _moment_finite_lower_mutant(text):
    """The finite-c lower-plate g term of the moment closure: '- beta B0 U' -> '+ beta B0 U' in the
    bottom branch only (the first of the two occurrences)."""
    old = "- (g[0][0] + g[0][1] + g[0][3]) -\n"
    assert text.count(old) == 1
    return text.replace(old, "- (g[0][0] + g[0][1] + g[0][3]) +\n")


def _compile(tmp_path, name, text):
    src = tmp_path / ("m_%s.c" % name)
    src.write_text(text)
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_run.argtypes = [ctypes.POINTER(oracle.OracleParams), dp, dp, ctypes.c_int64]
    L.orc_run.restype = ctypes.c_int
    return L


def _mirror_defect(L, closure, c_move, c_rest):
    """Largest departure from the mirror image, relative to each profile's scale (u_x and B_x)."""
    top, bot = _pair(closure, c_move, c_rest, 0.0, 0, lib=L)
    mt, mb = top.moments(), bot.moments()
    du = np.max(np.abs(mb[1] - mt[1][::-1])) / np.max(np.abs(mt[1]))
    db = np.max(np.abs(mb[3] + mt[3][::-1])) / np.max(np.abs(mt[3]))
    return max(du, db)


def _mutants():
    text = open(SRC).read()
    out = {}
    for name, (old, new) in LOWER_MUTANTS.items():
        assert text.count(old) == 1, name
        out[name] = text.replace(old, new)
    out["moment_g_moving_lower_sign_finite"] = _moment_finite_lower_mutant(text)
    return out


def test_unmutated_copy_is_mirror_symmetric(tmp_path):
    L = _compile(tmp_path, "none", open(SRC).read())
    for closure in (oracle.LINK, oracle.MOMENT):
        for c_move in (0.4, math.inf):
            assert _mirror_defect(L, closure, c_move, 0.0) < 1e-12


@pytest.mark.parametrize("name", ["link_ladd_lower_sign", "link_g_moving_lower_sign", "moment_g_moving_lower_sign_inf",
                                  "moment_f_lower_momentum_sign", "moment_g_moving_lower_sign_finite"])
def test_lower_wall_mutant_is_caught(tmp_path, name):
    L = _compile(tmp_path, name, _mutants()[name])
    worst = max(_mirror_defect(L, closure, c_move, 0.0) for closure in (oracle.LINK, oracle.MOMENT)
                for c_move in (0.4, math.inf))
    assert worst > 1e-3, (name, worst)


@pytest.mark.parametrize("name,old,new", [
    ("theta_without_half", "double theta = c * a / (tau_m - 0.5);", "double theta = c * a / tau_m;"),
    ("beta_uses_tau_minus_half", "const double beta_b = p->c_bot * a_half / (p->tau_m * CS2);",
     "const double beta_b = p->c_bot * a_half / ((p->tau_m - 0.5) * CS2);"),
])
def test_robin_pin_catches_wrong_closure_coefficients(tmp_path, name, old, new):
    """theta (link) with tau_m instead of tau_m - 1/2, or beta (moment) with tau_m - 1/2 instead of
    tau_m, changes the effective conductance of the plate and with it the decay rate."""
    text = open(SRC).read()
    assert text.count(old) == 1
    L = _compile(tmp_path, name, text.replace(old, new))
    closure = oracle.LINK if name == "theta_without_half" else oracle.MOMENT
    err = robin_decay_error(closure, 0.3, 0.3, 33, lib=L)
    assert abs(err) > 1e-2, err


@pytest.mark.parametrize("case", ["hartmann", "couette"])
def test_moment_closure_mass_change_saturates(case):
    """The moment-based closure sets rho at a wall node from the known populations (App. A) and so
    need not conserve total mass, unlike the link-based bounce-back.  The change is reported, and it
    is bounded: it settles with the flow (Hartmann 3 x 65, Ha = 5, c = 0.5: -1.45e-6; Couette, top
    plate at 0.05: +1.9e-5) instead of drifting."""
    ny, a = 65, 32.0
    b0 = an.b0_from_ha(5.0, a, 0.8, 0.8)
    if case == "hartmann":
        o = oracle.Oracle(3, ny, 0.8, 0.8, b0, an.force_for_centre_speed(0.01, 5.0, 0.5, a, 0.8), oracle.MOMENT,
                          0.5, 0.5)
    else:
        o = oracle.Oracle(3, ny, 0.8, 0.8, b0, 0.0, oracle.MOMENT, 0.0, 0.5, 0.0, 0.05)
    m0 = o.f.sum()
    o.step(16000)
    d16 = (o.f.sum() - m0) / m0
    o.step(4000)
    d20 = (o.f.sum() - m0) / m0
    assert abs(d20) < 5e-5
    assert abs(d20 - d16) < 1e-2 * abs(d20)

"""The pins are sharp enough: plausible one-token mistakes planted in a copy of the oracle's C
source (compiled on the CPU, never used elsewhere) make the steady-profile pins fail."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from oracle import analytic as an

SRC = os.path.join(os.path.dirname(oracle.__file__), "lks_oracle.c")

MUTANTS = {
    "maxwell_stress_sign": ("return W9[a] * (0.5 * b2 * e2 - eb * eb)", "return W9[a] * (eb * eb - 0.5 * b2 * e2)"),
    "theta_without_half": ("double theta = c * a / (tau_m - 0.5);", "double theta = c * a / tau_m;"),
    "half_force_shift_dropped": ("double ux = (mx + 0.5 * Fx) / rho", "double ux = (mx) / rho"),
    "moving_wall_g_sign": ("s * W5[a] * EY5[a] * B0 * uw / CS2;", "-s * W5[a] * EY5[a] * B0 * uw / CS2;"),
    "beta_uses_tau_minus_half": ("p->c_top * a_half / (p->tau_m * CS2)", "p->c_top * a_half / ((p->tau_m - 0.5) * CS2)"),
    "geq_antisymmetric_sign": ("s += e[j] * (u[j] * b[i] - b[j] * u[i]);", "s += e[j] * (b[j] * u[i] - u[j] * b[i]);"),
    "ladd_term_dropped": ("+ 2.0 * W9[a] * EX9[a] * uw / CS2;", ";"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    src = tmp_path / ("m_%s.c" % name)
    src.write_text(text.replace(old, new))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    return ctypes.CDLL(str(so))


def _errors(L, closure, couette_case):
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_init.argtypes = [ctypes.POINTER(oracle.OracleParams), ctypes.c_uint64, ctypes.c_double, dp, dp]
    L.orc_run.argtypes = [ctypes.POINTER(oracle.OracleParams), dp, dp, ctypes.c_int64]
    L.orc_moments.argtypes = [ctypes.POINTER(oracle.OracleParams), dp, dp, dp]
    ny, ha, c = 33, 5.0, 0.5
    a = ny / 2 if closure == oracle.LINK else (ny - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    if couette_case:
        fx, cl, cu, ut = 0.0, 0.0, 0.5, 0.05
    else:
        fx, cl, cu, ut = an.force_for_centre_speed(0.01, ha, c, a, 0.8), c, c, 0.0
    p = oracle.OracleParams(nx=2, ny=ny, closure=closure, tau_f=0.8, tau_m=0.8, B0=b0, Fx=fx,
                            c_bot=cl, c_top=cu, u_bot=0.0, u_top=ut)
    f = np.zeros((9, ny, 2))
    g = np.zeros((2, 5, ny, 2))
    P = lambda x: x.ctypes.data_as(dp)
    L.orc_init(ctypes.byref(p), 0, 0.0, P(f), P(g))
    L.orc_run(ctypes.byref(p), P(f), P(g), 12000)
    m = np.zeros((5, ny, 2))
    L.orc_moments(ctypes.byref(p), P(f), P(g), P(m))
    u, b = m[1].mean(axis=1), m[3].mean(axis=1)
    j = np.arange(ny)
    y = (-a + j + 0.5) if closure == oracle.LINK else (-a + j)
    if couette_case:
        ua, ba = an.couette_profiles(y, a, ha, cl, cu, ut, 0.8, 0.8)
    else:
        ua, ba = an.hartmann_profiles(y, a, ha, c, fx, 0.8, 0.8)
    if not (np.all(np.isfinite(u)) and np.all(np.isfinite(b))):
        return np.inf
    return max(an.rel_l2(u, ua), an.rel_l2(b, ba))


def test_unmutated_copy_passes(tmp_path):
    text = open(SRC).read()
    src = tmp_path / "m_none.c"
    src.write_text(text)
    so = tmp_path / "m_none.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    for closure in (oracle.LINK, oracle.MOMENT):
        for cc in (False, True):
            assert _errors(L, closure, cc) < 1e-2


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    L = _build_mutant(tmp_path, name)
    worst = max(_errors(L, cl, cc) for cl in (oracle.LINK, oracle.MOMENT) for cc in (False, True))
    assert worst > 2e-2, (name, worst)


# ---- the paper's Lorentz-force coupling (coupling = 1, Sec. IV-V) --------------------------------
# Planted mistakes in the force branch: each must move the steady Hartmann channel away from the
# closed forms (A13/A14) or break its total-pressure balance (rho c_s^2 + B_x^2/2 uniform across
# the channel, since F_y = J_z B_x = -d/dy (B_x^2/2)).
LORENTZ_MUTANTS = {
    # J x B with the wrong sign along the flow: the field drives instead of brakes
    "lorentz_jxb_x_sign": ("Fx = p->Fx - jz * by;", "Fx = p->Fx + jz * by;"),
    # the wall-normal Lorentz force with the wrong sign (u_x and B_x unaffected: only the pressure
    # balance sees it)
    "lorentz_fy_sign": ("Fy = jz * bx;", "Fy = -jz * bx;"),
    # J_z = -(1/(tau_m c_sm^2)) eps Lambda^(1) without its 1/tau_m
    "lorentz_j_without_tau": ("eps_zjk Lambda^(1)_jk */\n                        const double jz = ((lyx - l0yx) - (lxy - l0xy)) / (p->tau_m * CS2);",
                              "eps_zjk Lambda^(1)_jk */\n                        const double jz = ((lyx - l0yx) - (lxy - l0xy)) / CS2;"),
    # the equilibrium Lambda^(0)_yx = u_y B_x - B_y u_x with the wrong sign in the step
    "lorentz_lambda0_sign": ("(Eq. rank2antisymmtensoreq) */\n                        const double l0yx = uy * bx - by * ux,",
                             "(Eq. rank2antisymmtensoreq) */\n                        const double l0yx = by * ux - uy * bx,"),
}


def _lorentz_defect(L, closure):
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_init.argtypes = [ctypes.POINTER(oracle.OracleParams), ctypes.c_uint64, ctypes.c_double, dp, dp]
    L.orc_run.argtypes = [ctypes.POINTER(oracle.OracleParams), dp, dp, ctypes.c_int64]
    L.orc_moments.argtypes = [ctypes.POINTER(oracle.OracleParams), dp, dp, dp]
    ny, ha, c = 33, 5.0, 0.5
    a = ny / 2 if closure == oracle.LINK else (ny - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
    p = oracle.OracleParams(nx=2, ny=ny, closure=closure, coupling=1, tau_f=0.8, tau_m=0.8, B0=b0, Fx=fx,
                            c_bot=c, c_top=c, u_bot=0.0, u_top=0.0)
    f = np.zeros((9, ny, 2))
    g = np.zeros((2, 5, ny, 2))
    P = lambda x: x.ctypes.data_as(dp)
    L.orc_init(ctypes.byref(p), 0, 0.0, P(f), P(g))
    L.orc_run(ctypes.byref(p), P(f), P(g), 20000)
    m = np.zeros((5, ny, 2))
    L.orc_moments(ctypes.byref(p), P(f), P(g), P(m))
    rho, u, b = m[0].mean(axis=1), m[1].mean(axis=1), m[3].mean(axis=1)
    if not (np.all(np.isfinite(u)) and np.all(np.isfinite(b)) and np.all(np.isfinite(rho))):
        return np.inf
    j = np.arange(ny)
    y = (-a + j + 0.5) if closure == oracle.LINK else (-a + j)
    ua, ba = an.hartmann_profiles(y, a, ha, c, fx, 0.8, 0.8)
    total = rho / 3.0 + 0.5 * b ** 2
    spread = (total.max() - total.min()) / (0.5 * np.max(b ** 2))
    return max(an.rel_l2(u, ua), an.rel_l2(b, ba), spread)


def test_unmutated_copy_passes_lorentz(tmp_path):
    text = open(SRC).read()
    src = tmp_path / "m_none.c"
    src.write_text(text)
    so = tmp_path / "m_none.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    for closure in (oracle.LINK, oracle.MOMENT):
        assert _lorentz_defect(L, closure) < 1e-2


@pytest.mark.parametrize("name", sorted(LORENTZ_MUTANTS))
def test_lorentz_mutant_is_caught(tmp_path, name):
    old, new = LORENTZ_MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    src = tmp_path / ("m_%s.c" % name)
    src.write_text(text.replace(old, new))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    worst = max(_lorentz_defect(L, cl) for cl in (oracle.LINK, oracle.MOMENT))
    assert worst > 2e-2, (name, worst)

"""Pins of the three-dimensional oracle (oracle/lks3d_oracle.c: D3Q19 f with the 3D Maxwell stress,
D3Q7 g per component of B, link-based Shercliff walls at the y planes, periodic in x and z).

The paper prints the 2D scheme only; the 3D channel flow between plates is the same 1D problem, so
the closed forms of Sec. VIII / App. C pin the steady state, with the magnetic diffusivity of the
D3Q7 lattice, eta = (tau_m - 1/2)/4.  Further pins: exact mass conservation (which the 3D stress
satisfies only with its trace term), invariance in x and z, the rest state as a fixed point, decay
of a transverse field B_z, and planted one-token mistakes in a copy of the source failing them.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import analytic as an

SRC3 = os.path.join(os.path.dirname(oracle.__file__), "lks3d_oracle.c")


def tau_m_2d(tau_m):
    """tau_m of the D2Q5 closed-form helpers with the same eta as D3Q7 at tau_m."""
    return 0.5 + 0.75 * (tau_m - 0.5)


def hartmann3(ny, ha, c, nx=2, nz=2, tau=0.8, u_c=0.01):
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, tau, tau_m_2d(tau))
    fx = an.force_for_centre_speed(u_c, ha, c, a, tau)
    return oracle.Oracle3D(nx, ny, nz, tau, tau, b0, fx, c, c), a, fx


@pytest.mark.parametrize("ha,c", [(5.0, 0.0), (5.0, 0.5), (10.0, 0.1), (5.0, math.inf)])
def test_hartmann_steady_profiles_3d(ha, c):
    o, a, fx = hartmann3(48, ha, c)
    r = o.run_to_steady(1e-9, 200, 400_000)
    assert r < 1e-9
    u, b = o.profiles()
    ua, ba = an.hartmann_profiles(o.y(), a, ha, c, fx, 0.8, tau_m_2d(0.8))
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3


@pytest.mark.parametrize("ha,cl,cu", [(5.0, 0.0, 0.5), (10.0, 0.1, 1e4)])
def test_couette_steady_profiles_3d(ha, cl, cu):
    ny, tau = 48, 0.8
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, tau, tau_m_2d(tau))
    o = oracle.Oracle3D(2, ny, 2, tau, tau, b0, 0.0, cl, cu, 0.0, 0.05)
    r = o.run_to_steady(1e-9, 200, 400_000)
    assert r < 1e-9
    u, b = o.profiles()
    ua, ba = an.couette_profiles(o.y(), a, ha, cl, cu, 0.05, tau, tau_m_2d(tau))
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3


def test_hartmann_different_walls_3d():
    ny, ha, cl, cu = 48, 5.0, 0.0, 0.5
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, 0.8, tau_m_2d(0.8))
    fx = an.force_for_centre_speed(0.01, ha, 0.25, a, 0.8)
    o = oracle.Oracle3D(2, ny, 2, 0.8, 0.8, b0, fx, cl, cu)
    assert o.run_to_steady(1e-9, 200, 400_000) < 1e-9
    u, b = o.profiles()
    ua, ba = an.hartmann_walls_profiles(o.y(), a, ha, cl, cu, fx, 0.8, tau_m_2d(0.8))
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3


def test_second_order_convergence_3d():
    errs = []
    for ny in (24, 48):
        o, a, fx = hartmann3(ny, 5.0, 0.5, nx=1, nz=1, u_c=0.01 * 24 / ny)
        o.run_to_steady(1e-10, 200, 1_000_000)
        u, b = o.profiles()
        ua, _ = an.hartmann_profiles(o.y(), a, 5.0, 0.5, fx, 0.8, tau_m_2d(0.8))
        errs.append(an.rel_l2(u, ua))
    order = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert 1.7 < order < 2.3, errs


def _perturb(o, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    o.f += amp * rng.uniform(-1, 1, o.f.shape) * np.abs(o.f)
    o.g += amp * 1e-2 * rng.uniform(-1, 1, o.g.shape)


def test_rest_state_is_a_fixed_point():
    o = oracle.Oracle3D(5, 7, 3, 0.8, 0.7, 0.05, 0.0, 0.3, 2.0)
    f0, g0 = o.f.copy(), o.g.copy()
    o.step(20)
    assert np.max(np.abs(o.f - f0)) < 1e-15 and np.max(np.abs(o.g - g0)) < 1e-15


def test_mass_conservation_3d():
    """Every population that meets a wall is reflected and the collision conserves mass, so the
    total mass is constant to roundoff, with moving walls, a body force and a field."""
    o = oracle.Oracle3D(6, 9, 4, 0.8, 0.7, 0.05, 1e-5, 0.3, math.inf, -0.02, 0.04)
    _perturb(o, 1)
    m0 = o.moments()[0].sum()
    o.step(60)
    assert abs(o.moments()[0].sum() - m0) < 1e-12 * m0


def test_x_and_z_invariance():
    o = oracle.Oracle3D(4, 10, 3, 0.8, 0.8, 0.03, 2e-6, 0.5, 0.1, 0.0, 0.05)
    o.step(300)
    m = o.moments()
    for k in range(7):
        assert np.max(np.abs(m[k] - m[k][:1, :, :1])) == 0.0
    assert np.max(np.abs(m[5] - 0.03)) < 1e-15          # B_y = B0 everywhere in a 1D flow
    assert np.max(np.abs(m[6])) == 0.0 and np.max(np.abs(m[3])) == 0.0


def test_transverse_field_decays():
    """A B_z perturbation with insulating walls diffuses away (no source for it)."""
    o = oracle.Oracle3D(2, 16, 2, 0.8, 0.8, 0.0, 0.0, 0.0, 0.0)
    y = o.y() / o.a
    prof = np.cos(0.5 * math.pi * y)
    for a in range(7):
        o.g[2, a] += (0.25 if a == 0 else 0.125) * 1e-3 * prof[None, :, None]
    b0 = np.abs(o.moments()[6]).max()
    o.step(2000)
    b1 = np.abs(o.moments()[6]).max()
    assert b1 < 0.5 * b0


def _by_offset_decay(L, steps=3000):
    """Shift B_y by a uniform delta (adding W_a delta to every g_y population) and return the
    remaining fraction of the shift after `steps` steps: the walls hold the normal component at
    B0 (anti-bounce-back), so the shift diffuses out through them."""
    dp = ctypes.POINTER(ctypes.c_double)
    P = lambda x: x.ctypes.data_as(dp)
    ny, b0, d = 16, 0.02, 1e-3
    p = oracle.Oracle3DParams(nx=1, ny=ny, nz=1, pad=0, tau_f=0.8, tau_m=0.8, B0=b0, Fx=0.0, c_bot=0.5,
                              c_top=0.5, u_bot=0.0, u_top=0.0)
    f = np.zeros((19, 1, ny, 1))
    g = np.zeros((3, 7, 1, ny, 1))
    L.o3_init(ctypes.byref(p), P(f), P(g))
    for a in range(7):
        g[1, a] += (0.25 if a == 0 else 0.125) * d
    L.o3_run(ctypes.byref(p), P(f), P(g), steps)
    m = np.zeros((7, 1, ny, 1))
    L.o3_moments(ctypes.byref(p), P(f), P(g), P(m))
    return float(np.mean(m[5] - b0)) / d


def test_normal_component_held_at_b0():
    assert _by_offset_decay(oracle.lib()) < 0.5


MUTANTS = {
    "stress_trace_dropped": ("(0.5 * B2 * e2 - eB * eB - B2 / 6.0)", "(0.5 * B2 * e2 - eB * eB)"),
    "theta_without_half": ("const double th = c * a / (p->tau_m - 0.5);", "const double th = c * a / p->tau_m;"),
    "d3q7_uses_cs2_of_d2q5": ("return w7(a) * (B[i] + 4.0 * s);", "return w7(a) * (B[i] + 3.0 * s);"),
    "moving_wall_g_sign": ("r * go_out - 2.0 * k * w7(a)", "r * go_out + 2.0 * k * w7(a)"),
    "normal_component_bounce_back": ("gp[i][a] = -go_out + 2.0 * w7(a) * p->B0;", "gp[i][a] = go_out;"),
}


def _load(so):
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(oracle.Oracle3DParams)
    L.o3_init.argtypes = [pp, dp, dp]
    L.o3_run.argtypes = [pp, dp, dp, ctypes.c_int64]
    L.o3_moments.argtypes = [pp, dp, dp, dp]
    return L


def _compile(tmp_path, name, text):
    src = tmp_path / ("m3_%s.c" % name)
    src.write_text(text)
    so = tmp_path / ("m3_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", "-o", str(so), str(src), "-lm"],
                   check=True)
    return _load(so)


def _pins_pass(L):
    """The Couette profile, mass conservation and B_y = B0 pins, run on library L."""
    dp = ctypes.POINTER(ctypes.c_double)
    P = lambda x: x.ctypes.data_as(dp)
    ny, ha, cl, cu = 32, 5.0, 0.0, 0.5
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, 0.8, tau_m_2d(0.8))
    p = oracle.Oracle3DParams(nx=1, ny=ny, nz=1, pad=0, tau_f=0.8, tau_m=0.8, B0=b0, Fx=0.0, c_bot=cl, c_top=cu,
                              u_bot=0.0, u_top=0.05)
    f = np.zeros((19, 1, ny, 1))
    g = np.zeros((3, 7, 1, ny, 1))
    L.o3_init(ctypes.byref(p), P(f), P(g))
    L.o3_run(ctypes.byref(p), P(f), P(g), 20000)
    m = np.zeros((7, 1, ny, 1))
    L.o3_moments(ctypes.byref(p), P(f), P(g), P(m))
    y = -a + np.arange(ny) + 0.5
    ua, ba = an.couette_profiles(y, a, ha, cl, cu, 0.05, 0.8, tau_m_2d(0.8))
    ok_profile = (an.rel_l2(m[1].mean(axis=(0, 2)), ua) < 5e-3 and an.rel_l2(m[4].mean(axis=(0, 2)), ba) < 5e-3)
    ok_by = np.max(np.abs(m[5] - b0)) < 1e-12
    # mass with a field and a body force
    p2 = oracle.Oracle3DParams(nx=3, ny=8, nz=3, pad=0, tau_f=0.8, tau_m=0.7, B0=0.05, Fx=1e-5, c_bot=0.3,
                               c_top=0.3, u_bot=0.0, u_top=0.04)
    f2 = np.zeros((19, 3, 8, 3))
    g2 = np.zeros((3, 7, 3, 8, 3))
    L.o3_init(ctypes.byref(p2), P(f2), P(g2))
    m0 = f2.sum()
    L.o3_run(ctypes.byref(p2), P(f2), P(g2), 50)
    ok_mass = abs(f2.sum() - m0) < 1e-12 * m0
    ok_normal = _by_offset_decay(L) < 0.5
    return ok_profile and ok_by and ok_mass and ok_normal


def test_unmutated_source_passes_the_mutant_pins(tmp_path):
    assert _pins_pass(_compile(tmp_path, "none", open(SRC3).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC3).read()
    assert text.count(old) == 1, name
    assert not _pins_pass(_compile(tmp_path, name, text.replace(old, new)))


def test_steady_channel_total_pressure_is_uniform():
    """Nothing varies along x or z in the steady channel, so d/dy Pi_yy = 0.  With the Maxwell stress
    in the D3Q19 equilibrium (trace part included), Pi_yy = rho c_s^2 + |B|^2/2 - B_y^2 with B_y = B0
    uniform, so rho c_s^2 + B_x^2/2 is the same at every y, exactly on the lattice; the density
    carries the induced field's magnetic pressure."""
    ny = 33
    a = ny / 2
    b0 = an.b0_from_ha(5.0, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, 5.0, 0.5, a, 0.8)
    o = oracle.Oracle3D(1, ny, 1, 0.8, 0.8, b0, fx, c_bot=0.5, c_top=0.5)
    o.run_to_steady(1e-12, 200, 3_000_000)
    m = o.moments()
    rho, bx = m[0][0, :, 0], m[4][0, :, 0]
    mag = 0.5 * np.max(bx ** 2)
    total = rho / 3.0 + 0.5 * bx ** 2
    assert (total.max() - total.min()) < 1e-9 * mag
    assert (rho.max() - rho.min()) / 3.0 > 0.99 * mag

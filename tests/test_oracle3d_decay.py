"""Decay pins of the 3D oracle's wall closures for the components of B that the fully developed duct
leaves near their applied values (B_z near 0, B_y near B0), so that its profiles pin little about
them (oracle/lks3d_oracle.c), and for B_x at all four walls of a duct.

At rest (u = 0) with no applied field (B0 = 0) and B = (0, 0, B_z), every Lambda_ji = u_j B_i - B_j u_i
vanishes, and each D3Q7 distribution of the induction scheme (Sec. IV) advances its component by pure
diffusion, dB_z/dt = eta lap B_z with eta = c_sm^2 (tau_m - 1/2), c_sm^2 = 1/4.  A uniform B_z
therefore decays, after its higher modes have died out, at the rate eta k^2 of the lowest mode that
the walls allow:

- side walls of the duct (the planes z = +-b, b = nz/2; B_z is normal to them): the induced field's
  normal component vanishes at a wall parallel to the applied field (the reading of the side walls
  taken for the duct), a Dirichlet condition, so k = pi/(2b); the Hartmann walls are made perfectly
  conducting (c = inf: bounce-back, a Neumann condition for a tangential component) so that B_z
  stays uniform in y;
- Hartmann walls (the planes y = +-a, a = ny/2, periodic in z; B_z is tangential to them): the
  Shercliff condition of Eq. ShercliffBClocalcoordinate, B + c a dB/dn = 0, so k is the smallest
  positive root of the textbook Robin condition k tan(k a) = 1/(c a).

In a square duct (b = a) a uniform B_y or B_x decays as the lowest separable mode
cos(k_y y) cos(k_z z): B_y is normal to the Hartmann walls (anti-bounce-back to B0 = 0, Dirichlet)
and tangential to the side walls (Robin with the side wall's length c a); B_x is tangential to all
four (Robin).

Planted mistakes in these branches (bounce-back for the normal component, the tangential Robin
ratio for it, the Robin weighting with the wrong sign, no weighting) move the rate by tens of per
cent or more and are caught.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle

TAU = 0.8
ETA = 0.25 * (TAU - 0.5)
W7 = np.array([0.25] + [0.125] * 6)   # D3Q7 weights (Sec. IV)
AMP = 1e-4


def _side_duct(nz):
    o = oracle.Oracle3D(1, 4, nz, TAU, TAU, 0.0, 0.0, c_bot=math.inf, c_top=math.inf, side=True, c_back=1.0,
                        c_front=1.0)
    o.g[2] = AMP * W7[:, None, None, None]     # B_z = AMP at rest: g_a = W_a B_z
    return o


def _hartmann_channel(ny, c):
    o = oracle.Oracle3D(1, ny, 4, TAU, TAU, 0.0, 0.0, c_bot=c, c_top=c)
    o.g[2] = AMP * W7[:, None, None, None]
    return o


def _rate_of(o, comp, t1, t2, run=None):
    """Decay rate of the mean of component comp of B between steps t1 and t2 (B_i = sum_a g_ai of the
    stored state)."""
    run = run or (lambda n: o.step(n))
    run(t1)
    m1 = float(o.g[comp].sum(axis=0).mean())
    run(t2 - t1)
    m2 = float(o.g[comp].sum(axis=0).mean())
    return math.log(m1 / m2) / (t2 - t1)


def _robin_k(a, c):
    x = brentq(lambda x: x * math.tan(x) - 1.0 / c, 1e-9, 0.5 * math.pi - 1e-12)
    return x / a


def test_side_wall_bz_decays_as_dirichlet_at_second_order():
    err = {}
    for nz in (16, 32):
        s = (nz / 16) ** 2
        lam = _rate_of(_side_duct(nz), 2, int(1000 * s), int(3000 * s))
        err[nz] = lam / (ETA * (math.pi / nz) ** 2) - 1.0
    assert abs(err[16]) < 5e-3 and abs(err[32]) < 1.5e-3, err
    assert 3.5 < err[16] / err[32] < 4.5, err     # second order in 1/nz


@pytest.mark.parametrize("c", [0.1, 1.0, 10.0])
def test_hartmann_wall_bz_decays_as_robin(c):
    ny = 16
    lam = _rate_of(_hartmann_channel(ny, c), 2, 1000, 3000)
    exact = ETA * _robin_k(ny / 2, c) ** 2
    assert abs(lam / exact - 1.0) < 2e-3, (lam, exact)


def _square_duct(n, comp, c_side, c_hartmann):
    """A square duct (b = a = n/2) holding a uniform component comp of B at rest, B0 = 0."""
    o = oracle.Oracle3D(1, n, n, TAU, TAU, 0.0, 0.0, c_bot=c_hartmann, c_top=c_hartmann, side=True,
                        c_back=c_side, c_front=c_side)
    o.g[comp] = AMP * W7[:, None, None, None]
    return o


def _duct_exact(n, comp, c):
    """Rate of the lowest separable mode cos(k_y y) cos(k_z z): B_y is normal to the Hartmann walls
    (anti-bounce-back to B0 = 0: Dirichlet, k_y = pi/(2a)) and tangential to the side walls (Robin
    with the side wall's length c a); B_x is tangential to both (Robin, the same c on all four)."""
    a = n / 2
    kz = _robin_k(a, c)
    ky = math.pi / (2 * a) if comp == 1 else _robin_k(a, c)
    return ETA * (ky * ky + kz * kz)


@pytest.mark.parametrize("comp", [0, 1])
@pytest.mark.parametrize("c", [0.2, 1.0])
def test_duct_tangential_components_decay_at_second_order(comp, c):
    err = {}
    for n in (16, 32):
        s = (n / 16) ** 2
        o = _square_duct(n, comp, c, math.inf if comp == 1 else c)
        err[n] = _rate_of(o, comp, int(1000 * s), int(3000 * s)) / _duct_exact(n, comp, c) - 1.0
    assert abs(err[16]) < 3e-3 and abs(err[32]) < 8e-4, err
    assert 3.5 < err[16] / err[32] < 4.5, err


SRC3 = os.path.join(os.path.dirname(oracle.__file__), "lks3d_oracle.c")

MUTANTS = {
    # the normal component at a side wall: bounce-back (Neumann) instead of anti-bounce-back to 0
    "side_bz_bounce_back": ("side", "gp[i][a] = -go_out;", "gp[i][a] = go_out;"),
    # the normal component at a side wall closed like a tangential one (the side wall's Robin ratio)
    "side_bz_robin": ("side", "gp[i][a] = -go_out;", "gp[i][a] = r * go_out;"),
    # B_z at a Hartmann wall: the Robin weighting with the wrong sign
    "hartmann_bz_sign": ("hartmann", "gp[i][a] = r * go_out; /* B_z", "gp[i][a] = -r * go_out; /* B_z"),
    # B_z at a Hartmann wall: plain bounce-back whatever the wall's conductance
    "hartmann_bz_unweighted": ("hartmann", "gp[i][a] = r * go_out; /* B_z", "gp[i][a] = go_out; /* B_z"),
    # B_y at a side wall: the Robin weighting with the wrong sign
    "side_by_sign": ("duct_by", "gp[i][a] = r * go_out + (1.0 - r) * w7(a) * p->B0;",
                     "gp[i][a] = -r * go_out + (1.0 - r) * w7(a) * p->B0;"),
    # B_y at a side wall: plain bounce-back whatever the wall's conductance
    "side_by_unweighted": ("duct_by", "gp[i][a] = r * go_out + (1.0 - r) * w7(a) * p->B0;",
                           "gp[i][a] = go_out + (1.0 - r) * w7(a) * p->B0;"),
}


def _compile(tmp_path, name, text):
    src = tmp_path / ("bz_%s.c" % name)
    src.write_text(text)
    so = tmp_path / ("bz_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", "-o", str(so), str(src),
                    "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.o3_run.argtypes = [ctypes.POINTER(oracle.Oracle3DParams), dp, dp, ctypes.c_int64]
    L.o3_run.restype = ctypes.c_int
    return L


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_closure_mutant_is_caught(tmp_path, name):
    case, old, new = MUTANTS[name]
    text = open(SRC3).read()
    assert text.count(old) == 1, name
    L = _compile(tmp_path, name, text.replace(old, new))
    comp = 2
    if case == "side":
        o, exact = _side_duct(16), ETA * (math.pi / 16) ** 2
    elif case == "hartmann":
        o, exact = _hartmann_channel(16, 1.0), ETA * _robin_k(8.0, 1.0) ** 2
    else:
        comp = 1
        o, exact = _square_duct(16, 1, 1.0, math.inf), _duct_exact(16, 1, 1.0)
    P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def run(n):
        assert L.o3_run(ctypes.byref(o.p), P(o.f), P(o.g), n) == 0

    lam = _rate_of(o, comp, 1000, 3000, run)
    assert abs(lam / exact - 1.0) > 0.1, (name, lam, exact)

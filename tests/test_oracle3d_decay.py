"""Decay pins of the 3D oracle's wall closures for B_z (oracle/lks3d_oracle.c), the component that
the fully developed duct leaves near zero, so that its profiles pin nothing about it.

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

Planted mistakes in either branch (bounce-back for the normal component, the tangential Robin ratio
for it, the Robin weighting with the wrong sign, no weighting) move the rate by tens of per cent or
more and are caught.
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


def _rate(o, t1, t2, run=None):
    """Decay rate of the mean of B_z between steps t1 and t2 (B_z = sum_a g_a of the stored state)."""
    run = run or (lambda n: o.step(n))
    run(t1)
    m1 = float(o.g[2].sum(axis=0).mean())
    run(t2 - t1)
    m2 = float(o.g[2].sum(axis=0).mean())
    return math.log(m1 / m2) / (t2 - t1)


def _robin_k(a, c):
    x = brentq(lambda x: x * math.tan(x) - 1.0 / c, 1e-9, 0.5 * math.pi - 1e-12)
    return x / a


def test_side_wall_bz_decays_as_dirichlet_at_second_order():
    err = {}
    for nz in (16, 32):
        s = (nz / 16) ** 2
        lam = _rate(_side_duct(nz), int(1000 * s), int(3000 * s))
        err[nz] = lam / (ETA * (math.pi / nz) ** 2) - 1.0
    assert abs(err[16]) < 5e-3 and abs(err[32]) < 1.5e-3, err
    assert 3.5 < err[16] / err[32] < 4.5, err     # second order in 1/nz


@pytest.mark.parametrize("c", [0.1, 1.0, 10.0])
def test_hartmann_wall_bz_decays_as_robin(c):
    ny = 16
    lam = _rate(_hartmann_channel(ny, c), 1000, 3000)
    exact = ETA * _robin_k(ny / 2, c) ** 2
    assert abs(lam / exact - 1.0) < 2e-3, (lam, exact)


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
def test_bz_closure_mutant_is_caught(tmp_path, name):
    case, old, new = MUTANTS[name]
    text = open(SRC3).read()
    assert text.count(old) == 1, name
    L = _compile(tmp_path, name, text.replace(old, new))
    if case == "side":
        o, exact = _side_duct(16), ETA * (math.pi / 16) ** 2
    else:
        o, exact = _hartmann_channel(16, 1.0), ETA * _robin_k(8.0, 1.0) ** 2
    P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def run(n):
        assert L.o3_run(ctypes.byref(o.p), P(o.f), P(o.g), n) == 0

    lam = _rate(o, 1000, 3000, run)
    assert abs(lam / exact - 1.0) > 0.1, (name, lam, exact)

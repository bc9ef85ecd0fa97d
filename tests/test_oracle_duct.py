"""Pins of the duct references (oracle/duct.py) and of the oracle's duct (oracle/lks3d_oracle.c with
walls at the z planes): fully developed MHD flow along x in the cross-section |y| <= a (Hartmann
walls, normal to B0) x |z| <= b (side walls, parallel to B0), every wall with the Shercliff thin-wall
condition of Eq. ShercliffBClocalcoordinate and the link-based closure of Eq. linkbasedBCschemefinal.

- The Hunt-type series (insulating side walls) reduces to the textbook series of rectangular-duct
  Poiseuille flow at B0 = 0 (written here as the expansion along the other axis, so it shares nothing
  with the series code), and at the centre of a very wide duct to the Hartmann closed form (Sec. VIII.A).
- The finite-difference solver converges at second order to the series, both with the field along y
  (its Hartmann-wall code) and turned along z (its side-wall code).
- The oracle's duct converges at second order to the finite-difference solution, keeps B_y = B0 and
  B_z = 0 (the fully developed field), is symmetric in y and z, and conserves mass; planted mistakes in
  the side-wall closure are caught.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import analytic as an
from oracle import duct

NU = ETA = 0.1


def test_series_is_textbook_poiseuille_at_zero_field():
    a, b, F = 10.0, 7.0, 1e-5
    y = np.linspace(-a, a, 11)[:, None]
    z = np.linspace(-b, b, 9)[None, :]
    u, B = duct.hunt_series(y, z, a, b, 0.0, NU, ETA, F, 0.5)
    # the same flow expanded in cos modes of y: u = (16 F a^2/(nu pi^3)) sum_k (-1)^k/n^3
    #   [1 - cosh(n pi z/(2a))/cosh(n pi b/(2a))] cos(n pi y/(2a)),  n = 2k + 1
    ref = np.zeros(np.broadcast(y, z).shape)
    for k in range(3000):
        n = 2 * k + 1
        q = n * math.pi / (2 * a)
        ratio = np.exp(q * (np.abs(z) - b)) * (1 + np.exp(-2 * q * np.abs(z))) / (1 + math.exp(-2 * q * b))
        ref = ref + 16 * F * a * a / (NU * math.pi ** 3) * (-1) ** k / n ** 3 * (1 - ratio) * np.cos(q * y)
    np.testing.assert_allclose(u, ref, rtol=0, atol=1e-9 * np.max(np.abs(ref)))
    assert np.max(np.abs(B)) == 0.0


@pytest.mark.parametrize("ha,c", [(5.0, 0.5), (10.0, 0.0), (10.0, math.inf), (20.0, 0.1)])
def test_series_wide_duct_centre_is_hartmann(ha, c):
    a, F = 16.0, 1e-5
    B0 = ha * math.sqrt(NU * ETA) / a
    y = np.linspace(-a, a, 33)
    u, B = duct.hunt_series(y, 0.0 * y, a, 40.0 * a, B0, NU, ETA, F, c, nterms=20000)
    ua, ba = an.hartmann_profiles(y, a, ha, c, F, 3 * NU + 0.5, 3 * ETA + 0.5)
    assert np.max(np.abs(u - ua)) < 1e-8 * np.max(np.abs(ua))
    assert np.max(np.abs(B - ba)) < 1e-8 * np.max(np.abs(ba))


def _fd_vs_series(ha, c, n, field_axis):
    a, b, F = 16.0, 12.0, 1e-5
    B0 = ha * math.sqrt(NU * ETA) / a
    if field_axis == "y":
        y, z, u, B = duct.fd_solve(a, b, B0, NU, ETA, F, c, c, 0.0, 0.0, n, int(n * b / a))
        Y, Z = np.meshgrid(y, z, indexing="ij")
        us, bs = duct.hunt_series(Y, Z, a, b, B0, NU, ETA, F, c, nterms=600)
    else:
        # field along z: the z walls are the Hartmann walls (half-width b), the y walls the side walls;
        # a ratio c relative to a is c a/b relative to b
        y, z, u, B = duct.fd_solve(a, b, B0, NU, ETA, F, 0.0, 0.0, c, c, n, int(n * b / a), field_axis="z")
        Y, Z = np.meshgrid(y, z, indexing="ij")
        us, bs = duct.hunt_series(Z, Y, b, a, B0, NU, ETA, F, c * a / b, nterms=600)
    return np.max(np.abs(u - us)) / np.max(np.abs(us)), np.max(np.abs(B - bs)) / np.max(np.abs(bs))


@pytest.mark.parametrize("field_axis", ["y", "z"])
@pytest.mark.parametrize("ha,c", [(5.0, 0.5), (8.0, math.inf), (5.0, 0.0)])
def test_fd_converges_to_series(field_axis, ha, c):
    e48 = _fd_vs_series(ha, c, 48, field_axis)
    e96 = _fd_vs_series(ha, c, 96, field_axis)
    for k in range(2):
        order = math.log(e48[k] / e96[k], 2)
        assert 1.7 < order < 2.3, (k, e48, e96)
        assert e96[k] < 4e-3


# ---- the oracle's duct ----

TAU = 0.8
NU3, ETA3 = (TAU - 0.5) / 3, (TAU - 0.5) / 4   # D3Q19 and D3Q7 diffusivities


def _duct(n, ha, ch, cs, lib=None, cs_front=None, max_steps=200_000):
    a = n / 2
    B0 = ha * math.sqrt(NU3 * ETA3) / a
    F = 1e-6 * (16 / n) ** 2
    cf = cs if cs_front is None else cs_front
    o = oracle.Oracle3D(1, n, n, TAU, TAU, B0, F, ch, ch, side=True, c_back=cs, c_front=cf)
    if lib is None:
        o.run_to_steady(1e-10, 200, max_steps)
    else:
        P = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        assert lib.o3_run(ctypes.byref(o.p), P(o.f), P(o.g), 6000) == 0
    m = o.moments()
    uf, Bf = duct.fd_on_lattice(n, n, B0, NU3, ETA3, F, ch, ch, cs, cf, refine=4)
    return o, m, uf, Bf


def _err(m, uf, Bf):
    u, B = m[1][:, :, 0].T, m[4][:, :, 0].T     # (ny, nz)
    return (math.sqrt(np.mean((u - uf) ** 2)) / np.max(np.abs(uf)),
            math.sqrt(np.mean((B - Bf) ** 2)) / np.max(np.abs(Bf)))


@pytest.mark.parametrize("ha,ch,cs", [(5.0, 0.5, 0.3), (8.0, math.inf, 1.0), (4.0, 0.0, 0.0)])
def test_duct_steady_profiles_second_order(ha, ch, cs):
    e16 = _err(*_duct(16, ha, ch, cs)[1:])
    e32 = _err(*_duct(32, ha, ch, cs)[1:])
    for k in range(2):
        order = math.log(e16[k] / e32[k], 2)
        assert 1.8 < order < 2.2, (k, e16, e32)
        assert e32[k] < 5e-3


def test_duct_field_symmetry_and_mass():
    """The fully developed field: B_y = B0 and B_z = 0, up to the tiny secondary flow that the magnetic
    pressure grad(B_x^2/2) drives in the compressible lattice (u_y, u_z ~ 1e-6 of u_x here, which
    induces B_y - B0 ~ 1e-9 B0 and B_z of the same size); u even in y and z, B_x odd in y and even in z;
    total mass unchanged, since every cut link is reflected."""
    o, m, _, _ = _duct(16, 5.0, 0.5, 0.3)
    u, u_y, u_z = m[1][:, :, 0], m[2][:, :, 0], m[3][:, :, 0]
    B_x, B_y, B_z = m[4][:, :, 0], m[5][:, :, 0], m[6][:, :, 0]   # (nz, ny)
    su, sb = np.max(np.abs(u)), np.max(np.abs(B_x))
    assert max(np.max(np.abs(u_y)), np.max(np.abs(u_z))) < 1e-5 * su
    np.testing.assert_allclose(B_y, o.p.B0, rtol=1e-7)
    assert np.max(np.abs(B_z)) < 1e-5 * sb
    np.testing.assert_allclose(u, u[::-1, :], rtol=0, atol=1e-10 * su)       # even in z
    np.testing.assert_allclose(u, u[:, ::-1], rtol=0, atol=1e-10 * su)       # even in y
    np.testing.assert_allclose(B_x, B_x[::-1, :], rtol=0, atol=1e-10 * sb)   # even in z
    np.testing.assert_allclose(B_x, -B_x[:, ::-1], rtol=0, atol=1e-10 * sb)  # odd in y
    assert abs(o.f.sum() - o.f.shape[1] * o.f.shape[2] * o.f.shape[3]) < 1e-10  # every cut link reflected


SRC3 = os.path.join(os.path.dirname(oracle.__file__), "lks3d_oracle.c")

DUCT_MUTANTS = {
    # the side wall's ratio taken from the wrong wall
    "side_ratio_swapped": ("const double r = szr < 0 ? rk : rf;", "const double r = szr < 0 ? rf : rk;"),
    # B_x at a side wall closed with the opposite weighting
    "side_bx_sign": ("                                gp[i][a] = r * go_out;\n                            else\n",
                     "                                gp[i][a] = -r * go_out;\n                            else\n"),
    # B_y at a side wall without the applied-field term of its anti-bounce-back half
    "side_by_without_B0": ("gp[i][a] = r * go_out + (1.0 - r) * w7(a) * p->B0;", "gp[i][a] = r * go_out;"),
}


def _compile3(tmp_path, name, text):
    src = tmp_path / ("d_%s.c" % name)
    src.write_text(text)
    so = tmp_path / ("d_%s.so" % name)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11", "-o", str(so), str(src),
                    "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    dp = ctypes.POINTER(ctypes.c_double)
    L.o3_run.argtypes = [ctypes.POINTER(oracle.Oracle3DParams), dp, dp, ctypes.c_int64]
    L.o3_run.restype = ctypes.c_int
    return L


def _defect(L, name):
    """Departure of a 6000-step duct run from the unmutated oracle's, relative to each field."""
    kw = dict(cs=0.2, cs_front=2.0) if name == "side_ratio_swapped" else dict(cs=0.3)
    ref = _duct(16, 5.0, 0.5, lib=_compile3.unmutated, **kw)[1]
    got = _duct(16, 5.0, 0.5, lib=L, **kw)[1]
    du = max(np.max(np.abs(got[k] - ref[k])) / np.max(np.abs(ref[k])) for k in (1, 4))
    dby = np.max(np.abs(got[5] - ref[5])) / ref[5].mean()
    return max(du, 1e3 * dby)   # B_y is B0 to 1e-9 in the unmutated duct


@pytest.mark.parametrize("name", sorted(DUCT_MUTANTS))
def test_duct_mutant_is_caught(tmp_path, name):
    text = open(SRC3).read()
    old, new = DUCT_MUTANTS[name]
    assert text.count(old) == 1, name
    _compile3.unmutated = _compile3(tmp_path, "none", text)
    L = _compile3(tmp_path, name, text.replace(old, new))
    assert _defect(L, name) > 1e-3


@pytest.mark.parametrize("ha,c", [(5.0, 0.5), (8.0, math.inf)])
def test_extrapolated_fd_matches_series(ha, c):
    """The Richardson-extrapolated finite-difference solution on the lattice nodes of a 32^2 duct with
    insulating side walls agrees with the series to well below the scheme's own error there (~1e-3)."""
    n, nu, eta, F = 32, 0.1, 0.075, 1e-6
    a = n / 2
    B0 = ha * math.sqrt(nu * eta) / a
    y = -a + np.arange(n) + 0.5
    us, bs = duct.hunt_series(y[:, None], y[None, :], a, a, B0, nu, eta, F, c, nterms=2000)
    ue, be = duct.fd_on_lattice_extrapolated(n, n, B0, nu, eta, F, c, c, 0.0, 0.0, refine=2)
    assert np.max(np.abs(ue - us)) < 6e-5 * np.max(np.abs(us))
    assert np.max(np.abs(be - bs)) < 6e-5 * np.max(np.abs(bs))

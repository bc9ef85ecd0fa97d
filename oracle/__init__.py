"""FP64 CPU oracle of the LKS-MHD step with Shercliff wall closures.

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU-baseline
leg are the only users.  The product library never imports this package, and this
package imports nothing from the product library.

`lks_oracle.c` holds the scheme (see its header for the paper passages it follows),
`lks3d_oracle.c` the three-dimensional channel (D3Q19 + D3Q7, link-based walls);
`analytic.py` holds the closed-form profiles.  `build()` compiles the C file with
gcc (no fast-math, no FP contraction) into `_build/liboracle.so` beside this file.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lks_oracle.c")
_SRC3 = os.path.join(_HERE, "lks3d_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

LINK = 0
MOMENT = 1


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("closure", ctypes.c_int32),
        ("pi20_literal", ctypes.c_int32),
        ("freeze_u", ctypes.c_int32),
        ("coupling", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("B0", ctypes.c_double),
        ("Fx", ctypes.c_double),
        ("c_bot", ctypes.c_double),
        ("c_top", ctypes.c_double),
        ("u_bot", ctypes.c_double),
        ("u_top", ctypes.c_double),
    ]


class Oracle3DParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("B0", ctypes.c_double),
        ("Fx", ctypes.c_double),
        ("c_bot", ctypes.c_double),
        ("c_top", ctypes.c_double),
        ("u_bot", ctypes.c_double),
        ("u_top", ctypes.c_double),
        ("side", ctypes.c_int32),
        ("pad2", ctypes.c_int32),
        ("c_back", ctypes.c_double),
        ("c_front", ctypes.c_double),
    ]


def build(force=False):
    """Compile the oracle shared library (gcc -O2 -ffp-contract=off -fopenmp)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and all(
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src) for src in (_SRC, _SRC3)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-std=c11", "-o", tmp, _SRC, _SRC3, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(OracleParams)
        L.orc_init.argtypes = [pp, ctypes.c_uint64, ctypes.c_double, dp, dp]
        L.orc_init.restype = ctypes.c_int
        L.orc_step.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_run.argtypes = [pp, dp, dp, ctypes.c_int64]
        L.orc_run.restype = ctypes.c_int
        L.orc_moments.argtypes = [pp, dp, dp, dp]
        L.orc_moments.restype = None
        L.orc_half_width.argtypes = [pp]
        L.orc_half_width.restype = ctypes.c_double
        L.orc_threads.argtypes = []
        L.orc_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        p3 = ctypes.POINTER(Oracle3DParams)
        L.o3_init.argtypes = [p3, dp, dp]
        L.o3_init.restype = ctypes.c_int
        L.o3_step.argtypes = [p3, dp, dp, dp, dp]
        L.o3_step.restype = ctypes.c_int
        L.o3_run.argtypes = [p3, dp, dp, ctypes.c_int64]
        L.o3_run.restype = ctypes.c_int
        L.o3_moments.argtypes = [p3, dp, dp, dp]
        L.o3_moments.restype = None
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One channel lattice advanced by the FP64 reference scheme.

    State arrays: f (9, ny, nx) and g (2, 5, ny, nx), post-collision populations.
    """

    def __init__(self, nx, ny, tau_f, tau_m, B0, Fx=0.0, closure=LINK, c_bot=0.0, c_top=0.0,
                 u_bot=0.0, u_top=0.0, pi20_literal=False, freeze_u=False, seed=0, perturb_amp=0.0, coupling=0):
        self.p = OracleParams(nx=nx, ny=ny, closure=closure, pi20_literal=int(pi20_literal),
                              freeze_u=int(freeze_u), coupling=int(coupling), tau_f=tau_f, tau_m=tau_m, B0=B0, Fx=Fx,
                              c_bot=c_bot, c_top=c_top, u_bot=u_bot, u_top=u_top)
        self.nx, self.ny = nx, ny
        self.f = np.zeros((9, ny, nx))
        self.g = np.zeros((2, 5, ny, nx))
        rc = lib().orc_init(ctypes.byref(self.p), ctypes.c_uint64(seed), perturb_amp, _ptr(self.f), _ptr(self.g))
        if rc != 0:
            raise ValueError("oracle init rejected the parameters")
        self.steps = 0

    @property
    def a(self):
        return lib().orc_half_width(ctypes.byref(self.p))

    def y(self):
        """Wall-normal node coordinates y_j (link: -a + j + 1/2; moment: -a + j)."""
        j = np.arange(self.ny, dtype=np.float64)
        if self.p.closure == LINK:
            return -self.a + j + 0.5
        return -self.a + j

    def set_walls(self, c_bot, c_top, u_bot=0.0, u_top=0.0):
        self.p.c_bot, self.p.c_top, self.p.u_bot, self.p.u_top = c_bot, c_top, u_bot, u_top

    def step(self, n=1):
        rc = lib().orc_run(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g), int(n))
        if rc != 0:
            raise RuntimeError("oracle step failed (%d)" % rc)
        self.steps += n

    def step_detail(self):
        """One step returning (f_pre, g_pre, mom): post-closure pre-collision populations
        and the moments that entered the collision."""
        fo = np.empty_like(self.f)
        go = np.empty_like(self.g)
        fpre = np.empty_like(self.f)
        gpre = np.empty_like(self.g)
        mom = np.empty((5, self.ny, self.nx))
        rc = lib().orc_step(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g), _ptr(fo), _ptr(go),
                            _ptr(fpre), _ptr(gpre), _ptr(mom))
        if rc != 0:
            raise RuntimeError("oracle step failed (%d)" % rc)
        self.f, self.g = fo, go
        self.steps += 1
        return fpre, gpre, mom

    def moments(self):
        """(5, ny, nx): rho, u_x, u_y, B_x, B_y of the stored state."""
        mom = np.empty((5, self.ny, self.nx))
        lib().orc_moments(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g), _ptr(mom))
        return mom

    def profiles(self):
        """x-averaged u_x(y), B_x(y)."""
        m = self.moments()
        return m[1].mean(axis=1), m[3].mean(axis=1)

    def run_to_steady(self, tol=1e-10, check_every=100, max_steps=10_000_000):
        """Step until max(|du_x|_2/|u_x|_2, |dB_x|_2/|B_x|_2) over check_every steps < tol."""
        prev = self.moments()
        while self.steps < max_steps:
            self.step(check_every)
            cur = self.moments()
            r = residual(prev, cur)
            prev = cur
            if r < tol:
                return r
        return r


def residual(prev, cur):
    """Steady-state residual between two moment snapshots (u_x and B_x, relative L2)."""
    out = 0.0
    for m in (1, 3):
        num = float(np.sqrt(np.sum((cur[m] - prev[m]) ** 2)))
        den = float(np.sqrt(np.sum(cur[m] ** 2)))
        if den > 1e-30:
            out = max(out, num / den)
    return out


def set_threads(n):
    lib().orc_set_threads(int(n))


def threads_used():
    return lib().orc_threads()


class Oracle3D:
    """Three-dimensional channel (D3Q19 f + D3Q7 g per component of B, link-based walls at the
    y planes, periodic in x and z) advanced by the FP64 reference scheme of lks3d_oracle.c.

    State arrays: f (19, nz, ny, nx) and g (3, 7, nz, ny, nx), post-collision populations; they
    may be set directly (e.g. to a perturbed state) before stepping.
    """

    def __init__(self, nx, ny, nz, tau_f, tau_m, B0, Fx=0.0, c_bot=0.0, c_top=0.0, u_bot=0.0, u_top=0.0,
                 side=False, c_back=0.0, c_front=0.0):
        """side=True closes the channel into a duct: walls at the z planes (half-way outside planes 0
        and nz-1) with conductance ratios c_back (z = -b) and c_front (z = +b), relative to a."""
        self.p = Oracle3DParams(nx=nx, ny=ny, nz=nz, pad=0, tau_f=tau_f, tau_m=tau_m, B0=B0, Fx=Fx, c_bot=c_bot,
                                c_top=c_top, u_bot=u_bot, u_top=u_top, side=int(bool(side)), pad2=0,
                                c_back=c_back, c_front=c_front)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.f = np.zeros((19, nz, ny, nx))
        self.g = np.zeros((3, 7, nz, ny, nx))
        if lib().o3_init(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g)) != 0:
            raise ValueError("oracle init rejected the parameters")
        self.steps = 0

    @property
    def a(self):
        return 0.5 * self.ny

    def y(self):
        """Wall-normal node coordinates y_j = -a + j + 1/2."""
        return -self.a + np.arange(self.ny, dtype=np.float64) + 0.5

    def z(self):
        """Side-wall-normal node coordinates z_k = -b + k + 1/2, b = nz/2 (duct)."""
        return -0.5 * self.nz + np.arange(self.nz, dtype=np.float64) + 0.5

    def step(self, n=1):
        if lib().o3_run(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g), int(n)) != 0:
            raise RuntimeError("oracle step failed")
        self.steps += n

    def moments(self):
        """(7, nz, ny, nx): rho, u_x, u_y, u_z, B_x, B_y, B_z of the stored state."""
        mom = np.empty((7, self.nz, self.ny, self.nx))
        lib().o3_moments(ctypes.byref(self.p), _ptr(self.f), _ptr(self.g), _ptr(mom))
        return mom

    def profiles(self):
        """u_x(y), B_x(y) averaged over x and z."""
        m = self.moments()
        return m[1].mean(axis=(0, 2)), m[4].mean(axis=(0, 2))

    def run_to_steady(self, tol=1e-10, check_every=100, max_steps=10_000_000):
        """Step until the relative change of u_x and B_x over check_every steps is below tol."""
        prev = self.moments()
        r = float("inf")
        while self.steps < max_steps:
            self.step(check_every)
            cur = self.moments()
            r = 0.0
            for m in (1, 4):
                den = float(np.sqrt(np.sum(cur[m] ** 2)))
                if den > 1e-30:
                    r = max(r, float(np.sqrt(np.sum((cur[m] - prev[m]) ** 2))) / den)
            prev = cur
            if r < tol:
                return r
        return r

"""Thin ctypes binding of include/lks3d.h (argument marshalling only): the three-dimensional
channel, D3Q19 f + D3Q7 g per component of B with the link-based Shercliff walls at the y planes,
periodic in x and z.  PyTorch supplies device memory and the stream; every step runs in the
library's kernels."""
import ctypes

import numpy as np

from . import lks as _lks


class Lks3Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("B0", ctypes.c_double),
        ("Fx", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_buffer", ctypes.c_void_p),
        ("dev_buffer_bytes", ctypes.c_size_t),
    ]


_VP = ctypes.c_void_p
_PP = ctypes.POINTER(Lks3Params)
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_status = ctypes.c_int

# Every entry point declared in include/lks3d.h, with (restype, argtypes).
SIGNATURES = {
    "lks3_footprint_bytes": (ctypes.c_size_t, [_PP]),
    "lks3_create": (_status, [_PP, ctypes.POINTER(_VP)]),
    "lks3_set_walls": (_status, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "lks3_set_side_walls": (_status, [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double]),
    "lks3_step": (_status, [_VP, ctypes.c_int64]),
    "lks3_steps_taken": (ctypes.c_int64, [_VP]),
    "lks3_moments": (_status, [_VP, ctypes.c_int, _dp]),
    "lks3_residual": (_status, [_VP, _dp, _dp]),
    "lks3_run_to_steady": (_status, [_VP, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _i64p, _dp]),
    "lks3_get_state": (_status, [_VP, _dp, _dp]),
    "lks3_set_state": (_status, [_VP, _dp, _dp]),
    "lks3_sync": (_status, [_VP]),
    "lks3_selftest_wait_timeout": (_status, [_VP, ctypes.c_double]),
    "lks3_destroy": (_status, [_VP]),
    "lks3_last_error": (ctypes.c_char_p, [_VP]),
}

_bound = None


def lib():
    global _bound
    L = _lks.load()
    if _bound is not L:
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _bound = L
    return L


def _check(status, handle=None):
    if status != _lks.LKS_OK:
        msg = lib().lks3_last_error(handle)
        raise _lks.LksError(status, msg.decode() if msg else "")


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def make_params(nx, ny, nz, tau_f, tau_m, B0, Fx=0.0, storage="f64", stream=0, dev_buffer=0, dev_buffer_bytes=0):
    st = _lks.STORAGES[storage]
    return Lks3Params(nx=nx, ny=ny, nz=nz, storage=st, tau_f=tau_f, tau_m=tau_m, B0=B0, Fx=Fx,
                      cuda_stream=stream or None, dev_buffer=dev_buffer or None, dev_buffer_bytes=dev_buffer_bytes)


def footprint_bytes(nx, ny, nz, storage="f64", tau_f=0.8, tau_m=0.8):
    p = make_params(nx, ny, nz, tau_f, tau_m, 0.0, storage=storage)
    return int(lib().lks3_footprint_bytes(ctypes.byref(p)))


class Lattice3D:
    """One three-dimensional channel resident on the GPU (a wrapped lks3_handle)."""

    def __init__(self, nx, ny, nz, tau_f, tau_m, B0, Fx=0.0, storage="f64", stream=None, torch_memory=True):
        import torch
        L = lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        p = make_params(nx, ny, nz, tau_f, tau_m, B0, Fx, storage, stream.cuda_stream)
        self.nbytes = int(L.lks3_footprint_bytes(ctypes.byref(p)))
        if self.nbytes == 0:
            raise _lks.LksError(_lks.LKS_EINVAL, "invalid lattice parameters")
        self._buf = None
        if torch_memory:
            self._buf = torch.empty(self.nbytes, dtype=torch.uint8, device=stream.device)
            p.dev_buffer = self._buf.data_ptr()
            p.dev_buffer_bytes = self.nbytes
        h = ctypes.c_void_p()
        _check(L.lks3_create(ctypes.byref(p), ctypes.byref(h)))
        self._h = h

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    @property
    def a(self):
        return 0.5 * self.ny

    def y(self):
        """Wall-normal node coordinates y_j = -a + j + 1/2."""
        return -self.a + np.arange(self.ny, dtype=np.float64) + 0.5

    def set_walls(self, c_bottom, c_top, u_bottom=0.0, u_top=0.0):
        _check(lib().lks3_set_walls(self._h, c_bottom, c_top, u_bottom, u_top), self._h)

    def set_side_walls(self, c_back, c_front, enable=True):
        """Close the channel into a duct: walls at the z planes with conductance ratios c_back
        (z = -b) and c_front (z = +b), relative to the Hartmann half-width a."""
        _check(lib().lks3_set_side_walls(self._h, int(bool(enable)), c_back, c_front), self._h)

    def z(self):
        """Side-wall-normal node coordinates z_k = -b + k + 1/2, b = nz/2 (duct)."""
        return -0.5 * self.nz + np.arange(self.nz, dtype=np.float64) + 0.5

    def step(self, n=1):
        _check(lib().lks3_step(self._h, int(n)), self._h)

    @property
    def steps(self):
        return int(lib().lks3_steps_taken(self._h))

    def moments(self):
        """(7, nz, ny, nx): rho, u_x, u_y, u_z, B_x, B_y, B_z."""
        out = np.empty((7, self.nz, self.ny, self.nx))
        _check(lib().lks3_moments(self._h, _lks.MOMENTS_NODES, _ptr(out)), self._h)
        return out

    def profiles(self):
        """u_x(y), B_x(y) averaged over x and z."""
        out = np.empty((7, self.ny))
        _check(lib().lks3_moments(self._h, _lks.MOMENTS_PROFILES, _ptr(out)), self._h)
        return out[1].copy(), out[4].copy()

    def residual(self):
        ru, rb = ctypes.c_double(), ctypes.c_double()
        _check(lib().lks3_residual(self._h, ctypes.byref(ru), ctypes.byref(rb)), self._h)
        return ru.value, rb.value

    def run_to_steady(self, tol, check_every=100, max_steps=10_000_000, raise_on_fail=True):
        steps, r = ctypes.c_int64(), ctypes.c_double()
        st = lib().lks3_run_to_steady(self._h, tol, int(check_every), int(max_steps), ctypes.byref(steps),
                                      ctypes.byref(r))
        if raise_on_fail:
            _check(st, self._h)
        return steps.value, r.value, st

    def get_state(self):
        f = np.empty((19, self.nz, self.ny, self.nx))
        g = np.empty((3, 7, self.nz, self.ny, self.nx))
        _check(lib().lks3_get_state(self._h, _ptr(f), _ptr(g)), self._h)
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (19, self.nz, self.ny, self.nx) and g.shape == (3, 7, self.nz, self.ny, self.nx)
        _check(lib().lks3_set_state(self._h, _ptr(f), _ptr(g)), self._h)

    def sync(self):
        _check(lib().lks3_sync(self._h), self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lks3_destroy(self._h)
            self._h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

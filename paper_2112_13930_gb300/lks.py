"""Thin ctypes binding of the C ABI in include/lks.h (argument marshalling only).

Every step of the method runs in the CUDA library liblks.so; this module only converts
arguments.  Device memory comes from PyTorch (a uint8 tensor handed to the library as
lks_params.dev_buffer) and work is enqueued on PyTorch's current CUDA stream unless a stream
is given.  Importing works without a GPU; creating a Lattice needs one and the built library.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblks.so")

(LKS_OK, LKS_EINVAL, LKS_ENOMEM, LKS_ECUDA, LKS_EUNSTABLE, LKS_ETIMEOUT, LKS_ENOTCONVERGED, LKS_EBUSY,
 LKS_ESTALLED) = range(9)
LINK, MOMENT = 0, 1
F64, F32, BF16_DEV, F16_DEV = 0, 1, 2, 3
MOMENTS_NODES, MOMENTS_PROFILES = 0, 1

CLOSURES = {"link": LINK, "moment": MOMENT, LINK: LINK, MOMENT: MOMENT}
MAXWELL, LORENTZ = 0, 1
COUPLINGS = {"maxwell": MAXWELL, "lorentz": LORENTZ, MAXWELL: MAXWELL, LORENTZ: LORENTZ}
STORAGES = {"f64": F64, "f32": F32, "bf16": BF16_DEV, "f16": F16_DEV,
            F64: F64, F32: F32, BF16_DEV: BF16_DEV, F16_DEV: F16_DEV}
STORAGE_BYTES = {F64: 8, F32: 4, BF16_DEV: 2, F16_DEV: 2}
# FP16 deviation storage holds each deviation times this power of two (include/lks.h, lks_storage)
F16_SCALE = 2.0 ** 14

# Every entry point declared in include/lks.h, with (restype, argtypes).
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


class LksParams(ctypes.Structure):
    """Mirror of struct lks_params."""
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("closure", ctypes.c_int32),
        ("storage", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("B0", ctypes.c_double),
        ("Fx", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("perturb_amp", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_buffer", ctypes.c_void_p),
        ("dev_buffer_bytes", ctypes.c_size_t),
        ("coupling", ctypes.c_int32),
        ("inplace", ctypes.c_int32),
    ]


_PP = ctypes.POINTER(LksParams)
SIGNATURES = {
    "lks_footprint_bytes": (ctypes.c_size_t, [_PP]),
    "lks_create": (ctypes.c_int, [_PP, ctypes.POINTER(ctypes.c_void_p)]),
    "lks_set_walls": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double]),
    "lks_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "lks_steps_taken": (ctypes.c_int64, [ctypes.c_void_p]),
    "lks_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp]),
    "lks_moments_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "lks_residual": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "lks_run_to_steady": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, _i64p,
                                         _dp]),
    "lks_get_state": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "lks_set_state": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "lks_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "lks_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "lks_get_state_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lks_set_state_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "lks_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "lks_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lks_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lks_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lks_residual_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                            ctypes.c_double, ctypes.c_void_p, _dp, ctypes.c_void_p]),
}

_lib = None


class LksError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_status_name(status), message))
        self.status = status


def _status_name(s):
    names = ["LKS_OK", "LKS_EINVAL", "LKS_ENOMEM", "LKS_ECUDA", "LKS_EUNSTABLE", "LKS_ETIMEOUT",
             "LKS_ENOTCONVERGED", "LKS_EBUSY", "LKS_ESTALLED"]
    return names[s] if 0 <= s < len(names) else "LKS_%d" % s


def load(path=None):
    """Load liblks.so.  Raises if it has not been built: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("liblks.so not found at %s: build it with paper_2112_13930_gb300.build.build()" % path)
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status, handle=None):
    if status != LKS_OK:
        msg = load().lks_last_error(handle)
        raise LksError(status, msg.decode() if msg else "")


def _dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def make_params(nx, ny, tau_f, tau_m, B0, Fx=0.0, closure="link", storage="f64", seed=0, perturb_amp=0.0,
                stream=0, dev_buffer=0, dev_buffer_bytes=0, coupling="maxwell", inplace=False):
    return LksParams(nx=nx, ny=ny, closure=CLOSURES[closure], storage=STORAGES[storage], tau_f=tau_f, tau_m=tau_m,
                     B0=B0, Fx=Fx, seed=seed, perturb_amp=perturb_amp, cuda_stream=stream or None,
                     dev_buffer=dev_buffer or None, dev_buffer_bytes=dev_buffer_bytes, coupling=COUPLINGS[coupling],
                     inplace=int(bool(inplace)))


def footprint_bytes(nx, ny, closure="link", storage="f64", tau_f=0.8, tau_m=0.8, inplace=False):
    p = make_params(nx, ny, tau_f, tau_m, 0.0, closure=closure, storage=storage, inplace=inplace)
    return int(load().lks_footprint_bytes(ctypes.byref(p)))


class Lattice:
    """One channel lattice resident on the GPU (a wrapped lks_handle)."""

    def __init__(self, nx, ny, tau_f, tau_m, B0, Fx=0.0, closure="link", storage="f64", seed=0, perturb_amp=0.0,
                 stream=None, torch_memory=True, coupling="maxwell", inplace=False):
        """inplace=True: one population buffer updated in place, steps in pairs (even counts)."""
        import torch
        L = load()
        self.nx, self.ny = int(nx), int(ny)
        self.closure = CLOSURES[closure]
        self.storage = STORAGES[storage]
        self.Fx = Fx
        self.B0 = B0
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        p = make_params(nx, ny, tau_f, tau_m, B0, Fx, closure, storage, seed, perturb_amp, stream.cuda_stream,
                        coupling=coupling, inplace=inplace)
        self.inplace = bool(inplace)
        self.nbytes = int(L.lks_footprint_bytes(ctypes.byref(p)))
        if self.nbytes == 0:
            raise LksError(LKS_EINVAL, "invalid lattice parameters")
        self._buf = None
        if torch_memory:
            self._buf = torch.empty(self.nbytes, dtype=torch.uint8, device=stream.device)
            p.dev_buffer = self._buf.data_ptr()
            p.dev_buffer_bytes = self.nbytes
        h = ctypes.c_void_p()
        status = L.lks_create(ctypes.byref(p), ctypes.byref(h))
        if status != LKS_OK:
            msg = L.lks_last_error(None)
            raise LksError(status, msg.decode() if msg else "")
        self._h = h
        self.params = p

    @property
    def a(self):
        """Channel half-width: ny/2 (link-based walls half-way outside the rows) or (ny-1)/2."""
        return self.ny / 2 if self.closure == LINK else (self.ny - 1) / 2

    def y(self):
        j = np.arange(self.ny, dtype=np.float64)
        return (-self.a + j + 0.5) if self.closure == LINK else (-self.a + j)

    def set_walls(self, c_bottom, c_top, u_bottom=0.0, u_top=0.0):
        _check(load().lks_set_walls(self._h, c_bottom, c_top, u_bottom, u_top), self._h)

    def step(self, n=1):
        _check(load().lks_step(self._h, int(n)), self._h)

    @property
    def steps(self):
        return int(load().lks_steps_taken(self._h))

    def moments(self, what=MOMENTS_NODES):
        shape = (5, self.ny, self.nx) if what == MOMENTS_NODES else (5, self.ny)
        out = np.empty(shape, dtype=np.float64)
        _check(load().lks_moments(self._h, what, _dptr(out)), self._h)
        return out

    def moments_device(self, out, what=MOMENTS_NODES):
        """Write the moments into a caller-allocated float64 CUDA tensor (asynchronous)."""
        _check(load().lks_moments_device(self._h, what, ctypes.c_void_p(out.data_ptr())), self._h)
        return out

    def profiles(self):
        """x-averaged u_x(y), B_x(y)."""
        m = self.moments(MOMENTS_PROFILES)
        return m[1], m[3]

    def residual(self):
        ru, rb = ctypes.c_double(), ctypes.c_double()
        _check(load().lks_residual(self._h, ctypes.byref(ru), ctypes.byref(rb)), self._h)
        return ru.value, rb.value

    def run_to_steady(self, tol, check_every=100, max_steps=10_000_000, raise_on_fail=True):
        steps, r = ctypes.c_int64(), ctypes.c_double()
        st = load().lks_run_to_steady(self._h, tol, int(check_every), int(max_steps), ctypes.byref(steps),
                                      ctypes.byref(r))
        if raise_on_fail:
            _check(st, self._h)
        return steps.value, r.value, st

    def get_state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((2, 5, self.ny, self.nx))
        _check(load().lks_get_state(self._h, _dptr(f), _dptr(g)), self._h)
        return f, g

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, self.ny, self.nx) and g.shape == (2, 5, self.ny, self.nx)
        _check(load().lks_set_state(self._h, _dptr(f), _dptr(g)), self._h)

    def state_bytes(self):
        return int(load().lks_state_bytes(self._h))

    def get_state_raw(self, out=None):
        """The state in the library's storage image (uint8, lks_state_bytes long): a bit-exact
        checkpoint.  out: optional uint8 numpy array or (pinned) CPU torch tensor to write into."""
        n = self.state_bytes()
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        ptr = out.ctypes.data if isinstance(out, np.ndarray) else out.data_ptr()
        _check(load().lks_get_state_raw(self._h, ctypes.c_void_p(ptr), n), self._h)
        return out

    def set_state_raw(self, image):
        """Replace the state by a storage image from get_state_raw (numpy uint8 or CPU torch tensor)."""
        ptr = image.ctypes.data if isinstance(image, np.ndarray) else image.data_ptr()
        n = image.nbytes if isinstance(image, np.ndarray) else image.numel() * image.element_size()
        _check(load().lks_set_state_raw(self._h, ctypes.c_void_p(ptr), n), self._h)

    def save(self, path, **meta):
        """Checkpoint: the state (FP64 absolute populations via lks_get_state) and the step count."""
        f, g = self.get_state()
        np.savez(path, f=f, g=g, steps=self.steps, nx=self.nx, ny=self.ny, **meta)

    def load(self, path):
        """Resume from a checkpoint written by save() for a lattice of the same shape."""
        d = np.load(path)
        if int(d["nx"]) != self.nx or int(d["ny"]) != self.ny:
            raise ValueError("checkpoint shape %dx%d does not match %dx%d" % (d["nx"], d["ny"], self.nx, self.ny))
        self.set_state(d["f"], d["g"])
        return int(d["steps"])

    def sync(self):
        _check(load().lks_sync(self._h), self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lks_destroy(self._h)
            self._h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

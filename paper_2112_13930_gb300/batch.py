"""Thin ctypes binding of include/lks_batch.h (argument marshalling only): many independent
channel instances advanced by one persistent kernel launch per run() call."""
import ctypes
import json
import math
import os

import numpy as np

from . import lks as _lks

INST_FREE, INST_RUNNING, INST_CONVERGED, INST_MAX_STEPS, INST_UNSTABLE, INST_STALLED = -1, 0, 1, 2, 3, 4
STATE_NAMES = {INST_FREE: "free", INST_RUNNING: "running", INST_CONVERGED: "converged",
               INST_MAX_STEPS: "max_steps", INST_UNSTABLE: "unstable", INST_STALLED: "stalled"}


class BatchConfig(ctypes.Structure):
    _fields_ = [
        ("storage", ctypes.c_int32),
        ("max_instances", ctypes.c_int32),
        ("pool_bytes", ctypes.c_size_t),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_buffer", ctypes.c_void_p),
        ("dev_buffer_bytes", ctypes.c_size_t),
        ("threads_per_group", ctypes.c_int32),
        ("groups_per_cta", ctypes.c_int32),
        ("cluster_ctas", ctypes.c_int32),
        ("coupling", ctypes.c_int32),
        ("inplace", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class InstanceDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32),
        ("closure", ctypes.c_int32),
        ("coupling", ctypes.c_int32),
        ("tau_f", ctypes.c_double),
        ("tau_m", ctypes.c_double),
        ("B0", ctypes.c_double),
        ("Fx", ctypes.c_double),
        ("c_bottom", ctypes.c_double),
        ("c_top", ctypes.c_double),
        ("u_bottom", ctypes.c_double),
        ("u_top", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("perturb_amp", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("check_every", ctypes.c_int64),
        ("max_steps", ctypes.c_int64),
    ]


class InstanceResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("pad", ctypes.c_int32), ("steps", ctypes.c_int64),
                ("residual", ctypes.c_double)]


_VP = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_DP = ctypes.POINTER(ctypes.c_double)
_SZP = ctypes.POINTER(ctypes.c_size_t)
SIGNATURES = {
    "lks_instance_footprint_bytes": (ctypes.c_size_t, [ctypes.POINTER(InstanceDesc), ctypes.c_int32,
                                                       ctypes.c_int32]),
    "lks_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchConfig), ctypes.POINTER(_VP)]),
    "lks_batch_add": (ctypes.c_int, [_VP, ctypes.POINTER(InstanceDesc), _I32P]),
    "lks_batch_run": (ctypes.c_int, [_VP, ctypes.c_int64, _I32P]),
    "lks_batch_result": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(InstanceResult)]),
    "lks_batch_moments": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int, _DP]),
    "lks_batch_get_state": (ctypes.c_int, [_VP, ctypes.c_int32, _DP, _DP]),
    "lks_batch_set_state": (ctypes.c_int, [_VP, ctypes.c_int32, _DP, _DP]),
    "lks_batch_remove": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "lks_batch_set_shape": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "lks_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int64, _I32P, _I32P, _I32P, ctypes.c_int32, _DP, _I32P]),
    "lks_batch_memory": (ctypes.c_int, [_VP, _SZP, _SZP]),
    "lks_batch_destroy": (ctypes.c_int, [_VP]),
    "lks_batch_last_error": (ctypes.c_char_p, [_VP]),
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


def make_desc(nx, ny, closure, tau_f, tau_m, B0, Fx=0.0, c_bottom=0.0, c_top=0.0, u_bottom=0.0, u_top=0.0, seed=0,
              perturb_amp=0.0, tol=1e-10, check_every=100, max_steps=10_000_000, coupling="maxwell"):
    return InstanceDesc(nx=nx, ny=ny, closure=_lks.CLOSURES[closure], coupling=_lks.COUPLINGS[coupling], tau_f=tau_f,
                        tau_m=tau_m, B0=B0, Fx=Fx,
                        c_bottom=c_bottom, c_top=c_top, u_bottom=u_bottom, u_top=u_top, seed=seed,
                        perturb_amp=perturb_amp, tol=tol, check_every=check_every, max_steps=max_steps)


def instance_footprint(desc, storage, inplace=False):
    return int(lib().lks_instance_footprint_bytes(ctypes.byref(desc), _lks.STORAGES[storage], int(bool(inplace))))


class Batch:
    """A pool of resident channel instances (wrapped lks_batch)."""

    def __init__(self, storage="f32", max_instances=4096, pool_bytes=1 << 30, threads_per_group=0,
                 groups_per_cta=0, cluster_ctas=0, stream=None, torch_memory=True, coupling="maxwell",
                 inplace=False):
        import torch
        L = lib()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.storage = _lks.STORAGES[storage]
        self._pool = None
        cfg = BatchConfig(storage=self.storage, max_instances=max_instances, pool_bytes=pool_bytes,
                          cuda_stream=stream.cuda_stream or None, dev_buffer=None, dev_buffer_bytes=0,
                          threads_per_group=threads_per_group, groups_per_cta=groups_per_cta,
                          cluster_ctas=cluster_ctas, coupling=_lks.COUPLINGS[coupling],
                          inplace=int(bool(inplace)), pad=0)
        self.inplace = bool(inplace)
        if torch_memory:
            self._pool = torch.empty(pool_bytes, dtype=torch.uint8, device=stream.device)
            cfg.dev_buffer = self._pool.data_ptr()
            cfg.dev_buffer_bytes = pool_bytes
        h = ctypes.c_void_p()
        st = L.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != _lks.LKS_OK:
            raise _lks.LksError(st, (L.lks_batch_last_error(None) or b"").decode())
        self._h = h
        self.max_instances = max_instances
        self.shapes = {}

    def _check(self, st):
        if st != _lks.LKS_OK:
            raise _lks.LksError(st, (lib().lks_batch_last_error(self._h) or b"").decode())

    def add(self, desc):
        """Admit an instance; returns its slot, or None when the batch is full (LKS_EBUSY)."""
        slot = ctypes.c_int32(-1)
        st = lib().lks_batch_add(self._h, ctypes.byref(desc), ctypes.byref(slot))
        if st == _lks.LKS_EBUSY:
            return None
        self._check(st)
        self.shapes[slot.value] = (desc.nx, desc.ny)
        return slot.value

    def run(self, quantum):
        n = ctypes.c_int32(0)
        self._check(lib().lks_batch_run(self._h, int(quantum), ctypes.byref(n)))
        return n.value

    def result(self, slot):
        r = InstanceResult()
        self._check(lib().lks_batch_result(self._h, slot, ctypes.byref(r)))
        return r.state, r.steps, r.residual

    def moments(self, slot, what=_lks.MOMENTS_NODES):
        nx, ny = self.shapes[slot]
        shape = (5, ny, nx) if what == _lks.MOMENTS_NODES else (5, ny)
        out = np.empty(shape)
        self._check(lib().lks_batch_moments(self._h, slot, what, out.ctypes.data_as(_DP)))
        return out

    def profiles(self, slot):
        m = self.moments(slot, _lks.MOMENTS_PROFILES)
        return m[1], m[3]

    def get_state(self, slot):
        """FP64 absolute populations (f (9, ny, nx), g (2, 5, ny, nx)) of one instance."""
        nx, ny = self.shapes[slot]
        f = np.empty((9, ny, nx))
        g = np.empty((2, 5, ny, nx))
        self._check(lib().lks_batch_get_state(self._h, slot, f.ctypes.data_as(_DP), g.ctypes.data_as(_DP)))
        return f, g

    def set_state(self, slot, f, g):
        """Replace one instance's state (FP64 absolute populations) and restart its bookkeeping."""
        nx, ny = self.shapes[slot]
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.shape == (9, ny, nx) and g.shape == (2, 5, ny, nx)
        self._check(lib().lks_batch_set_state(self._h, slot, f.ctypes.data_as(_DP), g.ctypes.data_as(_DP)))

    def remove(self, slot):
        self._check(lib().lks_batch_remove(self._h, slot))
        self.shapes.pop(slot, None)

    def set_shape(self, threads_per_group, groups_per_cta, cluster_ctas=1):
        self._check(lib().lks_batch_set_shape(self._h, threads_per_group, groups_per_cta, cluster_ctas))

    def autotune(self, candidates, probe_steps=200):
        """Time each (threads_per_group, groups_per_cta[, cluster_ctas]) candidate on the current
        instances (state is restored after each); keeps and returns the fastest plus all timings."""
        n = len(candidates)
        T = (ctypes.c_int32 * n)(*[c[0] for c in candidates])
        G = (ctypes.c_int32 * n)(*[c[1] for c in candidates])
        C = (ctypes.c_int32 * n)(*[(c[2] if len(c) > 2 else 1) for c in candidates])
        secs = (ctypes.c_double * n)()
        best = ctypes.c_int32(-1)
        self._check(lib().lks_batch_autotune(self._h, int(probe_steps), T, G, C, n, secs, ctypes.byref(best)))
        return candidates[best.value], list(secs)

    def memory(self):
        fr, us = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(lib().lks_batch_memory(self._h, ctypes.byref(fr), ctypes.byref(us)))
        return fr.value, us.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().lks_batch_destroy(self._h)
            self._h = None
            self._pool = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Shapes the autotuner tries (threads per instance group, groups per CTA, CTAs per cluster).
DEFAULT_CANDIDATES = [(64, 8, 1), (128, 4, 1), (256, 2, 1), (512, 1, 1), (128, 2, 1), (256, 1, 1), (64, 4, 1),
                      (32, 8, 1), (256, 1, 2), (512, 1, 2), (256, 1, 4), (512, 1, 4), (128, 1, 8), (256, 1, 8)]


def tuned_shape(batch, cache_path, key, probe_steps=200, candidates=None):
    """Autotune once per key (e.g. storage + size class) and cache the choice as JSON."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if key in cache:
        shape = cache[key]["shape"]
        batch.set_shape(*shape)
        return tuple(shape), cache[key]
    best, secs = batch.autotune(candidates or DEFAULT_CANDIDATES, probe_steps)
    entry = {"shape": list(best), "candidates": [list(c) for c in (candidates or DEFAULT_CANDIDATES)],
             "seconds": secs, "probe_steps": probe_steps}
    cache[key] = entry
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, entry

"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports every entry
point include/lks.h declares, and validates parameters (no device work: no GPU is needed)."""
import ctypes
import math
import os
import re

import pytest

from paper_2112_13930_gb300 import build as lks_build
from paper_2112_13930_gb300 import lks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lks_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    lks_build.build()
    return lks.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("lks.h")
    assert "lks_create" in names and "lks_step" in names and "lks_set_walls" in names and "lks_moments" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in lks.SIGNATURES, "binding lacks " + n


def test_every_batch_symbol_is_exported(lib):
    from paper_2112_13930_gb300 import batch
    names = _declared("lks_batch.h")
    assert "lks_batch_run" in names and "lks_batch_autotune" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in batch.SIGNATURES, "binding lacks " + n


def test_instance_footprint_and_batch_config_validation(lib):
    from paper_2112_13930_gb300 import batch
    d = batch.make_desc(4, 1025, "link", 0.8, 0.8, 0.01)
    fp = batch.instance_footprint(d, "f32")
    assert 2 * 19 * 4 * 4100 + 16 * 4100 <= fp < 2 * 19 * 4 * 4100 + 16 * 4100 + 5 * 256
    bad = batch.make_desc(4, 2, "moment", 0.8, 0.8, 0.01)
    assert batch.instance_footprint(bad, "f32") == 0
    bad = batch.make_desc(4, 20, "link", 0.8, 0.8, 0.01, c_top=-1.0)
    assert batch.instance_footprint(bad, "f32") == 0
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=48, groups_per_cta=1)
    h = ctypes.c_void_p()
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL and not h.value
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=256, groups_per_cta=4)
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=128, groups_per_cta=2,
                            cluster_ctas=2)
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=128, groups_per_cta=1,
                            cluster_ctas=3)
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=128, groups_per_cta=1,
                            coupling=2)
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL
    lor = batch.make_desc(4, 20, "link", 0.8, 1.02, 0.01, coupling="lorentz")   # |tau_m - 1| < 0.05
    assert batch.instance_footprint(lor, "f32") == 0
    cfg = batch.BatchConfig(storage=1, max_instances=4, pool_bytes=1 << 20, threads_per_group=128, groups_per_cta=1,
                            inplace=2)
    assert lib.lks_batch_create(ctypes.byref(cfg), ctypes.byref(h)) == lks.LKS_EINVAL
    # in place: one population buffer per instance, and even check/step counts
    d = batch.make_desc(8, 100, "moment", 0.8, 0.8, 0.01, check_every=100, max_steps=1000)
    two, one = batch.instance_footprint(d, "f32"), batch.instance_footprint(d, "f32", inplace=True)
    assert two - one == 28928 + 32000    # the f (9 x 800 x 4 B) and g (10 x 800 x 4 B) planes, 256-byte aligned
    odd = batch.make_desc(8, 100, "moment", 0.8, 0.8, 0.01, check_every=101)
    assert batch.instance_footprint(odd, "f32") > 0 and batch.instance_footprint(odd, "f32", inplace=True) == 0
    assert lib.lks_batch_destroy(None) == lks.LKS_OK


def test_footprint_counts_both_buffers(lib):
    nx, ny = 4096, 4096
    for storage, sb in (("f64", 8), ("f32", 4), ("bf16", 2), ("f16", 2)):
        fp = lks.footprint_bytes(nx, ny, "moment", storage)
        pops = 2 * 19 * nx * ny * sb
        snap = 2 * nx * ny * 8
        assert pops + snap <= fp < pops + snap + 1 << 20


def test_inplace_footprint_is_one_population_buffer(lib):
    nx, ny = 4096, 4096
    for storage, sb in (("f64", 8), ("f32", 4), ("bf16", 2), ("f16", 2)):
        two = lks.footprint_bytes(nx, ny, "moment", storage)
        one = lks.footprint_bytes(nx, ny, "moment", storage, inplace=True)
        assert two - one == 19 * nx * ny * sb   # 9 f + 10 g planes, 256-byte multiples here
    p = lks.make_params(8, 8, 0.8, 0.8, 0.01)
    p.inplace = 2
    assert lib.lks_footprint_bytes(ctypes.byref(p)) == 0


@pytest.mark.parametrize("kw,ok", [
    (dict(nx=4, ny=65, closure="link"), True),
    (dict(nx=4, ny=1, closure="link"), False),
    (dict(nx=4, ny=2, closure="link"), True),
    (dict(nx=4, ny=2, closure="moment"), False),
    (dict(nx=0, ny=8, closure="link"), False),
    (dict(nx=4, ny=8, closure="link", tau_f=0.5), False),
    (dict(nx=4, ny=8, closure="link", tau_m=0.4), False),
    (dict(nx=4, ny=8, closure="link", tau_m=math.nan), False),
    (dict(nx=4, ny=8, closure="moment", tau_m=0.8, coupling="lorentz"), True),
    (dict(nx=4, ny=8, closure="moment", tau_m=1.0, coupling="lorentz"), False),
    (dict(nx=4, ny=8, closure="moment", tau_m=1.0, coupling="maxwell"), True),
])
def test_parameter_validation(lib, kw, ok):
    p = lks.make_params(kw.get("nx"), kw.get("ny"), kw.get("tau_f", 0.8), kw.get("tau_m", 0.8), 0.01,
                        closure=kw["closure"], coupling=kw.get("coupling", "maxwell"))
    assert (lib.lks_footprint_bytes(ctypes.byref(p)) > 0) == ok


def test_create_rejects_bad_parameters_without_touching_the_device(lib):
    p = lks.make_params(4, 1, 0.8, 0.8, 0.01, closure="link")
    h = ctypes.c_void_p()
    st = lib.lks_create(ctypes.byref(p), ctypes.byref(h))
    assert st == lks.LKS_EINVAL and not h.value
    assert b"ny" in lib.lks_last_error(None)
    assert lib.lks_create(None, ctypes.byref(h)) == lks.LKS_EINVAL
    assert lib.lks_status_string(lks.LKS_EUNSTABLE) == b"LKS_EUNSTABLE"
    assert lib.lks_destroy(None) == lks.LKS_OK


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lks_step(None, 1) == lks.LKS_EINVAL
    assert lib.lks_set_walls(None, 0.0, 0.0, 0.0, 0.0) == lks.LKS_EINVAL
    assert lib.lks_sync(None) == lks.LKS_EINVAL
    assert lib.lks_steps_taken(None) == -1


def test_binding_fails_loudly_without_the_library(tmp_path):
    with pytest.raises(ImportError):
        lks.Lattice.__init__  # noqa: B018 -- attribute exists
        import importlib
        mod = importlib.import_module("paper_2112_13930_gb300.lks")
        saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "missing.so"))
        finally:
            mod._lib = saved


def test_every_3d_symbol_is_exported(lib):
    from paper_2112_13930_gb300 import lks3d
    text = open(os.path.join(ROOT, "include", "lks3d.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = sorted(set(re.findall(r"\b(lks3_[a-z0-9_]+)\s*\(", text)))
    assert "lks3_create" in names and "lks3_step" in names and "lks3_run_to_steady" in names
    for n in names:
        assert hasattr(lib, n), n
        assert n in lks3d.SIGNATURES, "binding lacks " + n


@pytest.mark.parametrize("kw,ok", [
    (dict(nx=4, ny=2, nz=1), True),
    (dict(nx=4, ny=1, nz=1), False),
    (dict(nx=0, ny=8, nz=4), False),
    (dict(nx=4, ny=8, nz=0), False),
    (dict(nx=4, ny=8, nz=4, storage="bf16"), True),
    (dict(nx=4, ny=8, nz=4, tau_m=0.5), False),
    (dict(nx=1024, ny=1024, nz=1025), False),       # above 2^30 nodes
])
def test_3d_parameter_validation(lib, kw, ok):
    from paper_2112_13930_gb300 import lks3d
    p = lks3d.make_params(kw["nx"], kw["ny"], kw["nz"], 0.8, kw.get("tau_m", 0.8), 0.01,
                          storage=kw.get("storage", "f64"))
    assert (lib.lks3_footprint_bytes(ctypes.byref(p)) > 0) == ok


def test_3d_footprint_counts_both_buffers(lib):
    from paper_2112_13930_gb300 import lks3d
    n = 256 ** 3
    for storage, sb in (("f64", 8), ("f32", 4)):
        fp = lks3d.footprint_bytes(256, 256, 256, storage)
        pops = 2 * 40 * n * sb
        assert pops + 2 * n * 8 <= fp < pops + 2 * n * 8 + (1 << 20)


def test_newer_entry_points_validate_before_device_work(lib):
    """The raw state image, the allocation-free residual, the duct's side walls and the batch state
    transfer and shape calls reject a NULL handle or bad arguments before any device work."""
    buf = (ctypes.c_double * 16)()
    vp = ctypes.cast(buf, ctypes.c_void_p)
    dp = ctypes.cast(buf, ctypes.POINTER(ctypes.c_double))
    assert lib.lks_state_bytes(None) == 0
    assert lib.lks_get_state_raw(None, vp, 16) == lks.LKS_EINVAL
    assert lib.lks_set_state_raw(None, vp, 16) == lks.LKS_EINVAL

    def noalloc(f=vp, g=vp, storage=lks.F64, nx=4, ny=8, coupling=lks.MAXWELL, tau_m=0.8, snap=vp, out=dp):
        return lib.lks_residual_noalloc(f, g, storage, nx, ny, 0.01, 0.0, coupling, tau_m, snap, out, None)

    assert noalloc(f=None) == lks.LKS_EINVAL
    assert noalloc(snap=None) == lks.LKS_EINVAL
    assert noalloc(out=None) == lks.LKS_EINVAL
    assert noalloc(storage=7) == lks.LKS_EINVAL
    assert noalloc(nx=0) == lks.LKS_EINVAL
    assert noalloc(coupling=5) == lks.LKS_EINVAL
    assert noalloc(coupling=lks.LORENTZ, tau_m=1.02) == lks.LKS_EINVAL   # J cannot be read back at tau_m = 1
    assert noalloc(nx=1 << 16, ny=(1 << 14) + 1) == lks.LKS_EINVAL       # above 2^30 nodes
    assert b"lks_residual_noalloc" in lib.lks_last_error(None)

    from paper_2112_13930_gb300 import lks3d  # noqa: F401 -- the 3D signatures are set on load
    assert lib.lks3_set_side_walls(None, 1, 0.1, 0.1) == lks.LKS_EINVAL
    assert lib.lks_batch_get_state(None, 0, dp, dp) == lks.LKS_EINVAL
    assert lib.lks_batch_set_state(None, 0, dp, dp) == lks.LKS_EINVAL
    assert lib.lks_batch_set_shape(None, 128, 1, 8) == lks.LKS_EINVAL

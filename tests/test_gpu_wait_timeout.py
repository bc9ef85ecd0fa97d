"""Failure detection of the staged kernels' bounded waits, on the GPU, without a GPU fault.

Every wait of the staged kernels (on an mbarrier phase) gives up after a time limit, records the
timeout in the handle's error word and returns; the next synchronising call reports LKS_ETIMEOUT.
lks_selftest_wait_timeout makes such a wait run out on purpose: one warp waits, with the same
bounded-wait helper, on a freshly initialised barrier that nothing arrives on (no copy is in flight
to it), gives up after the limit and sets the error word.  The host must then see LKS_ETIMEOUT from
the next synchronising calls, the wait must have lasted about its limit, and the CUDA context must
stay usable for a new handle.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks as mod
    build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def l3(lks):
    from paper_2112_13930_gb300 import lks3d
    return lks3d


def _staged(lks):
    # BF16, nx a multiple of 8 and >= 1024: the staged two-buffer step
    return lks.Lattice(1032, 8, 0.8, 0.8, 0.02, 1e-6, "moment", "bf16", seed=3, perturb_amp=1e-3)


def test_wait_that_runs_out_reports_etimeout(lks):
    L = lks.load()
    lat = _staged(lks)
    lat.step(4)
    lat.sync()
    limit = 0.05
    t0 = time.perf_counter()
    assert L.lks_selftest_wait_timeout(lat._h, limit) == lks.LKS_OK  # enqueued only
    st = L.lks_sync(lat._h)
    dt = time.perf_counter() - t0
    assert st == lks.LKS_ETIMEOUT
    assert b"wait ran out" in L.lks_last_error(lat._h)
    assert limit <= dt < 5.0
    # the handle stays in its error state
    with pytest.raises(lks.LksError) as err:
        lat.moments()
    assert err.value.status == lks.LKS_ETIMEOUT
    lat.close()
    # the context is intact: a new handle steps, synchronises and reads finite moments
    b = _staged(lks)
    b.step(6)
    b.sync()
    assert np.all(np.isfinite(b.moments()))
    b.close()


def test_selftest_rejects_unstaged_handles_and_bad_limits(lks):
    L = lks.load()
    f32 = lks.Lattice(1032, 8, 0.8, 0.8, 0.02, 1e-6, "moment", "f32")
    assert L.lks_selftest_wait_timeout(f32._h, 0.05) == lks.LKS_EINVAL
    f32.close()
    lat = _staged(lks)
    for bad in (0.0, -1.0, 2.0, float("nan")):
        assert L.lks_selftest_wait_timeout(lat._h, bad) == lks.LKS_EINVAL
    lat.sync()  # nothing was enqueued: still healthy
    lat.close()


def test_3d_wait_that_runs_out_reports_etimeout(lks, l3):
    L = l3.lib()
    lat = l3.Lattice3D(24, 8, 4, 0.8, 0.7, 0.02, 1e-6, "bf16")  # staged: BF16, nx % 8 == 0, nx <= 512
    lat.step(3)
    lat.sync()
    limit = 0.05
    t0 = time.perf_counter()
    assert L.lks3_selftest_wait_timeout(lat._h, limit) == lks.LKS_OK
    st = L.lks3_sync(lat._h)
    dt = time.perf_counter() - t0
    assert st == lks.LKS_ETIMEOUT
    assert b"wait ran out" in L.lks3_last_error(lat._h)
    assert limit <= dt < 5.0
    lat.close()
    f32 = l3.Lattice3D(24, 8, 4, 0.8, 0.7, 0.02, 1e-6, "f32")
    assert L.lks3_selftest_wait_timeout(f32._h, limit) == lks.LKS_EINVAL
    f32.step(3)
    f32.sync()
    assert np.all(np.isfinite(f32.moments()))
    f32.close()

"""A driven channel whose 16-bit state stops changing is reported as stalled, not converged.

The 4 x 513 body-force Hartmann channel (Ha = 30, c = 0.5, tau = 0.8, centreline speed 0.01) gains
about 1e-9 of velocity per step from the body force, far below one unit in the last place of its
BF16 deviations (8-bit significand, ~1e-5 here): after a few thousand steps the stored state is a
fixed point of the rounded update, u_x and B_x no longer change by a single bit, and the
steady-state residual is exactly 0 while the profiles are still far from the steady solution.
lks_run_to_steady must return LKS_ESTALLED there (not LKS_OK), and the batched engine must end such
an instance STALLED."""
import math

import numpy as np
import pytest

from oracle import analytic as an

pytestmark = pytest.mark.gpu

NY, HA, C, TAU = 513, 30.0, 0.5, 0.8


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import batch, build, lks
    build.build()
    lks.load()
    return lks, batch


def _channel():
    a = NY / 2
    b0 = an.b0_from_ha(HA, a, TAU, TAU)
    fx = an.force_for_centre_speed(0.01, HA, C, a, TAU)
    return a, b0, fx


@pytest.mark.parametrize("storage", ["bf16"])
def test_single_lattice_reports_stall(mods, storage):
    lks, _ = mods
    a, b0, fx = _channel()
    lat = lks.Lattice(4, NY, TAU, TAU, b0, fx, "link", storage)
    lat.set_walls(C, C)
    steps, r, status = lat.run_to_steady(1e-9, 1000, 400_000, raise_on_fail=False)
    assert status == lks.LKS_ESTALLED, (lks._status_name(status), steps, r)
    assert r == 0.0 and steps < 400_000
    assert b"stopped changing" in lks.load().lks_last_error(lat._h)
    # the stagnant profile is not the steady solution
    u, _ = lat.profiles()
    ua, _ = an.hartmann_profiles(lat.y(), a, HA, C, fx, TAU, TAU)
    assert an.rel_l2(u, ua) > 1e-2
    lat.close()


def test_fp32_same_channel_is_not_reported_as_stalled_early(mods):
    """FP32 resolves the increments on this channel: it keeps changing over the same number of steps."""
    lks, _ = mods
    a, b0, fx = _channel()
    lat = lks.Lattice(4, NY, TAU, TAU, b0, fx, "link", "f32")
    lat.set_walls(C, C)
    steps, r, status = lat.run_to_steady(1e-9, 1000, 30_000, raise_on_fail=False)
    assert status == lks.LKS_ENOTCONVERGED and r > 0.0
    lat.close()


@pytest.mark.parametrize("storage", ["bf16"])
def test_batch_reports_stall(mods, storage):
    lks, batch = mods
    a, b0, fx = _channel()
    b = batch.Batch(storage, max_instances=2, pool_bytes=16 << 20)
    d = batch.make_desc(4, NY, "link", TAU, TAU, b0, fx, C, C, tol=1e-9, check_every=1000, max_steps=400_000)
    s = b.add(d)
    while b.run(20_000):
        pass
    st, steps, r = b.result(s)
    assert st == batch.INST_STALLED, (st, steps, r)
    assert r == 0.0 and steps < 400_000
    b.close()

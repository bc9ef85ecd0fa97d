"""Batched engine (lks_batch.h) on the GPU: per-instance parity with the FP64 oracle and with the
single-lattice API, results independent of the mix, admission by pool footprint, statuses, and
an autotune pass that leaves every state untouched."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as an

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import batch, build, lks
    build.build()
    lks.load()
    return lks, batch


def _descs(batch, n=6, max_steps=10**7, tol=1e-30, check_every=50):
    """A mixed set: link/moment, body force/shear, c = 0 / finite / inf, nx in {1, 4, 37}."""
    out = []
    rng = np.random.default_rng(7)
    for k in range(n):
        closure = "link" if k % 2 == 0 else "moment"
        ny = int(rng.integers(12, 70))
        nx = [4, 1, 37][k % 3]
        a = ny / 2 if closure == "link" else (ny - 1) / 2
        ha = float(rng.uniform(1, 0.3 * a))  # B0 = Ha sqrt(nu eta)/a <= 0.03: stable Alfven speed
        b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
        c = [0.0, 0.3, math.inf][k % 3]
        if k % 2 == 0:
            fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
            d = batch.make_desc(nx, ny, closure, 0.8, 0.8, b0, fx, c, c, 0.0, 0.0, seed=k, perturb_amp=1e-3,
                                tol=tol, check_every=check_every, max_steps=max_steps)
        else:
            d = batch.make_desc(nx, ny, closure, 0.8, 0.8, b0, 0.0, 0.0, c, 0.0, 0.05, seed=k, perturb_amp=1e-3,
                                tol=tol, check_every=check_every, max_steps=max_steps)
        out.append(d)
    return out


def _oracle_for(d):
    return oracle.Oracle(d.nx, d.ny, d.tau_f, d.tau_m, d.B0, d.Fx, d.closure, d.c_bottom, d.c_top, d.u_bottom,
                         d.u_top, seed=d.seed, perturb_amp=d.perturb_amp)


@pytest.mark.parametrize("shape", [(128, 2, 1), (128, 1, 4)])
def test_batch_fp64_matches_oracle(mods, shape):
    lks, batch = mods
    b = batch.Batch("f64", max_instances=16, pool_bytes=64 << 20, threads_per_group=shape[0], groups_per_cta=shape[1],
                    cluster_ctas=shape[2])
    descs = _descs(batch)
    slots = [b.add(d) for d in descs]
    for q in (7, 93):
        b.run(q)
        for d, s in zip(descs, slots):
            o = _oracle_for(d)
            o.step(7 if q == 7 else 100)
            mo, mg = o.moments(), b.moments(s)
            for m in (0, 1, 3):
                scale = np.max(np.abs(mo[m]))
                assert np.max(np.abs(mg[m] - mo[m])) <= 1e-11 * scale, (d.closure, m)
            st, steps, r = b.result(s)
            assert st == batch.INST_RUNNING and steps == (7 if q == 7 else 100)
    b.close()


@pytest.mark.parametrize("shape", [(64, 4, 1), (128, 1, 2), (64, 1, 8)])
def test_batch_matches_single_lattice_bitwise(mods, shape):
    """Same device update as lks_step: FP32 batch instances equal single-lattice runs bit for bit,
    with groups inside a CTA and with thread-block clusters spanning 2 or 8 SMs."""
    lks, batch = mods
    b = batch.Batch("f32", max_instances=16, pool_bytes=64 << 20, threads_per_group=shape[0],
                    groups_per_cta=shape[1], cluster_ctas=shape[2])
    descs = _descs(batch)
    slots = [b.add(d) for d in descs]
    b.run(250)
    for d, s in zip(descs, slots):
        g = lks.Lattice(d.nx, d.ny, d.tau_f, d.tau_m, d.B0, d.Fx, d.closure, "f32", seed=d.seed,
                        perturb_amp=d.perturb_amp)
        g.set_walls(d.c_bottom, d.c_top, d.u_bottom, d.u_top)
        g.step(250)
        assert np.array_equal(g.moments(), b.moments(s))
        g.close()
    b.close()


@pytest.mark.parametrize("cluster", [1, 4])
def test_alone_equals_in_the_mix(mods, cluster):
    """Each instance's result is the same alone and in a mixed batch (bitwise, same group size)."""
    lks, batch = mods
    descs = _descs(batch, n=8, tol=1e-9, check_every=100, max_steps=3000)
    g = 2 if cluster == 1 else 1
    mix = batch.Batch("f32", max_instances=16, pool_bytes=64 << 20, threads_per_group=128, groups_per_cta=g,
                      cluster_ctas=cluster)
    slots = [mix.add(d) for d in descs]
    while mix.run(700):
        pass
    for d, s in zip(descs, slots):
        alone = batch.Batch("f32", max_instances=1, pool_bytes=8 << 20, threads_per_group=128, groups_per_cta=1,
                            cluster_ctas=cluster)
        a = alone.add(d)
        while alone.run(300):
            pass
        assert alone.result(a)[:2] == mix.result(s)[:2]
        assert alone.result(a)[0] in (batch.INST_CONVERGED, batch.INST_MAX_STEPS)
        m = mix.moments(s)
        assert np.all(np.isfinite(m)) and np.array_equal(alone.moments(a), m)
        alone.close()
    mix.close()


def test_statuses_and_residual(mods):
    """CONVERGED at tol, MAX_STEPS at max_steps; the residual equals the single-lattice one."""
    lks, batch = mods
    b = batch.Batch("f64", max_instances=4, pool_bytes=16 << 20)
    ny, ha, c = 33, 10.0, 0.5
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
    d1 = batch.make_desc(4, ny, "link", 0.8, 0.8, b0, fx, c, c, tol=1e-9, check_every=100, max_steps=10**6)
    d2 = batch.make_desc(4, ny, "link", 0.8, 0.8, b0, fx, c, c, tol=1e-30, check_every=100, max_steps=500)
    s1, s2 = b.add(d1), b.add(d2)
    while b.run(5000):
        pass
    st1, steps1, r1 = b.result(s1)
    st2, steps2, r2 = b.result(s2)
    assert st1 == batch.INST_CONVERGED and r1 < 1e-9 and steps1 % 100 == 0
    assert st2 == batch.INST_MAX_STEPS and steps2 == 500
    g = lks.Lattice(4, ny, 0.8, 0.8, b0, fx, "link", "f64")
    g.set_walls(c, c)
    n, r, status = g.run_to_steady(1e-9, 100, 10**6)
    assert n == steps1 and r == pytest.approx(r1, rel=1e-9)
    u, bx = b.profiles(s1)
    ua, ba = an.hartmann_profiles(g.y(), a, ha, c, fx, 0.8, 0.8)
    assert an.rel_l2(u, ua) < 1e-2 and an.rel_l2(bx, ba) < 1e-2   # 33-node channel: ~6e-3
    g.close()
    b.close()


def test_admission_by_footprint_and_slots(mods):
    lks, batch = mods
    d = batch.make_desc(4, 100, "moment", 0.8, 0.8, 0.01)
    fp = batch.instance_footprint(d, "f32")
    assert fp >= 2 * 19 * 4 * 400 + 16 * 400
    b = batch.Batch("f32", max_instances=3, pool_bytes=2 * fp + 1024)
    s0, s1 = b.add(d), b.add(d)
    assert s0 is not None and s1 is not None
    assert b.add(d) is None                       # pool full -> LKS_EBUSY
    free0, used0 = b.memory()
    assert used0 == 2 * fp
    b.remove(s0)
    assert b.memory()[1] == fp
    s2 = b.add(d)
    assert s2 == s0
    small = batch.make_desc(4, 5, "moment", 0.8, 0.8, 0.01)
    assert b.add(small) is None or b.memory()[0] >= 0
    b.close()
    c = batch.Batch("f32", max_instances=1, pool_bytes=8 << 20)
    assert c.add(small) is not None
    assert c.add(small) is None                   # no slot -> LKS_EBUSY
    c.close()


def test_autotune_leaves_states_untouched(mods):
    lks, batch = mods
    descs = _descs(batch, n=6)
    ref = batch.Batch("f32", max_instances=8, pool_bytes=32 << 20, threads_per_group=128, groups_per_cta=1)
    tun = batch.Batch("f32", max_instances=8, pool_bytes=32 << 20, threads_per_group=128, groups_per_cta=1)
    rs = [ref.add(d) for d in descs]
    ts = [tun.add(d) for d in descs]
    ref.run(100)
    tun.run(100)
    best, secs = tun.autotune([(64, 2, 1), (128, 1, 1), (256, 1, 1), (32, 8, 1), (128, 1, 4), (64, 1, 8)],
                              probe_steps=50)
    assert len(secs) == 6 and all(s > 0 for s in secs)
    tun.set_shape(128, 1)
    ref.run(100)
    tun.run(100)
    for a, c in zip(rs, ts):
        assert ref.result(a)[:2] == tun.result(c)[:2]
        assert np.array_equal(ref.moments(a), tun.moments(c))
    ref.close()
    tun.close()


def _lorentz_descs(batch, **kw):
    descs = _descs(batch, **kw)
    for d in descs:
        d.coupling = 1
    return descs


@pytest.mark.parametrize("shape", [(128, 2, 1), (128, 1, 4)])
def test_batch_lorentz_fp64_matches_oracle(mods, shape):
    """The Lorentz-force coupling (Sec. III source term, J from the non-equilibrium moment of g)
    in the batched engine: FP64 instances equal the oracle with coupling 1 within 1e-11."""
    lks, batch = mods
    b = batch.Batch("f64", max_instances=16, pool_bytes=64 << 20, threads_per_group=shape[0], groups_per_cta=shape[1],
                    cluster_ctas=shape[2], coupling="lorentz")
    descs = _lorentz_descs(batch)
    slots = [b.add(d) for d in descs]
    b.run(60)
    for d, s in zip(descs, slots):
        o = oracle.Oracle(d.nx, d.ny, d.tau_f, d.tau_m, d.B0, d.Fx, d.closure, d.c_bottom, d.c_top, d.u_bottom,
                          d.u_top, seed=d.seed, perturb_amp=d.perturb_amp, coupling=1)
        o.step(60)
        mo, mg = o.moments(), b.moments(s)
        for m in (0, 1, 3):
            scale = np.max(np.abs(mo[m]))
            assert np.max(np.abs(mg[m] - mo[m])) <= 1e-11 * scale, (d.closure, m)
    b.close()


@pytest.mark.parametrize("shape", [(64, 4, 1), (64, 1, 8)])
def test_batch_lorentz_matches_single_lattice_bitwise(mods, shape):
    lks, batch = mods
    b = batch.Batch("f32", max_instances=16, pool_bytes=64 << 20, threads_per_group=shape[0],
                    groups_per_cta=shape[1], cluster_ctas=shape[2], coupling="lorentz")
    descs = _lorentz_descs(batch)
    slots = [b.add(d) for d in descs]
    b.run(250)
    for d, s in zip(descs, slots):
        g = lks.Lattice(d.nx, d.ny, d.tau_f, d.tau_m, d.B0, d.Fx, d.closure, "f32", seed=d.seed,
                        perturb_amp=d.perturb_amp, coupling="lorentz")
        g.set_walls(d.c_bottom, d.c_top, d.u_bottom, d.u_top)
        g.step(250)
        assert np.array_equal(g.moments(), b.moments(s))
        g.close()
    b.close()


def test_batch_rejects_mixed_coupling(mods):
    lks, batch = mods
    b = batch.Batch("f32", max_instances=4, pool_bytes=8 << 20)
    d = batch.make_desc(4, 20, "link", 0.8, 0.8, 0.01, coupling="lorentz")
    with pytest.raises(lks.LksError):
        b.add(d)
    b.close()


def test_state_transfer_between_batches(mods):
    """lks_batch_get_state / lks_batch_set_state: an FP64 instance copied into another batch continues
    as the original does (to the rounding of the FP64 absolute populations), and its bookkeeping
    restarts (steps 0, RUNNING)."""
    lks, batch = mods
    d = _descs(batch, n=2, check_every=50)[0]
    a = batch.Batch("f64", max_instances=2, pool_bytes=8 << 20)
    b = batch.Batch("f64", max_instances=2, pool_bytes=8 << 20)
    sa = a.add(d)
    a.run(400)
    f, g = a.get_state(sa)
    sb = b.add(d)
    b.set_state(sb, f, g)
    st, steps, _ = b.result(sb)
    assert st == batch.INST_RUNNING and steps == 0
    f2, g2 = b.get_state(sb)
    np.testing.assert_allclose(f2, f, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g2, g, rtol=0, atol=1e-15)
    a.run(300)
    b.run(300)
    ma, mb = a.moments(sa), b.moments(sb)
    for k in (1, 3):
        assert np.max(np.abs(ma[k] - mb[k])) <= 1e-12 * np.max(np.abs(ma[k]))
    a.close()
    b.close()


def test_fp32_floor_finished_in_fp64(mods):
    """The mixed-precision lane: an FP32 solve run to a hand-off tolerance of 1e-5 (or stopped at its
    rounding floor, STALLED), moved into an FP64 batch, converges there to 1e-10 and agrees with a
    pure FP64 solve of the same instance."""
    lks, batch = mods
    ny, ha, c = 129, 10.0, 0.5
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01 * 64 / (ny - 1), ha, c, a, 0.8)
    d32 = batch.make_desc(4, ny, "link", 0.8, 0.8, b0, fx, c, c, tol=1e-5, check_every=100, max_steps=4_000_000)
    d64 = batch.make_desc(4, ny, "link", 0.8, 0.8, b0, fx, c, c, tol=1e-10, check_every=100, max_steps=4_000_000)
    b32 = batch.Batch("f32", max_instances=1, pool_bytes=8 << 20)
    s32 = b32.add(d32)
    while b32.run(100_000):
        pass
    st32, steps32, r32 = b32.result(s32)
    assert st32 in (batch.INST_CONVERGED, batch.INST_STALLED), (st32, steps32, r32)
    b64 = batch.Batch("f64", max_instances=2, pool_bytes=16 << 20)
    sf = b64.add(d64)
    b64.set_state(sf, *b32.get_state(s32))
    sp = b64.add(d64)
    while b64.run(100_000):
        pass
    stf, stepsf, rf = b64.result(sf)
    stp, stepsp, rp = b64.result(sp)
    assert stf == batch.INST_CONVERGED and stp == batch.INST_CONVERGED
    uf, bf = b64.profiles(sf)
    up, bp = b64.profiles(sp)
    assert np.max(np.abs(uf - up)) <= 1e-6 * np.max(np.abs(up))
    assert np.max(np.abs(bf - bp)) <= 1e-6 * np.max(np.abs(bp))
    assert stepsf < stepsp   # the FP32 phase already covered part of the way
    b32.close()
    b64.close()


def test_mixed_lane_equals_solo_handoffs(mods):
    """sweep.run_mixed: every instance's result equals the same hand-off done alone (an FP32 batch of
    one to the hand-off residual, then, if it converged or stalled within its budget, an FP64 batch of
    one from that state with what is left of the budget) -- bit for bit, although the batches change
    shape on the way; each instance's time-to-steady is recorded once and lies within the run."""
    lks, batch = mods
    from paper_2112_13930_gb300 import sweep, workloads
    specs = workloads.sweep_instances(n=6, seed=11, ny_range=(33, 65), ha_range=(1.0, 4.0))
    budget, shape = 12_000, (64, 2)
    # tail_below=4: each batch runs in the base shape while 4 or more of its instances run, then on
    # clusters of 8 CTAs per instance
    out = sweep.run_mixed(specs, handoff_tol=1e-5, tol=1e-9, check_every=100, quantum=1000, max_steps=budget,
                          shape=shape, tail_shape=(128, 1, 8), tail_below=4)
    kw = dict(threads_per_group=shape[0], groups_per_cta=shape[1])
    for spec, rec in zip(specs, out["records"]):
        assert rec["t_done"] is not None and 0.0 <= rec["t_done"] <= out["wall"]
        b32 = batch.Batch("f32", max_instances=1, pool_bytes=64 << 20, **kw)
        s = b32.add(sweep.make_desc(spec, 1e-5, 100, budget))
        while b32.run(1000):
            pass
        st32, steps32, _ = b32.result(s)
        assert rec["fp32_state"] == batch.STATE_NAMES[st32] and rec["steps_fp32"] == steps32
        if st32 in (batch.INST_CONVERGED, batch.INST_STALLED) and steps32 < budget:
            b64 = batch.Batch("f64", max_instances=1, pool_bytes=64 << 20, **kw)
            s64 = b64.add(sweep.make_desc(spec, 1e-9, 100, budget - steps32))
            b64.set_state(s64, *b32.get_state(s))
            while b64.run(1000):
                pass
            st, steps64, _ = b64.result(s64)
            u, bx = b64.profiles(s64)
            assert rec["state"] == batch.STATE_NAMES[st] and rec["steps_fp64"] == steps64
            b64.close()
        else:
            u, bx = b32.profiles(s)
            assert rec["state"] == "fp32_" + batch.STATE_NAMES[st32] and rec["steps_fp64"] == 0
        b32.close()
        assert np.array_equal(u, rec["u"]) and np.array_equal(bx, rec["b"])

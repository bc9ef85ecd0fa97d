"""Serving loop on the GPU: requests that arrive while others run are admitted and finish; each
result equals the same request solved alone (small lane: lks_batch with one instance; large lane:
a single lattice), bit for bit."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import batch, build, lks, serve, sweep, workloads
    build.build()
    lks.load()
    return lks, batch, serve, sweep, workloads


def _trace(workloads):
    tr = workloads.serve_trace(14, rate=400.0, seed=21, ny_median=40, ny_sigma=0.4, ny_clamp=(33, 80),
                               nx_choices=(4, 96))
    for r in tr:  # keep the Alfven speed B0 = Ha sqrt(nu eta)/a small enough for a stable lattice
        r["ha"] = min(r["ha"], 0.3 * (r["ny"] - 1) / 2)
    return tr


@pytest.mark.parametrize("inplace", [False, True])
def test_served_results_equal_solo_results(mods, inplace):
    """Served (two-buffer or in-place) results equal the two-buffer solo solves bit for bit."""
    lks, batch, serve, sweep, workloads = mods
    tr = _trace(workloads)
    srv = serve.Server("f32", budget_bytes=1 << 30, small_pool_bytes=256 << 20, small_max_nodes=400,
                       large_workers=2, tol=1e-7, check_every=100, quantum=300, max_steps=4000, shape=(64, 2),
                       inplace=inplace)
    recs = srv.serve(tr, time_limit=300)
    srv.close()
    assert len(recs) == len(tr)
    lanes = {r["lane"] for r in recs}
    assert lanes == {"small", "large"}
    for rec in recs:
        req = rec["req"]
        assert rec["state"] in ("converged", "max_steps"), rec["state"]
        assert rec["t_done"] >= rec["t_arrival"] and rec["t_admit"] >= rec["t_arrival"] - 1e-9
        if rec["lane"] == "small":
            b = batch.Batch("f32", max_instances=1, pool_bytes=64 << 20, threads_per_group=64, groups_per_cta=1)
            s = b.add(sweep.make_desc(req, 1e-7, 100, 4000))
            while b.run(300):
                pass
            u, bx = b.profiles(s)
            st, steps, r = b.result(s)
            b.close()
        else:
            p = sweep.lattice_params(req)
            lat = lks.Lattice(req["nx"], req["ny"], 0.8, 0.8, p["B0"], p["Fx"], req["closure"], "f32")
            lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
            steps, r, status = lat.run_to_steady(1e-7, 100, 4000, raise_on_fail=False)
            u, bx = lat.profiles()
            lat.close()
        assert steps == rec["steps"]
        assert np.array_equal(u, rec["u"]) and np.array_equal(bx, rec["b"])


def test_admission_waits_for_memory(mods):
    """A pool that holds one request at a time still serves the whole trace, in order."""
    lks, batch, serve, sweep, workloads = mods
    tr = [r for r in _trace(workloads) if r["nx"] * r["ny"] <= 400][:4]
    fp = max(batch.instance_footprint(sweep.make_desc(r, 1e-7, 100, 1000), "f32") for r in tr)
    srv = serve.Server("f32", budget_bytes=1 << 30, small_pool_bytes=fp + 512, small_max_nodes=400,
                       large_workers=1, tol=1e-7, check_every=100, quantum=200, max_steps=1000)
    recs = srv.serve(tr, time_limit=300)
    srv.close()
    assert len(recs) == len(tr)
    admits = sorted(r["t_admit"] for r in recs)
    dones = sorted(r["t_done"] for r in recs)
    for k in range(1, len(tr)):
        assert admits[k] >= dones[k - 1] - 1e-9   # the next one got in only after one left


def test_served_fp64_finish_equals_solo_mixed_solves(mods):
    """With finish_tol the server hands each request from FP32 (at residual 1e-5) to FP64 (to 1e-9,
    with what is left of its 40 000-step budget);
    every result equals the same hand-off done alone: small lane, an FP32 batch then an FP64 batch
    through lks_batch_get_state / lks_batch_set_state; large lane, an FP32 lattice then an FP64
    lattice through lks_get_state / lks_set_state -- bit for bit."""
    lks, batch, serve, sweep, workloads = mods
    tr = _trace(workloads)[:8]
    kw = dict(tol=1e-9, check_every=100, max_steps=40_000)
    srv = serve.Server("f32", budget_bytes=1 << 30, small_pool_bytes=128 << 20, small_max_nodes=400,
                       large_workers=2, quantum=2000, shape=(64, 2), finish_tol=1e-5, **kw)
    recs = srv.serve(tr, time_limit=600)
    srv.close()
    assert len(recs) == len(tr)
    for rec in recs:
        req = rec["req"]
        if rec["lane"] == "small":
            b32 = batch.Batch("f32", max_instances=1, pool_bytes=64 << 20, threads_per_group=64, groups_per_cta=1)
            s = b32.add(sweep.make_desc(req, 1e-5, 100, 40_000))
            while b32.run(2000):
                pass
            st32, steps32, _ = b32.result(s)
            if st32 in (batch.INST_CONVERGED, batch.INST_STALLED) and steps32 < 40_000:
                b64 = batch.Batch("f64", max_instances=1, pool_bytes=64 << 20, threads_per_group=64,
                                  groups_per_cta=1)
                s64 = b64.add(sweep.make_desc(req, 1e-9, 100, 40_000 - steps32))
                b64.set_state(s64, *b32.get_state(s))
                while b64.run(2000):
                    pass
                st, steps64, _ = b64.result(s64)
                u, bx = b64.profiles(s64)
                steps = steps32 + steps64
                b64.close()
            else:
                st, steps = st32, steps32
                u, bx = b32.profiles(s)
            b32.close()
            assert rec["state"] == batch.STATE_NAMES[st]
        else:
            p = sweep.lattice_params(req)
            lat = lks.Lattice(req["nx"], req["ny"], 0.8, 0.8, p["B0"], p["Fx"], req["closure"], "f32")
            lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
            steps, r, status = lat.run_to_steady(1e-5, 100, 40_000, raise_on_fail=False)
            if status in (lks.LKS_OK, lks.LKS_ESTALLED) and steps < 40_000:
                f, g = lat.get_state()
                lat.close()
                lat = lks.Lattice(req["nx"], req["ny"], 0.8, 0.8, p["B0"], p["Fx"], req["closure"], "f64")
                lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
                lat.set_state(f, g)
                s64, r, status = lat.run_to_steady(1e-9, 100, 40_000 - steps, raise_on_fail=False)
                steps += s64
            u, bx = lat.profiles()
            lat.close()
        assert steps == rec["steps"]
        assert np.array_equal(u, rec["u"]) and np.array_equal(bx, rec["b"])

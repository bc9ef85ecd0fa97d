"""Parameter-sweep driver: many channel instances solved to steady state by the batched engine
(include/lks_batch.h), and the one-at-a-time FP64 baseline through the single-lattice API."""
import math
import time

import numpy as np

from . import batch as _batch
from . import lks as _lks
from . import profiles

TAU = 0.8
U_WALL = 0.05


def lattice_params(spec, tau=TAU):
    """Lattice parameters of one instance: B0 from Ha, body force for an analytic centreline speed
    u_c = 0.01 * 64/(ny - 1) (diffusive scaling), shear instances' top plate at U_w = 0.05."""
    a, _ = profiles.node_y(spec["ny"], spec["closure"])
    nu = eta = (tau - 0.5) / 3.0
    b0 = spec["ha"] * math.sqrt(nu * eta) / a
    if spec["kind"] == "body":
        fx = profiles.hartmann_force(0.01 * 64.0 / (spec["ny"] - 1), spec["ha"], spec["c"], a, tau)
        return dict(B0=b0, Fx=fx, c_bottom=spec["c"], c_top=spec["c"], u_bottom=0.0, u_top=0.0)
    return dict(B0=b0, Fx=0.0, c_bottom=0.0, c_top=spec["c"], u_bottom=0.0, u_top=U_WALL)


def make_desc(spec, tol, check_every, max_steps, tau=TAU):
    p = lattice_params(spec, tau)
    return _batch.make_desc(spec["nx"], spec["ny"], spec["closure"], tau, tau, p["B0"], p["Fx"], p["c_bottom"],
                            p["c_top"], p["u_bottom"], p["u_top"], tol=tol, check_every=check_every,
                            max_steps=max_steps)


def analytic_error(spec, u, b, tau=TAU):
    """Relative L2 errors of u_x and B_x profiles against the closed form."""
    p = lattice_params(spec, tau)
    a, y = profiles.node_y(spec["ny"], spec["closure"])
    if spec["kind"] == "body":
        ua, ba = profiles.hartmann(y, a, spec["ha"], spec["c"], p["Fx"], tau, tau)
    else:
        ua, ba = profiles.couette(y, a, spec["ha"], 0.0, spec["c"], U_WALL, tau, tau)
    return profiles.rel_l2(u, ua), profiles.rel_l2(b, ba)


def run_batched(specs, storage="f32", tol=1e-10, check_every=100, quantum=20000, max_steps=10**9, shape=None,
                tune_candidates=None, time_budget=None, tail_shape=(128, 1, 8), tail_below=None):
    """Admit every instance into one batch and run persistent launches of `quantum` steps until
    none is running.  Returns per-instance records and the wall time.  An instance's
    time-to-steady is the wall time at the end of the launch in which it left RUNNING.

    Shape policy: the autotuned (or given) shape while many instances run; once fewer than
    `tail_below` (default: the number of SMs) remain, `tail_shape` -- clusters of CTAs on several
    SMs per instance -- so the last, longest instances advance faster per step."""
    import torch
    descs = [make_desc(s, tol, check_every, max_steps) for s in specs]
    pool = sum(_batch.instance_footprint(d, storage) for d in descs) + (1 << 20)
    b = _batch.Batch(storage, max_instances=len(descs), pool_bytes=pool,
                     threads_per_group=shape[0] if shape else 0, groups_per_cta=shape[1] if shape else 0,
                     cluster_ctas=shape[2] if shape and len(shape) > 2 else 0)
    slots = [b.add(d) for d in descs]
    tune = None
    if tune_candidates:
        best, secs = b.autotune(tune_candidates, probe_steps=200)
        tune = {"best": list(best), "seconds": secs, "candidates": [list(c) for c in tune_candidates]}
    if tail_below is None:
        tail_below = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_at = [None] * len(slots)
    running = len(slots)
    launches = 0
    tail_at = None
    while running:
        if tail_shape and tail_at is None and running < tail_below:
            b.set_shape(*tail_shape)
            tail_at = time.perf_counter() - t0
        running = b.run(quantum)
        launches += 1
        now = time.perf_counter() - t0
        for k, s in enumerate(slots):
            if done_at[k] is None and b.result(s)[0] != _batch.INST_RUNNING:
                done_at[k] = now
        if time_budget is not None and now > time_budget:
            break
    wall = time.perf_counter() - t0
    recs = []
    for k, (spec, s) in enumerate(zip(specs, slots)):
        st, steps, r = b.result(s)
        u, bx = b.profiles(s)
        eu, eb = analytic_error(spec, u, bx)
        recs.append({"index": spec["index"], "ny": spec["ny"], "ha": spec["ha"], "c": spec["c"], "kind": spec["kind"],
                     "state": _batch.STATE_NAMES[st], "steps": int(steps), "residual": r,
                     "t_done": done_at[k], "l2_u": eu, "l2_b": eb, "nodes": spec["nx"] * spec["ny"],
                     "u": u, "b": bx})
    b.close()
    return {"records": recs, "wall": wall, "launches": launches, "tune": tune, "tail_shape_at": tail_at}


def run_one_at_a_time(specs, storage="f64", tol=1e-10, check_every=100, max_steps=10**9, time_limit=None):
    """The baseline: for each instance in order, lks_create -> lks_set_walls -> lks_run_to_steady
    -> lks_moments -> lks_destroy on the same GPU.  Latency of instance k = sum of solve times
    up to k (first-in first-out, all present at t = 0).  time_limit: stop starting new instances
    after that many seconds (the records then cover the first instances only)."""
    import torch
    recs = []
    t0 = time.perf_counter()
    for spec in specs:
        if time_limit is not None and time.perf_counter() - t0 > time_limit:
            break
        p = lattice_params(spec)
        ts = time.perf_counter()
        lat = _lks.Lattice(spec["nx"], spec["ny"], TAU, TAU, p["B0"], p["Fx"], spec["closure"], storage)
        lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
        steps, r, status = lat.run_to_steady(tol, check_every, max_steps, raise_on_fail=False)
        u, bx = lat.profiles()
        lat.close()
        torch.cuda.synchronize()
        te = time.perf_counter()
        eu, eb = analytic_error(spec, u, bx)
        recs.append({"index": spec["index"], "steps": int(steps), "residual": r, "status": int(status),
                     "solve_s": te - ts, "t_done": te - t0, "l2_u": eu, "l2_b": eb, "u": u, "b": bx})
    return {"records": recs, "wall": time.perf_counter() - t0}


def run_mixed(specs, handoff_tol=1e-5, tol=1e-10, check_every=100, quantum=20000, max_steps=10**9,
              shape=None, time_budget=None, tail_shape=(128, 1, 8), tail_below=None):
    """The mixed-precision lane: every instance starts in an FP32 batch with tolerance handoff_tol;
    as soon as it leaves RUNNING there (converged at handoff_tol, or stalled at FP32's rounding floor)
    its state moves (lks_batch_get_state / lks_batch_set_state) into an FP64 batch that runs it to
    tol, a residual FP32 storage cannot certify, with what is left of its max_steps (the budget covers
    both phases).  The two batches' launches alternate on the GPU.
    Unstable instances and instances at max_steps end in the FP32 lane.  Time-to-steady of an instance
    is the wall time at the end of the FP64 launch in which it left RUNNING.

    Shape policy, per batch: `shape` (default 128 threads per instance, one instance per CTA) while
    the batch holds at least `tail_below` running instances (default: the number of SMs), else
    `tail_shape` -- each instance on a cluster of CTAs, so that few instances still occupy the GPU.
    Results do not depend on the shape."""
    import torch
    d32 = [make_desc(s, handoff_tol, check_every, max_steps) for s in specs]
    d64 = [make_desc(s, tol, check_every, max_steps) for s in specs]
    pool32 = sum(_batch.instance_footprint(d, "f32") for d in d32) + (1 << 20)
    pool64 = sum(_batch.instance_footprint(d, "f64") for d in d64) + (1 << 20)
    kw = {}
    if shape:
        kw = dict(threads_per_group=shape[0], groups_per_cta=shape[1], cluster_ctas=shape[2] if len(shape) > 2 else 0)
    b32 = _batch.Batch("f32", max_instances=len(specs), pool_bytes=pool32, **kw)
    b64 = _batch.Batch("f64", max_instances=len(specs), pool_bytes=pool64, **kw)
    base = tuple(shape[:3]) + (1,) * (3 - len(shape)) if shape else (128, 1, 1)
    if tail_below is None:
        tail_below = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    cur = {id(b32): base if shape else None, id(b64): base if shape else None}

    def fit_shape(b, running):
        want = tuple(tail_shape) if tail_shape and running < tail_below else base
        if cur[id(b)] != want:
            b.set_shape(*want)
            cur[id(b)] = want
    s32 = [b32.add(d) for d in d32]
    left32 = [False] * len(specs)  # the instance left the FP32 batch (moved on, or ended there)
    s64 = [None] * len(specs)
    steps32 = [0] * len(specs)
    state32 = [None] * len(specs)
    done_at = [None] * len(specs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    running32, running64, launches = len(specs), 0, 0
    while running32 or running64:
        if running32:
            fit_shape(b32, running32)
            running32 = b32.run(quantum)
            launches += 1
            for k, s in enumerate(s32):
                if s is None or left32[k]:
                    continue
                st, steps, r = b32.result(s)
                if st == _batch.INST_RUNNING:
                    continue
                left32[k] = True
                steps32[k], state32[k] = int(steps), _batch.STATE_NAMES[st]
                if st in (_batch.INST_CONVERGED, _batch.INST_STALLED) and steps < max_steps:
                    # the FP64 phase gets what is left of the instance's step budget
                    f, g = b32.get_state(s)
                    d64[k].max_steps = max_steps - int(steps)
                    s64[k] = b64.add(d64[k])
                    b64.set_state(s64[k], f, g)
                    b32.remove(s)
                    s32[k] = None
                else:
                    done_at[k] = time.perf_counter() - t0  # ends in the FP32 lane
        fit_shape(b64, sum(1 for k, s in enumerate(s64) if s is not None and done_at[k] is None))
        running64 = b64.run(quantum)
        launches += 1
        now = time.perf_counter() - t0
        for k, s in enumerate(s64):
            if s is not None and done_at[k] is None and b64.result(s)[0] != _batch.INST_RUNNING:
                done_at[k] = now
        running64 = sum(1 for k, s in enumerate(s64) if s is not None and done_at[k] is None)
        if time_budget is not None and now > time_budget:
            break
    wall = time.perf_counter() - t0
    recs = []
    for k, spec in enumerate(specs):
        if s64[k] is not None:
            st, steps, r = b64.result(s64[k])
            u, bx = b64.profiles(s64[k])
            state, steps64 = _batch.STATE_NAMES[st], int(steps)
        else:
            st, steps, r = b32.result(s32[k])
            u, bx = b32.profiles(s32[k])
            state, steps64 = "fp32_" + _batch.STATE_NAMES[st], 0
            steps32[k] = int(steps)
        eu, eb = analytic_error(spec, u, bx)
        recs.append({"index": spec["index"], "ny": spec["ny"], "ha": spec["ha"], "c": spec["c"], "kind": spec["kind"],
                     "state": state, "fp32_state": state32[k], "steps_fp32": steps32[k], "steps_fp64": steps64,
                     "residual": r, "t_done": done_at[k], "l2_u": eu, "l2_b": eb,
                     "nodes": spec["nx"] * spec["ny"], "u": u, "b": bx})
    b32.close()
    b64.close()
    return {"records": recs, "wall": wall, "launches": launches}

"""Continuous-batching solve server for channel requests.

Requests (one channel problem each: size, Ha, c, forcing kind) arrive over time.  Two lanes share
the GPU:

- small lane: requests of at most `small_max_nodes` nodes are admitted into one lks_batch pool
  (admission by device-memory footprint and free slots, done natively by lks_batch_add) and
  advanced together by persistent launches of `quantum` steps; a request that arrives while others
  are on the GPU joins at the next launch, and a finished one leaves the pool at once;
- large lane: bigger requests each run as their own lattice (lks_create / lks_run_to_steady with
  CUDA-graph stepping) on their own CUDA stream in a worker thread, up to `large_workers` at a
  time, admitted while the large-lane share of the memory budget allows.

Every result is the same as the request solved alone: the per-node update and the per-instance
residual reduction do not depend on what else is resident.

FP64 finish (finish_tol set): the lanes run in the server's storage type (FP32) only to a hand-off
residual `finish_tol` (or until they stall at FP32's rounding floor), then continue in FP64 to `tol`,
a residual FP32 cannot certify: small-lane instances move into a second, FP64 batch
(lks_batch_get_state / lks_batch_set_state), large-lane lattices are replaced by an FP64 lattice
with the same state (lks_get_state / lks_set_state).  max_steps is the request's whole budget: the
FP64 phase gets what the FP32 phase left.

Failure handling (all on the host): a request the library rejects (LKS_EINVAL) is recorded as
"rejected" and the server continues; an exception while solving a large-lane request is recorded
as "error" and its stream and memory share are released; a request can be cancelled while queued
or while in the small lane (its pool memory is freed at once) -- a large-lane request that is
already solving finishes and is then reported as "cancelled".
"""
import collections
import concurrent.futures
import math
import threading
import time

import numpy as np

from . import batch as _batch
from . import lks as _lks
from . import sweep as _sweep

TAU = _sweep.TAU


def _finish_fp64(lat32, req, stream, tol, check_every, max_steps):
    """Continue a lattice's state in FP64 to tol (at most max_steps more steps): lks_get_state ->
    FP64 lattice -> lks_set_state."""
    f, g = lat32.get_state()
    lat32.close()
    lat = _default_lattice(req, "f64", stream)
    try:
        lat.set_state(f, g)
        steps, r, status = lat.run_to_steady(tol, check_every, max_steps, raise_on_fail=False)
        u, b = lat.profiles()
    finally:
        lat.close()
    return steps, r, status, u, b


def _default_lattice(req, storage, stream, inplace=False):
    p = _sweep.lattice_params(req)
    lat = _lks.Lattice(req["nx"], req["ny"], TAU, TAU, p["B0"], p["Fx"], req["closure"], storage, stream=stream,
                       inplace=inplace)
    lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
    return lat


class Server:
    def __init__(self, storage="f32", budget_bytes=120 << 30, small_pool_bytes=8 << 30, small_max_nodes=32768,
                 max_small=8192, large_workers=6, tol=1e-9, check_every=100, quantum=2000, max_steps=10**9,
                 shape=None, batch=None, lattice_factory=None, streams=None, inplace=False, finish_tol=None,
                 tail_shape=(128, 1, 8), tail_below=None):
        """inplace=True: every request keeps one population buffer (in-place pairs of steps, same
        results), so the memory budget admits about twice the requests; quantum, check_every and
        max_steps must then be even.  finish_tol: hand-off residual of the FP64 finish (None: off).
        Shape policy of the small lane's batches: `shape` (default 256 threads per instance, one
        instance per CTA) while a batch holds at least `tail_below` requests (default: the number of
        SMs), else `tail_shape` (each request on a cluster of CTAs; None: never).  A batch passed
        in as `batch` keeps the shape its caller gave it.  Results do not depend on the shape."""
        self.storage = storage
        self.inplace = bool(inplace)
        self.tol, self.check_every, self.quantum, self.max_steps = tol, check_every, quantum, max_steps
        self.finish_tol = finish_tol
        self.small_max_nodes = small_max_nodes
        small_pool_bytes = min(small_pool_bytes, budget_bytes // (4 if finish_tol else 2))
        self.large_budget = budget_bytes - small_pool_bytes * (2 if finish_tol else 1)
        self.large_used = 0
        self.batch64 = None
        self.small64 = {}  # FP64-batch slot -> request record
        if finish_tol:
            self.batch64 = _batch.Batch("f64", max_instances=max_small, pool_bytes=small_pool_bytes,
                                        threads_per_group=shape[0] if shape else 0,
                                        groups_per_cta=shape[1] if shape else 0,
                                        cluster_ctas=shape[2] if shape and len(shape) > 2 else 0)
        self._own_batch = batch is None
        if batch is None:
            batch = _batch.Batch(storage, max_instances=max_small, pool_bytes=small_pool_bytes,
                                 threads_per_group=shape[0] if shape else 0, groups_per_cta=shape[1] if shape else 0,
                                 cluster_ctas=shape[2] if shape and len(shape) > 2 else 0, inplace=inplace)
        self.batch = batch
        self.base_shape = (tuple(shape[:3]) + (1,) * (3 - len(shape))) if shape else (256, 1, 1)
        self.tail_shape = tuple(tail_shape) if tail_shape else None
        self.tail_below = tail_below  # None: the number of SMs, looked up at first use
        self._shape = {}  # id(batch) -> the shape last set (absent: base_shape, as the batch was created)
        self.lattice_factory = lattice_factory or (
            lambda req, stream: _default_lattice(req, storage, stream, inplace))
        if streams is None:
            import torch
            streams = [torch.cuda.Stream() for _ in range(large_workers)]
        self.streams = streams
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=large_workers)
        self.large_workers = large_workers
        self.large_active = {}
        self.free_streams = list(range(large_workers))
        self.small_slots = {}  # slot -> request record
        self.cancelled = set()

    def is_small(self, req):
        return req["nx"] * req["ny"] <= self.small_max_nodes

    def footprint(self, req):
        d = _sweep.make_desc(req, self.tol, self.check_every, self.max_steps)
        if self.is_small(req):
            return _batch.instance_footprint(d, self.storage, self.inplace)
        fp = _lks.footprint_bytes(req["nx"], req["ny"], req["closure"], self.storage, inplace=self.inplace)
        if self.finish_tol:  # the FP64 lattice replaces the first one: the larger of the two
            fp = max(fp, _lks.footprint_bytes(req["nx"], req["ny"], req["closure"], "f64"))
        return fp

    # -- small lane ------------------------------------------------------------------------
    def try_admit_small(self, req, now, out):
        """True when the request left the queue (admitted or rejected), False when it must wait."""
        d = _sweep.make_desc(req, self.finish_tol or self.tol, self.check_every, self.max_steps)
        try:
            slot = self.batch.add(d)
        except _lks.LksError as e:
            out.append({"req": req, "t_admit": now, "lane": "small", "state": "rejected", "error": str(e),
                        "steps": 0, "residual": math.inf, "t_done": now, "u": None, "b": None})
            return True
        if slot is None:
            return False
        self.small_slots[slot] = {"req": req, "t_admit": now, "lane": "small"}
        return True

    def collect_small(self, now, out):
        for slot in list(self.small_slots):
            rec = self.small_slots[slot]
            if rec["req"]["index"] in self.cancelled:
                self.batch.remove(slot)
                del self.small_slots[slot]
                rec.update({"state": "cancelled", "steps": 0, "residual": math.inf, "t_done": now, "u": None,
                            "b": None})
                out.append(rec)
                continue
            st, steps, r = self.batch.result(slot)
            if st == _batch.INST_RUNNING:
                continue
            if self.batch64 is not None and st in (_batch.INST_CONVERGED, _batch.INST_STALLED) \
                    and steps < self.max_steps:
                # hand the state over to the FP64 batch with what is left of the step budget; wait
                # there for a slot and memory
                left = self.max_steps - int(steps)
                if self.inplace:
                    left -= left & 1
                d = _sweep.make_desc(rec["req"], self.tol, self.check_every, left)
                s64 = self.batch64.add(d)
                if s64 is None:
                    continue
                self.batch64.set_state(s64, *self.batch.get_state(slot))
                self.batch.remove(slot)
                del self.small_slots[slot]
                rec["steps_fp32"] = int(steps)
                self.small64[s64] = rec
                continue
            del self.small_slots[slot]
            u, b = self.batch.profiles(slot)
            self.batch.remove(slot)
            rec.update({"state": _batch.STATE_NAMES[st], "steps": int(steps), "residual": r, "t_done": now,
                        "u": u, "b": b})
            out.append(rec)
        for slot in list(self.small64):
            st, steps, r = self.batch64.result(slot)
            if st == _batch.INST_RUNNING:
                continue
            rec = self.small64.pop(slot)
            u, b = self.batch64.profiles(slot)
            self.batch64.remove(slot)
            rec.update({"state": _batch.STATE_NAMES[st], "steps": rec["steps_fp32"] + int(steps), "residual": r,
                        "t_done": now, "u": u, "b": b})
            out.append(rec)

    # -- large lane ------------------------------------------------------------------------
    def _solve_large(self, req, sidx):
        lat = self.lattice_factory(req, self.streams[sidx])
        try:
            if self.finish_tol:
                steps, r, status = lat.run_to_steady(self.finish_tol, self.check_every, self.max_steps,
                                                     raise_on_fail=False)
                if status in (_lks.LKS_OK, _lks.LKS_ESTALLED) and steps < self.max_steps:
                    # the FP64 phase gets what is left of the request's step budget
                    s64, r, status, u, b = _finish_fp64(lat, req, self.streams[sidx], self.tol, self.check_every,
                                                        self.max_steps - steps)
                    steps += s64
                else:
                    u, b = lat.profiles()
            else:
                steps, r, status = lat.run_to_steady(self.tol, self.check_every, self.max_steps,
                                                     raise_on_fail=False)
                u, b = lat.profiles()
        finally:
            lat.close()
        state = {_lks.LKS_OK: "converged", _lks.LKS_ENOTCONVERGED: "max_steps", _lks.LKS_ESTALLED: "stalled",
                 _lks.LKS_EUNSTABLE: "unstable"}.get(status, "error")
        return {"state": state, "steps": int(steps), "residual": r, "u": u, "b": b}

    def try_admit_large(self, req, now, out):
        fp = self.footprint(req)
        if fp == 0:
            out.append({"req": req, "t_admit": now, "lane": "large", "state": "rejected",
                        "error": "invalid parameters", "steps": 0, "residual": math.inf, "t_done": now,
                        "u": None, "b": None})
            return True
        if not self.free_streams or self.large_used + fp > self.large_budget:
            return False
        sidx = self.free_streams.pop()
        self.large_used += fp
        fut = self.pool.submit(self._solve_large, req, sidx)
        self.large_active[fut] = ({"req": req, "t_admit": now, "lane": "large"}, sidx, fp)
        return True

    def collect_large(self, now, out):
        for fut in [f for f in self.large_active if f.done()]:
            rec, sidx, fp = self.large_active.pop(fut)
            try:
                rec.update(fut.result())
            except Exception as e:  # the lattice could not be created or solved
                rec.update({"state": "error", "error": "%s: %s" % (type(e).__name__, e), "steps": 0,
                            "residual": math.inf, "u": None, "b": None})
            if rec["req"]["index"] in self.cancelled:
                rec["state"] = "cancelled"
            rec["t_done"] = now
            self.large_used -= fp
            self.free_streams.append(sidx)
            out.append(rec)

    def cancel(self, index):
        """Cancel request `index` (queued, in the small lane, or -- reported only -- in the large lane)."""
        self.cancelled.add(index)

    # -- the loop ----------------------------------------------------------------------------
    def serve(self, trace, time_limit=None):
        """Replay a trace (requests with t_arrival in seconds, sorted; optional `cancel_after` seconds).
        Returns one record per request with arrival, admission and completion times (seconds from
        the start) and its state."""
        t0 = time.perf_counter()
        q_small, q_large = collections.deque(), collections.deque()
        out = []
        i = 0
        n = len(trace)
        while len(out) < n:
            now = time.perf_counter() - t0
            while i < n and trace[i]["t_arrival"] <= now:
                (q_small if self.is_small(trace[i]) else q_large).append(trace[i])
                i += 1
            for req in trace[:i]:
                ca = req.get("cancel_after")
                if ca is not None and now >= req["t_arrival"] + ca:
                    self.cancel(req["index"])
            for q in (q_small, q_large):
                for req in [r for r in q if r["index"] in self.cancelled]:
                    q.remove(req)
                    out.append({"req": req, "t_admit": None, "lane": "queue", "state": "cancelled", "steps": 0,
                                "residual": math.inf, "t_done": now, "u": None, "b": None})
            while q_small and self.try_admit_small(q_small[0], now, out):
                q_small.popleft()
            while q_large and self.try_admit_large(q_large[0], now, out):
                q_large.popleft()
            if self.small_slots or self.small64:
                if self.small_slots:
                    self._fit_shape(self.batch, len(self.small_slots))
                    self.batch.run(self.quantum)
                if self.small64:
                    self._fit_shape(self.batch64, len(self.small64))
                    self.batch64.run(self.quantum)
            else:
                time.sleep(0.0005)
            now = time.perf_counter() - t0
            self.collect_small(now, out)
            self.collect_large(now, out)
            if time_limit is not None and now > time_limit:
                break
        for rec in out:
            rec["t_arrival"] = rec["req"]["t_arrival"]
            rec["latency"] = rec["t_done"] - rec["t_arrival"]
        return out

    def _fit_shape(self, b, n):
        """Clusters of CTAs per request while the batch holds fewer than tail_below requests."""
        if b is self.batch and not self._own_batch:
            return
        if self.tail_below is None:
            import torch
            self.tail_below = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        want = self.tail_shape if self.tail_shape and n < self.tail_below else self.base_shape
        if self._shape.get(id(b), self.base_shape) != want:
            b.set_shape(*want)
            self._shape[id(b)] = want

    def close(self):
        self.pool.shutdown(wait=True)
        self.batch.close()
        if self.batch64 is not None:
            self.batch64.close()


def serve_one_at_a_time(trace, storage="f64", tol=1e-9, check_every=100, max_steps=10**9, time_limit=None):
    """Baseline: the same trace solved first-in first-out, one request at a time, through
    lks_create / lks_run_to_steady / lks_destroy."""
    import torch
    t0 = time.perf_counter()
    out = []
    for req in trace:
        now = time.perf_counter() - t0
        if now < req["t_arrival"]:
            time.sleep(req["t_arrival"] - now)
        p = _sweep.lattice_params(req)
        lat = _lks.Lattice(req["nx"], req["ny"], TAU, TAU, p["B0"], p["Fx"], req["closure"], storage)
        lat.set_walls(p["c_bottom"], p["c_top"], p["u_bottom"], p["u_top"])
        steps, r, status = lat.run_to_steady(tol, check_every, max_steps, raise_on_fail=False)
        u, b = lat.profiles()
        lat.close()
        torch.cuda.synchronize()
        t_done = time.perf_counter() - t0
        state = {_lks.LKS_OK: "converged", _lks.LKS_ENOTCONVERGED: "max_steps", _lks.LKS_ESTALLED: "stalled",
                 _lks.LKS_EUNSTABLE: "unstable"}.get(status, "error")
        out.append({"req": req, "t_arrival": req["t_arrival"], "t_done": t_done, "latency": t_done - req["t_arrival"],
                    "steps": int(steps), "residual": r, "status": int(status), "state": state, "u": u, "b": b})
        if time_limit is not None and t_done > time_limit:
            break
    return out


STEADY_STATES = ("converged", "stalled")


def summarize(records, n_offered):
    """Throughput and latency over the requests that finished.  `completed` counts every request
    the server ran to an end (steady state, its step cap, or instability); `steady` counts those
    that reached steady state (residual below tol, or stalled at the storage's rounding floor),
    with their own rate and latency percentiles."""
    done = [r for r in records if r.get("state") not in ("rejected", "cancelled", "error")]
    steady = [r for r in done if r.get("state") in STEADY_STATES]
    lat = np.array([r["latency"] for r in done]) if done else np.array([np.nan])
    lat_s = np.array([r["latency"] for r in steady]) if steady else np.array([np.nan])
    t_first = min(r["t_arrival"] for r in done) if done else 0.0
    t_last = max(r["t_done"] for r in done) if done else 0.0
    span = max(1e-9, t_last - t_first)
    states = collections.Counter(r.get("state", "done") for r in records)
    return {"offered": n_offered, "completed": len(done),
            "solves_per_s": len(done) / span,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "steady": len(steady), "steady_per_s": len(steady) / span,
            "steady_latency_p50_s": float(np.percentile(lat_s, 50)),
            "steady_latency_p99_s": float(np.percentile(lat_s, 99)),
            "makespan_s": t_last - t_first, "states": dict(states)}

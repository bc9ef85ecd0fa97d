"""Host-side scheduling and failure handling of the serving loop, with fake lanes (no GPU):
FIFO admission under a full pool, a rejected (malformed) request, cancellation while queued or
running, a large-lane request whose solver raises, and the large lane's memory budget."""
import math
import threading
import time

import numpy as np
import pytest

from paper_2112_13930_gb300 import batch as B
from paper_2112_13930_gb300 import build, lks, serve


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lks.load()


class FakeBatch:
    """Stands in for lks_batch: `capacity` slots; an instance finishes after 10*ny steps."""

    def __init__(self, capacity):
        self.capacity = capacity
        self.slots = {}
        self.removed = []

    def add(self, desc):
        if desc.closure == lks.MOMENT and desc.ny < 3:
            raise lks.LksError(lks.LKS_EINVAL, "ny must be >= 3 for the moment-based closure")
        if len(self.slots) >= self.capacity:
            return None
        slot = min(set(range(self.capacity)) - set(self.slots))
        self.slots[slot] = {"ny": desc.ny, "steps": 0}
        return slot

    def run(self, quantum):
        for s in self.slots.values():
            s["steps"] = min(s["steps"] + quantum, 10 * s["ny"])
        return sum(1 for s in self.slots.values() if s["steps"] < 10 * s["ny"])

    def result(self, slot):
        s = self.slots[slot]
        done = s["steps"] >= 10 * s["ny"]
        return (B.INST_CONVERGED if done else B.INST_RUNNING), s["steps"], (1e-12 if done else 1.0)

    def profiles(self, slot):
        ny = self.slots[slot]["ny"]
        return np.zeros(ny), np.zeros(ny)

    def remove(self, slot):
        del self.slots[slot]
        self.removed.append(slot)

    def close(self):
        pass


class FakeLattice:
    active = 0
    peak = 0
    lock = threading.Lock()

    def __init__(self, req, stream):
        if req.get("fail"):
            raise lks.LksError(lks.LKS_ENOMEM, "cudaMalloc failed (injected)")
        self.ny = req["ny"]
        with FakeLattice.lock:
            FakeLattice.active += 1
            FakeLattice.peak = max(FakeLattice.peak, FakeLattice.active)

    def run_to_steady(self, tol, check_every, max_steps, raise_on_fail=True):
        time.sleep(0.02)
        return 100, 1e-12, lks.LKS_OK

    def profiles(self):
        return np.zeros(self.ny), np.zeros(self.ny)

    def close(self):
        with FakeLattice.lock:
            FakeLattice.active -= 1


def _req(i, t=0.0, nx=4, ny=40, closure="moment", **kw):
    r = {"index": i, "t_arrival": t, "nx": nx, "ny": ny, "ha": 5.0, "c": 0.5, "kind": "shear", "closure": closure}
    r.update(kw)
    return r


def _server(capacity=2, workers=2, budget=1 << 30, small_max_nodes=1000):
    FakeLattice.active = FakeLattice.peak = 0
    return serve.Server("f32", budget_bytes=budget, small_pool_bytes=budget // 2, small_max_nodes=small_max_nodes,
                        large_workers=workers, tol=1e-9, quantum=100, batch=FakeBatch(capacity),
                        lattice_factory=FakeLattice, streams=[None] * workers)


def test_fifo_admission_waits_for_capacity():
    srv = _server(capacity=1)
    trace = [_req(i, ny=30 + i) for i in range(4)]
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    assert [r["state"] for r in recs] == ["converged"] * 4
    by = {r["req"]["index"]: r for r in recs}
    for i in range(1, 4):
        assert by[i]["t_admit"] >= by[i - 1]["t_done"] - 1e-9


def test_rejected_request_does_not_stop_the_server():
    srv = _server(capacity=2)
    trace = [_req(0), _req(1, ny=2), _req(2)]
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    states = {r["req"]["index"]: r["state"] for r in recs}
    assert states == {0: "converged", 1: "rejected", 2: "converged"}


def test_cancel_queued_and_running():
    srv = _server(capacity=1, small_max_nodes=10**8)
    trace = [_req(0, ny=10**6, cancel_after=0.05),      # would run for ages: cancelled while running
             _req(1, ny=30, cancel_after=0.0),          # cancelled while still queued
             _req(2, ny=30)]
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    states = {r["req"]["index"]: r for r in recs}
    assert states[0]["state"] == "cancelled" and states[0]["lane"] == "small"
    assert states[1]["state"] == "cancelled" and states[1]["t_admit"] is None
    assert states[2]["state"] == "converged"
    assert srv.batch.slots == {}


def test_large_lane_failure_is_contained():
    srv = _server(workers=2, small_max_nodes=10)
    trace = [_req(0, nx=256, ny=64), _req(1, nx=256, ny=64, fail=True), _req(2, nx=256, ny=64)]
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    states = {r["req"]["index"]: r["state"] for r in recs}
    assert states == {0: "converged", 1: "error", 2: "converged"}
    assert "injected" in [r for r in recs if r["req"]["index"] == 1][0]["error"]
    assert sorted(srv.free_streams) == [0, 1] and srv.large_used == 0


def test_large_lane_memory_budget_serialises():
    one = lks.footprint_bytes(256, 64, "moment", "f32")
    srv = _server(workers=4, small_max_nodes=10, budget=2 * (one + 1024))
    trace = [_req(i, nx=256, ny=64) for i in range(4)]
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    assert all(r["state"] == "converged" for r in recs)
    assert FakeLattice.peak == 1          # the large-lane share holds one lattice at a time


class ShapedFakeBatch(FakeBatch):
    """FakeBatch that the server creates itself (it stands in for batch.Batch) and that records
    every shape the server sets."""
    made = []

    def __init__(self, storage, max_instances, pool_bytes, threads_per_group=0, groups_per_cta=0, cluster_ctas=0,
                 inplace=False, **kw):
        super().__init__(max_instances)
        self.shapes = []
        ShapedFakeBatch.made.append(self)

    def set_shape(self, threads_per_group, groups_per_cta, cluster_ctas=1):
        self.shapes.append(((threads_per_group, groups_per_cta, cluster_ctas), len(self.slots)))


def test_small_lane_moves_to_clusters_below_tail(monkeypatch):
    """The server's own small-lane batch keeps its base shape while it holds tail_below or more
    requests and moves to tail_shape (clusters of CTAs) once fewer remain; a batch handed in by
    the caller is never reshaped."""
    ShapedFakeBatch.made = []
    monkeypatch.setattr(serve._batch, "Batch", ShapedFakeBatch)
    FakeLattice.active = FakeLattice.peak = 0
    trace = [_req(i, ny=30 + 10 * i) for i in range(5)]   # done after 300, 400, ..., 700 steps
    srv = serve.Server("f32", budget_bytes=1 << 30, small_pool_bytes=1 << 29, small_max_nodes=1000, max_small=8,
                       large_workers=1, tol=1e-9, quantum=100, lattice_factory=FakeLattice, streams=[None],
                       shape=(64, 2), tail_shape=(128, 1, 8), tail_below=3)
    recs = srv.serve(trace, time_limit=30)
    srv.close()
    assert sorted(r["state"] for r in recs) == ["converged"] * 5
    assert len(ShapedFakeBatch.made) == 1
    # 5, 4, 3 resident: the base shape (64, 2, 1), set at creation; 2 resident: the clusters, once
    assert ShapedFakeBatch.made[0].shapes == [((128, 1, 8), 2)]

    given = ShapedFakeBatch("f32", 8, 1 << 29)
    srv = serve.Server("f32", budget_bytes=1 << 30, small_pool_bytes=1 << 29, small_max_nodes=1000, max_small=8,
                       large_workers=1, tol=1e-9, quantum=100, lattice_factory=FakeLattice, streams=[None],
                       batch=given, tail_shape=(128, 1, 8), tail_below=3)
    recs = srv.serve([_req(i, ny=30 + 10 * i) for i in range(5)], time_limit=30)
    srv.close()
    assert sorted(r["state"] for r in recs) == ["converged"] * 5
    assert given.shapes == []

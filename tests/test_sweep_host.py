"""Host-side bookkeeping of the mixed-precision lane (sweep.run_mixed) with fake batches (no GPU):
hand-offs carry what is left of each instance's step budget, an instance that ends in the FP32
lane keeps the time of the launch in which it ended, and each batch moves to clusters of CTAs
once it holds fewer running instances than tail_below."""
import types

import numpy as np
import pytest

from paper_2112_13930_gb300 import batch as B
from paper_2112_13930_gb300 import build, lks, sweep


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()   # instance_footprint is computed by the library (host code, no device work)
    lks.load()


class Clock:
    """Stands in for the time module: one second per batch launch."""

    def __init__(self):
        self.t = 0.0

    def perf_counter(self):
        return self.t


class FakeBatch:
    """Stands in for lks_batch.  An instance needs 10 ny steps to reach the hand-off residual in the
    FP32 batch and 4 ny more in the FP64 batch; an instance with ny = 37 turns unstable in its first
    FP32 launch.  Every run() is one second of the clock."""

    made = {}
    clock = None

    def __init__(self, storage, max_instances, pool_bytes, **kw):
        self.storage = storage
        self.inst = {}
        self.shapes = []
        FakeBatch.made[storage] = self

    def set_shape(self, *shape):
        self.shapes.append((tuple(shape), sum(1 for i in self.inst.values() if i["state"] == B.INST_RUNNING)))

    def add(self, d):
        slot = len(self.inst)
        self.inst[slot] = {"ny": d.ny, "cap": d.max_steps, "steps": 0, "state": B.INST_RUNNING, "set": False}
        return slot

    def run(self, quantum):
        for i in self.inst.values():
            if i["state"] != B.INST_RUNNING:
                continue
            if self.storage == "f32" and i["ny"] == 37:
                i["steps"], i["state"] = quantum, B.INST_UNSTABLE
                continue
            need = (10 if self.storage == "f32" else 4) * i["ny"]
            i["steps"] = min(i["steps"] + quantum, need, i["cap"])
            if i["steps"] >= need:
                i["state"] = B.INST_CONVERGED
            elif i["steps"] >= i["cap"]:
                i["state"] = B.INST_MAX_STEPS
        FakeBatch.clock.t += 1.0
        return sum(1 for i in self.inst.values() if i["state"] == B.INST_RUNNING)

    def result(self, slot):
        i = self.inst[slot]
        return i["state"], i["steps"], 1e-12

    def get_state(self, slot):
        return np.zeros(1), np.zeros(1)

    def set_state(self, slot, f, g):
        self.inst[slot]["set"] = True

    def remove(self, slot):
        self.inst[slot]["state"] = "removed"

    def profiles(self, slot):
        ny = self.inst[slot]["ny"]
        return np.full(ny, 1e-3), np.full(ny, 1e-4)

    def close(self):
        pass


def test_mixed_lane_bookkeeping(monkeypatch):
    import torch
    clock = Clock()
    FakeBatch.clock, FakeBatch.made = clock, {}
    monkeypatch.setattr(sweep, "time", types.SimpleNamespace(perf_counter=clock.perf_counter))
    monkeypatch.setattr(sweep._batch, "Batch", FakeBatch)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    # ny 40: hand-off after 400 steps, FP64 done 160 later; ny 37: unstable at once; ny 90: reaches
    # the 1000-step budget in FP32 (needs 900 to hand off, then 360 in FP64 with 100 left: capped);
    # ny 200: the budget runs out in FP32
    specs = [{"index": k, "nx": 4, "ny": ny, "ha": 2.0, "c": 0.5, "kind": "body", "closure": "link"}
             for k, ny in enumerate((40, 37, 90, 200))]
    out = sweep.run_mixed(specs, handoff_tol=1e-5, tol=1e-10, check_every=100, quantum=100, max_steps=1000,
                          shape=(128, 1, 1), tail_shape=(128, 1, 8), tail_below=3)
    r = {rec["ny"]: rec for rec in out["records"]}

    assert r[40]["state"] == "converged" and r[40]["fp32_state"] == "converged"
    assert (r[40]["steps_fp32"], r[40]["steps_fp64"]) == (400, 160)
    assert r[37]["state"] == "fp32_unstable" and r[37]["steps_fp64"] == 0
    assert r[90]["state"] == "max_steps" and (r[90]["steps_fp32"], r[90]["steps_fp64"]) == (900, 100)
    assert r[200]["state"] == "fp32_max_steps" and r[200]["steps_fp32"] == 1000

    f32, f64 = FakeBatch.made["f32"], FakeBatch.made["f64"]
    # the FP64 phase was given what the FP32 phase left of the 1000-step budget, and the state
    assert f64.inst[0]["cap"] == 600 and f64.inst[1]["cap"] == 100
    assert f64.inst[0]["set"] and f64.inst[1]["set"]
    # the unstable instance ended in the first FP32 launch (clock 1): its time stays 1, although
    # the FP32 batch kept running for 9 more launches
    assert r[37]["t_done"] == 1.0
    # an FP32 instance that ends at its budget keeps the time of that launch: the 10th FP32 launch,
    # at clock 19
    assert r[200]["t_done"] == 19.0
    # each loop is one FP32 launch (odd clock) and one FP64 launch (even clock): the ny 40 instance
    # handed off after FP32 launch 4 (clock 7), and its 160 FP64 steps took FP64 launches 4 and 5
    # (clocks 8 and 10)
    assert r[40]["t_done"] == 10.0
    assert all(0.0 < rec["t_done"] <= out["wall"] for rec in out["records"])
    # each batch's shape: the base while it held 3 or more running instances, then clusters
    assert f32.shapes == [((128, 1, 8), 2)]
    assert f64.shapes and f64.shapes[0][0] == (128, 1, 8)

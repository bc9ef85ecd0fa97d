"""Benchmark of the fused LKS-MHD collide-stream step on GB300.

Default workload (one "step" = one time step of the whole lattice: pull-stream, wall closures,
moments, equilibria, collision and store in one fused kernel): shear-driven Hartmann-Couette channel, 4096 x 4096 nodes, periodic in x,
moment-based Shercliff closure on both walls (c = 1), top wall at U_w = 0.05, Ha = 20,
tau_f = tau_m = 0.8, rest start, FP32 deviation storage.  Inputs (2.5 GB of populations) are far
larger than the 129 MB L2, so no flush is needed between steps.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the host cores instead.
Multi-GPU runs (torchrun) are independent replicas, one lattice per GPU (the path does not shard).
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS (f+g)"
UNIT = "MLUPS"
BYTES_PER_NODE = {"f64": 304, "f32": 152, "bf16": 76, "f16": 76}


def _workload(args):
    n = args.n
    return {
        "workload": "Hartmann-Couette %dx%d, moment-based closure, U_w=0.05, Ha=20, c=1 both walls, "
                    "tau_f=tau_m=0.8, rest start" % (n, n),
        "nx": n, "ny": n, "closure": "moment", "storage": args.storage,
        "buffers": "one, in place (pairs of steps)" if getattr(args, "inplace", False) else "two (ping-pong)",
        "l2": "inputs larger than L2 (%.2f GB of populations read per step vs 129 MB L2)"
              % (BYTES_PER_NODE[args.storage] / 2 * n * n / 1e9),
    }


def _physics(n):
    a = (n - 1) / 2
    nu = eta = (0.8 - 0.5) / 3
    b0 = 20.0 * math.sqrt(nu * eta) / a
    return dict(tau_f=0.8, tau_m=0.8, B0=b0, Fx=0.0, c=1.0, u_w=0.05)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(text):
    """C++ source without comments and blank space, so that a comment edit does not change the hash."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _kernel_hash():
    """sha256 (first 16 hex digits) of the step kernel's code (lks_step.cu + lks_device.cuh, comments
    and spacing removed)."""
    h = hashlib.sha256()
    for rel in ("paper_2112_13930_gb300/csrc/lks_step.cu", "paper_2112_13930_gb300/csrc/lks_device.cuh"):
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _ncu_traffic(storage, n):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it was taken on
    the current kernel source (same hash) for this storage type; else None."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    for m in re.finditer(r"^traffic storage=(\w+) nodes=(\d+) kernel_hash=(\w+) dram_bytes=([0-9.eE+]+)$", text, re.M):
        st, nodes, kh, b = m.group(1), int(m.group(2)), m.group(3), float(m.group(4))
        if st == storage and kh == _kernel_hash():
            return b * (n * n) / nodes
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_oracle_sample(n, seconds, phys):
    """FP64 CPU oracle on the same lattice, as many whole steps as fit in about `seconds`."""
    import numpy as np
    import oracle
    o = oracle.Oracle(n, n, phys["tau_f"], phys["tau_m"], phys["B0"], phys["Fx"], oracle.MOMENT,
                      phys["c"], phys["c"], 0.0, phys["u_w"])
    o.step(1)  # warm-up (page-in)
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    mlups = n * n * steps / dt / 1e6
    cores = oracle.threads_used()
    out = {"value": round(mlups, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%d full steps of the %dx%d lattice (FP64, OpenMP over rows), %.1f s" % (steps, n, n, dt)}
    # the same oracle on one thread: whole steps for about half the budget (at least one)
    oracle.set_threads(1)
    try:
        s1, t0 = 0, time.perf_counter()
        while True:
            o.step(1)
            s1 += 1
            if time.perf_counter() - t0 >= seconds / 2:
                break
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    out["single_thread"] = {"value": round(n * n * s1 / dt1 / 1e6, 3), "unit": UNIT, "cores": 1,
                            "sample": "%d full steps of the %dx%d lattice, %.1f s" % (s1, n, n, dt1)}
    return out


def bench_reference(args):
    """The FP64 oracle on the host cores.  Each timed step is one oracle step over a bounded sample
    of the lattice: the full 4096-wide channel cut to r rows (walls included), r chosen so that the
    whole warm-up + timed run takes about --ref-seconds."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    phys = _physics(args.n)

    def make(rows):
        return oracle.Oracle(args.n, rows, phys["tau_f"], phys["tau_m"], phys["B0"], phys["Fx"], oracle.MOMENT,
                             phys["c"], phys["c"], 0.0, phys["u_w"])

    probe = make(256)
    probe.step(1)
    t0 = time.perf_counter()
    probe.step(1)
    t1 = time.perf_counter() - t0
    del probe
    per_step = args.ref_seconds / max(1, args.steps + args.warmup)
    rows = int(max(3, min(args.n, 256 * per_step / max(t1, 1e-6))))
    o = make(rows)
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    mlups = args.n * rows * args.steps / dt / 1e6
    cfg = _workload(args)
    cfg["storage"] = "f64"
    sample = "each step: one FP64 oracle step over %d x %d nodes of the %d x %d channel (walls included)" % (
        args.n, rows, args.n, args.n)
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": round(mlups, 3), "unit": UNIT, "cores": oracle.threads_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(mlups, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_max(x, world_size, device):
    """Max of a per-rank time over the process group (the slowest replica sets the job time)."""
    if world_size <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world_size, max_seconds):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank units in at
    most max_seconds."""
    return units_per_rank * world_size / max_seconds


def _time_steps(lat, steps, stream):
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    lat.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def bench_ours(args):
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    lks.load()
    n = args.n
    phys = _physics(n)
    stream = torch.cuda.current_stream()

    def make(storage, nn=n, inplace=False):
        lat = lks.Lattice(nn, nn, phys["tau_f"], phys["tau_m"], phys["B0"], phys["Fx"], "moment", storage,
                          inplace=inplace)
        lat.set_walls(phys["c"], phys["c"], 0.0, phys["u_w"])
        return lat

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return replica_max(x, ws, "cuda")

    # --- main measurement -------------------------------------------------------------------
    if args.inplace:  # in-place handles step in pairs
        args.steps += args.steps & 1
        args.warmup += args.warmup & 1
    lat = make(args.storage, inplace=args.inplace)
    lat.step(args.warmup)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    t = _time_steps(lat, args.steps, stream)
    barrier()
    clocks = sampler.stop()
    t = max_over_ranks(t)
    nodes = n * n
    value = replica_throughput(nodes * args.steps, ws, t) / 1e6
    per_launch = t / args.steps
    peak, peak_kind = _peaks()
    bpn = BYTES_PER_NODE[args.storage]
    achieved = bpn * nodes / per_launch / 1e9
    traffic = None if args.inplace else _ncu_traffic(args.storage, n)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured" else
                "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": bpn * nodes, "kernel": ("step_kernel_aa<%s,moment> (both phases)" if args.inplace else "step_kernel<%s,moment>")
                % args.storage}
    # sanity: the state must still be finite (lks_residual reports a non-finite state as LKS_EUNSTABLE)
    lat.residual()

    # --- end to end through the C ABI with host buffers -------------------------------------
    # The timed region: the state comes in from page-locked host memory (lks_set_state_raw: the
    # library's storage image, a bit-exact checkpoint), K steps run, and the result a caller of the
    # channel problem reads -- the x-averaged profiles rho, u_x, u_y, B_x, B_y(y) -- comes back to
    # the host.  The FP64 form of the same round trip (lks_set_state with absolute populations, per-
    # node moments out) is timed too and reported beside it.
    e2e = None
    if not args.skip_e2e:
        img = torch.empty(lat.state_bytes(), dtype=torch.uint8, pin_memory=True)
        lat.get_state_raw(img)              # a valid state to upload (taken outside the timed region)
        p_host = torch.empty((5, n), dtype=torch.float64, pin_memory=True).numpy()
        barrier()
        t0 = time.perf_counter()
        lat.set_state_raw(img)              # H2D from pinned host memory, the storage image
        lat.step(args.steps)
        lks._check(lks.load().lks_moments(lat._h, lks.MOMENTS_PROFILES, lks._dptr(p_host)), lat._h)  # D2H
        barrier()
        te = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": round(nodes * args.steps * ws / te / 1e6, 1), "unit": UNIT,
               "h2d_bytes_per_step": int(round(lat.state_bytes() / args.steps)),
               "d2h_bytes_per_step": int(round(5 * 8 * n / args.steps)),
               "timed": "lks_set_state_raw (the state's storage image, pinned host -> device) + lks_step(K) + "
                        "lks_moments (x-averaged profiles, device -> pinned host)"}
        # the FP64 form: absolute FP64 populations in (lks_set_state), per-node FP64 moments out
        f_host = torch.empty((9, n, n), dtype=torch.float64, pin_memory=True).numpy()
        g_host = torch.empty((2, 5, n, n), dtype=torch.float64, pin_memory=True).numpy()
        m_host = torch.empty((5, n, n), dtype=torch.float64, pin_memory=True).numpy()
        f0, g0 = lat.get_state()
        f_host[...] = f0
        g_host[...] = g0
        del f0, g0
        barrier()
        t0 = time.perf_counter()
        lat.set_state(f_host, g_host)       # H2D from pinned host memory + conversion
        lat.step(args.steps)
        lks._check(lks.load().lks_moments(lat._h, lks.MOMENTS_NODES, lks._dptr(m_host)), lat._h)  # D2H
        barrier()
        tf = max_over_ranks(time.perf_counter() - t0)
        e2e["fp64_state_and_node_moments"] = {
            "value": round(nodes * args.steps * ws / tf / 1e6, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(round(19 * 8 * nodes / args.steps)),
            "d2h_bytes_per_step": int(round(5 * 8 * nodes / args.steps)),
            "timed": "lks_set_state (FP64 host->device + conversion) + lks_step(K) + lks_moments (nodes)"}
        # the host transfers of both regions, each timed alone afterwards (best of 3, wall clock)
        ts = {"lks_set_state_raw": [], "lks_moments_profiles": [], "lks_set_state": [], "lks_moments_nodes": []}
        for _ in range(3):
            t1 = time.perf_counter()
            lat.set_state_raw(img)
            t2 = time.perf_counter()
            lks._check(lks.load().lks_moments(lat._h, lks.MOMENTS_PROFILES, lks._dptr(p_host)), lat._h)
            t3 = time.perf_counter()
            lat.set_state(f_host, g_host)
            t4 = time.perf_counter()
            lks._check(lks.load().lks_moments(lat._h, lks.MOMENTS_NODES, lks._dptr(m_host)), lat._h)
            t5 = time.perf_counter()
            for k, v in zip(ts, (t2 - t1, t3 - t2, t4 - t3, t5 - t4)):
                ts[k].append(v)
        e2e["breakdown_ms"] = {k: round(min(v) * 1e3, 2) for k, v in ts.items()}
        e2e["breakdown_ms"]["steps_at_device_rate"] = round(per_launch * args.steps * 1e3, 2)
        # the host link's own rate: a plain copy of the same pinned image into device memory (one
        # cudaMemcpyAsync, CUDA events, best of 3), beside the rate lks_set_state_raw reaches
        dev_img = torch.empty(img.numel(), dtype=torch.uint8, device="cuda")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_link = math.inf
        for _ in range(3):
            ev0.record()
            dev_img.copy_(img, non_blocking=True)
            ev1.record()
            ev1.synchronize()
            t_link = min(t_link, ev0.elapsed_time(ev1) / 1e3)
        e2e["host_link"] = {"h2d_gbs": round(img.numel() / t_link / 1e9, 1),
                            "lks_set_state_raw_gbs": round(img.numel() / min(ts["lks_set_state_raw"]) / 1e9, 1),
                            "what": "a plain copy of the pinned state image to device memory, against "
                                    "lks_set_state_raw of the same image (its snapshot pass and synchronisation included)"}
        del dev_img
        del f_host, g_host, m_host, img
    lat.close()
    del lat
    torch.cuda.empty_cache()

    # --- FP64 storage on the same workload (compute-bound on GB300's FP64 rate) --------------
    extra = {}
    if not args.skip_extra:
        k64 = max(10, min(args.steps, args.fp64_steps))
        l64 = make("f64")
        l64.step(3)
        barrier()
        t64 = max_over_ranks(_time_steps(l64, k64, stream))
        v64 = nodes * k64 * ws / t64 / 1e6
        a64 = 304 * nodes / (t64 / k64) / 1e9
        extra["fp64"] = {"value": round(v64, 1), "unit": UNIT, "steps": k64,
                         "roofline_hbm": {"achieved": round(a64, 1), "peak": peak, "unit": "GB/s",
                                          "frac": round(a64 / peak, 4)},
                         "roofline_alu": {"bound": "alu", "flops_per_node": FP64_FLOPS_PER_NODE,
                                          "achieved": round(FP64_FLOPS_PER_NODE * v64 * 1e6 / 1e12, 3),
                                          "peak": 1.25, "unit": "TFLOP/s",
                                          "frac": round(FP64_FLOPS_PER_NODE * v64 * 1e6 / 1.25e12, 4),
                                          "peak_source": "nominal GB300 FP64 rate"},
                         "roofline_fp64_pipe": {"bound": "fp64 pipe", "instr_per_node": FP64_PIPE_INSTR_PER_NODE,
                                                "achieved": round(FP64_PIPE_INSTR_PER_NODE * v64 * 1e6 / 1e12, 4),
                                                "peak": FP64_PIPE_PEAK / 1e12, "unit": "T FP64 instr/s",
                                                "frac": round(FP64_PIPE_INSTR_PER_NODE * v64 * 1e6 / FP64_PIPE_PEAK, 4),
                                                "source": "profiles/step_kernel_f64_2048sq_fp64_pipe.md"}}
        l64.close()
        del l64
        # the paper's own coupling (Lorentz force in the source), FP32, same workload
        ll = lks.Lattice(n, n, phys["tau_f"], phys["tau_m"], phys["B0"], phys["Fx"], "moment", "f32",
                         coupling="lorentz")
        ll.set_walls(phys["c"], phys["c"], 0.0, phys["u_w"])
        ll.step(3)
        barrier()
        kl = max(10, min(args.steps, 2000))
        tl = max_over_ranks(_time_steps(ll, kl, stream))
        vl = nodes * kl * ws / tl / 1e6
        al = 152 * nodes / (tl / kl) / 1e9
        extra["lorentz_f32"] = {"value": round(vl, 1), "unit": UNIT, "steps": kl,
                                "roofline": {"bound": "hbm", "achieved": round(al, 1), "peak": peak, "unit": "GB/s",
                                             "frac": round(al / peak, 4)}}
        ll.close()
        del ll
        # 16-bit deviation storage; then the in-place (one-buffer) step in FP32 and BF16
        for key, st, inplace in (("bf16", "bf16", False), ("f16", "f16", False), ("inplace_f32", "f32", True),
                                 ("inplace_bf16", "bf16", True)):
            lr = make(st, inplace=inplace)
            lr.step(4)
            barrier()
            kr = max(10, min(args.steps, 2000))
            kr += kr & 1
            tr = max_over_ranks(_time_steps(lr, kr, stream))
            vr = nodes * kr * ws / tr / 1e6
            ar = BYTES_PER_NODE[st] * nodes / (tr / kr) / 1e9
            extra[key] = {"value": round(vr, 1), "unit": UNIT, "steps": kr,
                          "roofline": {"bound": "hbm", "achieved": round(ar, 1), "peak": peak, "unit": "GB/s",
                                       "frac": round(ar / peak, 4)}}
            if inplace:
                extra[key]["footprint_bytes"] = lr.nbytes
            lr.close()
            del lr
        # three-dimensional channel (D3Q19 + 3 x D3Q7, link-based walls), FP32, 256^3
        from paper_2112_13930_gb300 import lks3d
        n3 = 256
        l3 = lks3d.Lattice3D(n3, n3, n3, phys["tau_f"], phys["tau_m"], 20.0 * 0.1 / (n3 / 2), 0.0, "f32")
        l3.set_walls(phys["c"], phys["c"], 0.0, phys["u_w"])
        l3.step(3)
        barrier()
        k3 = max(10, min(args.steps, 200))
        t3 = max_over_ranks(_time_steps(l3, k3, stream))
        nodes3 = n3 ** 3
        v3 = nodes3 * k3 * ws / t3 / 1e6
        a3 = 320 * nodes3 / (t3 / k3) / 1e9
        extra["d3q19_f32"] = {"value": round(v3, 1), "unit": UNIT, "steps": k3,
                              "config": "256^3, Hartmann-Couette, link-based walls c = 1, U_w = 0.05",
                              "roofline": {"bound": "hbm", "achieved": round(a3, 1), "peak": peak, "unit": "GB/s",
                                           "frac": round(a3 / peak, 4), "bytes_per_node": 320}}
        l3.close()
        del l3
        # the same channel with BF16 deviations (rows staged through shared memory by bulk copies)
        l3 = lks3d.Lattice3D(n3, n3, n3, phys["tau_f"], phys["tau_m"], 20.0 * 0.1 / (n3 / 2), 0.0, "bf16")
        l3.set_walls(phys["c"], phys["c"], 0.0, phys["u_w"])
        l3.step(3)
        barrier()
        t3 = max_over_ranks(_time_steps(l3, k3, stream))
        v3 = nodes3 * k3 * ws / t3 / 1e6
        a3 = 160 * nodes3 / (t3 / k3) / 1e9
        extra["d3q19_bf16"] = {"value": round(v3, 1), "unit": UNIT, "steps": k3,
                               "roofline": {"bound": "hbm", "achieved": round(a3, 1), "peak": peak, "unit": "GB/s",
                                            "frac": round(a3 / peak, 4), "bytes_per_node": 160}}
        l3.close()
        del l3
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.skip_cpu:
        cpu = run_oracle_sample(n, args.cpu_seconds, phys)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(per_launch * 1e3, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.storage != "f64" else "f64",
                "data": "synthetic", "config": _workload(args), "roofline": roofline, "cpu_baseline": cpu,
                "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks,
                "parallelism": "replicas" if ws > 1 else "single GPU"}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def bench_precision(args):
    """Reduced-precision storage: body-force Hartmann flow on 8192 x 8192 (Ha = 30, c = 0.5,
    tau = 0.8, seeded +-1e-3 velocity perturbation), link-based closure.  Reports MLUPS per storage
    type, the error of each storage type against the FP64 GPU run after 1000 steps (the FP64 path
    itself checked against the oracle on sampled rows after 2 steps), and the error against the
    analytic profile of a 4 x 513 channel of the same physics run to steady state."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    n = args.n if args.n != 4096 else 8192
    ha, c, tau = 30.0, 0.5, 0.8
    closure = "link"
    a = n / 2
    nu = (tau - 0.5) / 3
    b0 = ha * nu / a
    ustar0 = (1.0 / ha) * ((c + 1.0) / (ha * c + math.tanh(ha))) * (1.0 - 1.0 / math.cosh(ha))
    fx = 0.01 * nu / (a * a * ustar0)
    seed, amp = 20211227, 1e-3
    out = {"workload": "precision", "config": {"nx": n, "ny": n, "closure": closure, "Ha": ha, "c": c, "tau": tau,
                                               "B0": b0, "Fx": fx, "seed": seed, "perturb_amp": amp}}

    stream = torch.cuda.current_stream()
    steps_err = args.precision_steps

    def run(cl, b0c, fxc, check_oracle):
        """MLUPS per storage type and the error of each against the FP64 run after steps_err steps."""
        mlups, fields = {}, {}
        for st in ("f64", "f32", "f16", "bf16"):
            lat = lks.Lattice(n, n, tau, tau, b0c, fxc, cl, st, seed=seed, perturb_amp=amp)
            lat.set_walls(c, c)
            if st == "f64" and check_oracle and not args.skip_cpu:
                # parity of the FP64 path on sampled rows against the oracle (2 steps of the full lattice)
                import oracle
                o = oracle.Oracle(n, n, tau, tau, b0c, fxc, oracle.LINK if cl == "link" else oracle.MOMENT, c, c,
                                  seed=seed, perturb_amp=amp)
                t_or = time.perf_counter()
                o.step(2)
                t_or = time.perf_counter() - t_or
                out["oracle_host"] = {"kind": "oracle", "mlups": round(n * n * 2 / t_or / 1e6, 3),
                                      "cores": oracle.threads_used(),
                                      "sample": "2 FP64 oracle steps of the full %d x %d lattice (%.1f s)" % (n, n, t_or)}
                lat.step(2)
                mo = o.moments()
                mg = torch.empty((5, n, n), dtype=torch.float64, device="cuda")
                lat.moments_device(mg)
                rows = [0, 1, n // 3, n // 2, n - 2, n - 1]
                mgr = mg[:, rows, :].cpu().numpy()
                err = max(float(np.max(np.abs(mgr[m] - mo[m][rows])) / np.max(np.abs(mo[m][rows])))
                          for m in (1, 3))
                out["fp64_vs_oracle_2_steps_sampled_rows"] = err
                del o, mo, mg
                lat.close()
                lat = lks.Lattice(n, n, tau, tau, b0c, fxc, cl, st, seed=seed, perturb_amp=amp)
                lat.set_walls(c, c)
            k = 50 if st == "f64" else 200
            lat.step(5)
            t = _time_steps(lat, k, stream)
            mlups[st] = round(n * n * k / t / 1e6, 1)
            lat.step(steps_err - 5 - k)
            m = torch.empty((5, n, n), dtype=torch.float64, device="cuda")
            lat.moments_device(m)
            torch.cuda.synchronize()
            fields[st] = (m[1].clone(), m[3].clone())
            del m
            lat.close()
            torch.cuda.empty_cache()
        errs = {}
        u64, b64 = fields["f64"]
        for st in ("f32", "f16", "bf16"):
            u, b = fields[st]
            errs[st] = {"u_x_relmax": float((u - u64).abs().max() / u64.abs().max()),
                        "u_x_rel_rms": float(((u - u64) ** 2).mean().sqrt() / u64.abs().max()),
                        "B_x_relmax": float((b - b64).abs().max() / b64.abs().max()),
                        "B_x_rel_rms": float(((b - b64) ** 2).mean().sqrt() / b64.abs().max())}
        del fields
        torch.cuda.empty_cache()
        return mlups, errs

    mlups, errs = run(closure, b0, fx, True)
    # the same physics with the moment-based closure (walls on the node rows: a = (n - 1)/2)
    am = (n - 1) / 2
    b0m = ha * nu / am
    fxm = 0.01 * nu / (am * am * ustar0)
    mlups_m, errs_m = run("moment", b0m, fxm, False)
    out["moment"] = {"B0": b0m, "Fx": fxm, "mlups": mlups_m,
                     "error_vs_fp64_after_%d_steps" % steps_err: errs_m}
    # analytic comparison on a 4 x 513 channel of the same physics (Ha, c, tau, u_c = 0.01)
    ny = 513
    a2 = ny / 2
    b02 = ha * nu / a2
    fx2 = 0.01 * nu / (a2 * a2 * ustar0)
    y = -a2 + np.arange(ny) + 0.5
    xi = y / a2
    fac = (c + 1.0) / (ha * c + math.tanh(ha)) / ha
    ua = (a2 * a2 * fx2 / nu) * fac * (1.0 - np.cosh(ha * xi) / math.cosh(ha))
    ba = (a2 * a2 * fx2 / nu) * (-xi / ha + fac * np.sinh(ha * xi) / math.cosh(ha))
    analytic = {}
    for st in ("f64", "f32", "f16", "bf16"):
        lat = lks.Lattice(4, ny, tau, tau, b02, fx2, closure, st)
        lat.set_walls(c, c)
        steps, r, status = lat.run_to_steady(1e-9, 1000, args.precision_max_steps, raise_on_fail=False)
        u, b = lat.profiles()
        analytic[st] = {"steps": steps, "residual": r, "status": int(status),
                        "u_rel_l2": float(np.sqrt(np.mean((u - ua) ** 2)) / np.max(np.abs(ua))),
                        "B_rel_l2": float(np.sqrt(np.mean((b - ba) ** 2)) / np.max(np.abs(ba)))}
        lat.close()
    out.update({"mlups": mlups, "error_vs_fp64_after_%d_steps" % steps_err: errs,
                "analytic_4x513": analytic,
                "roofline_hbm_frac": {st: round(mlups[st] * 1e6 * BYTES_PER_NODE[st] / 1e9 / _peaks()[0], 4)
                                      for st in mlups}})
    print(json.dumps(out), flush=True)
    return 0


def bench_sweep(args):
    """Batched sweep: a seeded sample of the 4096-instance parameter-sweep set (nx = 4, ny in
    33..1025, Ha log-uniform in [1, 200], c log-uniform in [1e-3, 1e3] plus 5% each of 0 and inf,
    half body-force/link-based, half shear/moment-based), residual tolerance 1e-10.

    Arms: (1) the mixed-precision lane -- FP32 batch to a hand-off residual of 1e-5 (or its rounding
    floor), then each instance continued in an FP64 batch to 1e-10 -- the headline; (2) FP32 alone
    (stalls at its floor); (3) FP64 through the batched engine on the first instances; and, on the
    same first --sweep-baseline instances, (4) the mixed lane run on just those and (5) one-at-a-time
    FP64 solving through the single-lattice API, with p50/p99 time-to-steady of both arms and the
    accuracy gates (rel. L2 <= 1e-4 against the FP64 solve on the same grid, and against the closed
    form where the FP64 solve itself meets it)."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks, sweep, workloads
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    specs = workloads.sweep_instances(4096, seed=4096)
    sample = specs[: args.sweep_sample]
    cands = [(64, 8, 1), (128, 4, 1), (256, 2, 1), (512, 1, 1), (256, 1, 2), (512, 1, 2), (256, 1, 4),
             (512, 1, 4), (128, 1, 8), (256, 1, 8)]

    def pct(x, q):
        x = [v for v in x if v is not None]
        return float(np.percentile(x, q)) if x else None

    def rel(a, b):
        return max(float(np.sqrt(np.mean((a["u"] - b["u"]) ** 2)) / max(1e-300, np.max(np.abs(b["u"])))),
                   float(np.sqrt(np.mean((a["b"] - b["b"]) ** 2)) / max(1e-300, np.max(np.abs(b["b"])))))

    def states_of(recs):
        out = {}
        for r in recs:
            out[r["state"]] = out.get(r["state"], 0) + 1
        return out

    # (1) mixed lane on the whole sample
    mix = sweep.run_mixed(sample, handoff_tol=1e-5, tol=1e-10, check_every=100, quantum=args.sweep_quantum,
                          max_steps=args.sweep_max_steps, shape=(128, 1, 1), time_budget=args.sweep_time)
    mrecs = mix["records"]
    mconv = [r for r in mrecs if r["state"] == "converged"]
    mnodes = sum(r["nodes"] * (r["steps_fp32"] + r["steps_fp64"]) for r in mrecs)
    # (2) FP32 alone
    res = sweep.run_batched(sample, "f32", tol=1e-10, check_every=100, quantum=args.sweep_quantum,
                            max_steps=args.sweep_max_steps, tune_candidates=cands, time_budget=args.sweep_time)
    recs = res["records"]
    done = [r for r in recs if r["t_done"] is not None]
    node_updates = sum(r["nodes"] * r["steps"] for r in recs)
    # (3) FP64 through the batched engine on the first instances
    nb64 = max(args.sweep_baseline, args.sweep_fp64_sample)
    res64 = sweep.run_batched(sample[:nb64], "f64", tol=1e-10, check_every=100, quantum=args.sweep_quantum,
                              max_steps=args.sweep_max_steps, tune_candidates=cands, time_budget=args.sweep_time)
    r64 = res64["records"]
    # (4), (5) the same first K instances, both arms
    K = args.sweep_baseline
    base = sweep.run_one_at_a_time(sample[:K], "f64", tol=1e-10, check_every=100, max_steps=args.sweep_max_steps,
                                   time_limit=args.sweep_time)
    brecs = base["records"]
    K = len(brecs)   # the instances the baseline reached within its time limit: both arms solve those
    mixK = sweep.run_mixed(sample[:K], handoff_tol=1e-5, tol=1e-10, check_every=100, quantum=args.sweep_quantum,
                           max_steps=args.sweep_max_steps, shape=(128, 1, 1), time_budget=args.sweep_time)
    gate = {"instances": K, "fp64_one_at_a_time_unstable": 0, "fp64_one_at_a_time_converged": 0,
            "mixed_vs_fp64_same_grid_le_1e-4": 0, "fp32_vs_fp64_same_grid_le_1e-4": 0,
            "fp64_meets_analytic_le_1e-4": 0, "mixed_meets_analytic_where_fp64_does": 0,
            "mixed_vs_fp64_same_grid_rel_l2": [], "fp32_vs_fp64_same_grid_rel_l2": [],
            "fp64_vs_analytic_rel_l2": []}
    for m, f32r, bb in zip(mixK["records"], recs[:K], brecs):
        if bb["status"] == lks.LKS_EUNSTABLE:
            gate["fp64_one_at_a_time_unstable"] += 1
            gate["mixed_vs_fp64_same_grid_rel_l2"].append(None)
            gate["fp32_vs_fp64_same_grid_rel_l2"].append(None)
            gate["fp64_vs_analytic_rel_l2"].append(None)
            continue
        gate["fp64_one_at_a_time_converged"] += int(bb["status"] == lks.LKS_OK)
        dm = rel(m, bb) if m["state"] != "fp32_unstable" else float("inf")
        d32 = rel(f32r, bb) if f32r["state"] != "unstable" else float("inf")
        da = max(bb["l2_u"], bb["l2_b"])
        gate["mixed_vs_fp64_same_grid_rel_l2"].append(dm)
        gate["fp32_vs_fp64_same_grid_rel_l2"].append(d32)
        gate["fp64_vs_analytic_rel_l2"].append(da)
        gate["mixed_vs_fp64_same_grid_le_1e-4"] += int(dm <= 1e-4)
        gate["fp32_vs_fp64_same_grid_le_1e-4"] += int(d32 <= 1e-4)
        if da <= 1e-4:
            gate["fp64_meets_analytic_le_1e-4"] += 1
            gate["mixed_meets_analytic_where_fp64_does"] += int(max(m["l2_u"], m["l2_b"]) <= 1e-4)
    # The FP64 oracle on the host cores: 2000 steps of each of the first instances (until about
    # --cpu-seconds of CPU work), extrapolated by node-updates to the steps the one-at-a-time FP64
    # arm needed for its instances.  Marked as an extrapolation.
    oracle_est = None
    if not args.skip_cpu:
        import oracle
        t_or, nu_or, used, k_or = 0.0, 0, 0, 2000
        for spec in sample[:K]:
            if t_or > args.cpu_seconds:
                break
            p = sweep.lattice_params(spec)
            o = oracle.Oracle(spec["nx"], spec["ny"], sweep.TAU, sweep.TAU, p["B0"], p["Fx"],
                              oracle.LINK if spec["closure"] == "link" else oracle.MOMENT, p["c_bottom"], p["c_top"],
                              p["u_bottom"], p["u_top"])
            t1 = time.perf_counter()
            o.step(k_or)
            t_or += time.perf_counter() - t1
            nu_or += spec["nx"] * spec["ny"] * k_or
            used += 1
            del o
    if not args.skip_cpu and used > 0:
        rate = nu_or / t_or
        need = sum(spec["nx"] * spec["ny"] * bb["steps"] for spec, bb in zip(sample[:K], brecs))
        oracle_est = {"kind": "oracle", "extrapolated": True, "cores": oracle.threads_used(),
                      "mlups": round(rate / 1e6, 3), "est_wall_s": round(need / rate, 1),
                      "node_updates": int(need),
                      "sample": "%d FP64 oracle steps of each of the first %d instances (%.1f s), scaled to the "
                                "step counts the one-at-a-time FP64 arm needed on its %d instances" % (
                                    k_or, used, t_or, K)}
    # L2-resident copy bandwidth (2 x 24 MB, well inside the 129 MB L2), the roofline of the batched
    # kernel whose small instances stay in L2 while resident
    a = torch.empty(6 << 20, dtype=torch.float32, device="cuda")
    bbuf = torch.empty_like(a)
    for _ in range(20):
        bbuf.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = None
    for _ in range(5):
        e0.record()
        for _ in range(200):
            bbuf.copy_(a)
        e1.record()
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / 200
        best = dt if best is None else min(best, dt)
    l2_gbs = 2 * a.numel() * 4 / best / 1e9
    del a, bbuf
    out = {"workload": "sweep", "metric": "sweep solves/s", "unit": "solves/s", "higher_is_better": True,
           "sample": len(sample), "of": len(specs), "dtype": "f32->f64",
           "value": round(len(mconv) / mix["wall"], 3),
           "mixed_lane": {"handoff_tol": 1e-5, "tol": 1e-10, "wall_s": round(mix["wall"], 3),
                          "converged": len(mconv), "states": states_of(mrecs),
                          "fp32_states": states_of([{"state": r["fp32_state"]} for r in mrecs]),
                          "time_to_steady_p50_s": pct([r["t_done"] for r in mconv], 50),
                          "time_to_steady_p99_s": pct([r["t_done"] for r in mconv], 99),
                          "glups": round(mnodes / mix["wall"] / 1e9, 2), "launches": mix["launches"],
                          "steps_fp32_total": int(sum(r["steps_fp32"] for r in mrecs)),
                          "steps_fp64_total": int(sum(r["steps_fp64"] for r in mrecs))},
           "fp32_only": {"wall_s": round(res["wall"], 3), "solves_per_s": round(len(done) / res["wall"], 3),
                         "time_to_steady_p50_s": pct([r["t_done"] for r in done], 50),
                         "time_to_steady_p99_s": pct([r["t_done"] for r in done], 99),
                         "states": states_of(recs), "glups": round(node_updates / res["wall"] / 1e9, 2),
                         "roofline_l2": {"bound": "l2", "achieved": round(node_updates / res["wall"] * 152 / 1e9, 1),
                                         "peak": round(l2_gbs, 1), "unit": "GB/s",
                                         "frac": round(node_updates / res["wall"] * 152 / 1e9 / l2_gbs, 4),
                                         "peak_source": "measured here: torch copy of 24 MB within L2, best of 5",
                                         "note": "whole sweep wall time, launch gaps and the tail included"},
                         "launches": res["launches"], "autotune": res["tune"],
                         "tail_shape_at_s": res["tail_shape_at"]},
           "fp64_batched": {"instances": len(r64), "wall_s": round(res64["wall"], 3),
                            "solves_per_s": round(sum(r["t_done"] is not None for r in r64) / res64["wall"], 4),
                            "time_to_steady_p50_s": pct([r["t_done"] for r in r64], 50),
                            "time_to_steady_p99_s": pct([r["t_done"] for r in r64], 99),
                            "states": states_of(r64)},
           "same_sample": {
               "instances": K,
               "mixed_lane": {"wall_s": round(mixK["wall"], 3), "states": states_of(mixK["records"]),
                              "solves_per_s": round(sum(r["state"] == "converged" for r in mixK["records"])
                                                    / mixK["wall"], 4),
                              "time_to_steady_p50_s": pct([r["t_done"] for r in mixK["records"]], 50),
                              "time_to_steady_p99_s": pct([r["t_done"] for r in mixK["records"]], 99)},
               "one_at_a_time_fp64": {"wall_s": round(base["wall"], 3),
                                      "solves_per_s": round(sum(r["status"] == lks.LKS_OK for r in brecs)
                                                            / base["wall"], 4),
                                      "time_to_steady_p50_s": pct([r["t_done"] for r in brecs], 50),
                                      "time_to_steady_p99_s": pct([r["t_done"] for r in brecs], 99),
                                      "statuses": {lks._status_name(k): sum(r["status"] == k for r in brecs)
                                                   for k in {r["status"] for r in brecs}}},
               "gate": gate,
               "oracle_host": oracle_est},
           "settings": {"quantum": args.sweep_quantum, "max_steps": args.sweep_max_steps, "check_every": 100,
                        "time_budget_s": args.sweep_time, "mixed_shape": [128, 1, 1],
                        "mixed_tail_shape": [128, 1, 8], "mixed_tail_below": "number of SMs"}}
    print(json.dumps(out), flush=True)
    return 0


def bench_serve(args):
    """Serving stream: Poisson arrivals at 2000 req/s (seed 5) of Hartmann / Hartmann-Couette
    solves, nx in {4, 256}, ny lognormal (median 256, sigma 1, clamp 33..4096), Ha and c as in the
    sweep, FP32 storage, residual tolerance 1e-9, a 120 GB device-memory budget.  A finite prefix of
    the trace is replayed with a per-request step cap; the FIFO one-at-a-time FP64 baseline replays
    the first requests of the same prefix."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks, serve, workloads
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    from paper_2112_13930_gb300 import sweep

    finish = args.serve_finish_tol if args.serve_finish_tol > 0 else None

    def replay(rate, n=None):
        trace = workloads.serve_trace(args.serve_requests, rate=rate, seed=5)
        if n is not None:
            trace = trace[:n]
        srv = serve.Server("f32", budget_bytes=120 << 30, small_pool_bytes=16 << 30, small_max_nodes=32768,
                           large_workers=args.serve_workers, tol=1e-9, check_every=100, quantum=args.serve_quantum,
                           max_steps=args.serve_max_steps, inplace=args.serve_inplace, finish_tol=finish)
        recs = srv.serve(trace, time_limit=args.serve_time)
        srv.close()
        summ = serve.summarize(recs, len(trace))
        summ["_records"] = recs
        errs = [max(sweep.analytic_error(r["req"], r["u"], r["b"])) for r in recs
                if r.get("state") in serve.STEADY_STATES]
        if errs:
            summ["steady_vs_analytic_rel_l2"] = {"median": float(np.median(errs)), "max": float(np.max(errs)),
                                                 "le_1e-4": int(sum(e <= 1e-4 for e in errs))}
        lanes = {}
        for r in recs:
            lanes[r["lane"]] = lanes.get(r["lane"], 0) + 1
        summ["lanes"] = lanes
        summ["offered_rate_per_s"] = rate
        return trace, summ

    trace, summ = replay(args.serve_rate)
    summ.pop("_records")
    # the same first K requests through both arms: the server alone on them, and FIFO one-at-a-time FP64
    K = args.serve_baseline
    _, ssum = replay(args.serve_rate, K)
    srecs = {r["req"]["index"]: r for r in ssum.pop("_records")}
    base = serve.serve_one_at_a_time(trace[:K], "f64", tol=1e-9, check_every=100,
                                     max_steps=args.serve_max_steps, time_limit=args.serve_time)
    bsum = serve.summarize(base, K)
    gate = {"requests": K, "fp64_steady": 0, "served_vs_fp64_same_grid_le_1e-4": 0,
            "fp64_meets_analytic_le_1e-4": 0, "served_meets_analytic_where_fp64_does": 0,
            "served_vs_fp64_same_grid_rel_l2": []}
    for b in base:
        r = srecs.get(b["req"]["index"])
        if r is None or r.get("u") is None or b["state"] not in serve.STEADY_STATES:
            gate["served_vs_fp64_same_grid_rel_l2"].append(None)
            continue
        gate["fp64_steady"] += 1
        d = max(float(np.sqrt(np.mean((r["u"] - b["u"]) ** 2)) / max(1e-300, np.max(np.abs(b["u"])))),
                float(np.sqrt(np.mean((r["b"] - b["b"]) ** 2)) / max(1e-300, np.max(np.abs(b["b"])))))
        gate["served_vs_fp64_same_grid_rel_l2"].append(d)
        gate["served_vs_fp64_same_grid_le_1e-4"] += int(d <= 1e-4)
        if max(sweep.analytic_error(b["req"], b["u"], b["b"])) <= 1e-4:
            gate["fp64_meets_analytic_le_1e-4"] += 1
            gate["served_meets_analytic_where_fp64_does"] += int(max(sweep.analytic_error(r["req"], r["u"], r["b"]))
                                                                 <= 1e-4)
    out = {"workload": "serve", "metric": "served solves/s", "unit": "solves/s", "higher_is_better": True,
           "dtype": "f32->f64" if finish else "f32", "value": round(summ["solves_per_s"], 3), "summary": summ,
           "offered_rate_per_s": args.serve_rate,
           "same_sample": {"requests": K, "served": ssum, "one_at_a_time_fp64_fifo": bsum, "gate": gate},
           "settings": {"requests": args.serve_requests, "max_steps": args.serve_max_steps,
                        "buffers": "one, in place" if args.serve_inplace else "two", "finish_tol": finish,
                        "quantum": args.serve_quantum, "large_workers": args.serve_workers,
                        "time_limit_s": args.serve_time}}
    if args.serve_underload > 0:
        # the same requests offered below capacity: latency is then solve time, not queueing
        _, under = replay(args.serve_underload * summ["solves_per_s"])
        under.pop("_records")
        out["underload"] = under
    print(json.dumps(out), flush=True)
    return 0


def bench_d3(args):
    """The three-dimensional channel alone: n^3 nodes (default 256^3), Hartmann-Couette set-up
    (link-based walls, c = 1, top wall at 0.05, Ha = 20), FP64, FP32, BF16 or FP16 storage, K timed
    steps.  Algorithmic bytes per node: 40 populations read and written once, 8, 4 or 2 bytes each."""
    import torch
    from paper_2112_13930_gb300 import build, lks, lks3d
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    n = args.n if args.n != 4096 else 256
    storage = args.storage if args.storage in ("f64", "f32", "bf16", "f16") else "f32"
    lat = lks3d.Lattice3D(n, n, n, 0.8, 0.8, 20.0 * 0.1 / (n / 2), 0.0, storage)
    lat.set_walls(1.0, 1.0, 0.0, 0.05)
    lat.step(args.warmup)
    stream = torch.cuda.current_stream()
    t = _time_steps(lat, args.steps, stream)
    nodes = n ** 3
    bpn = 80 * {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage]
    peak, _ = _peaks()
    achieved = bpn * nodes / (t / args.steps) / 1e9
    v = nodes * args.steps / t / 1e6
    out = {"workload": "d3q19", "metric": METRIC, "unit": UNIT, "value": round(v, 1),
           "config": {"n": n, "storage": storage, "steps": args.steps, "bytes_per_node": bpn},
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4)}}
    if storage == "f64":  # FP64 arithmetic, not HBM, bounds this kernel on GB300
        ipn = FP64_PIPE_INSTR_PER_NODE_3D
        out["roofline_fp64_pipe"] = {"bound": "fp64 pipe", "instr_per_node": ipn,
                                     "achieved": round(ipn * v * 1e6 / 1e12, 4), "peak": FP64_PIPE_PEAK / 1e12,
                                     "unit": "T FP64 instr/s", "frac": round(ipn * v * 1e6 / FP64_PIPE_PEAK, 4),
                                     "source": "profiles/step3_kernel_f64_128cube_fp64_pipe.md"}
    lat.close()
    print(json.dumps(out), flush=True)
    return 0


def bench_duct(args):
    """The rectangular duct (3D channel with side walls at the z planes, lks3_set_side_walls), fully
    developed: nx = 1, ny = nz = n (default 1024), Hartmann walls c = 0.5, side walls c = 0.1, Ha = 20,
    body force, tau = 0.8, FP32 (or --storage) storage, K timed steps of the flattened one-node
    kernel.  Algorithmic bytes per node: 40 populations read and written once."""
    import torch
    from paper_2112_13930_gb300 import build, lks, lks3d
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    n = args.n if args.n != 4096 else 1024
    storage = args.storage
    nu, eta = 0.1, 0.075
    B0 = 20.0 * math.sqrt(nu * eta) / (n / 2)
    lat = lks3d.Lattice3D(1, n, n, 0.8, 0.8, B0, 1e-6 * (64.0 / n) ** 2, storage)
    lat.set_walls(0.5, 0.5)
    lat.set_side_walls(0.1, 0.1)
    lat.step(args.warmup)
    stream = torch.cuda.current_stream()
    t = _time_steps(lat, args.steps, stream)
    nodes = n * n
    bpn = 80 * {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[storage]
    peak, _ = _peaks()
    achieved = bpn * nodes / (t / args.steps) / 1e9
    v = nodes * args.steps / t / 1e6
    out = {"workload": "duct", "metric": METRIC, "unit": UNIT, "value": round(v, 1),
           "config": {"nx": 1, "ny": n, "nz": n, "storage": storage, "steps": args.steps, "bytes_per_node": bpn,
                      "c_hartmann": 0.5, "c_side": 0.1, "Ha": 20.0,
                      "l2": "inputs larger than L2" if bpn * nodes > 129e6 else "inputs within L2"},
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "kernel": "step3_duct_kernel<%s>" % storage}}
    lat.close()
    print(json.dumps(out), flush=True)
    return 0


def bench_validation(args):
    """The paper's E1-E6 experiments on the GPU (FP64 batch, residual 1e-10); CSV profiles in
    --validation-out; prints a JSON summary of the errors and convergence orders."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks, validation
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    t0 = time.perf_counter()
    rows, orders = validation.run(args.validation_out)
    wall = time.perf_counter() - t0
    per_exp = {}
    for r in rows:
        e = per_exp.setdefault(r["exp"], {"cases": 0, "max_l2_u": 0.0, "max_l2_b": 0.0, "states": {}})
        e["cases"] += 1
        e["max_l2_u"] = max(e["max_l2_u"], r["l2_u"])
        e["max_l2_b"] = max(e["max_l2_b"], r["l2_b"])
        e["states"][r["state"]] = e["states"].get(r["state"], 0) + 1
    out = {"workload": "validation", "wall_s": round(wall, 2), "experiments": per_exp,
           "convergence_orders": [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in o.items()}
                                  for o in orders],
           "csv_dir": args.validation_out}
    if args.validation_record:
        # the record kept with the sources: per-case errors, E3 orders and the per-experiment table
        import shutil
        os.makedirs(args.validation_record, exist_ok=True)
        for name in ("summary.csv", "convergence.csv"):
            shutil.copy(os.path.join(args.validation_out, name),
                        os.path.join(args.validation_record, "validation_" + name))
        with open(os.path.join(args.validation_record, "validation_table.csv"), "w") as fh:
            fh.write("exp,cases,converged,max_l2_u_or_min_order,max_l2_b_or_max_order\n")
            for t in validation.table(rows, orders):
                fh.write("%s,%d,%d,%.4g,%.4g\n" % (t["exp"], t["cases"], t["converged"], t["max_l2_u"],
                                                    t["max_l2_b"]))
        out["record_dir"] = args.validation_record
    print(json.dumps(out), flush=True)
    return 0


def bench_c2(args):
    """The timing matrix of the shear-driven 4096 x 4096 channel: moment-based closure, top wall at
    U_w = 0.05, bottom at rest, tau_f = tau_m = 0.8, Ha in {5, 20, 50} (B0 = Ha 0.1 / 2047.5) and the
    same c on both walls in {0, 0.01, 1, 100, 1e6}, from rest: 200 warm-up steps, then the median of
    3 timed runs (FP32: 5000 steps each; FP64, bound by the FP64 pipe: --c2-fp64-steps each)."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    stream = torch.cuda.current_stream()
    n, a = 4096, 2047.5
    rows = []
    for storage, steps in (("f32", 5000), ("f64", args.c2_fp64_steps)):
        for ha in (5.0, 20.0, 50.0):
            lat = lks.Lattice(n, n, 0.8, 0.8, ha * 0.1 / a, 0.0, "moment", storage)
            for c in (0.0, 0.01, 1.0, 100.0, 1e6):
                lat.set_walls(c, c, 0.0, 0.05)
                lat.step(200)
                t = sorted(_time_steps(lat, steps, stream) for _ in range(3))[1]
                rows.append({"storage": storage, "Ha": ha, "c": c, "steps": steps,
                             "mlups": round(n * n * steps / t / 1e6, 1)})
            lat.close()
            del lat
            torch.cuda.empty_cache()
    out = {"workload": "c2", "config": {"n": n, "closure": "moment", "u_top": 0.05, "tau": 0.8,
                                        "warmup": 200, "repeats": 3}, "points": rows}
    for st in ("f32", "f64"):
        v = [r["mlups"] for r in rows if r["storage"] == st]
        out[st] = {"min": min(v), "median": float(np.median(v)), "max": max(v)}
    print(json.dumps(out), flush=True)
    return 0


def bench_c1(args):
    """Body-force Hartmann channel, 4 x 65 nodes, walls at y = +-a with the Shercliff condition
    (link-based closure), B0 from Ha = 10, c = 0.1, tau_f = tau_m = 0.8, FP64, 2e4 steps: GPU wall
    time for the 2e4 steps, parity with the FP64 oracle, and the profile against the closed form."""
    import numpy as np
    import torch
    from paper_2112_13930_gb300 import build, lks, profiles
    torch.cuda.set_device(0)
    build.build()
    lks.load()
    nx, ny, ha, c, tau, steps = 4, 65, 10.0, 0.1, 0.8, 20000
    a, y = profiles.node_y(ny, "link")
    nu = (tau - 0.5) / 3.0
    b0 = ha * nu / a
    fx = profiles.hartmann_force(0.01, ha, c, a, tau)
    lat = lks.Lattice(nx, ny, tau, tau, b0, fx, "link", "f64")
    lat.set_walls(c, c)
    lat.step(64)
    lat2 = lks.Lattice(nx, ny, tau, tau, b0, fx, "link", "f64")
    lat2.set_walls(c, c)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat2.step(steps)
    lat2.sync()
    t_gpu = time.perf_counter() - t0
    u, b = lat2.profiles()
    ua, ba = profiles.hartmann(y, a, ha, c, fx, tau, tau)
    out = {"workload": "c1", "config": {"nx": nx, "ny": ny, "Ha": ha, "c": c, "tau": tau, "B0": b0, "Fx": fx,
                                        "closure": "link", "storage": "f64", "steps": steps},
           "gpu_wall_s": round(t_gpu, 4), "gpu_mlups": round(nx * ny * steps / t_gpu / 1e6, 2),
           "gpu_us_per_step": round(t_gpu / steps * 1e6, 3),
           "l2_vs_closed_form": {"u": profiles.rel_l2(u, ua), "B": profiles.rel_l2(b, ba)}}
    if not args.skip_cpu:
        import oracle
        o = oracle.Oracle(nx, ny, tau, tau, b0, fx, oracle.LINK, c, c)
        t0 = time.perf_counter()
        o.step(steps)
        t_cpu = time.perf_counter() - t0
        fg, gg = lat2.get_state()
        out["oracle_wall_s"] = round(t_cpu, 3)
        out["oracle_cores"] = oracle.threads_used()
        out["fp64_parity_max_rel"] = max(float(np.max(np.abs(fg - o.f)) / np.max(np.abs(o.f))),
                                         float(np.max(np.abs(gg - o.g)) / np.max(np.abs(o.g))))
    steps_ss, r, status = lat.run_to_steady(1e-10, 100, 2_000_000, raise_on_fail=False)
    u2, b2 = lat.profiles()
    out["to_steady"] = {"steps": steps_ss + 64, "residual": r, "status": int(status),
                        "l2_u": profiles.rel_l2(u2, ua), "l2_B": profiles.rel_l2(b2, ba)}
    lat.close()
    lat2.close()
    print(json.dumps(out), flush=True)
    return 0


# FP64 arithmetic per bulk node per step in collide_node, counted from the source with an FMA as
# 2 flops: moments and 1/rho (Newton) 40, equilibrium set-up 23, nine directions 116, g 33.
FP64_FLOPS_PER_NODE = 212
# FP64 pipe instructions per node of the FP64 step kernel (ncu sm__inst_executed_pipe_fp64.sum x 32
# / nodes at 2048^2) and the pipe's nominal rate (1.25 TFLOP/s = 0.625e12 DFMA/s on GB300)
FP64_PIPE_INSTR_PER_NODE = 153
FP64_PIPE_INSTR_PER_NODE_3D = 336
FP64_PIPE_PEAK = 0.625e12


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f64", "bf16", "f16"], default="f32")
    ap.add_argument("--c2-fp64-steps", type=int, default=300, help="--workload c2: FP64 steps per timed run")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--inplace", action="store_true",
                    help="time the in-place (one-buffer) step instead of the two-buffer step")
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-extra", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--workload", choices=["main", "c1", "c2", "precision", "sweep", "serve", "validation", "d3",
                                           "duct"],
                    default="main")
    ap.add_argument("--config", type=int, choices=[1, 2, 3, 4, 5], default=None,
                    help="preset of the five benchmark configurations: 1 = c1, 2 = main, 3 = precision, "
                         "4 = sweep, 5 = serve")
    ap.add_argument("--validation-out", default="validation_out")
    ap.add_argument("--validation-record", default="",
                    help="--workload validation: also write the summary CSVs into this directory")
    ap.add_argument("--precision-steps", type=int, default=1000)
    ap.add_argument("--precision-max-steps", type=int, default=3_000_000)
    ap.add_argument("--sweep-sample", type=int, default=512)
    ap.add_argument("--sweep-baseline", type=int, default=64)
    ap.add_argument("--sweep-fp64-sample", type=int, default=64)
    ap.add_argument("--sweep-quantum", type=int, default=20000)
    ap.add_argument("--sweep-max-steps", type=int, default=2_000_000)
    ap.add_argument("--sweep-time", type=float, default=600.0)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-baseline", type=int, default=64)
    ap.add_argument("--serve-finish-tol", type=float, default=1e-5,
                    help="hand-off residual of the FP64 finish (0: FP32 only)")
    ap.add_argument("--serve-quantum", type=int, default=2000)
    ap.add_argument("--serve-max-steps", type=int, default=200_000)
    ap.add_argument("--serve-workers", type=int, default=6)
    ap.add_argument("--serve-time", type=float, default=600.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-inplace", action="store_true",
                    help="serve with one population buffer per request (in-place pairs of steps)")
    ap.add_argument("--serve-underload", type=float, default=0.0,
                    help="if > 0, replay the trace again at this fraction of the measured solves/s")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.config is not None:
        args.workload = {1: "c1", 2: "main", 3: "precision", 4: "sweep", 5: "serve"}[args.config]
    if args.impl == "reference":
        return bench_reference(args)
    if args.workload == "c2":
        return bench_c2(args)
    if args.workload == "c1":
        return bench_c1(args)
    if args.workload == "precision":
        return bench_precision(args)
    if args.workload == "sweep":
        return bench_sweep(args)
    if args.workload == "serve":
        return bench_serve(args)
    if args.workload == "d3":
        return bench_d3(args)
    if args.workload == "validation":
        return bench_validation(args)
    if args.workload == "duct":
        return bench_duct(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())

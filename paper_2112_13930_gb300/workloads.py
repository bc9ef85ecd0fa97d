"""Seeded synthetic workloads: the parameter-sweep instance set and the serving arrival trace.

Only random draws live here (sizes, Hartmann numbers, wall conductance ratios, forcing kinds,
arrival times); converting them to lattice parameters is done by the solvers.
"""
import math

import numpy as np


def _c_draw(rng):
    """Wall conductance ratio: 5% insulating (0), 5% perfectly conducting (inf), else log-uniform
    in [1e-3, 1e3]."""
    u = rng.uniform()
    if u < 0.05:
        return 0.0
    if u < 0.10:
        return math.inf
    return float(math.exp(rng.uniform(math.log(1e-3), math.log(1e3))))


def sweep_instances(n=4096, seed=4096, ny_range=(33, 1025), ha_range=(1.0, 200.0), nx=4):
    """Batched-sweep set: nx = 4, ny uniform in ny_range, Ha log-uniform in ha_range, c as _c_draw;
    even index: body-force flow with the link-based closure and c on both plates; odd index:
    shear flow (top plate at U_w = 0.05) with the moment-based closure, c on the moving plate and
    the other plate insulating."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        ha = float(math.exp(rng.uniform(math.log(ha_range[0]), math.log(ha_range[1]))))
        c = _c_draw(rng)
        kind = "body" if k % 2 == 0 else "shear"
        out.append({"index": k, "nx": nx, "ny": ny, "ha": ha, "c": c, "kind": kind,
                    "closure": "link" if kind == "body" else "moment"})
    return out


def serve_trace(n, rate=2000.0, seed=5, ny_median=256, ny_sigma=1.0, ny_clamp=(33, 4096), nx_choices=(4, 256)):
    """Poisson arrivals (rate per second) of solve requests: nx from nx_choices with equal
    probability, ny = clamp(round(ny_median * exp(N(0, ny_sigma)))), Ha, c and forcing kind as in
    the sweep (kind drawn with equal probability)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += float(rng.exponential(1.0 / rate))
        nx = int(nx_choices[int(rng.integers(0, len(nx_choices)))])
        ny = int(min(max(round(ny_median * math.exp(rng.normal(0.0, ny_sigma))), ny_clamp[0]), ny_clamp[1]))
        ha = float(math.exp(rng.uniform(0.0, math.log(200.0))))
        c = _c_draw(rng)
        kind = "body" if rng.uniform() < 0.5 else "shear"
        out.append({"index": k, "t_arrival": t, "nx": nx, "ny": ny, "ha": ha, "c": c, "kind": kind,
                    "closure": "link" if kind == "body" else "moment"})
    return out

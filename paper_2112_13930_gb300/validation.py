"""The paper's validation experiments on the GPU (Sec. VIII), solved with the batched engine in FP64:

E1/E2  body-force Hartmann flow, link-based / moment-based closure, 3 x 101 nodes, tau = 0.57,
       tau_m = 0.75, Ha in {5, 20}, c in {0, 0.1, 0.5, 1, 1e4}, compared with the Chang & Lundgren
       profiles (Sec. VIII.A);
E3     grid convergence, Ha = 20, tau = 0.9, tau_m = 0.95, N in {50, 100, 200}, c in {0, 0.1, 0.5, 1},
       both closures, diffusive scaling of the velocity (Sec. VIII.A);
E4/E5  Hartmann-Couette flow, top plate at U_w = 0.05, 3 x 101 nodes, tau = 0.6, tau_m = 0.65,
       Ha in {5, 20}, (c_u, c_l) in {(0, 0), (0.5, 0.5), (0, 0.5)}, link- / moment-based (Sec. VIII.B);
E6     Hartmann-Couette, Ha = 5, c_l = 0, c_u in {0, 0.1, 0.5, 1, 1e4}, both closures (Sec. VIII.B).
E7     body-force Hartmann flow with a different conductance ratio on each plate (not in the paper:
       the closed form is solved here like App. C's shear-driven case), 3 x 101, tau = 0.57,
       tau_m = 0.75, Ha in {5, 20}, (c_l, c_u) in {(0, 0.5), (0.1, 2), (0, 1e4)}, both closures.

Every case runs to a residual of 1e-10 (FP64).  Profiles are written as CSV (y, u_x, u_x closed
form, B_x, B_x closed form) with a summary CSV of the relative L2 errors and the measured
convergence orders.
"""
import csv
import math
import os

import numpy as np

from . import batch as _batch
from . import profiles

HA_E1 = (5.0, 20.0)
C_E1 = (0.0, 0.1, 0.5, 1.0, 1e4)


def cases():
    out = []
    for closure, tag in (("link", "E1"), ("moment", "E2")):
        for ha in HA_E1:
            for c in C_E1:
                out.append(dict(exp=tag, kind="body", closure=closure, ny=101, nx=3, ha=ha, c_l=c, c_u=c, tau_f=0.57,
                                tau_m=0.75, u_c=0.01))
    for closure in ("link", "moment"):
        for c in (0.0, 0.1, 0.5, 1.0):
            for ny in (50, 100, 200):
                out.append(dict(exp="E3", kind="body", closure=closure, ny=ny, nx=3, ha=20.0, c_l=c, c_u=c,
                                tau_f=0.9, tau_m=0.95, u_c=0.01 * 50.0 / ny))
    for closure, tag in (("link", "E4"), ("moment", "E5")):
        for ha in (5.0, 20.0):
            for cu, cl in ((0.0, 0.0), (0.5, 0.5), (0.0, 0.5)):
                out.append(dict(exp=tag, kind="shear", closure=closure, ny=101, nx=3, ha=ha, c_l=cl, c_u=cu,
                                tau_f=0.6, tau_m=0.65, u_w=0.05))
    for closure in ("link", "moment"):
        for cu in C_E1:
            out.append(dict(exp="E6", kind="shear", closure=closure, ny=101, nx=3, ha=5.0, c_l=0.0, c_u=cu,
                            tau_f=0.6, tau_m=0.65, u_w=0.05))
    for closure in ("link", "moment"):
        for ha in HA_E1:
            for cl, cu in ((0.0, 0.5), (0.1, 2.0), (0.0, 1e4)):
                out.append(dict(exp="E7", kind="body", closure=closure, ny=101, nx=3, ha=ha, c_l=cl, c_u=cu,
                                tau_f=0.57, tau_m=0.75, u_c=0.01))
    return out


def _desc(case, tol, max_steps):
    a, _ = profiles.node_y(case["ny"], case["closure"])
    nu = (case["tau_f"] - 0.5) / 3.0
    eta = (case["tau_m"] - 0.5) / 3.0
    b0 = case["ha"] * math.sqrt(nu * eta) / a
    if case["kind"] == "body":
        fx = profiles.hartmann_walls_force(case["u_c"], case["ha"], case["c_l"], case["c_u"], a, case["tau_f"])
        d = _batch.make_desc(case["nx"], case["ny"], case["closure"], case["tau_f"], case["tau_m"], b0, fx,
                             case["c_l"], case["c_u"], tol=tol, check_every=100, max_steps=max_steps)
    else:
        fx = 0.0
        d = _batch.make_desc(case["nx"], case["ny"], case["closure"], case["tau_f"], case["tau_m"], b0, 0.0,
                             case["c_l"], case["c_u"], 0.0, case["u_w"], tol=tol, check_every=100,
                             max_steps=max_steps)
    return d, a, fx


def case_name(case):
    return "%s_%s_Ha%g_cl%g_cu%g_N%d" % (case["exp"], case["closure"], case["ha"], case["c_l"], case["c_u"],
                                         case["ny"])


def run(out_dir, tol=1e-10, max_steps=20_000_000, quantum=50_000, storage="f64", select=None):
    """Solve every case (or those for which select(case) is true) in one batch; write CSVs to
    out_dir; return the summary rows and the E3 convergence orders.  With fewer cases than SMs each
    case runs on a cluster of 8 CTAs (the results do not depend on the shape)."""
    import torch
    os.makedirs(out_dir, exist_ok=True)
    cs = [c for c in cases() if select is None or select(c)]
    descs = [_desc(c, tol, max_steps) for c in cs]
    pool = sum(_batch.instance_footprint(d, storage) for d, _, _ in descs) + (1 << 20)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    b = _batch.Batch(storage, max_instances=len(cs), pool_bytes=pool, threads_per_group=128, groups_per_cta=1,
                     cluster_ctas=8 if len(cs) < sms else 1)
    slots = [b.add(d) for d, _, _ in descs]
    while b.run(quantum):
        pass
    rows = []
    for case, (d, a, fx), s in zip(cs, descs, slots):
        st, steps, r = b.result(s)
        u, bx = b.profiles(s)
        _, y = profiles.node_y(case["ny"], case["closure"])
        if case["kind"] == "body":
            ua, ba = profiles.hartmann_walls(y, a, case["ha"], case["c_l"], case["c_u"], fx, case["tau_f"],
                                             case["tau_m"])
        else:
            ua, ba = profiles.couette(y, a, case["ha"], case["c_l"], case["c_u"], case["u_w"], case["tau_f"],
                                      case["tau_m"])
        name = case_name(case)
        with open(os.path.join(out_dir, name + ".csv"), "w", newline="") as fh:
            w = csv.writer(fh)
            w.writerow(["y", "xi", "u_x", "u_x_closed_form", "B_x", "B_x_closed_form"])
            for k in range(case["ny"]):
                w.writerow(["%.6f" % y[k], "%.8f" % (y[k] / a), "%.12e" % u[k], "%.12e" % ua[k], "%.12e" % bx[k],
                            "%.12e" % ba[k]])
        rows.append(dict(case=name, exp=case["exp"], closure=case["closure"], ha=case["ha"], c_l=case["c_l"],
                         c_u=case["c_u"], ny=case["ny"], state=_batch.STATE_NAMES[st], steps=int(steps), residual=r,
                         l2_u=profiles.rel_l2(u, ua), l2_b=profiles.rel_l2(bx, ba), u=u, b=bx))
    b.close()
    # E3 convergence orders between consecutive resolutions (relative errors; a = N/2 or (N-1)/2)
    orders = []
    for closure in ("link", "moment"):
        for c in (0.0, 0.1, 0.5, 1.0):
            sub = [r for r in rows if r["exp"] == "E3" and r["closure"] == closure and r["c_u"] == c]
            sub.sort(key=lambda r: r["ny"])
            for r0, r1 in zip(sub[:-1], sub[1:]):
                a0 = r0["ny"] / 2 if closure == "link" else (r0["ny"] - 1) / 2
                a1 = r1["ny"] / 2 if closure == "link" else (r1["ny"] - 1) / 2
                orders.append(dict(closure=closure, c=c, n0=r0["ny"], n1=r1["ny"],
                                   order_u=-math.log(r1["l2_u"] / r0["l2_u"]) / math.log(a1 / a0),
                                   order_b=-math.log(r1["l2_b"] / r0["l2_b"]) / math.log(a1 / a0)))
    fields = [k for k in rows[0] if k not in ("u", "b")]
    with open(os.path.join(out_dir, "summary.csv"), "w", newline="") as fh:
        w = csv.DictWriter(fh, fieldnames=fields, extrasaction="ignore")
        w.writeheader()
        w.writerows(rows)
    if orders:
        with open(os.path.join(out_dir, "convergence.csv"), "w", newline="") as fh:
            w = csv.DictWriter(fh, fieldnames=list(orders[0].keys()))
            w.writeheader()
            w.writerows(orders)
    return rows, orders


def table(rows, orders):
    """Per experiment: cases, converged cases, max relative L2 errors of u_x and B_x; E3 order range."""
    out = []
    for exp in sorted({r["exp"] for r in rows}):
        sub = [r for r in rows if r["exp"] == exp]
        out.append(dict(exp=exp, cases=len(sub), converged=sum(r["state"] == "converged" for r in sub),
                        max_l2_u=max(r["l2_u"] for r in sub), max_l2_b=max(r["l2_b"] for r in sub)))
    for closure in ("link", "moment"):
        sub = [o for o in orders if o["closure"] == closure]
        if sub:
            out.append(dict(exp="E3 order (%s)" % closure, cases=len(sub), converged=len(sub),
                            max_l2_u=min(min(o["order_u"], o["order_b"]) for o in sub),
                            max_l2_b=max(max(o["order_u"], o["order_b"]) for o in sub)))
    return out

"""Writes the stored expected values under tests/golden/ -- computed by the FP64 oracle only.

c1_profiles.txt: the Hartmann channel of Sec. VI.A with the link-based closure (Sec. VI,
Eq. linkbasedBCschemefinal): 4 x 65 nodes, tau_f = tau_m = 0.8, Ha = 10 (B0 = Ha sqrt(nu eta)/a,
a = 32.5), c = 0.1 on both walls, body force F_x for an analytic centreline speed of 0.01, rest
start, 20000 steps; the x-averaged u_x(y) and B_x(y) of the stored state.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.abspath(os.path.join(HERE, "..", "..")))

import oracle  # noqa: E402
from oracle import analytic as an  # noqa: E402

C1 = dict(nx=4, ny=65, tau=0.8, ha=10.0, c=0.1, u_c=0.01, steps=20000)


def c1_oracle():
    a = C1["ny"] / 2
    b0 = an.b0_from_ha(C1["ha"], a, C1["tau"], C1["tau"])
    fx = an.force_for_centre_speed(C1["u_c"], C1["ha"], C1["c"], a, C1["tau"])
    o = oracle.Oracle(C1["nx"], C1["ny"], C1["tau"], C1["tau"], b0, fx, oracle.LINK, C1["c"], C1["c"])
    o.step(C1["steps"])
    return o, b0, fx


def main():
    o, b0, fx = c1_oracle()
    u, bx = o.profiles()
    with open(os.path.join(HERE, "c1_profiles.txt"), "w") as fh:
        fh.write("# Hartmann channel, link-based closure (Sec. VI.A, Eq. linkbasedBCschemefinal): 4 x 65,\n")
        fh.write("# tau_f = tau_m = 0.8, Ha = 10, c = 0.1 both walls, B0 = %.17g, Fx = %.17g, rest start,\n" % (b0, fx))
        fh.write("# 20000 steps, FP64 oracle (tests/golden/make_golden.py).  Columns: j  u_x  B_x\n")
        for j in range(len(u)):
            fh.write("%d %.17e %.17e\n" % (j, u[j], bx[j]))


if __name__ == "__main__":
    main()

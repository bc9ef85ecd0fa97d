"""The stored C1 profiles (tests/golden/c1_profiles.txt, written by tests/golden/make_golden.py
from the oracle): the oracle still reproduces them, they lie within the discretisation error of the
closed-form Hartmann profiles (App. C / Sec. VI.A), and the header's B0 and F_x are the values the
configuration defines (Ha = 10, u_c = 0.01, a = 32.5, nu = eta = 0.1)."""
import importlib.util
import math
import os

import numpy as np

from oracle import analytic as an

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "c1_profiles.txt")


def load_golden():
    data = np.loadtxt(GOLDEN)
    return data[:, 1], data[:, 2]


def _maker():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_golden():
    u_g, b_g = load_golden()
    o, b0, fx = _maker().c1_oracle()
    u, bx = o.profiles()
    assert np.max(np.abs(u - u_g)) <= 1e-13 * np.max(np.abs(u_g))
    assert np.max(np.abs(bx - b_g)) <= 1e-13 * np.max(np.abs(b_g))


def test_golden_parameters_and_closed_form():
    a, nu = 32.5, 0.1
    b0 = an.b0_from_ha(10.0, a, 0.8, 0.8)
    assert math.isclose(b0, 10.0 * nu / a, rel_tol=1e-15)          # Ha sqrt(nu eta)/a with nu = eta
    assert abs(b0 - 0.0307692) < 5e-8
    fx = an.force_for_centre_speed(0.01, 10.0, 0.1, a, 0.8)
    assert abs(fx - 1.72151e-5) < 5e-11
    u_g, b_g = load_golden()
    y = -a + np.arange(65) + 0.5
    ua, ba = an.hartmann_profiles(y, a, 10.0, 0.1, fx, 0.8, 0.8)
    assert an.rel_l2(u_g, ua) < 3e-3 and an.rel_l2(b_g, ba) < 3e-3   # discretisation error at 65 nodes

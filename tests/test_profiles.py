"""The product-side closed forms (paper_2112_13930_gb300/profiles.py) agree with the pinned oracle
closed forms (oracle/analytic.py), which are independent code."""
import math

import numpy as np
import pytest

from oracle import analytic as an
from paper_2112_13930_gb300 import profiles


@pytest.mark.parametrize("ha,c", [(1.0, 0.0), (5.0, 0.5), (30.0, 0.5), (200.0, 1e-3), (10.0, math.inf)])
def test_hartmann_agrees(ha, c):
    y = np.linspace(-32.5, 32.5, 66)
    u1, b1 = profiles.hartmann(y, 32.5, ha, c, 1e-5, 0.8, 0.8)
    u2, b2 = an.hartmann_profiles(y, 32.5, ha, c, 1e-5, 0.8, 0.8)
    np.testing.assert_allclose(u1, u2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b1, b2, rtol=1e-12, atol=1e-15)
    assert profiles.hartmann_force(0.01, ha, c, 32.5, 0.8) == pytest.approx(
        an.force_for_centre_speed(0.01, ha, c, 32.5, 0.8), rel=1e-12)


@pytest.mark.parametrize("ha,cl,cu", [(5.0, 0.0, 0.0), (5.0, 0.5, 0.5), (20.0, 0.0, 0.5), (3.0, 0.0, math.inf),
                                      (2.0, math.inf, 0.1), (150.0, 0.0, 100.0)])
def test_couette_agrees(ha, cl, cu):
    y = np.linspace(-40, 40, 81)
    u1, b1 = profiles.couette(y, 40.0, ha, cl, cu, 0.05, 0.8, 0.8)
    u2, b2 = an.couette_profiles(y, 40.0, ha, cl, cu, 0.05, 0.8, 0.8)
    np.testing.assert_allclose(u1, u2, rtol=1e-11, atol=1e-15)
    np.testing.assert_allclose(b1, b2, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("ha,cl,cu", [(5.0, 0.0, 0.5), (20.0, 0.1, 2.0), (3.0, math.inf, 0.3), (7.0, 0.5, math.inf),
                                      (10.0, 0.4, 0.4), (2.0, math.inf, math.inf)])
def test_hartmann_walls_agrees(ha, cl, cu):
    y = np.linspace(-32.5, 32.5, 66)
    u1, b1 = profiles.hartmann_walls(y, 32.5, ha, cl, cu, 1e-5, 0.8, 0.8)
    u2, b2 = an.hartmann_walls_profiles(y, 32.5, ha, cl, cu, 1e-5, 0.8, 0.8)
    np.testing.assert_allclose(u1, u2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b1, b2, rtol=1e-12, atol=1e-15)
    fx = profiles.hartmann_walls_force(0.01, ha, cl, cu, 32.5, 0.8)
    u0, _ = an.hartmann_walls_profiles([0.0], 32.5, ha, cl, cu, fx, 0.8, 0.8)
    assert u0[0] == pytest.approx(0.01, rel=1e-12)


def test_node_coordinates():
    a, y = profiles.node_y(65, "link")
    assert a == 32.5 and y[0] == -32.0 and y[-1] == 32.0
    a, y = profiles.node_y(65, "moment")
    assert a == 32.0 and y[0] == -32.0 and y[-1] == 32.0

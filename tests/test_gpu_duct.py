"""The duct on the GPU (lks3_set_side_walls): the 3D channel closed by walls at the z planes, against
the FP64 oracle's duct and the finite-difference reference of fully developed duct flow.

FP64 storage: populations within 1e-11 of the largest deviation from rest and moments within 1e-11 of
each field's scale, after 1 and 40 steps from the same perturbed state, on ducts whose flattened node
count spans several 256-thread blocks with a ragged tail, nx = 1 (fully developed) and nx > 1, every
wall setting (insulating, finite, perfectly conducting, unequal side walls, a moving Hartmann wall).
FP32 within 1e-4 after 40 steps; FP32, BF16 and FP16 one step within 8 u_s.  Steady FP64 profiles
converge at second order to the finite-difference solution."""
import math

import numpy as np
import pytest

import oracle
from oracle import duct

pytestmark = pytest.mark.gpu

REL64 = 1e-11


@pytest.fixture(scope="module")
def l3():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks, lks3d
    build.build()
    lks.load()
    return lks3d


CASES = [
    # nx, ny, nz, (c_bot, c_top), (c_back, c_front), (u_bot, u_top)
    (1, 40, 30, (0.5, 0.5), (0.0, 0.0), (0.0, 0.0)),
    (1, 23, 17, (math.inf, 0.2), (0.3, 2.0), (0.0, 0.0)),
    (5, 17, 9, (0.0, 1e4), (math.inf, 0.0), (0.0, 0.04)),
    (3, 2, 2, (0.4, 0.4), (0.7, 0.7), (-0.02, 0.0)),
]


def _pair(l3, case, storage, seed=0):
    nx, ny, nz, c, cs, u = case
    B0, Fx = 0.02, 2e-6
    o = oracle.Oracle3D(nx, ny, nz, 0.8, 0.7, B0, Fx, c[0], c[1], u[0], u[1], side=True, c_back=cs[0],
                        c_front=cs[1])
    f_rest, g_rest = o.f.copy(), o.g.copy()
    # a perturbation large enough that the deviations the parity bound is relative to (>~1e-4) sit well
    # above the FP64 rounding of the O(1) absolute populations the oracle works in (~1e-15)
    rng = np.random.default_rng(seed)
    o.f += 1e-2 * rng.uniform(-1, 1, o.f.shape) * np.abs(o.f)
    o.g += 1e-4 * rng.uniform(-1, 1, o.g.shape)
    gpu = l3.Lattice3D(nx, ny, nz, 0.8, 0.7, B0, Fx, storage)
    gpu.set_walls(c[0], c[1], u[0], u[1])
    gpu.set_side_walls(cs[0], cs[1])
    gpu.set_state(o.f, o.g)
    return o, gpu, f_rest, g_rest


def _fields_close(mo, mg, rel):
    u_scale = float(np.max(np.abs(mo[1:4])))
    b_scale = max(float(np.max(np.abs(mo[4]))), float(np.max(np.abs(mo[6]))))
    by_scale = float(np.max(np.abs(mo[5] - np.mean(mo[5]))) + 1e-300)
    assert np.max(np.abs(mg[0] - mo[0])) <= rel * np.max(np.abs(mo[0]))
    assert np.max(np.abs(mg[1:4] - mo[1:4])) <= rel * u_scale
    assert np.max(np.abs(mg[[4, 6]] - mo[[4, 6]])) <= rel * b_scale
    assert np.max(np.abs(mg[5] - mo[5])) <= rel * max(by_scale, b_scale)


@pytest.mark.parametrize("case", CASES)
def test_duct_fp64_matches_oracle(l3, case):
    o, gpu, f_rest, g_rest = _pair(l3, case, "f64")
    for n in (1, 39):
        o.step(n)
        gpu.step(n)
        fg, gg = gpu.get_state()
        df = float(np.max(np.abs(o.f - f_rest)))
        dg = float(np.max(np.abs(o.g - g_rest)))
        # relative to the largest deviation, with a floor at the FP64 rounding of the absolute
        # populations the oracle steps (64 ulp of max |f|): nx = 1 ducts damp the perturbation fast
        floor_f = 64 * np.finfo(np.float64).eps * float(np.max(np.abs(o.f)))
        floor_g = 64 * np.finfo(np.float64).eps * float(np.max(np.abs(o.g)))
        assert np.max(np.abs(fg - o.f)) <= REL64 * df + floor_f
        assert np.max(np.abs(gg - o.g)) <= REL64 * dg + floor_g
        _fields_close(o.moments(), gpu.moments(), REL64)
    gpu.close()


@pytest.mark.parametrize("case", CASES[:3])
def test_duct_fp32_matches_oracle(l3, case):
    o, gpu, _, _ = _pair(l3, case, "f32")
    o.step(40)
    gpu.step(40)
    _fields_close(o.moments(), gpu.moments(), 1e-4)
    gpu.close()


@pytest.mark.parametrize("storage,us", [("f32", 2.0 ** -24), ("bf16", 2.0 ** -9), ("f16", 2.0 ** -11)])
def test_duct_reduced_precision_one_step(l3, storage, us):
    case = CASES[1]
    o, gpu, f_rest, g_rest = _pair(l3, case, storage)
    o.step(1)
    gpu.step(1)
    fg, gg = gpu.get_state()
    df = float(np.max(np.abs(o.f - f_rest)))
    dg = float(np.max(np.abs(o.g - g_rest)))
    assert np.max(np.abs(fg - o.f)) <= 8 * us * df
    assert np.max(np.abs(gg - o.g)) <= 8 * us * dg
    gpu.close()


def test_duct_side_walls_reopen(l3):
    """enable = 0 returns the handle to the periodic channel: the same bits as a handle that never had
    side walls."""
    case = (4, 9, 6, (0.3, 0.3), (0.5, 0.5), (0.0, 0.0))
    _, a, _, _ = _pair(l3, case, "f64")
    _, b, _, _ = _pair(l3, case, "f64")
    b.set_side_walls(0.0, 0.0, enable=False)
    a.set_side_walls(0.5, 0.5)
    a.set_side_walls(0.0, 0.0, enable=False)
    a.step(10)
    b.step(10)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


@pytest.mark.parametrize("ha,ch,cs", [(5.0, 0.5, 0.3), (8.0, math.inf, 1.0)])
def test_duct_steady_second_order(l3, ha, ch, cs):
    """Errors against the Richardson-extrapolated finite-difference solution (itself within ~3e-5 of
    the series where that applies) on 12^2, 24^2 and 48^2 ducts."""
    tau = 0.8
    nu, eta = (tau - 0.5) / 3, (tau - 0.5) / 4
    errs = []
    for n in (12, 24, 48):
        a = n / 2
        B0 = ha * math.sqrt(nu * eta) / a
        F = 1e-6 * (16 / n) ** 2
        gpu = l3.Lattice3D(1, n, n, tau, tau, B0, F, "f64")
        gpu.set_walls(ch, ch)
        gpu.set_side_walls(cs, cs)
        steps, r, status = gpu.run_to_steady(1e-11, 200, 2_000_000)
        m = gpu.moments()
        u, B = m[1][:, :, 0].T, m[4][:, :, 0].T
        uf, Bf = duct.fd_on_lattice_extrapolated(n, n, B0, nu, eta, F, ch, ch, cs, cs, refine=2)
        errs.append((math.sqrt(np.mean((u - uf) ** 2)) / np.max(np.abs(uf)),
                     math.sqrt(np.mean((B - Bf) ** 2)) / np.max(np.abs(Bf))))
        gpu.close()
    for k in range(2):
        for i in range(2):
            order = math.log(errs[i][k] / errs[i + 1][k], 2)
            assert 1.8 < order < 2.2, (k, errs)
    assert max(errs[-1]) < 3e-3

"""Three-dimensional channel on the GPU (include/lks3d.h) against the 3D FP64 oracle.

FP64 storage: moments per field within 1e-11 of max|field| and populations within 1e-11 of the
largest deviation from rest, after 1 and after 40 steps from the same perturbed state, on lattices
with a ragged x block (300 = 256 + 44), nx = 1, ny = 2 (both rows are wall rows) and every wall
setting (insulating, finite, perfectly conducting, moving).  FP32 storage: within 1e-4 of the field
scale after 40 steps (FP32 rounding of deviations ~1e-3 over a few tens of steps).  FP32, BF16 and
FP16 storage after one step: populations within 8 u_s of the largest deviation from rest (u_s the
storage's unit roundoff), and FP16 over 2000 steps of a Hartmann flow within the bounds of the
two-dimensional channel.  Steady state: closed-form Hartmann profiles with the D3Q7 diffusivity."""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as an

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
    # nx, ny, nz, (c_bot, c_top), (u_bot, u_top)
    (37, 9, 5, (0.3, math.inf), (0.0, 0.05)),
    (300, 6, 3, (0.0, 2.0), (-0.02, 0.04)),
    (1, 12, 1, (1e4, 0.1), (0.03, 0.0)),
    (4, 2, 7, (0.5, 0.5), (0.0, -0.03)),
]


def _pair(l3, nx, ny, nz, c, u, storage, seed=0):
    B0, Fx = 0.02, 2e-6
    o = oracle.Oracle3D(nx, ny, nz, 0.8, 0.7, B0, Fx, c[0], c[1], u[0], u[1])
    f_rest, g_rest = o.f.copy(), o.g.copy()
    rng = np.random.default_rng(seed)
    o.f += 1e-3 * rng.uniform(-1, 1, o.f.shape) * np.abs(o.f)
    o.g += 1e-5 * rng.uniform(-1, 1, o.g.shape)
    gpu = l3.Lattice3D(nx, ny, nz, 0.8, 0.7, B0, Fx, storage)
    gpu.set_walls(c[0], c[1], u[0], u[1])
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
def test_fp64_matches_oracle(l3, case):
    nx, ny, nz, c, u = case
    o, gpu, f_rest, g_rest = _pair(l3, nx, ny, nz, c, u, "f64")
    for n in (1, 39):
        o.step(n)
        gpu.step(n)
        fg, gg = gpu.get_state()
        df = float(np.max(np.abs(o.f - f_rest)))
        dg = float(np.max(np.abs(o.g - g_rest)))
        assert np.max(np.abs(fg - o.f)) <= REL64 * df
        assert np.max(np.abs(gg - o.g)) <= REL64 * dg
        _fields_close(o.moments(), gpu.moments(), REL64)
    gpu.close()


@pytest.mark.parametrize("case", CASES[:2])
def test_fp32_close_to_oracle(l3, case):
    nx, ny, nz, c, u = case
    o, gpu, _, _ = _pair(l3, nx, ny, nz, c, u, "f32", seed=1)
    o.step(40)
    gpu.step(40)
    _fields_close(o.moments(), gpu.moments(), 1e-4)
    gpu.close()


def test_profiles_and_residual_consistent(l3):
    o, gpu, _, _ = _pair(l3, 37, 9, 5, (0.3, 0.3), (0.0, 0.05), "f64", seed=2)
    gpu.residual()
    m0 = gpu.moments()
    gpu.step(10)
    m1 = gpu.moments()
    u, b = gpu.profiles()
    assert np.allclose(u, m1[1].mean(axis=(0, 2)), rtol=1e-13, atol=1e-18)
    assert np.allclose(b, m1[4].mean(axis=(0, 2)), rtol=1e-13, atol=1e-18)
    ru, rb = gpu.residual()
    ru_h = np.sqrt(np.sum((m1[1] - m0[1]) ** 2) / np.sum(m1[1] ** 2))
    rb_h = np.sqrt(np.sum((m1[4] - m0[4]) ** 2) / np.sum(m1[4] ** 2))
    assert ru == pytest.approx(ru_h, rel=1e-9) and rb == pytest.approx(rb_h, rel=1e-9)
    gpu.close()


@pytest.mark.parametrize("ha,c", [(5.0, 0.5), (10.0, math.inf)])
def test_steady_hartmann_profiles(l3, ha, c):
    ny, tau = 48, 0.8
    a = ny / 2
    tm2 = 0.5 + 0.75 * (tau - 0.5)     # D2Q5 tau_m with the D3Q7 diffusivity
    b0 = an.b0_from_ha(ha, a, tau, tm2)
    fx = an.force_for_centre_speed(0.01, ha, c, a, tau)
    gpu = l3.Lattice3D(3, ny, 2, tau, tau, b0, fx, "f64")
    gpu.set_walls(c, c)
    steps, r, status = gpu.run_to_steady(1e-9, 200, 400_000)
    assert r < 1e-9
    u, b = gpu.profiles()
    ua, ba = an.hartmann_profiles(gpu.y(), a, ha, c, fx, tau, tm2)
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3
    gpu.close()


# One step of a 16-bit (or FP32) handle against the FP64 oracle from the same state: the stored
# deviations carry a rounding error <= u_s |d| each, the collision maps them with coefficients of
# magnitude <= 1 (|1 - 1/tau_f| = 0.25, |1 - 1/tau_m| = 0.43, equilibrium weights summing to 1), the
# FP32 moments, equilibria and wall terms add a few roundings of that size and the result is
# rounded once more: max|d_gpu - d_oracle| <= 8 u_s max|d|.
ONE_STEP = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}


# 16-bit storage with nx a multiple of 8 and nx <= 512 is staged through shared memory in tasks of
# R = min(ny, 512 // nx) whole rows: nx = 8 (R = ny: both wall rows in one task), 16 with nz = 1
# (the z pull wraps onto the same plane), 128 with ny = 10 (R = 4, a ragged last task of 2 rows),
# 264 (R = 1) and 512 (the widest staged rows).  Other nx run one node per thread: 37, 300, 2, 4,
# 518 and 520 (wider than a task).
STORAGE_CASES = CASES[:2] + [
    (2, 5, 3, (0.2, 1.0), (0.01, -0.02)),
    (518, 3, 2, (math.inf, 0.0), (0.0, 0.03)),
    (4, 2, 7, (0.5, 0.5), (0.0, -0.03)),
    (8, 4, 3, (0.3, 2.0), (0.02, 0.0)),
    (264, 3, 2, (1.0, math.inf), (0.0, 0.04)),
    (16, 5, 1, (0.0, 0.7), (-0.03, 0.02)),
    (128, 10, 3, (0.4, 0.4), (0.01, 0.02)),
    (512, 3, 2, (2.0, 0.0), (0.0, -0.01)),
    (520, 2, 2, (0.1, 0.9), (0.02, 0.0)),
]


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", STORAGE_CASES)
def test_reduced_precision_one_step(l3, case, storage):
    nx, ny, nz, c, u = case
    o, gpu, f_rest, g_rest = _pair(l3, nx, ny, nz, c, u, storage, seed=5)
    o.step(1)
    gpu.step(1)
    fg, gg = gpu.get_state()
    df = float(np.max(np.abs(o.f - f_rest)))
    dg = float(np.max(np.abs(o.g - g_rest)))
    assert np.max(np.abs(fg - o.f)) <= 8 * ONE_STEP[storage] * df
    assert np.max(np.abs(gg - o.g)) <= 8 * ONE_STEP[storage] * dg
    gpu.close()


# Long run: each step adds a relative error ~u_s to every stored deviation; the error of u_x and
# B_x behaves like a random walk damped on the diffusive time a^2/nu, plus the loss of sub-ulp
# increments.  FP16 bounds relative to max|field| as in the two-dimensional channel: 1e-1 for u_x,
# 5e-2 for B_x; FP32 1e-4 for both.
@pytest.mark.parametrize("storage,bounds", [("f32", (1e-4, 1e-4)), ("f16", (1e-1, 5e-2))])
def test_reduced_precision_long_run(l3, storage, bounds):
    nx, ny, nz, ha, c, tau = 8, 33, 2, 10.0, 0.5, 0.8
    a = ny / 2
    tm2 = 0.5 + 0.75 * (tau - 0.5)
    b0 = an.b0_from_ha(ha, a, tau, tm2)
    fx = an.force_for_centre_speed(0.01, ha, c, a, tau)
    o = oracle.Oracle3D(nx, ny, nz, tau, tau, b0, fx, c, c, 0.0, 0.0)
    rng = np.random.default_rng(11)
    o.f += 1e-3 * rng.uniform(-1, 1, o.f.shape) * np.abs(o.f)
    gpu = l3.Lattice3D(nx, ny, nz, tau, tau, b0, fx, storage)
    gpu.set_walls(c, c)
    gpu.set_state(o.f, o.g)
    o.step(2000)
    gpu.step(2000)
    mo, mg = o.moments(), gpu.moments()
    assert np.max(np.abs(mg[1] - mo[1])) <= bounds[0] * np.max(np.abs(mo[1]))
    assert np.max(np.abs(mg[4] - mo[4])) <= bounds[1] * np.max(np.abs(mo[4]))
    gpu.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_staged_pair_path_bitwise_equals_one_node_kernel(l3, storage):
    """16-bit storage with nx = 40 runs the staged kernel (two nodes per thread, packed FP32x2
    arithmetic), nx = 37 the one-node kernel.  On a flow that depends on y only (rest start, body
    force, moving wall) every (x, z) column of both must be bit-identical: the per-node arithmetic
    is the same sequence of individually rounded operations."""
    out = []
    for nx in (37, 40):
        g = l3.Lattice3D(nx, 21, 3, 0.7, 0.9, 0.02, 2e-5, storage)
        g.set_walls(0.4, math.inf, 0.0, 0.04)
        g.step(150)
        f, gg = g.get_state()
        assert np.all(f == f[..., :1]) and np.all(f == f[:, :1])
        assert np.all(gg == gg[..., :1]) and np.all(gg == gg[:, :, :1])
        assert np.max(np.abs(f[:, 0, :, 0] - f[:, 0, :1, 0])) > 0  # the flow is not the rest state
        out.append((f[:, 0, :, 0].copy(), gg[:, :, 0, :, 0].copy()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_kernels_agree_bitwise_on_a_tiled_perturbed_state(l3, storage):
    """nx = 12 runs the one-node kernel, nx = 24 the staged one (two nodes per thread on FP32x2): the
    wide lattice started from the narrow one's perturbed state tiled twice in x stays that state
    tiled, bit for bit, with every node carrying its own values."""
    o, a, _, _ = _pair(l3, 12, 6, 3, (0.3, 2.0), (0.01, 0.04), storage, seed=9)
    b = l3.Lattice3D(24, 6, 3, 0.8, 0.7, 0.02, 2e-6, storage)
    b.set_walls(0.3, 2.0, 0.01, 0.04)
    f, g = a.get_state()
    b.set_state(np.concatenate([f, f], axis=-1), np.concatenate([g, g], axis=-1))
    for n in (1, 9):
        a.step(n)
        b.step(n)
        fa, ga = a.get_state()
        fb, gb = b.get_state()
        assert np.array_equal(fb, np.concatenate([fa, fa], axis=-1)), n
        assert np.array_equal(gb, np.concatenate([ga, ga], axis=-1)), n
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_full_size_one_step(l3, storage):
    """The 3D benchmark size (256^3; FP32: the one-node kernel, BF16: the staged kernel with ~100
    tasks per persistent block) with both walls at c = 1 and the top one moving, from a perturbed
    state: one step against the FP64 oracle over the whole lattice, every population of the planes
    y = 0, 1, 127, 254, 255 within 8 u_s of the largest deviation from rest."""
    n = 256
    o, gpu, f_rest, g_rest = _pair(l3, n, n, n, (1.0, 1.0), (0.0, 0.05), storage, seed=6)
    o.step(1)
    gpu.step(1)
    fg, gg = gpu.get_state()
    gpu.close()
    ys = [0, 1, 127, 254, 255]
    df = float(np.max(np.abs(o.f - f_rest)))
    dg = float(np.max(np.abs(o.g - g_rest)))
    assert np.max(np.abs(fg[:, :, ys] - o.f[:, :, ys])) <= 8 * ONE_STEP[storage] * df
    assert np.max(np.abs(gg[:, :, :, ys] - o.g[:, :, :, ys])) <= 8 * ONE_STEP[storage] * dg

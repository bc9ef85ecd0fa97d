"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

FP64 storage: element-wise, max|GPU - oracle| / max|oracle| <= 1e-11 per field (the bound the
scheme's specification sets; the two differ only in rounding order and FMA contraction).
FP32 / BF16 / FP16 storage of deviations with FP32 arithmetic: tolerances derived in the test
docstrings from the storage precision.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as an

pytestmark = pytest.mark.gpu

REL64 = 1e-11


@pytest.fixture(scope="module")
def lks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks as mod
    build.build()
    mod.load()
    return mod


def _pair(lks, nx, ny, closure, storage="f64", tau_f=0.8, tau_m=0.8, B0=0.03, Fx=0.0, c=(0.0, 0.0), u=(0.0, 0.0),
          seed=0, amp=0.0):
    cl = oracle.LINK if closure == "link" else oracle.MOMENT
    o = oracle.Oracle(nx, ny, tau_f, tau_m, B0, Fx, cl, c[0], c[1], u[0], u[1], seed=seed, perturb_amp=amp)
    g = lks.Lattice(nx, ny, tau_f, tau_m, B0, Fx, closure, storage, seed=seed, perturb_amp=amp)
    g.set_walls(c[0], c[1], u[0], u[1])
    return o, g


def _relmax(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (scale if scale > 0 else 1.0)


def _compare_fields(o, g, rel, rel_pop=None):
    fo, go = o.f, o.g
    fg, gg = g.get_state()
    mo, mg = o.moments(), g.moments()
    # fields: rho - 1, u (vector), B_x, B_y - B0
    errs = {
        "rho": _relmax(mg[0], mo[0]),
        "u": max(_relmax(mg[1], mo[1]), float(np.max(np.abs(mg[2] - mo[2]))) / max(1e-300, float(np.max(np.abs(mo[1:3]))))),
        "bx": _relmax(mg[3], mo[3]) if np.max(np.abs(mo[3])) > 0 else float(np.max(np.abs(mg[3]))),
        "by": float(np.max(np.abs(mg[4] - mo[4]))) / max(1e-300, float(np.max(np.abs(mo[4])))),
    }
    if rel_pop is not None:
        errs["f"] = float(np.max(np.abs(fg - fo))) / float(np.max(np.abs(fo)))
        errs["g"] = float(np.max(np.abs(gg - go))) / max(1e-300, float(np.max(np.abs(go))))
    for k, v in errs.items():
        lim = rel_pop if k in ("f", "g") else rel
        assert v <= lim, (k, v, lim, errs)
    return errs


@pytest.mark.parametrize("closure", ["link", "moment"])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_initial_state_matches_oracle(lks, closure, storage):
    """Init (equilibria at rho = 1, B = (0, B0), seeded u0) equals the oracle's, up to the
    storage rounding of the deviations."""
    o, g = _pair(lks, 37, 5, closure, storage, seed=1234, amp=1e-3)
    fg, gg = g.get_state()
    tol = {"f64": 1e-16, "f32": 1e-9, "bf16": 2e-5, "f16": 3e-6}[storage]
    assert np.max(np.abs(fg - o.f)) <= tol
    assert np.max(np.abs(gg - o.g)) <= tol


def test_hartmann_channel_fp64_parity_20000_steps(lks):
    """4 x 65 link-based Hartmann channel, Ha = 10, c = 0.1, tau_f = tau_m = 0.8, 2e4 steps (FP64)."""
    ny, ha, c = 65, 10.0, 0.1
    a = ny / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
    o, g = _pair(lks, 4, ny, "link", "f64", B0=b0, Fx=fx, c=(c, c))
    o.step(20000)
    g.step(20000)
    errs = _compare_fields(o, g, REL64, REL64)
    u, b = g.profiles()
    ua, ba = an.hartmann_profiles(g.y(), a, ha, c, fx, 0.8, 0.8)
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3


CASES = [
    # nx spans several 256-thread blocks with a ragged tail; moving walls, finite / zero / infinite c
    dict(nx=300, ny=7, closure="link", c=(0.3, 2.0), u=(0.0, 0.04), Fx=1e-5, amp=1e-2),
    dict(nx=300, ny=7, closure="moment", c=(0.3, 2.0), u=(-0.02, 0.04), Fx=1e-5, amp=1e-2),
    dict(nx=33, ny=40, closure="link", c=(0.0, math.inf), u=(0.01, -0.03), Fx=0.0, amp=5e-3),
    dict(nx=33, ny=40, closure="moment", c=(math.inf, 0.0), u=(0.0, 0.05), Fx=2e-5, amp=5e-3),
    dict(nx=1, ny=3, closure="moment", c=(0.5, 0.5), u=(0.0, 0.05), Fx=0.0, amp=0.0),
    dict(nx=1, ny=2, closure="link", c=(1e4, 0.0), u=(0.0, 0.05), Fx=1e-4, amp=0.0),
    dict(nx=257, ny=9, closure="link", c=(0.0, 0.0), u=(0.0, 0.0), Fx=0.0, amp=1e-2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dx%d" % (c["closure"], c["nx"], c["ny"]))
def test_fp64_parity_cases(lks, case):
    o, g = _pair(lks, case["nx"], case["ny"], case["closure"], "f64", tau_f=0.7, tau_m=0.9, B0=0.02,
                 Fx=case["Fx"], c=case["c"], u=case["u"], seed=99, amp=case["amp"])
    for n in (1, 7, 130):  # 130 > the graph length: exercises graph launch plus direct launches
        o.step(n)
        g.step(n)
        _compare_fields(o, g, REL64, REL64)


def test_graph_steps_equal_direct_steps(lks):
    """Steps launched through the captured CUDA graph are bitwise the same as direct launches."""
    a = lks.Lattice(50, 11, 0.7, 0.9, 0.02, 1e-5, "moment", "f32", seed=3, perturb_amp=1e-2)
    b = lks.Lattice(50, 11, 0.7, 0.9, 0.02, 1e-5, "moment", "f32", seed=3, perturb_amp=1e-2)
    for h in (a, b):
        h.set_walls(0.2, 0.7, 0.0, 0.03)
    a.step(200)
    for _ in range(200):
        b.step(1)
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_moments_profiles_and_residual(lks):
    """lks_moments (nodes, profiles) and lks_residual against the oracle's state."""
    o, g = _pair(lks, 70, 12, "moment", "f64", B0=0.02, Fx=1e-5, c=(0.2, 0.9), u=(0.0, 0.03), seed=5, amp=1e-2)
    prev = o.moments()
    o.step(25)
    g.step(25)
    mo, mg = o.moments(), g.moments()
    np.testing.assert_allclose(mg, mo, rtol=1e-11, atol=1e-14)
    pg = g.moments(lks.MOMENTS_PROFILES)
    np.testing.assert_allclose(pg, mo.mean(axis=2), rtol=1e-11, atol=1e-14)
    ru, rb = g.residual()
    ru_o = np.sqrt(np.sum((mo[1] - prev[1]) ** 2) / np.sum(mo[1] ** 2))
    rb_o = np.sqrt(np.sum((mo[3] - prev[3]) ** 2) / np.sum(mo[3] ** 2))
    assert ru == pytest.approx(ru_o, rel=1e-9) and rb == pytest.approx(rb_o, rel=1e-9)


def test_set_state_roundtrip_and_continue(lks):
    """lks_set_state loads an oracle state; continuing on the GPU tracks the oracle."""
    o, g = _pair(lks, 40, 9, "link", "f64", B0=0.02, Fx=1e-5, c=(0.5, 0.5), seed=8, amp=1e-2)
    o.step(10)
    g.set_state(o.f, o.g)
    fg, gg = g.get_state()
    assert np.max(np.abs(fg - o.f)) < 1e-16 and np.max(np.abs(gg - o.g)) < 1e-16
    o.step(40)
    g.step(40)
    _compare_fields(o, g, REL64, REL64)


# Reduced precision.  Deviations d = f - f_rest are stored rounded to nearest in the storage type
# (unit roundoff u_s: 2^-24 FP32, 2^-11 FP16, 2^-8 BF16) and all arithmetic is FP32.
#
# One step: the inputs carry |error| <= u_s |d|; the collision maps them with coefficients of
# magnitude <= 1 (|1 - 1/tau| = 0.25 and the equilibrium weights sum to 1 over the node), the FP32
# arithmetic of the moments, equilibria and closures adds a few roundings of the same size, and the
# result is rounded once more: max|d_gpu - d_oracle| <= 8 u_s max|d| after one step (measured up
# to 5.3 u_s).
#
# Long runs: every step adds a fresh relative error u_s to every stored deviation; the error of u
# then behaves like a random walk damped on the channel's diffusive time a^2/nu (~2700 steps
# here), i.e. u_s * sqrt(2700) ~ 50 u_s, plus the systematic loss of sub-ulp increments in 16-bit
# storage.  Bounds after 2000 steps (relative to max|field|): FP32 1e-4 (measured 2-3e-5), FP16
# 1e-1 for u_x and 5e-2 for B_x (measured 3e-2 and 1e-2).  BF16 carries only 8 bits: its long-run
# error (0.6 in u_x, 0.1 in B_x on this case) is reported by the benchmark, not gated here.
ONE_STEP = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
LONG_RUN = {"f32": (1e-4, 1e-4), "f16": (1e-1, 5e-2)}


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
def test_reduced_precision_one_step(lks, storage, closure):
    o, g = _pair(lks, 37, 11, closure, storage, B0=0.02, Fx=1e-5, c=(0.4, 3.0), u=(0.0, 0.04), seed=17, amp=1e-2)
    o0 = oracle.Oracle(37, 11, 0.8, 0.8, 0.02, 1e-5, oracle.LINK if closure == "link" else oracle.MOMENT,
                       seed=0, perturb_amp=0.0)
    f_rest, g_rest = o0.f, o0.g          # rest equilibrium (rho = 1, u = 0, B = (0, B0))
    o.step(1)
    g.step(1)
    fg, gg = g.get_state()
    df = np.max(np.abs(o.f - f_rest))
    dg = np.max(np.abs(o.g - g_rest))
    assert np.max(np.abs(fg - o.f)) <= 8 * ONE_STEP[storage] * df
    assert np.max(np.abs(gg - o.g)) <= 8 * ONE_STEP[storage] * dg


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
def test_reduced_precision_long_run(lks, storage, closure):
    ny, ha, c = 33, 10.0, 0.5
    a = ny / 2 if closure == "link" else (ny - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
    o, g = _pair(lks, 16, ny, closure, storage, B0=b0, Fx=fx, c=(c, c), u=(0.0, 0.0), seed=11, amp=1e-3)
    o.step(2000)
    g.step(2000)
    mo, mg = o.moments(), g.moments()
    eu = _relmax(mg[1], mo[1])
    eb = _relmax(mg[3], mo[3])
    tu, tb = LONG_RUN[storage]
    assert eu <= tu and eb <= tb, (eu, eb)


def test_full_size_lattice_columns_match_oracle(lks):
    """4096 x 4096 moment-based Hartmann-Couette channel (the timed configuration) from rest: the
    solution does not depend on x, so every column of the GPU lattice must equal the oracle's
    4 x 4096 run (FP64, 20 steps), and all columns must agree."""
    import torch
    n, ha, c = 4096, 20.0, 1.0
    a = (n - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    o = oracle.Oracle(4, n, 0.8, 0.8, b0, 0.0, oracle.MOMENT, c, c, 0.0, 0.05)
    g = lks.Lattice(n, n, 0.8, 0.8, b0, 0.0, "moment", "f64")
    g.set_walls(c, c, 0.0, 0.05)
    o.step(20)
    g.step(20)
    out = torch.empty((5, n, n), dtype=torch.float64, device="cuda")
    g.moments_device(out)
    torch.cuda.synchronize()
    mo = o.moments()
    for m in (1, 3):
        col = out[m].cpu().numpy()
        assert np.max(np.abs(col - col[:, :1])) == 0.0
        assert _relmax(col[:, 1234], mo[m][:, 0]) <= REL64
    del out
    g.close()


def test_full_size_perturbed_fp64_sampled_rows(lks):
    """4096 x 4096 with a seeded perturbation, 3 steps: the oracle computes the full lattice (OpenMP)
    and rows near both walls and in the interior are compared element by element."""
    n = 4096
    o, g = _pair(lks, n, n, "moment", "f64", B0=0.001, Fx=1e-6, c=(1.0, 1.0), u=(0.0, 0.05), seed=20211227,
                 amp=1e-3)
    o.step(3)
    g.step(3)
    mo, mg = o.moments(), g.moments()
    rows = [0, 1, 2, 1000, 2047, 4093, 4094, 4095]
    for m in (1, 2, 3):
        assert _relmax(mg[m][rows], mo[m][rows]) <= REL64
    g.close()


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_full_size_timed_configuration_one_step(lks, storage):
    """The benchmark's timed configuration itself (4096 x 4096, moment-based closure, c = 1 on both
    walls, top wall moving) in its FP32 storage and the 16-bit extras' (staged kernel, ~108 tasks
    per persistent block), from a seeded perturbation: one step against the FP64 oracle over the
    whole lattice, every population of rows at both walls and in the interior within the one-step
    bound 8 u_s max|d| derived above."""
    n = 4096
    o, g = _pair(lks, n, n, "moment", storage, B0=0.001, Fx=1e-6, c=(1.0, 1.0), u=(0.0, 0.05), seed=20211228,
                 amp=1e-3)
    rest = oracle.Oracle(4, 4, 0.8, 0.8, 0.001, 1e-6, oracle.MOMENT, seed=0, perturb_amp=0.0)
    f_rest = rest.f[:, :1, :1]            # the rest state is the same at every node
    g_rest = rest.g[:, :, :1, :1]
    o.step(1)
    g.step(1)
    fg, gg = g.get_state()
    g.close()
    rows = [0, 1, 2, 1000, 2047, 4093, 4094, 4095]
    df = np.max(np.abs(o.f - f_rest))
    dg = np.max(np.abs(o.g - g_rest))
    assert np.max(np.abs(fg[:, rows] - o.f[:, rows])) <= 8 * ONE_STEP[storage] * df
    assert np.max(np.abs(gg[:, :, rows] - o.g[:, :, rows])) <= 8 * ONE_STEP[storage] * dg


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
def test_pair_kernel_bitwise_equals_single_node_kernel(lks, storage, closure):
    """16-bit storage with even nx runs the two-nodes-per-thread kernel, odd nx the one-node kernel,
    and nx a multiple of 8 of at least 1024 the staged kernel (rows through shared memory, packed
    FP32x2 arithmetic): 1032 (a full and a ragged segment, wrapped halos), 2056 (a middle segment
    with both halos in one copy).  On an x-independent flow (rest start, body force and moving wall)
    every column of all of them must be bit-identical: the per-node arithmetic is the same."""
    out = []
    for nx in (37, 38, 64, 1032, 2056):
        g = lks.Lattice(nx, 21, 0.7, 0.9, 0.02, 2e-5, closure, storage)
        g.set_walls(0.4, math.inf, 0.0, 0.04)
        g.step(150)
        f, gg = g.get_state()
        for a in range(9):
            assert np.all(f[a] == f[a][:, :1])
        out.append((f[:, :, 0].copy(), gg[:, :, :, 0].copy()))
        g.close()
    for f, gg in out[1:]:
        assert np.array_equal(f, out[0][0]) and np.array_equal(gg, out[0][1])


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
def test_pair_kernel_perturbed_matches_oracle_one_step(lks, storage, closure):
    """Perturbed lattice with even nx spanning several warps and rows that do not fill a warp, and
    the staged kernel's segment layouts (1032, 2056): one step against the oracle within the one-step
    bound of the storage type."""
    for nx, ny in ((38, 7), (130, 5), (2, 9), (1032, 6), (2056, 3)):
        o, g = _pair(lks, nx, ny, closure, storage, B0=0.02, Fx=1e-5, c=(0.4, 3.0), u=(0.0, 0.04), seed=3,
                     amp=1e-2)
        o0 = oracle.Oracle(nx, ny, 0.8, 0.8, 0.02, 1e-5, oracle.LINK if closure == "link" else oracle.MOMENT)
        o.step(1)
        g.step(1)
        fg, gg = g.get_state()
        assert np.max(np.abs(fg - o.f)) <= 8 * ONE_STEP[storage] * np.max(np.abs(o.f - o0.f))
        assert np.max(np.abs(gg - o.g)) <= 8 * ONE_STEP[storage] * np.max(np.abs(o.g - o0.g))
        g.close()


# ---- the paper's own coupling (Lorentz force in the source), kernel variant ----

def _pair_lorentz(lks, nx, ny, closure, storage="f64", tau_f=0.7, tau_m=0.9, B0=0.03, Fx=0.0, c=(0.0, 0.0),
                  u=(0.0, 0.0), seed=0, amp=0.0):
    cl = oracle.LINK if closure == "link" else oracle.MOMENT
    o = oracle.Oracle(nx, ny, tau_f, tau_m, B0, Fx, cl, c[0], c[1], u[0], u[1], seed=seed, perturb_amp=amp,
                      coupling=1)
    g = lks.Lattice(nx, ny, tau_f, tau_m, B0, Fx, closure, storage, seed=seed, perturb_amp=amp, coupling="lorentz")
    g.set_walls(c[0], c[1], u[0], u[1])
    return o, g


@pytest.mark.parametrize("case", CASES[:5], ids=lambda c: "%s-%dx%d" % (c["closure"], c["nx"], c["ny"]))
def test_lorentz_fp64_parity_cases(lks, case):
    """Lorentz-force coupling (the oracle iterates u and J to a fixed point, the kernel solves the
    linear system exactly): FP64 parity <= 1e-11 on populations and moments."""
    o, g = _pair_lorentz(lks, case["nx"], case["ny"], case["closure"], "f64", B0=0.04, Fx=case["Fx"], c=case["c"],
                         u=case["u"], seed=99, amp=case["amp"])
    for n in (1, 7, 130):
        o.step(n)
        g.step(n)
        _compare_fields(o, g, REL64, REL64)


@pytest.mark.parametrize("closure", ["link", "moment"])
def test_lorentz_hartmann_channel_fp64_and_analytic(lks, closure):
    ny, ha, c = 65, 10.0, 0.5
    a = ny / 2 if closure == "link" else (ny - 1) / 2
    b0 = an.b0_from_ha(ha, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, ha, c, a, 0.8)
    o, g = _pair_lorentz(lks, 4, ny, closure, "f64", tau_f=0.8, tau_m=0.8, B0=b0, Fx=fx, c=(c, c))
    o.step(20000)
    g.step(20000)
    _compare_fields(o, g, REL64, REL64)
    u, b = g.profiles()
    ua, ba = an.hartmann_profiles(g.y(), a, ha, c, fx, 0.8, 0.8)
    assert an.rel_l2(u, ua) < 5e-3 and an.rel_l2(b, ba) < 5e-3


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
def test_lorentz_reduced_precision(lks, storage, closure):
    """Same bounds as the Maxwell-stress coupling: one step within 8 u_s, 2000 steps within the
    long-run bounds."""
    o, g = _pair_lorentz(lks, 38, 11, closure, storage, B0=0.02, Fx=1e-5, c=(0.4, 3.0), u=(0.0, 0.04), seed=17,
                         amp=1e-2)
    o0 = oracle.Oracle(38, 11, 0.7, 0.9, 0.02, 1e-5, oracle.LINK, coupling=1)
    o.step(1)
    g.step(1)
    fg, gg = g.get_state()
    assert np.max(np.abs(fg - o.f)) <= 8 * ONE_STEP[storage] * np.max(np.abs(o.f - o0.f))
    assert np.max(np.abs(gg - o.g)) <= 8 * ONE_STEP[storage] * np.max(np.abs(o.g - o0.g))
    o.step(1999)
    g.step(1999)
    mo, mg = o.moments(), g.moments()
    tu, tb = LONG_RUN[storage]
    assert _relmax(mg[1], mo[1]) <= tu and _relmax(mg[3], mo[3]) <= tb


def test_lorentz_pair_kernel_bitwise(lks):
    out = []
    for nx in (37, 38, 1032):
        g = lks.Lattice(nx, 21, 0.7, 0.9, 0.02, 2e-5, "moment", "f16", coupling="lorentz")
        g.set_walls(0.4, math.inf, 0.0, 0.04)
        g.step(150)
        f, gg = g.get_state()
        out.append((f[:, :, 0].copy(), gg[:, :, :, 0].copy()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_checkpoint_resume(lks, tmp_path):
    """save() / load() round trip: a run resumed from a checkpoint continues like the original."""
    o, g = _pair(lks, 40, 12, "moment", "f64", B0=0.02, Fx=1e-5, c=(0.3, 2.0), u=(0.0, 0.03), seed=4, amp=1e-2)
    g.step(37)
    path = str(tmp_path / "ckpt.npz")
    g.save(path)
    h = lks.Lattice(40, 12, 0.8, 0.8, 0.02, 1e-5, "moment", "f64")
    h.set_walls(0.3, 2.0, 0.0, 0.03)
    assert h.load(path) == 37
    g.step(50)
    h.step(50)
    fg, gg = g.get_state()
    fh, gh = h.get_state()
    assert np.max(np.abs(fg - fh)) < 1e-15 and np.max(np.abs(gg - gh)) < 1e-15


def test_c1_matches_stored_golden_profiles(lks):
    """The 4 x 65 Hartmann channel (link-based, Ha = 10, c = 0.1, 2e4 FP64 steps) against the
    profiles stored in tests/golden/c1_profiles.txt (written by the oracle): within 1e-11."""
    import os
    data = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_profiles.txt"))
    a = 32.5
    b0 = an.b0_from_ha(10.0, a, 0.8, 0.8)
    fx = an.force_for_centre_speed(0.01, 10.0, 0.1, a, 0.8)
    g = lks.Lattice(4, 65, 0.8, 0.8, b0, fx, "link", "f64")
    g.set_walls(0.1, 0.1)
    g.step(20000)
    u, bx = g.profiles()
    assert np.max(np.abs(u - data[:, 1])) <= REL64 * np.max(np.abs(data[:, 1]))
    assert np.max(np.abs(bx - data[:, 2])) <= REL64 * np.max(np.abs(data[:, 2]))
    g.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
@pytest.mark.parametrize("coupling", ["maxwell", "lorentz"])
def test_kernels_agree_bitwise_on_a_tiled_perturbed_state(lks, storage, closure, coupling):
    """A lattice of width 2 nx started from the perturbed state of a width-nx lattice tiled twice in x
    stays that state tiled, bit for bit, although the two widths run different kernels: nx = 516 the
    two-node kernel and 1032 the staged one; nx = 517 the one-node kernel and 1034 the two-node one.
    Unlike an x-independent flow, every node carries its own values, so any difference in the
    per-node arithmetic between the kernels shows."""
    for nx in (516, 517):
        a = lks.Lattice(nx, 7, 0.7, 0.9, 0.02, 2e-5, closure, storage, seed=5, perturb_amp=1e-2, coupling=coupling)
        b = lks.Lattice(2 * nx, 7, 0.7, 0.9, 0.02, 2e-5, closure, storage, coupling=coupling)
        for lat in (a, b):
            lat.set_walls(0.4, 3.0, 0.02, -0.04)
        f, g = a.get_state()
        b.set_state(np.concatenate([f, f], axis=-1), np.concatenate([g, g], axis=-1))
        for n in (1, 9):
            a.step(n)
            b.step(n)
            fa, ga = a.get_state()
            fb, gb = b.get_state()
            assert np.array_equal(fb, np.concatenate([fa, fa], axis=-1)), (nx, n)
            assert np.array_equal(gb, np.concatenate([ga, ga], axis=-1)), (nx, n)
        a.close()
        b.close()

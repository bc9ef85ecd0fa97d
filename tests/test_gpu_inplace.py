"""In-place (one-buffer, AA-pattern) stepping: after every pair of steps the single buffer holds
bit for bit the state the two-buffer step reaches, for every storage type, closure, coupling and
launch grid (1D for narrow lattices, 2D with a ragged last block for wide ones); FP64 in-place
runs match the oracle within 1e-11; odd step counts are refused."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

STORAGE_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}


@pytest.fixture(scope="module")
def lks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks as mod
    build.build()
    mod.load()
    return mod


def _raw(lat, storage):
    """The stored populations as raw bit patterns in node order: f planes, then g planes (the
    first buffer of the footprint, where a two-buffer handle's state sits after an even number of
    steps).  An in-place handle with 16-bit storage and even nx keeps its rows interleaved (word w
    holds nodes w and w + nx/2), so node x sits in slot 2 (x mod nx/2) + (x >= nx/2)."""
    lat.sync()
    sb = STORAGE_BYTES[storage]
    nx, ny = lat.nx, lat.ny
    n = nx * ny * sb
    f_bytes = (9 * n + 255) // 256 * 256
    buf = lat._buf.cpu().numpy()
    dt = {8: np.uint64, 4: np.uint32, 2: np.uint16}[sb]
    f = buf[: 9 * n].view(dt).reshape(9, ny, nx)
    g = buf[f_bytes: f_bytes + 10 * n].view(dt).reshape(10, ny, nx)
    if lat.inplace and sb == 2 and nx % 2 == 0:
        h = nx // 2
        slot = [2 * x if x < h else 2 * (x - h) + 1 for x in range(nx)]
        f, g = f[:, :, slot], g[:, :, slot]
    return np.concatenate([f.ravel(), g.ravel()])


def _make(lks, nx, ny, closure, storage, coupling, inplace, c, u, amp=1e-3, Fx=2e-6, tau_m=0.8):
    lat = lks.Lattice(nx, ny, 0.8, tau_m, 0.02, Fx, closure, storage, seed=11, perturb_amp=amp, coupling=coupling,
                      inplace=inplace)
    lat.set_walls(c[0], c[1], u[0], u[1])
    return lat


CASES = [
    # nx, ny: 1D grid with odd nx; nx = 1 (the x-neighbours are the node itself); 2D grid with a
    # ragged last block (300 = 256 + 44); ny = 3, the smallest moment-based channel.  16-bit
    # storage with even nx takes the two-nodes-per-thread kernels: 24 pairs per row on the 1D grid
    # (warps spanning two rows), 65 pairs on the 2D grid (one active lane in the last warp).  16-bit
    # storage with nx a multiple of 8 and at least 1024 stages rows through shared memory (phase 0
    # in place, the whole step with two buffers): 1032 (a full and a ragged segment, halos wrapped
    # across the row edges), 2056 (a middle segment with both halos in one copy)
    (37, 9), (1, 12), (300, 7), (64, 3), (48, 10), (130, 5), (1032, 5), (2056, 3),
]


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("closure", ["link", "moment"])
@pytest.mark.parametrize("coupling", ["maxwell", "lorentz"])
def test_inplace_equals_two_buffer_bitwise(lks, storage, closure, coupling):
    walls = [((0.3, float("inf")), (0.0, 0.05)), ((0.0, 2.0), (-0.02, 0.04))]
    for k, (nx, ny) in enumerate(CASES):
        if closure == "link" and ny == 3:
            ny = 2  # the smallest link-based channel
        c, u = walls[k % 2]
        a = _make(lks, nx, ny, closure, storage, coupling, False, c, u)
        b = _make(lks, nx, ny, closure, storage, coupling, True, c, u)
        for n in (2, 6, 128):          # 128 steps go through the captured graph (64 per launch)
            a.step(n)
            b.step(n)
            assert np.array_equal(_raw(a, storage), _raw(b, storage)), (nx, ny, n)
        assert np.array_equal(a.moments(), b.moments())
        a.close()
        b.close()


def test_inplace_fp64_matches_oracle(lks):
    nx, ny = 21, 17
    o = oracle.Oracle(nx, ny, 0.8, 0.8, 0.02, 2e-6, oracle.MOMENT, 0.3, 5.0, 0.0, 0.05, seed=3, perturb_amp=1e-3)
    g = lks.Lattice(nx, ny, 0.8, 0.8, 0.02, 2e-6, "moment", "f64", seed=3, perturb_amp=1e-3, inplace=True)
    g.set_walls(0.3, 5.0, 0.0, 0.05)
    o.step(200)
    g.step(200)
    mo, mg = o.moments(), g.moments()
    for m in (0, 1, 3):
        scale = float(np.max(np.abs(mo[m])))
        assert float(np.max(np.abs(mg[m] - mo[m]))) <= 1e-11 * scale, m
    g.close()


def test_inplace_run_to_steady_and_checkpoint(lks, tmp_path):
    a = _make(lks, 4, 40, "link", "f64", "maxwell", False, (0.5, 0.5), (0.0, 0.0), amp=0.0, Fx=1e-5)
    b = _make(lks, 4, 40, "link", "f64", "maxwell", True, (0.5, 0.5), (0.0, 0.0), amp=0.0, Fx=1e-5)
    ra = a.run_to_steady(1e-8, 100, 200_000)
    rb = b.run_to_steady(1e-8, 100, 200_000)
    assert ra == rb
    path = str(tmp_path / "aa.npz")
    b.save(path)
    c = _make(lks, 4, 40, "link", "f64", "maxwell", True, (0.5, 0.5), (0.0, 0.0), amp=0.0, Fx=1e-5)
    c.load(path)
    # the checkpoint holds FP64 absolute populations (deviation + rest), so the reloaded
    # deviations agree to the rounding of that sum; both then continue alike
    b.step(100)
    c.step(100)
    fb, gb = b.get_state()
    fc, gc = c.get_state()
    assert np.max(np.abs(fb - fc)) < 1e-15 and np.max(np.abs(gb - gc)) < 1e-15
    for x in (a, b, c):
        x.close()


def test_inplace_rejects_odd_step_counts(lks):
    lat = _make(lks, 8, 8, "moment", "f32", "maxwell", True, (0.1, 0.1), (0.0, 0.0))
    with pytest.raises(lks.LksError):
        lat.step(3)
    with pytest.raises(lks.LksError):
        lat.run_to_steady(1e-6, 101, 1000)
    with pytest.raises(lks.LksError):
        lat.run_to_steady(1e-6, 100, 1001)
    lat.step(4)                       # the handle is still usable
    assert lat.steps == 4
    lat.close()


def _batch_descs(batch, coupling):
    out = []
    rng = np.random.default_rng(5)
    for k in range(6):
        closure = "link" if k % 2 == 0 else "moment"
        ny = int(rng.integers(12, 60))
        nx = [4, 1, 37][k % 3]
        c = [0.0, 0.3, float("inf")][k % 3]
        out.append(batch.make_desc(nx, ny, closure, 0.8, 0.7, 0.01, 2e-6 if k % 2 == 0 else 0.0, c, c, 0.0,
                                   0.0 if k % 2 == 0 else 0.04, seed=k, perturb_amp=1e-3, tol=1e-30,
                                   check_every=50, max_steps=10**6, coupling=coupling))
    return out


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("coupling", ["maxwell", "lorentz"])
@pytest.mark.parametrize("shape", [(64, 4, 1), (128, 1, 4)])
def test_inplace_batch_equals_two_buffer_batch(lks, storage, coupling, shape):
    """The batched engine with one buffer per instance: every instance's state and residual equal
    the two-buffer batch's bit for bit (CTA thread groups, and clusters of CTAs on several SMs)."""
    from paper_2112_13930_gb300 import batch
    descs = _batch_descs(batch, coupling)
    two = batch.Batch(storage, max_instances=8, pool_bytes=32 << 20, threads_per_group=shape[0],
                      groups_per_cta=shape[1], cluster_ctas=shape[2], coupling=coupling)
    one = batch.Batch(storage, max_instances=8, pool_bytes=32 << 20, threads_per_group=shape[0],
                      groups_per_cta=shape[1], cluster_ctas=shape[2], coupling=coupling, inplace=True)
    s2 = [two.add(d) for d in descs]
    s1 = [one.add(d) for d in descs]
    assert one.memory()[1] < two.memory()[1]
    for q in (2, 300):
        two.run(q)
        one.run(q)
        for a, b in zip(s2, s1):
            assert two.result(a) == one.result(b)
            assert np.array_equal(two.moments(a), one.moments(b))
    two.close()
    one.close()


def test_inplace_batch_rejects_odd_counts(lks):
    from paper_2112_13930_gb300 import batch
    b = batch.Batch("f32", max_instances=4, pool_bytes=8 << 20, inplace=True)
    with pytest.raises(lks.LksError):
        b.add(batch.make_desc(4, 20, "link", 0.8, 0.8, 0.01, check_every=51))
    s = b.add(batch.make_desc(4, 20, "link", 0.8, 0.8, 0.01, check_every=50, max_steps=1000))
    with pytest.raises(lks.LksError):
        b.run(7)
    b.run(8)
    assert b.result(s)[1] == 8
    b.close()

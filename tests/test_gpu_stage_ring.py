"""The staged 16-bit kernels over many tasks per block, on the GPU.

The staged kernels run one persistent block per SM (152 on GB300) that takes tasks t0, t0 + G, ...
and cycles them through five shared-memory stages, each with a `full` and an `empty` mbarrier whose
phase parity flips every time the stage is reused.  Lattices of a few rows give fewer tasks than
blocks, so they never reuse a stage.  Here every block takes 13-20 tasks, so each stage is filled
and released three times or more, and the result must still equal, bit for bit, that of a kernel
that does not stage:
  - 2D two buffers: width 1032 (staged) from a width-516 state tiled twice (two-node kernel);
  - 2D in place: the staged phase 0 against the two-buffer staged step, pair by pair;
  - 3D: width 24 (staged, 21 whole rows per task) from a width-12 state tiled twice (one-node
    kernel).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NY = 1500  # 2D: 2 segments x 1500 rows = 3000 tasks, ~20 per block


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks, lks3d
    build.build()
    lks.load()
    return lks, lks3d


@pytest.mark.parametrize("storage,closure,coupling", [
    ("bf16", "link", "maxwell"), ("bf16", "moment", "maxwell"), ("f16", "link", "maxwell"),
    ("f16", "moment", "maxwell"), ("bf16", "moment", "lorentz")])
def test_2d_staged_ring_equals_two_node_kernel(mods, storage, closure, coupling):
    lks, _ = mods
    a = lks.Lattice(516, NY, 0.7, 0.9, 0.02, 2e-5, closure, storage, seed=21, perturb_amp=1e-2, coupling=coupling)
    b = lks.Lattice(1032, NY, 0.7, 0.9, 0.02, 2e-5, closure, storage, coupling=coupling)
    try:
        for lat in (a, b):
            lat.set_walls(0.4, 3.0, 0.02, -0.04)
        f, g = a.get_state()
        b.set_state(np.concatenate([f, f], axis=-1), np.concatenate([g, g], axis=-1))
        for n in (1, 7):
            a.step(n)
            b.step(n)
            fa, ga = a.get_state()
            fb, gb = b.get_state()
            assert np.array_equal(fb, np.concatenate([fa, fa], axis=-1)), n
            assert np.array_equal(gb, np.concatenate([ga, ga], axis=-1)), n
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("storage,closure", [("bf16", "link"), ("f16", "moment")])
def test_2d_inplace_staged_ring_equals_two_buffer(mods, storage, closure):
    lks, _ = mods
    kw = dict(seed=22, perturb_amp=1e-2)
    a = lks.Lattice(1032, NY, 0.7, 0.9, 0.02, 2e-5, closure, storage, **kw)
    b = lks.Lattice(1032, NY, 0.7, 0.9, 0.02, 2e-5, closure, storage, inplace=True, **kw)
    try:
        for lat in (a, b):
            lat.set_walls(0.4, 3.0, 0.02, -0.04)
        for n in (2, 8):
            a.step(n)
            b.step(n)
            fa, ga = a.get_state()
            fb, gb = b.get_state()
            assert np.array_equal(fa, fb) and np.array_equal(ga, gb), n
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_3d_staged_ring_equals_one_node_kernel(mods, storage):
    _, l3 = mods
    ny, nz = 42, 1000  # width 24: 21 rows per task, 2 x 1000 = 2000 tasks, ~13 per block
    a = l3.Lattice3D(12, ny, nz, 0.8, 0.7, 0.02, 2e-6, storage)
    b = l3.Lattice3D(24, ny, nz, 0.8, 0.7, 0.02, 2e-6, storage)
    try:
        for lat in (a, b):
            lat.set_walls(0.3, 2.0, 0.01, 0.04)
        f, g = a.get_state()
        rng = np.random.default_rng(23)
        f = f + 1e-3 * rng.uniform(-1, 1, f.shape) * np.abs(f)
        g = g + 1e-5 * rng.uniform(-1, 1, g.shape)
        a.set_state(f, g)
        f, g = a.get_state()
        b.set_state(np.concatenate([f, f], axis=-1), np.concatenate([g, g], axis=-1))
        for n in (1, 7):
            a.step(n)
            b.step(n)
            fa, ga = a.get_state()
            fb, gb = b.get_state()
            assert np.array_equal(fb, np.concatenate([fa, fa], axis=-1)), n
            assert np.array_equal(gb, np.concatenate([ga, ga], axis=-1)), n
    finally:
        a.close()
        b.close()

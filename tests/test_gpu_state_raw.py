"""lks_get_state_raw / lks_set_state_raw: the state in the library's own storage image -- a bit-exact
checkpoint at the storage type's size -- and its relation to the FP64 absolute populations of
lks_get_state."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lks():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks
    build.build()
    lks.load()
    return lks


ARGS = dict(tau_f=0.7, tau_m=0.85, B0=0.03, Fx=2e-5, closure="moment")


@pytest.mark.parametrize("storage,inplace", [("f64", False), ("f32", False), ("bf16", False), ("f16", False),
                                             ("f16", True)])
def test_raw_round_trip_continues_bit_for_bit(lks, storage, inplace):
    nx, ny = 66, 13
    a = lks.Lattice(nx, ny, storage=storage, seed=3, perturb_amp=1e-2, inplace=inplace, **ARGS)
    a.set_walls(0.3, 1.5, 0.0, 0.04)
    a.step(10)
    img = a.get_state_raw()
    assert img.nbytes == 19 * nx * ny * lks.STORAGE_BYTES[lks.STORAGES[storage]]
    b = lks.Lattice(nx, ny, storage=storage, inplace=inplace, **ARGS)
    b.set_walls(0.3, 1.5, 0.0, 0.04)
    b.set_state_raw(img)
    assert b.steps == 0
    a.step(30)
    b.step(30)
    assert np.array_equal(a.get_state_raw(), b.get_state_raw())
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
def test_raw_image_is_the_stored_deviations(lks, storage):
    """Decoded in the storage type (FP16 divided by 2^14), the image plus the rest populations is the
    FP64 state lks_get_state returns, to the one rounding of that FP64 sum (the conversion kernel may
    fuse it with the rest value's product)."""
    nx, ny = 40, 9
    rest = lks.Lattice(nx, ny, storage=storage, **ARGS)
    f_rest, g_rest = rest.get_state()
    rest.close()
    lat = lks.Lattice(nx, ny, storage=storage, seed=5, perturb_amp=1e-2, **ARGS)
    lat.step(7)
    img = lat.get_state_raw()
    if storage == "f64":
        dev = img.view(np.float64)
    elif storage == "f32":
        dev = img.view(np.float32).astype(np.float64)
    elif storage == "bf16":
        dev = (img.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        dev = img.view(np.float16).astype(np.float64) / lks.F16_SCALE
    f, g = lat.get_state()
    np.testing.assert_allclose(dev[:9 * nx * ny].reshape(9, ny, nx) + f_rest, f, rtol=0, atol=1e-15)
    np.testing.assert_allclose(dev[9 * nx * ny:].reshape(2, 5, ny, nx) + g_rest, g, rtol=0, atol=1e-15)
    lat.close()


def test_raw_size_is_checked(lks):
    lat = lks.Lattice(8, 5, storage="f32", **ARGS)
    bad = np.zeros(lat.state_bytes() - 4, dtype=np.uint8)
    with pytest.raises(lks.LksError) as e:
        lat.set_state_raw(bad)
    assert e.value.status == lks.LKS_EINVAL
    lat.close()

"""lks_residual_noalloc -- the residual entry point for callers that cannot allocate device memory
(applications that reserve the whole device for their own pools, latency-critical loops where
cudaMalloc/cudaFree may synchronise the device, plugin hosts that forbid allocation calls).  It
keeps its partial sums in a static device array instead of allocated scratch.

Checked through the C ABI against the existing lks_residual on the same state, two calls in a
row (the second call reuses the array the first one left behind), within the FP64 parity
tolerance of the other GPU tests, for every storage type and both couplings of the field to the
flow.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL64 = 1e-11


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks
    build.build()
    lks.load()
    return torch, lks


def _encode(torch, lks, storage, dev):
    """Deviations (recovered exactly from FP64 absolute populations) in the library's storage format,
    as a CUDA tensor: FP64, FP32, BF16 (the upper half of the FP32 bits: the values are exactly
    representable) or FP16 holding the deviation times lks.F16_SCALE."""
    if storage == lks.F64:
        return torch.tensor(dev, dtype=torch.float64, device="cuda")
    if storage == lks.F32:
        return torch.tensor(dev.astype(np.float32), device="cuda")
    if storage == lks.BF16_DEV:
        bits = dev.astype(np.float32).view(np.uint32)
        assert np.all(bits & 0xFFFF == 0)
        return torch.tensor((bits >> 16).astype(np.int16), device="cuda")
    scaled = dev * lks.F16_SCALE
    h = scaled.astype(np.float16)
    assert np.array_equal(h.astype(np.float64), scaled)
    return torch.tensor(h.view(np.int16), device="cuda")


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16"])
@pytest.mark.parametrize("coupling", ["maxwell", "lorentz"])
def test_noalloc_residual_matches_lks_residual(mods, storage, coupling):
    torch, lks = mods
    L = lks.load()
    nx, ny, b0, fx, tau_m = 70, 12, 0.02, 1e-5, 0.9
    code = lks.STORAGES[storage]
    args = dict(tau_f=0.7, tau_m=tau_m, B0=b0, Fx=fx, closure="moment", storage=storage, coupling=coupling)
    rest = lks.Lattice(nx, ny, **args)          # rest start: its state is the rest equilibrium
    f_rest, g_rest = rest.get_state()
    rest.close()
    lat = lks.Lattice(nx, ny, seed=5, perturb_amp=1e-2, **args)
    lat.set_walls(0.2, 0.9, 0.0, 0.03)
    lat.step(20)
    lat.residual()                               # lattice snapshot := state after 20 steps
    m = lat.moments()
    snap = torch.tensor(np.concatenate([m[1].ravel(), m[3].ravel()]), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    cpl = lks.COUPLINGS[coupling]
    for _ in range(2):
        lat.step(10)
        ru, rb = lat.residual()
        f, g = lat.get_state()
        fd = _encode(torch, lks, code, f - f_rest)
        gd = _encode(torch, lks, code, g - g_rest)
        torch.cuda.synchronize()
        out = np.zeros(2)
        st = L.lks_residual_noalloc(fd.data_ptr(), gd.data_ptr(), code, nx, ny, b0, fx, cpl, tau_m,
                                    snap.data_ptr(), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    stream.cuda_stream)
        assert st == lks.LKS_OK, L.lks_last_error(None)
        assert ru > 0 and rb > 0
        assert out[0] == pytest.approx(ru, rel=REL64) and out[1] == pytest.approx(rb, rel=REL64)
    # the snapshot now holds the last state's u_x, B_x (the same stored values, so the same moments)
    m = lat.moments()
    for k, field in enumerate((m[1], m[3])):
        got = snap.cpu().numpy()[k * nx * ny:(k + 1) * nx * ny]
        assert np.max(np.abs(got - field.ravel())) <= REL64 * np.max(np.abs(field))
    lat.close()


def test_noalloc_rejects_bad_arguments(mods):
    torch, lks = mods
    L = lks.load()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = np.zeros(2)
    op = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = L.lks_residual_noalloc(dummy.data_ptr(), dummy.data_ptr(), lks.F32, 1 << 16, (1 << 14) + 1, 0.0, 0.0,
                                lks.MAXWELL, 0.8, dummy.data_ptr(), op, None)
    assert st == lks.LKS_EINVAL
    assert b"2^30" in L.lks_last_error(None)
    # the Lorentz coupling reads J back from the stored g: tau_m near 1 is refused, as lks_create does
    st = L.lks_residual_noalloc(dummy.data_ptr(), dummy.data_ptr(), lks.F64, 2, 2, 0.0, 0.0, lks.LORENTZ, 1.02,
                                dummy.data_ptr(), op, None)
    assert st == lks.LKS_EINVAL and b"tau_m" in L.lks_last_error(None)
    st = L.lks_residual_noalloc(dummy.data_ptr(), dummy.data_ptr(), lks.F64, 2, 2, 0.0, 0.0, 7, 0.8,
                                dummy.data_ptr(), op, None)
    assert st == lks.LKS_EINVAL

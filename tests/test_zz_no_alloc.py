"""lks_residual_noalloc -- the residual entry point for callers that cannot allocate device memory
(applications that reserve the whole device for their own pools, latency-critical loops where
cudaMalloc/cudaFree may synchronise the device, plugin hosts that forbid allocation calls).  It
keeps its partial sums in a static device array instead of allocated scratch.

Checked through the C ABI against the existing lks_residual on the same state, two calls in a
row (the second call reuses the array the first one left behind), within the FP64 parity
tolerance of the other GPU tests.  This file is collected last on purpose."""
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


def test_noalloc_residual_matches_lks_residual(mods):
    torch, lks = mods
    L = lks.load()
    nx, ny, b0, fx = 70, 12, 0.02, 1e-5
    args = dict(tau_f=0.7, tau_m=0.9, B0=b0, Fx=fx, closure="moment", storage="f64")
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
    for _ in range(2):
        lat.step(10)
        ru, rb = lat.residual()
        f, g = lat.get_state()
        fd = torch.tensor(f - f_rest, dtype=torch.float64, device="cuda")
        gd = torch.tensor(g - g_rest, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        out = np.zeros(2)
        st = L.lks_residual_noalloc(fd.data_ptr(), gd.data_ptr(), lks.F64, nx, ny, b0, fx, snap.data_ptr(),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stream.cuda_stream)
        assert st == lks.LKS_OK, L.lks_last_error(None)
        assert ru > 0 and rb > 0
        assert out[0] == pytest.approx(ru, rel=REL64) and out[1] == pytest.approx(rb, rel=REL64)
    # the snapshot now holds the last state's u_x, B_x (the state passed in was rebuilt from FP64
    # absolute populations, so it agrees to the parity tolerance, not bit for bit)
    m = lat.moments()
    for k, field in enumerate((m[1], m[3])):
        got = snap.cpu().numpy()[k * nx * ny:(k + 1) * nx * ny]
        assert np.max(np.abs(got - field.ravel())) <= REL64 * np.max(np.abs(field))
    lat.close()


def test_noalloc_rejects_oversized_lattices(mods):
    torch, lks = mods
    L = lks.load()
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = np.zeros(2)
    st = L.lks_residual_noalloc(dummy.data_ptr(), dummy.data_ptr(), lks.F32, 1 << 16, (1 << 14) + 1, 0.0, 0.0,
                                dummy.data_ptr(), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None)
    assert st == lks.LKS_EINVAL
    assert b"2^30" in L.lks_last_error(None)

"""State transfers of lattices larger than one conversion chunk (2^20 nodes), on the GPU.

lks_get_state / lks_set_state (and the 3D pair) convert between stored deviations and FP64
absolute populations either directly in the caller's host arrays when they are page-locked (one
kernel over the mapped memory) or, for pageable arrays and with LKS_HOST_STAGING=1, 2^20 nodes at a
time through a staging buffer.  All three are run: page-locked, pageable, and page-locked with the
staging forced.  On lattices of a little more than 2^20 nodes (one full chunk and a ragged one)
every node must land where it belongs:
  - FP64 storage: get_state(set_state(x)) equals x to within one rounding of (x - rest) + rest;
  - 16-bit storage (two-buffer and the interleaved in-place layout): each deviation comes back
    within one unit roundoff of the storage type (FP16: plus half its subnormal spacing, 2^-25),
    and a second round trip returns the first one's result bit for bit (a stored value converts
    back exactly).
Per-node host moments (lks_moments / lks3_moments with what = nodes) go through the same chunks:
with FP64 storage and no body force they equal the plain sums rho = sum f, rho u = sum f e_a and
B = sum g of the returned populations to within a few FP64 roundings (1e-13 absolute).
A node misplaced by a chunk offset would be off by the size of the random perturbation (1e-3),
far above those bounds.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U_S = {"f64": 2.0 ** -53, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}
ABS = {"f64": 0.0, "bf16": 0.0, "f16": 2.0 ** -25}


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13930_gb300 import build, lks, lks3d
    build.build()
    lks.load()
    return lks, lks3d


E2 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=float)
E3 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
               (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)], dtype=float)


def _sum_moments(f, g, e, ncomp):
    """rho, u (ncomp components), B (ncomp components) per node from FP64 populations (F = 0)."""
    rho = f.sum(axis=0)
    u = [np.tensordot(e[:, k], f, axes=(0, 0)) / rho for k in range(ncomp)]
    b = [g[k].sum(axis=0) for k in range(ncomp)]
    return np.stack([rho] + u + b)


def _check_moments(mg, mo):
    # the sums run over terms of size <= 1 (rho ~ 1): a few FP64 roundings are ~1e-15 absolute
    for k in range(mo.shape[0]):
        assert float(np.max(np.abs(mg[k] - mo[k]))) <= 1e-13, k


class Host:
    """get/set_state and per-node moments through the C ABI into host arrays of one kind."""

    def __init__(self, mods, lat, mode):
        import torch
        self.pinned = mode != "pageable"
        self.lat = lat
        lks, l3 = mods
        if isinstance(lat, l3.Lattice3D):
            lib, self.ptr, self.check = l3.lib(), l3._ptr, l3._check
            self.get, self.set, self.mom = lib.lks3_get_state, lib.lks3_set_state, lib.lks3_moments
            n = (lat.nz, lat.ny, lat.nx)
            self.shapes = ((19,) + n, (3, 7) + n, (7,) + n)
        else:
            lib, self.ptr, self.check = lks.load(), lks._dptr, lks._check
            self.get, self.set, self.mom = lib.lks_get_state, lib.lks_set_state, lib.lks_moments
            n = (lat.ny, lat.nx)
            self.shapes = ((9,) + n, (2, 5) + n, (5,) + n)
        self.nodes_what = lks.MOMENTS_NODES
        self.torch = torch

    def empty(self, shape):
        if self.pinned:
            return self.torch.empty(shape, dtype=self.torch.float64, pin_memory=True).numpy()
        return np.empty(shape)

    def get_state(self):
        f, g = self.empty(self.shapes[0]), self.empty(self.shapes[1])
        self.check(self.get(self.lat._h, self.ptr(f), self.ptr(g)), self.lat._h)
        return f, g

    def set_state(self, f, g):
        hf, hg = self.empty(self.shapes[0]), self.empty(self.shapes[1])
        hf[...] = f
        hg[...] = g
        self.check(self.set(self.lat._h, self.ptr(hf), self.ptr(hg)), self.lat._h)

    def moments(self):
        m = self.empty(self.shapes[2])
        self.check(self.mom(self.lat._h, self.nodes_what, self.ptr(m)), self.lat._h)
        return m


def _perturbed(rest_f, rest_g, seed):
    rng = np.random.default_rng(seed)
    f = rest_f + 1e-3 * rng.uniform(-1, 1, rest_f.shape) * np.abs(rest_f)
    g = rest_g + 1e-3 * rng.uniform(-1, 1, rest_g.shape)
    return f, g


def _check_roundtrip(host, rest_f, rest_g, storage, seed):
    f, g = _perturbed(rest_f, rest_g, seed)
    host.set_state(f, g)
    f1, g1 = host.get_state()
    u = U_S[storage]
    for x, y, r in ((f, f1, rest_f), (g, g1, rest_g)):
        d = x - r
        if storage == "f64":
            assert np.max(np.abs(y - x) - 2 * u * np.abs(x)) <= 0.0
        else:
            # one rounding to FP32, then one to the 16-bit type
            assert np.max(np.abs((y - r) - d) - 1.01 * u * np.abs(d) - ABS[storage]) <= 0.0
    if storage != "f64":
        host.set_state(f1, g1)
        f2, g2 = host.get_state()
        assert np.array_equal(f2, f1) and np.array_equal(g2, g1)


@pytest.fixture(params=["pinned", "pageable", "pinned-staged"])
def host_mode(request, monkeypatch):
    """LKS_HOST_STAGING is read by every transfer."""
    monkeypatch.setenv("LKS_HOST_STAGING", "1" if request.param == "pinned-staged" else "0")
    return request.param


@pytest.mark.parametrize("storage,inplace", [("f64", False), ("bf16", False), ("f16", True)])
def test_2d_state_roundtrip_over_two_chunks(mods, host_mode, storage, inplace):
    lks, _ = mods
    nx, ny = 1032, 1023  # 1,055,736 nodes = 2^20 + 7160
    lat = lks.Lattice(nx, ny, 0.8, 0.8, 0.03, 0.0, "link", storage, inplace=inplace)
    try:
        host = Host(mods, lat, host_mode)
        rest_f, rest_g = host.get_state()
        _check_roundtrip(host, rest_f, rest_g, storage, seed=11)
        if storage == "f64":
            f, g = host.get_state()
            _check_moments(host.moments(), _sum_moments(f, g, E2, 2))
    finally:
        lat.close()


@pytest.mark.parametrize("storage", ["f64", "bf16"])
def test_3d_state_roundtrip_over_two_chunks(mods, host_mode, storage):
    _, l3 = mods
    nx, ny, nz = 128, 91, 91  # 1,059,968 nodes = 2^20 + 11392
    lat = l3.Lattice3D(nx, ny, nz, 0.8, 0.7, 0.02, 0.0, storage)
    try:
        host = Host(mods, lat, host_mode)
        rest_f, rest_g = host.get_state()
        _check_roundtrip(host, rest_f, rest_g, storage, seed=12)
        if storage == "f64":
            f, g = host.get_state()
            _check_moments(host.moments(), _sum_moments(f, g, E3, 3))
    finally:
        lat.close()

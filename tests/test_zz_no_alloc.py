"""lbehd_phase_moments_noalloc: the droplet reduction for callers that cannot let a
library allocate device memory (a program that owns all device memory through its own
pre-sized pool, a framework that forbids allocation inside foreign calls). It keeps its
scratch in a fixed file-scope device array instead of allocating.

Checked through the C ABI against what lbehd_observe reports for the same step, on two
calls in a row (the second reuses the scratch the first left behind), with the
tolerances of the parity tests: mass 1e-5 relative, centroid 1e-3 lattice units,
velocity 0.5 % of its magnitude; on lattices of one block (24x16x16), of 64 blocks (the
128x64x64 workload) and in 2D; and against an FP64 numpy sum on synthetic fields of exactly
2048 blocks (the cap), followed by a one-block call that must ignore the partials the large
call left behind. This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_12868_b300 import build, lbehd
    build.build()
    lib = lbehd.load()
    fn = lib.lbehd_phase_moments_noalloc
    fn.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 5
    fn.restype = ctypes.c_int
    return lbehd, lib, torch


def _device_ptr(lib, sim, which):
    ptr, nb = ctypes.c_void_p(), ctypes.c_size_t()
    assert lib.lbehd_device_ptr(sim._h, which, ctypes.byref(ptr), ctypes.byref(nb)) == 0
    return ptr.value


@pytest.mark.parametrize("case", ["small_3d", "droplet_3d_128x64x64", "small_2d"])
def test_noalloc_moments_match_observe_twice(gpu, case):
    lbehd, lib, torch = gpu
    w = getattr(W, case)()
    sim = lbehd.Simulation(w)
    nz, ny, nx = w.shape
    solid = torch.tensor(w.solid.reshape(-1), dtype=torch.uint8, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sim.step(7)
        o = sim.observe()   # synchronises the library's stream
        rc = lib.lbehd_phase_moments_noalloc(
            w.dim, nx, ny, nz, _device_ptr(lib, sim, lbehd.PHI), _device_ptr(lib, sim, lbehd.U),
            solid.data_ptr(), out.data_ptr(), None)
        assert rc == 0, lib.lbehd_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] / o["M1"] - 1) <= 1e-5
        assert np.abs(got[1:4] - o["centroid"]).max() <= 1e-3
        v = o["velocity"]
        assert np.abs(got[4:7] - v).max() <= 5e-3 * np.abs(v).max()
        assert np.abs(got[7:10] / o["mass"] - 1).max() <= 1e-5


def test_noalloc_rejects_oversized_lattice(gpu):
    lbehd, lib, torch = gpu
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = lib.lbehd_phase_moments_noalloc(3, 1024, 1024, 17, buf.data_ptr(), buf.data_ptr(),
                                         buf.data_ptr(), buf.data_ptr(), None)
    assert rc == -1
    assert b"static scratch" in lib.lbehd_last_error(None)


def _numpy_moments(dim, shape, phi, u, solid):
    """FP64 reference of the ten outputs from host copies of the fields."""
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    fl = (solid.reshape(shape) == 0)
    P = phi.reshape((3,) + shape).astype(np.float64) * fl
    U = u.reshape((3,) + shape).astype(np.float64)
    M1 = P[0].sum()
    cen = [(P[0] * c).sum() / M1 for c in (xx, yy, zz)]
    vel = [(P[0] * U[a]).sum() / M1 for a in range(3)]
    return np.array([M1, *cen, *vel, M1, P[1].sum(), P[2].sum()])


def test_noalloc_at_the_block_cap_then_small(gpu):
    """Synthetic fields on a 256^3 lattice (2048 blocks of 8192 sites, the most the static
    scratch holds), then a 24x16x16 lattice (one block) right after, whose call must read only
    its own partial and not the 2047 the large call left behind."""
    lbehd, lib, torch = gpu
    g = torch.Generator(device="cuda").manual_seed(5)
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    for shape in ((256, 256, 256), (16, 16, 24)):
        N = int(np.prod(shape))
        phi = torch.rand(3 * N, generator=g, device="cuda", dtype=torch.float32)
        u = torch.rand(3 * N, generator=g, device="cuda", dtype=torch.float32) - 0.5
        solid = (torch.rand(N, generator=g, device="cuda") < 0.2).to(torch.uint8)
        nz, ny, nx = shape
        rc = lib.lbehd_phase_moments_noalloc(3, nx, ny, nz, phi.data_ptr(), u.data_ptr(),
                                             solid.data_ptr(), out.data_ptr(), None)
        assert rc == 0, lib.lbehd_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = _numpy_moments(3, shape, phi.cpu().numpy(), u.cpu().numpy(),
                             solid.cpu().numpy())
        idx_mass = [0, 7, 8, 9]
        assert np.abs(got[idx_mass] / ref[idx_mass] - 1).max() <= 1e-10, (shape, got, ref)
        assert np.abs(got[1:4] - ref[1:4]).max() <= 1e-8, (shape, got, ref)
        assert np.abs(got[4:7] - ref[4:7]).max() <= 1e-10, (shape, got, ref)

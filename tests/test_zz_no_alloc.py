"""lbehd_phase_moments_noalloc: the droplet reduction for callers that cannot let a
library allocate device memory (a program that owns all device memory through its own
pre-sized pool, a framework that forbids allocation inside foreign calls). It keeps its
scratch in a fixed file-scope device array instead of allocating.

Checked through the C ABI against what lbehd_observe reports for the same step, on two
calls in a row (the second reuses the scratch the first left behind), with the
tolerances of the parity tests: mass 1e-5 relative, centroid 1e-3 lattice units,
velocity 0.5 % of its magnitude. This file is collected last on purpose.
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


def test_noalloc_moments_match_observe_twice(gpu):
    lbehd, lib, torch = gpu
    w = W.small_3d()
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

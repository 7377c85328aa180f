"""The start of each step's Gauss-law solve (Eq. 13), LBEHD_OPT_WARM_START: 1 (a handle's
default) starts from the combination of the last two increments with the least residual
(k_pcg_init_mr), 0 (a batch's default) from the increment of step s - 2 alone.

Both stop at the same tolerance, so they step the same physics within it; the minimal-residual
start converges without a CG iteration on more steps. The persistent and the multi-launch
solves give the same bits with either start (tests/test_gpu_poisson_persistent.py), and so
does a batch instance against a single handle (tests/test_gpu_batch.py).
"""
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
    return lbehd


def test_option_values(gpu):
    sim = gpu.Simulation(W.small_3d(), poisson_mode=gpu.POISSON_GRAPH)
    assert sim.get_option(gpu.OPT_WARM_START) == 1
    sim.set_option(gpu.OPT_WARM_START, 0)
    assert sim.get_option(gpu.OPT_WARM_START) == 0
    sim.set_option(gpu.OPT_WARM_START, 1)
    assert sim.get_option(gpu.OPT_WARM_START) == 1
    with pytest.raises(gpu.LBEHDError):
        sim.set_option(gpu.OPT_WARM_START, 2)
    sim.close()
    batch = gpu.Batch([W.small_3d(), W.small_3d(seed=9)])
    batch.set_option(gpu.OPT_WARM_START, 0)
    batch.set_option(gpu.OPT_WARM_START, 1)
    with pytest.raises(gpu.LBEHDError):
        batch.set_option(gpu.OPT_WARM_START, 2)
    batch.close()


@pytest.mark.parametrize("case", ["small_3d", "small_2d"])
def test_both_starts_step_the_same_physics(gpu, case):
    """300 steps with each start: no error status, potentials and populations equal to the
    size the 1e-7 solve tolerance leaves (the oracle parity bars are 1e-5)."""
    w = getattr(W, case)()
    sims = []
    for warm in (1, 0):
        s = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
        s.set_option(gpu.OPT_WARM_START, warm)
        s.step(300)
        assert s.observe()["status"] == 0
        sims.append(s)
    a, b = sims
    pa, pb = a.potential(), b.potential()
    assert np.abs(pa - pb).max() <= 1e-5 * np.abs(pb).max()
    for name in ("fphi", "frho", "g"):
        x, y = a.array(name).astype(np.float64), b.array(name)
        assert np.abs(x - y).max() <= 1e-5 * max(np.abs(y).max(), 1e-30), name
    for s in sims:
        s.close()


def test_fewer_iterating_steps_on_the_droplet(gpu):
    """droplet_3d_128x64x64 in steady state (steps 4000-5000): the minimal-residual start
    leaves fewer steps that need a CG iteration (measured 0.12 against 0.26 iterations per
    step)."""
    w = W.droplet_3d_128x64x64()
    rate = {}
    for warm in (1, 0):
        s = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
        s.set_option(gpu.OPT_WARM_START, warm)
        s.step(4000)
        it0 = s.stats()["poisson_iters"]
        s.step(1000)
        rate[warm] = (s.stats()["poisson_iters"] - it0) / 1000.0
        assert s.observe()["status"] == 0
        s.close()
    assert rate[1] <= 0.75 * rate[0], rate

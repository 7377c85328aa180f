"""lbehd_save_state / lbehd_load_state (checkpoint and restart) on the GPU.

A handle restored from a saved state, even one that has taken other steps, continues the
saved run bit for bit: populations, fields, the potential pair, and the observables (the
drag force uses the previous step's sums, which are part of the state). The save point
is deliberately not a multiple of the 16-step multigrid refresh, so the preconditioner must
be rebuilt from the saved permittivity for the iterates to repeat.
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu

ARRAYS = ("g", "fphi", "frho", "phi", "pot", "pot_lo", "u")
CASES = {"small_3d": lambda: W.small_3d(), "small_2d": lambda: W.small_2d(),
         "control_3d_96x64x64": lambda: W.control_3d_96x64x64()}


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_12868_b300 import build, lbehd
    build.build()
    return lbehd


@pytest.mark.parametrize("case", list(CASES))
def test_restart_repeats_the_run(gpu, case):
    w = CASES[case]()
    V = np.array([v for _, v in w.schedule])
    a = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    a.step(21)
    state = a.save_state()
    b = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    b.step(3)
    b.load_state(state)
    for s in (a, b):
        if len(V) > 1:
            s.set_electrodes(V[1])   # a switch after the restart point
        s.step(13)
    for name in ARRAYS:
        x, y = a.array(name), b.array(name)
        assert np.array_equal(x, y), (name, np.abs(x.astype(np.float64) - y).max())
    oa, ob = a.observe(), b.observe()
    for k in ("step", "centroid", "velocity", "f_ele", "f_drag", "mass", "poisson_iters"):
        assert np.array_equal(np.asarray(oa[k]), np.asarray(ob[k])), k


def test_load_rejects_foreign_buffers(gpu):
    import torch
    a = gpu.Simulation(W.small_3d(), poisson_mode=gpu.POISSON_GRAPH)
    a.step(2)
    other = gpu.Simulation(W.small_2d(), poisson_mode=gpu.POISSON_GRAPH)
    with pytest.raises(gpu.LBEHDError):
        other.load_state(a.save_state())          # another lattice
    zeros = torch.zeros(a.save_state().numel(), dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu.LBEHDError):
        a.load_state(zeros)                       # not a saved state
    assert a.observe()["status"] == 0


@pytest.mark.parametrize("variant", [1, 3])
def test_observables_do_not_depend_on_when_they_are_read(gpu, variant):
    """The collide kernel leaves each step's block partials in the partial set of its step
    parity, and they are summed when the observables are read. Reading after every few
    steps or only at the end gives the same sums, including the drag force, which uses the
    previous step's sums as well."""
    w = W.small_3d()
    a = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    b = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    for s in (a, b):
        s.set_option(gpu.OPT_COLLIDE, variant)
    for n in (7, 1, 2):
        a.step(n)
        oa = a.observe()
    b.step(10)
    ob = b.observe()
    assert oa["step"] == ob["step"] == 9
    for k, v in oa.items():
        assert np.array_equal(np.asarray(v), np.asarray(ob[k])), k
    assert np.any(np.asarray(ob["f_drag"]) != 0.0)

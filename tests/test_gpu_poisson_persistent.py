"""The persistent Gauss-law solve (one cooperative kernel per solve, LBEHD_OPT_POISSON_KERNEL
= 1, the default) against the multi-launch graph with conditional nodes (= 0), with either
multigrid smoother (LBEHD_OPT_MG_SMOOTHER: 1 block-local, the default; 0 whole-level
red-black sweeps).

Both forms run the same per-cell arithmetic in the same order (the dot products keep their
partition, the scalar sums their fixed order), so the state after many steps is equal bit
for bit, and so are the iteration counts. Lattices with one, two and three multigrid levels
above the shared-memory tail; 2D and 3D; mid-run electrode switches (large increments with
refinement passes); and the adjoint's solves. The two smoothers are then compared with each
other: both converge to the tolerance, so the potentials agree to it.
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu

ARRAYS = ("g", "fphi", "frho", "phi", "pot", "pot_lo", "u")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_12868_b300 import build, lbehd
    build.build()
    return lbehd


def pair(gpu, w, smoother=1, warm=1):
    a = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    b = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    b.set_option(gpu.OPT_POISSON_KERNEL, 0)
    assert a.get_option(gpu.OPT_POISSON_KERNEL) == 1   # the persistent kernel really runs
    assert b.get_option(gpu.OPT_POISSON_KERNEL) == 0
    for s in (a, b):
        s.set_option(gpu.OPT_MG_SMOOTHER, smoother)
        assert s.get_option(gpu.OPT_MG_SMOOTHER) == smoother
        s.set_option(gpu.OPT_WARM_START, warm)
        assert s.get_option(gpu.OPT_WARM_START) == warm
    return a, b


def assert_same(a, b):
    for name in ARRAYS:
        x, y = a.array(name), b.array(name)
        assert np.array_equal(x, y), (name, np.abs(x.astype(np.float64) - y).max())
    sa, sb = a.stats(), b.stats()
    assert sa["steps"] == sb["steps"] and sa["poisson_iters"] == sb["poisson_iters"]
    oa, ob = a.observe(), b.observe()
    assert oa["status"] == 0 and ob["status"] == 0
    assert oa["poisson_iters"] == ob["poisson_iters"]


CASES = {
    "small_2d": lambda: W.small_2d(),
    "small_3d": lambda: W.small_3d(),
    "droplet_3d_64x32x32": lambda: W.droplet_3d(64, 32, 32, R=9.0, pillar_h=4, seed=3,
                                                 name="droplet_3d_64x32x32"),
    "control_3d_96x64x64": lambda: W.control_3d_96x64x64(),
}


@pytest.mark.parametrize("smoother", [1, 0])
@pytest.mark.parametrize("case", list(CASES))
def test_persistent_solve_is_the_multi_launch_solve(gpu, case, smoother):
    w = CASES[case]()
    a, b = pair(gpu, w, smoother)
    steps = 40 if case != "control_3d_96x64x64" else 24
    a.step(steps)
    b.step(steps)
    assert_same(a, b)


@pytest.mark.parametrize("case", list(CASES))
def test_persistent_solve_is_the_multi_launch_solve_step_s2_start(gpu, case):
    """The same with each solve started from the increment of step s - 2 alone
    (LBEHD_OPT_WARM_START = 0, a batch's start)."""
    w = CASES[case]()
    a, b = pair(gpu, w, 1, warm=0)
    steps = 40 if case != "control_3d_96x64x64" else 24
    a.step(steps)
    b.step(steps)
    assert_same(a, b)


@pytest.mark.parametrize("smoother", [1, 0])
def test_persistent_solve_through_electrode_switches(gpu, smoother):
    """Switching the potentials mid-run makes large increments (refinement passes)."""
    w = W.droplet_3d(64, 32, 32, R=9.0, pillar_h=4, seed=3, V=[0.02])
    a, b = pair(gpu, w, smoother)
    for V in (0.02, 0.08, 0.0, 0.05):
        for s in (a, b):
            s.set_electrodes([V])
            s.step(9)
    assert_same(a, b)


def test_persistent_solve_in_the_adjoint(gpu):
    """The adjoint's Gauss-law solves through the persistent kernel give the gradient of
    the multi-launch solves bit for bit."""
    w = W.control_3d_24x16x16(segments=2, seg_steps=20)
    V = np.array([v for _, v in w.schedule])
    for smoother in (1, 0):
        grads = []
        for kernel in (1, 0):
            s = gpu.Simulation(w)
            s.set_option(gpu.OPT_POISSON_KERNEL, kernel)
            s.set_option(gpu.OPT_MG_SMOOTHER, smoother)
            assert s.get_option(gpu.OPT_POISSON_KERNEL) == kernel
            s.adjoint_forward(V, 20)
            grads.append(s.adjoint_backward())
            s.close()
        assert np.array_equal(grads[0], grads[1]), (smoother, np.abs(grads[0] - grads[1]).max())


@pytest.mark.parametrize("case", ["small_2d", "droplet_3d_64x32x32", "control_3d_96x64x64"])
def test_block_smoother_against_whole_level_sweeps(gpu, case):
    """The block-local smoother preconditions CG as well as whole-level sweeps: the first
    solve from phi = 0 (many iterations) needs at most a quarter more iterations, every solve
    converges, and the potentials of the two runs agree to the solve's tolerance after 30
    steps (the states differ only by what each solve leaves below its tolerance)."""
    w = CASES[case]()
    runs = {}
    for smoother in (1, 0):
        s = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
        s.set_option(gpu.OPT_MG_SMOOTHER, smoother)
        assert s.get_option(gpu.OPT_MG_SMOOTHER) == smoother
        s.step(1)
        it1 = s.stats()["poisson_iters"]
        s.step(29)
        o = s.observe()
        assert o["status"] == 0
        runs[smoother] = (it1, s.potential(), s.stats()["poisson_iters"])
        s.close()
    (it_b, pot_b, tot_b), (it_w, pot_w, tot_w) = runs[1], runs[0]
    print(case, "first solve", it_b, it_w, "30 steps", tot_b, tot_w)
    assert it_b <= 1.25 * it_w + 1, (it_b, it_w)
    assert tot_b <= 1.25 * tot_w + 3, (tot_b, tot_w)
    scale = np.abs(pot_w).max()
    assert np.abs(pot_b - pot_w).max() <= 1e-5 * scale, np.abs(pot_b - pot_w).max() / scale

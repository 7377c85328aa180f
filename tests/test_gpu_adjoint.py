"""The discrete adjoint (lbehd_adjoint_forward / lbehd_adjoint_backward) on the GPU.

* Against the FP64 discrete-adjoint reference (oracle/adjoint_ref.py: the oracle step in
  differentiable PyTorch) on tiny 3D and 2D lattices: the gradient of the droplet's x
  centroid with respect to a piecewise-constant electrode schedule, within 1e-3 of the
  largest gradient component (FP32 state against FP64).
* The 24x16x16 copy of the differentiable-control case against the same reference, and,
  over a 100-step schedule, component by component: within 1e-3 relative of the FP64
  discrete adjoint for every component above 2 % of the largest, and within 1e-3 relative of
  central differences (h = 1e-4) of the FP64 oracle's forward on sampled components (the FP64
  forward keeps finite differences free of the FP32 rounding that h = 1e-4 would amplify).
* Against central finite differences of the GPU forward itself: a 40x16x16 lattice (1e-2
  of the largest component), and the full 96x64x64 control case, 4000 steps and 320
  parameters, on 8 sampled parameters (1e-3 of the largest component).
* Through torch.autograd (schedule_loss), and with the handle left in the post-run state.
"""
import numpy as np
import pytest
import torch

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_12868_b300 import build, lbehd
    build.build()
    return lbehd


def tiny_3d():
    return W.droplet_3d(16, 8, 12, R=3.5, pillar_h=3, electrodes=[(4, 8, 2, 6), (8, 12, 2, 6)],
                        V=[0.03, 0.05], seed=5)


def reference_grad(oracle_mod, w, V, seg):
    from oracle import adjoint_ref as AR
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    m = AR.RefModel(w.dim, w.shape, w.solid, w.elec, w.params, orc.normal)
    Vt = torch.tensor(V, dtype=torch.float64, requires_grad=True)
    L = AR.schedule_loss(m, w.phi_init, Vt, seg)
    L.backward()
    return float(L.detach()), Vt.grad.numpy()


@pytest.mark.parametrize("case", ["3d_2steps", "3d_2x6", "3d_4x5", "2d_3x5"])
def test_adjoint_matches_fp64_reference(gpu, oracle_mod, case):
    if case.startswith("3d"):
        w = tiny_3d()
        V = np.array([[0.03, 0.05], [0.06, 0.01], [0.0, 0.04], [0.05, 0.05]])
    else:
        w = W.small_2d(nx=24, ny=16, R=5.0)
        V = np.array([[0.05], [0.02], [0.06]])
    S, seg = {"3d_2steps": (1, 2), "3d_2x6": (2, 6), "3d_4x5": (4, 5), "2d_3x5": (3, 5)}[case]
    V = V[:S]
    L_ref, g_ref = reference_grad(oracle_mod, w, V, seg)
    sim = gpu.Simulation(w)
    L = sim.adjoint_forward(V, seg)
    g = sim.adjoint_backward()
    assert abs(L - L_ref) <= 1e-6 * abs(L_ref)
    assert np.abs(g - g_ref).max() <= 1e-3 * np.abs(g_ref).max(), (g, g_ref)


def test_control_copy_24x16x16_matches_fp64_reference(gpu, oracle_mod):
    """The 24x16x16 copy of the differentiable-control case (4 electrodes x 4 segments of
    5 steps): loss and all 16 gradient components against the FP64 discrete adjoint."""
    w = W.control_3d_24x16x16(segments=4, seg_steps=5)
    V = np.array([v for _, v in w.schedule])
    L_ref, g_ref = reference_grad(oracle_mod, w, V, 5)
    sim = gpu.Simulation(w)
    L = sim.adjoint_forward(V, 5)
    g = sim.adjoint_backward()
    assert abs(L - L_ref) <= 1e-6 * abs(L_ref)
    assert np.abs(g - g_ref).max() <= 1e-3 * np.abs(g_ref).max(), (g, g_ref)


def _oracle_loss(oracle_mod, w, V, seg):
    """x centroid of the droplet after the schedule V (segments x electrodes, seg steps each)
    run by the FP64 oracle: the fields of the last step, as lbehd_adjoint_forward reports."""
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    for k in range(V.shape[0]):
        orc.set_electrodes(V[k])
        orc.step(seg)
    return orc.observables()["centroid"][0]


COMPONENT_FLOOR = 0.02   # components below 2 % of the largest are compared in absolute terms


def test_control_copy_100_steps_component_by_component(gpu, oracle_mod):
    """The 24x16x16 copy of the control case over 5 segments of 20 steps (4 electrodes, 20
    parameters, 100 steps). Every gradient component above COMPONENT_FLOOR of the largest
    within 1e-3 relative of the FP64 discrete adjoint (the rest within 1e-3 COMPONENT_FLOOR of
    the largest); on the four largest components, the GPU adjoint within 1e-3 relative of
    central differences of the FP64 oracle forward at h = 1e-4, and the FP64 adjoint within
    1e-5 relative of the same differences."""
    w = W.control_3d_24x16x16(segments=5, seg_steps=20)
    V = np.array([v for _, v in w.schedule])
    seg = 20
    L_ref, g_ref = reference_grad(oracle_mod, w, V, seg)
    sim = gpu.Simulation(w)
    L = sim.adjoint_forward(V, seg)
    g = sim.adjoint_backward()
    assert abs(L - L_ref) <= 1e-6 * abs(L_ref)
    scale = np.abs(g_ref).max()
    big = np.abs(g_ref) >= COMPONENT_FLOOR * scale
    rel = np.abs(g - g_ref)[big] / np.abs(g_ref)[big]
    assert rel.max() <= 1e-3, (rel.max(), g, g_ref)
    assert np.abs(g - g_ref)[~big].max(initial=0.0) <= 1e-3 * COMPONENT_FLOOR * scale
    h = 1e-4
    for flat in np.argsort(-np.abs(g_ref).ravel())[:4]:
        k, e = np.unravel_index(flat, V.shape)
        Vp, Vm = V.copy(), V.copy()
        Vp[k, e] += h
        Vm[k, e] -= h
        fd = (_oracle_loss(oracle_mod, w, Vp, seg) - _oracle_loss(oracle_mod, w, Vm, seg)) / (2 * h)
        assert abs(g_ref[k, e] - fd) <= 1e-5 * abs(fd), (k, e, g_ref[k, e], fd)
        assert abs(g[k, e] - fd) <= 1e-3 * abs(fd), (k, e, g[k, e], fd)


def test_control_96x64x64_matches_finite_differences(gpu):
    """The differentiable-control case at full size (96x64x64, 16 electrodes x 20 segments
    of 200 steps, 4000 steps): the adjoint gradient against central differences of the
    GPU forward on 8 sampled parameters (seeded, among those above 5 % of the largest).
    h = 1e-3: at h = 1e-4 the FP32 forward's rounding, divided by h, reaches 1e-3 of the
    largest component by itself."""
    w = W.control_3d_96x64x64()
    V = np.array([v for _, v in w.schedule])
    seg = 200
    sim = gpu.Simulation(w)
    sim.adjoint_forward(V, seg)
    g = sim.adjoint_backward()
    info = sim.adjoint_info()
    sim.close()
    assert info["steps"] == 4000 and info["checkpoint_every"] == 64
    assert info["steps_reversed"] == 4000 and info["steps_replayed"] == 4000
    scale = np.abs(g).max()
    cand = np.argwhere(np.abs(g) > 0.05 * scale)
    pick = cand[np.random.default_rng(11).choice(len(cand), 8, replace=False)]

    def loss(Vx):
        s = gpu.Simulation(w)
        L = s.adjoint_forward(Vx, seg)
        s.close()
        return L

    h = 1e-3
    for k, e in pick:
        Vp, Vm = V.copy(), V.copy()
        Vp[k, e] += h
        Vm[k, e] -= h
        fd = (loss(Vp) - loss(Vm)) / (2 * h)
        assert abs(fd - g[k, e]) <= 1e-3 * scale, (k, e, fd, g[k, e], scale)


def test_adjoint_matches_finite_differences(gpu):
    """A 40x16x16 lattice, 3 electrodes, 4 segments of 25 steps: the adjoint gradient against
    central differences (h = 2e-3) of the GPU forward on 4 sampled parameters."""
    w = W.droplet_3d(40, 16, 16, R=5.0, pillar_h=3,
                     electrodes=[(16, 22, 4, 12), (22, 28, 4, 12), (28, 34, 4, 12)],
                     V=[0.04, 0.04, 0.04], seed=9)
    rng = np.random.default_rng(3)
    V = rng.uniform(0.0, 0.06, size=(4, 3))
    seg = 25
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    sim.adjoint_forward(V, seg)
    g = sim.adjoint_backward()
    sim.close()

    def loss(Vx):
        s = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
        L = s.adjoint_forward(Vx, seg)
        s.close()
        return L

    h = 2e-3
    scale = np.abs(g).max()
    for k, e in [(0, 0), (1, 1), (2, 2), (3, 1)]:
        Vp, Vm = V.copy(), V.copy()
        Vp[k, e] += h
        Vm[k, e] -= h
        fd = (loss(Vp) - loss(Vm)) / (2 * h)
        assert abs(fd - g[k, e]) <= 1e-2 * scale, (k, e, fd, g[k, e], scale)


def test_schedule_loss_autograd_and_state(gpu):
    """torch.autograd through schedule_loss gives the adjoint gradient, and the handle is
    left in the state after the run: continuing gives the same fields as a plain run."""
    w = tiny_3d()
    V = torch.tensor([[0.03, 0.05], [0.06, 0.01]], dtype=torch.float64, requires_grad=True)
    sim = gpu.Simulation(w)
    L = gpu.schedule_loss(sim, V, 6)
    L.backward()
    ref = gpu.Simulation(w)
    ref.adjoint_forward(V.detach().numpy(), 6)
    g_ref = ref.adjoint_backward()
    assert np.allclose(V.grad.numpy(), g_ref, rtol=1e-6, atol=1e-12)
    plain = gpu.Simulation(w)
    for k in range(2):
        plain.set_electrodes(V.detach().numpy()[k])
        plain.step(6)
    for s in (sim, plain):
        s.set_electrodes([0.02, 0.02])
        s.step(4)
    for name in ("g", "fphi", "frho", "phi"):
        assert np.abs(sim.array(name) - plain.array(name)).max() <= 1e-6, name


def test_observables_after_the_backward_are_the_forward_runs(gpu):
    """The backward's replays overwrite the observable sums; afterwards the handle reports
    the sums of the forward run's last two steps again, bit for bit."""
    w = tiny_3d()
    V = np.array([[0.03, 0.05], [0.06, 0.01]])
    sim = gpu.Simulation(w)
    sim.adjoint_forward(V, 6)
    before = sim.observe()
    sim.adjoint_backward()
    after = sim.observe()
    for k in ("step", "M1", "centroid", "velocity", "f_ele", "f_ele_total", "f_drag", "mass",
              "charge"):
        assert np.array_equal(np.asarray(before[k]), np.asarray(after[k])), k


def test_recorded_potential_and_replayed_solve_agree(gpu):
    """Backward replays with the recorded potential trajectory, and replays that solve
    Gauss's law again (LBEHD_OPT_ADJ_TRAJECTORY = 0), give the same gradient bit for bit:
    the replayed solve reproduces the recorded potential exactly. 52 steps, so four
    checkpoint intervals, the last one short."""
    w = tiny_3d()
    V = np.array([[0.03, 0.05], [0.06, 0.01], [0.0, 0.04], [0.05, 0.05]])
    grads, losses = [], []
    for traj in (1, 0):
        sim = gpu.Simulation(w)
        sim.set_option(gpu.OPT_ADJ_TRAJECTORY, traj)
        losses.append(sim.adjoint_forward(V, 13))
        grads.append(sim.adjoint_backward())
        sim.close()
    assert losses[0] == losses[1]
    assert np.array_equal(grads[0], grads[1]), np.abs(grads[0] - grads[1]).max()

"""The paper's droplet-transport analysis on top of the CUDA step (Results, Eqs. 1-7):

* the electrode geometry of Fig. 1 (an electrode block above a grounded substrate): the
  Gauss-law solution far from the electrode is the strip's lowest mode with the decay rate
  of Eqs. 3-4, and a droplet in that geometry steps like the FP64 oracle and is pulled
  towards the electrode;
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


def rel_linf(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("ny,l_e,x0", [(24, 8, 110), (34, 12, 80)])
def test_strip_lowest_mode_on_the_gpu(gpu, oracle_mod, ny, l_e, x0):
    """Fig. 1 geometry, 2D, no droplet: the potential of the CUDA Gauss-law solve against the
    oracle's (1e-5 relative), and its decay far from the electrode against the strip's
    lowest mode: cosh(alpha) = 2 - cos(k), k = pi / (2 H), H = ny - 1.5 (Eqs. 3-4 on the
    lattice), from every three consecutive values of the middle row over 31 nodes starting
    at x0 (100-160 nodes from the electrode: the next mode below 1e-5 of the lowest one, the
    potential still well above the solve's tolerance)."""
    w = W.electrode_above(2, 256, ny, 1, l_e=l_e, x_e=240, w_e=8, V=0.05)
    w.params = dict(w.params, poisson_tol=1e-8)
    sim = gpu.Simulation(w)
    sim.step(1)
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    orc.step(1)
    fl = w.solid == 0
    pot = sim.potential()
    assert rel_linf(pot[fl], orc.pot[fl]) <= 1e-5
    H, v = ny - 1.5, ny // 2
    k = np.pi / (2 * H)
    alpha = np.arccosh(2 - np.cos(k))
    row = pot[0, v, x0:x0 + 31]
    est = np.arccosh((row[2:] + row[:-2]) / row[1:-1] / 2)
    assert np.abs(est / alpha - 1).max() < 1e-3, (est.min(), est.max(), alpha)


def test_droplet_in_the_fig1_geometry(gpu, oracle_mod):
    """A droplet on a micropillar film below the electrode block of Fig. 1 (3D, 48x16x20):
    populations after 100 steps within 1e-5 of the oracle, observables within 0.5 %, and the
    electric force pulls the droplet towards the electrode (+x)."""
    w = W.electrode_above(3, 48, 16, 20, l_e=6, x_e=38, w_e=6, V=0.08, droplet=(17.3, 6.0),
                          pillar_h=3, seed=9)
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    sim.step(100)
    orc.step(100)
    fl = orc.solid == 0
    assert rel_linf(sim.populations_g()[:, fl], orc.g[:, fl]) <= 1e-5
    assert rel_linf(sim.array("fphi")[:, :, fl], orc.fphi[:, :, fl]) <= 1e-5
    og, oo = sim.observe(), orc.observables()
    for key in ("f_ele", "velocity"):
        assert np.abs(og[key] - oo[key]).max() <= 5e-3 * np.abs(oo[key]).max(), key
    assert oo["f_ele"][0] > 0 and og["f_ele"][0] > 0
    assert og["status"] == 0


def _settled(gpu, w, steps):
    """A handle stepped `steps` steps with no drive (the droplet sinks into the film and
    settles), and its saved state, from which the runs below branch."""
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    sim.step(steps)
    return sim, sim.save_state()


def _branch(sim, state, steps, every, V=0.0, body_droplet=0.0):
    """Rows (step, M1, centroid[3], velocity[3], f_ele[3], f_drag[3]) every `every` steps of
    a run from `state` with electrode potential V and droplet body force (body_droplet, 0, 0)."""
    sim.load_state(state)
    sim.set_electrodes([V])
    sim.set_body_force(body_droplet=[body_droplet, 0.0, 0.0])
    rows = []
    for k in range(steps // every):
        sim.step(every)
        o = sim.observe()
        assert o["status"] == 0
        rows.append([every * (k + 1), o["M1"], *o["centroid"], *o["velocity"], *o["f_ele"],
                     *o["f_drag"]])
    return np.array(rows)


def test_sliding_droplet_drag_is_linear(gpu):
    """Sliding droplet (Results, Fig. 3a-b, droplet-dissipation regime; Methods, sliding on a
    lubricant-infused surface): a settled droplet (R0 = 7 on a micropillar film, equal
    viscosities of droplet and lubricant) pushed along x by a body force on the droplet phase,
    b = 2.5e-6, 5e-6 and 1e-5, for 6000 steps, against a run with no force from the same
    state. Over the last 2000 steps:
    * the drag the step reports (the force balance) equals the applied force M1 b within 2 %
      (the droplet no longer accelerates);
    * the droplet's velocity, less the undriven run's drift, is proportional to b: the
      simulated drag coefficient C_drag,sim = M1 b / (2 R0 mu_bar V) (Eq. 1's linear law,
      mu_bar the geometric mean of the phases' viscosities) agrees between the three forces
      within 5 %."""
    from paper_2608_12868_b300 import reduced_model as RM
    w = W.droplet_3d(64, 32, 32, R=7.0, xc=20.0, pillar_h=4, electrodes=[(0, 0, 0, 0)], V=[0.0],
                     seed=32, name="sliding_3d_64x32x32")
    sim, state = _settled(gpu, w, 20000)
    base = _branch(sim, state, 6000, 50)
    mu_bar = RM.effective_viscosity(w.params["nu"])
    C = []
    for b in (2.5e-6, 5e-6, 1e-5):
        a = _branch(sim, state, 6000, 50, body_droplet=b)
        late = a[:, 0] > 4000
        M1 = a[-1, 1]
        assert abs(a[late, 11].mean() / (M1 * b) - 1) < 0.02
        i0 = np.argmax(late)
        dS = (a[-1, 2] - a[i0 - 1, 2]) - (base[-1, 2] - base[i0 - 1, 2])
        V = dS / (a[-1, 0] - a[i0 - 1, 0])
        C.append(RM.drag_coefficient(M1 * b, V, 7.0, mu_bar))
    C = np.array(C)
    assert np.all(C > 0)
    assert np.abs(C / C.mean() - 1).max() < 0.05, C


def test_reduced_model_predicts_electrode_driven_motion(gpu):
    """The reduced-order model of the Results (Eq. 5) closed on simulated runs, then used to
    predict runs it was not fitted to. A droplet (R0 = 7) settled on a micropillar film
    9 lu in front of a bottom electrode patch (96x32x32), all runs from one saved state,
    displacements measured against an undriven run from the same state:
    * the drag coefficient c = C_drag 2 R0 mu_bar of Eq. 5 from a sliding run (droplet body
      force 5e-6: the drag the step reports over the velocity);
    * the force coefficient A = Lambda K_e C_ele from the run at phi0 = 0.08: the electric
      force F_ele = A e^{2 alpha0 S} (Eq. 5 with S0 - S = S_e), alpha0 = pi / (2 H) the strip
      decay rate of the channel (Eq. 4; H = nz - 1.5 from the grounded top wall to the floor),
      A averaged over steps 40 000 - 100 000. Before that the lubricant's charge relaxes
      (eps / sigma = 2e4 steps) and the force is not yet a function of position alone, which
      Eq. 5 assumes;
    * prediction for phi0 = 0.06 and 0.1 (A scales with phi0^2, Eq. 4): Eq. 5 integrated over
      steps 40 000 - 100 000 from the simulated state at 40 000, against the simulation: the
      displacement within 25 %, and the time to cover half of it (a switching criterion for
      the next electrode) within 25 %. (The bar reflects what the one-degree-of-freedom
      model captures at these small displacements, ~0.2 lu, where the undriven run's drift
      that is subtracted is of the same order.) (Longer runs this close to the electrode are not
      used: at phi0 = 0.1 the state turned non-finite between 100 000 and 150 000 steps.)"""
    from paper_2608_12868_b300 import reduced_model as RM
    w = W.droplet_3d(96, 32, 32, R=7.0, xc=40.0, pillar_h=4, electrodes=[(56, 72, 8, 24)],
                     V=[0.0], seed=31, name="rom_3d_96x32x32")
    sim, state = _settled(gpu, w, 20000)
    T, every, t0 = 100000, 2500, 40000
    base = _branch(sim, state, T, every)            # rows at steps 2500, 5000, ...
    slide = _branch(sim, state, 5000, 2500, body_droplet=5e-6)
    V_slide = ((slide[1, 2] - slide[0, 2]) - (base[1, 2] - base[0, 2])) / 2500.0
    c = slide[1, 11] / V_slide                      # drag over velocity, quasi-steady
    alpha0 = RM.strip_alpha0(w.shape[0] - 1.5, 0.0)
    t = base[:, 0]
    win = t >= t0
    ref = _branch(sim, state, T, every, V=0.08)
    S_ref = ref[:, 2] - base[:, 2]
    A_ref = float(np.mean(ref[win, 8] * np.exp(-2.0 * alpha0 * S_ref[win])))
    for phi0 in (0.06, 0.1):
        run = _branch(sim, state, T, every, V=phi0)
        S = run[:, 2] - base[:, 2]
        k0 = int(np.argmax(win))
        V0 = (S[k0 + 1] - S[k0 - 1]) / (2.0 * every)
        model = RM.ReducedModel(m=run[-1, 1], c=c, A=A_ref * (phi0 / 0.08) ** 2,
                                alpha0=alpha0, S0=0.0)
        S_pred, _ = model.trajectory(t[win] - t0, S_init=S[k0], V_init=V0, substeps=200)
        dS_sim, dS_pred = S[-1] - S[k0], S_pred[-1] - S[k0]
        print("phi0", phi0, "c", c, "A", A_ref, "dS_sim", dS_sim, "dS_pred", dS_pred)
        assert dS_sim > 0
        assert abs(dS_pred / dS_sim - 1) < 0.25, (phi0, dS_pred, dS_sim, c, A_ref)

        def first_time(Sx, tx, target):
            k = int(np.argmax(Sx >= target))
            return tx[k - 1] + (target - Sx[k - 1]) / (Sx[k] - Sx[k - 1]) * (tx[k] - tx[k - 1])

        half = S[k0] + 0.5 * dS_sim
        t_sim = first_time(S[win], t[win], half)
        t_pred = first_time(S_pred, t[win], half)
        print("phi0", phi0, "half-way time sim", t_sim, "pred", t_pred)
        assert abs((t_pred - t0) / (t_sim - t0) - 1) < 0.25, (phi0, t_pred, t_sim)

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs.

Bars (written here, derived from the target tolerances of the method):
* populations: relative L-infinity max|f_gpu - f_oracle| / max|f_oracle| <= 1e-5 per
  population set after up to 100 steps (FP32 state against FP64);
* fields Phi_i: absolute L-infinity <= 1e-5 (they are O(1));
* droplet observables (centroid velocity, electric force): 0.5 % of their magnitude; the
  drag (force balance: driving force minus M1 dV/dt) 0.5 % of max(|drag|, DRAG_FLOOR |f_ele|):
  while the droplet still accelerates the drag is a small difference of two large terms, and
  its FP32 error is set by that of f_ele and of M1 dV/dt, not by its own size;
* per-component mass: conserved to 1e-6 relative on the GPU.
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
OBS_TOL = 5e-3
DRAG_FLOOR = 0.1


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


def make_pair(gpu, oracle_mod, w, **kw):
    sim = gpu.Simulation(w, **kw)
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    return sim, orc


def compare_populations(sim, orc, tol=POP_TOL):
    """Populations at fluid nodes (solid-node slots are never read by either side)."""
    fl = orc.solid == 0
    errs = {
        "g": rel_linf(sim.populations_g()[:, fl], orc.g[:, fl]),
        "fphi": rel_linf(sim.array("fphi")[:, :, fl], orc.fphi[:, :, fl]),
        "frho": (rel_linf(sim.array("frho")[:, fl], orc.frho[:, fl])
                 if np.abs(orc.frho).max() > 0 else 0.0),
    }
    for k, v in errs.items():
        assert v <= tol, (k, errs)
    return errs


def compare_fields(sim, orc, phi_tol=1e-5):
    fluid = orc.solid == 0
    phi = sim.array("phi")
    assert np.abs(phi[:, fluid] - orc.Phi[:, fluid]).max() <= phi_tol
    bnd = orc.normal > 0
    if bnd.any():   # wetting ghosts (Eq. 20a)
        assert np.abs(phi[:, bnd] - orc.Phi[:, bnd]).max() <= phi_tol
    pot = sim.potential()
    if np.abs(orc.pot).max() > 0:
        assert rel_linf(pot[fluid], orc.pot[fluid]) <= 1e-5


def compare_obs(sim, orc, keys=("velocity", "f_ele", "f_ele_total", "f_drag"), tol=OBS_TOL):
    og, oo = sim.observe(), orc.observables()
    for k in keys:
        a, b = np.asarray(og[k]), np.asarray(oo[k])
        scale = np.abs(b).max()
        if k == "f_drag":
            scale = max(scale, DRAG_FLOOR * np.abs(oo["f_ele"]).max())
        assert np.abs(a - b).max() <= tol * scale, (k, a, b)
    assert np.abs(og["centroid"] - oo["centroid"]).max() <= 1e-3
    assert np.abs(og["mass"] / oo["mass"] - 1).max() <= 1e-5


@pytest.mark.parametrize("steps", [1, 10, 100])
def test_small_2d_populations(gpu, oracle_mod, steps):
    w = W.small_2d()
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.step(steps)
    orc.step(steps)
    compare_populations(sim, orc)
    compare_fields(sim, orc)


@pytest.mark.parametrize("steps", [1, 100])
def test_small_3d_populations(gpu, oracle_mod, steps):
    w = W.small_3d()
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.step(steps)
    orc.step(steps)
    compare_populations(sim, orc)
    compare_fields(sim, orc)


@pytest.mark.parametrize("variant", ["global", "staged"])
def test_collide_kernel_variants(gpu, oracle_mod, variant):
    """Both fused collide kernels (populations loaded from global memory, or staged into
    shared memory by bulk copies) against the oracle, on a 3D case with a ragged x tile."""
    w = W.droplet_3d(136, 16, 16, R=5.0, pillar_h=3, electrodes=[(90, 120, 4, 12)], seed=12)
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.set_option(gpu.OPT_COLLIDE, gpu.COLLIDE_GLOBAL if variant == "global" else gpu.COLLIDE_STAGED)
    sim.step(30)
    orc.step(30)
    compare_populations(sim, orc)
    compare_fields(sim, orc)
    assert sim.observe()["status"] == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_strong_uniform_acceleration_parity(gpu, oracle_mod, dim):
    """Periodic box, uniform mixture Phi = (0.3, 0.2, 0.5), uniform body force 1e-3: after
    100 steps u = 0.1, and the force's share of the non-equilibrium second moments that the
    shear relaxation acts on, (1 - s_nu) (u F + F u) / 2 with 1 - s_nu = -0.5 here, is ~5e-5 of
    the momentum populations. Those within 1e-6 of the oracle (measured 3e-8 in 3D, 1e-7 in
    2D; a sign slip in that share, which the ordinary cases' 1e-5 bar misses at their small
    u F, fails this by 50x), the other sets at the usual 1e-5 (at u = 0.1 the FP32 backward
    difference of Phi u in Eq. 17 cancels two digits: ~4e-6)."""
    shape = (1, 6, 8) if dim == 2 else (4, 6, 8)
    one = np.ones(shape)
    phi = np.stack([0.3 * one, 0.2 * one, 0.5 * one])
    p = W.make_params(V=(), body=(1e-3, -4e-4, 2e-4 if dim == 3 else 0.0))
    w = W.Workload(f"accel_{dim}d", dim, shape, np.zeros(shape, np.uint8),
                   np.full(shape, -1, np.int16), phi, p)
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.step(100)
    orc.step(100)
    assert np.abs(orc.u[0]).max() > 0.09
    errs = compare_populations(sim, orc)
    assert errs["g"] <= 1e-6, errs


def test_small_3d_observables(gpu, oracle_mod):
    w = W.small_3d()
    sim, orc = make_pair(gpu, oracle_mod, w)
    for _ in range(4):
        sim.step(25)
        orc.step(25)
        compare_obs(sim, orc)


def test_droplet_2d_128x64(gpu, oracle_mod):
    """The 2D 128x64 pillar-row workload: populations after 100 steps, observables every
    100 steps up to 600."""
    w = W.droplet_2d_128x64()
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.step(100)
    orc.step(100)
    compare_populations(sim, orc)
    compare_fields(sim, orc)
    compare_obs(sim, orc)
    for _ in range(5):
        sim.step(100)
        orc.step(100)
        compare_obs(sim, orc)


def test_droplet_2d_128x64_full_run(gpu, oracle_mod):
    """The 2D 128x64 workload over its full 2000 steps in the benchmark's launch
    configuration (step graphs, persistent Gauss-law solve): droplet velocity and electric
    forces within 0.5 % of the FP64 oracle every 250 steps, centroid within 1e-3 lu, component
    masses within 1e-5."""
    w = W.droplet_2d_128x64()
    sim, orc = make_pair(gpu, oracle_mod, w, poisson_mode=gpu.POISSON_GRAPH)
    assert sim.get_option(gpu.OPT_POISSON_KERNEL) == 1
    for _ in range(8):
        sim.step(250)
        orc.step(250)
        compare_obs(sim, orc)
    assert sim.observe()["step"] == 1999


def test_droplet_3d_128x64x64_full_size(gpu, oracle_mod):
    """The 3D 128x64x64 workload at full size, in the launch configuration the benchmark
    times (graph replay with the persistent Gauss-law solve, autotuned collide kernel):
    every population set, the fields and the droplet observables after 3 and after 100
    steps (the FP64 oracle's first 100 steps of this configuration)."""
    w = W.droplet_3d_128x64x64()
    sim, orc = make_pair(gpu, oracle_mod, w, poisson_mode=gpu.POISSON_GRAPH)
    sim.step(1)
    sim.autotune(reps=2)
    sim.step(2)
    orc.step(3)
    assert sim.stats()["graph_launches"] == 2
    compare_populations(sim, orc)
    compare_fields(sim, orc)
    compare_obs(sim, orc)
    sim.step(97)
    orc.step(97)
    compare_populations(sim, orc)
    compare_fields(sim, orc)
    compare_obs(sim, orc)


@pytest.mark.parametrize("case", ["small_2d", "small_3d"])
def test_graph_mode_parity(gpu, oracle_mod, case):
    """Graph replay (CG loop as device-side conditional nodes) against the oracle, and
    against eager launches with host convergence checks."""
    w = getattr(W, case)()
    sim, orc = make_pair(gpu, oracle_mod, w, poisson_mode=gpu.POISSON_GRAPH)
    host = gpu.Simulation(w, poisson_mode=gpu.POISSON_HOST)
    sim.step(100)
    orc.step(100)
    host.step(100)
    compare_populations(sim, orc)
    compare_fields(sim, orc)
    assert sim.stats()["graph_launches"] == 99
    assert rel_linf(sim.array("fphi"), host.array("fphi").astype(np.float64)) <= 1e-6
    assert rel_linf(sim.potential(), host.potential()) <= 1e-6
    o = sim.observe()
    assert o["status"] == 0 and o["poisson_iters"] >= 0


def test_electrode_switching_parity(gpu, oracle_mod):
    """lbehd_set_electrodes mid-run (graph replay) matches the oracle switching at the same
    step."""
    w = W.droplet_3d(32, 16, 16, R=5.0, pillar_h=3,
                     electrodes=[(4, 10, 4, 12), (20, 28, 4, 12)], V=[0.05, 0.0], seed=11)
    sim, orc = make_pair(gpu, oracle_mod, w, poisson_mode=gpu.POISSON_GRAPH)
    sim.step(20)
    orc.step(20)
    sim.set_electrodes([0.0, 0.06])
    orc.set_electrodes([0.0, 0.06])
    sim.step(30)
    orc.step(30)
    compare_populations(sim, orc)
    compare_fields(sim, orc)


def test_ragged_and_periodic_edge_cases(gpu, oracle_mod):
    """nx not a multiple of the block width; an all-fluid periodic box with no electrode
    (the Poisson right-hand side is zero: phi = 0). The drop sits off the lattice symmetry
    lines: in an exactly mirror-symmetric box the sharpening flux of Eq. 18 amplifies
    rounding-level symmetry breaking at the saddle points between periodic images, so FP32
    and FP64 runs part there by construction."""
    w = W.small_2d(nx=50, ny=30)
    sim, orc = make_pair(gpu, oracle_mod, w)
    sim.step(30)
    orc.step(30)
    compare_populations(sim, orc)

    n = 32
    shape = (1, n, n)
    _, yy, xx = np.meshgrid(np.arange(1), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((xx - 16.3) ** 2 + (yy - 16.15) ** 2)
    pd = 0.5 * (1 - np.tanh(2 * (r - 8) / 5))
    phi = np.stack([pd, 0 * pd, 1 - pd])
    wp = W.Workload("periodic", 2, shape, np.zeros(shape, np.uint8), np.full(shape, -1, np.int16),
                    phi, W.make_params(V=()))
    sim, orc = make_pair(gpu, oracle_mod, wp)
    sim.step(40)
    orc.step(40)
    compare_populations(sim, orc)
    assert np.abs(sim.array("pot")).max() == 0.0


def test_mass_conservation_long_run(gpu):
    """Per-component mass over the full 10 000 steps of the 3D 128x64x64 workload (FP32
    state, the benchmark's launch configuration), checked every 2500 steps."""
    w = W.droplet_3d_128x64x64()
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    sim.step(1)
    sim.autotune(reps=2)
    m0 = sim.observe()["mass"]
    for _ in range(4):
        sim.step(2500)
        o = sim.observe()
        assert np.abs(o["mass"] / m0 - 1).max() <= 1e-6, o["mass"] / m0 - 1
        assert o["status"] == 0


def test_mid_3d_observables_long_run(gpu, oracle_mod):
    """Droplet observables of a 40x24x24 copy of the 3D workload (pillars, film, droplet,
    electrode) against the oracle every 250 steps over 1000 steps, in the benchmark's launch
    configuration. (The populations' 1e-5 bar is the 100-step one: FP32 rounding against
    FP64 grows with the run, to ~5e-5 of the phase-field populations after 1000 steps.)"""
    w = W.droplet_3d(40, 24, 24, R=7.0, pillar_h=4, seed=21, name="mid_3d_40x24x24")
    sim, orc = make_pair(gpu, oracle_mod, w, poisson_mode=gpu.POISSON_GRAPH)
    for _ in range(4):
        sim.step(250)
        orc.step(250)
        compare_obs(sim, orc)


def test_largest_workload_runs(gpu):
    """384x128x96 long-transport lattice (4.7 M sites) in the benchmark's launch
    configuration: allocates, steps, stays finite and conserving; its persistent Gauss-law
    solve (four multigrid levels above the tail) gives the multi-launch solve's bits."""
    w = W.transport_3d_384x128x96()
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    assert sim.get_option(gpu.OPT_POISSON_KERNEL) == 1
    sim.step(2)
    m0 = sim.observe()["mass"]
    sim.step(20)
    o = sim.observe()
    assert o["status"] == 0
    assert np.abs(o["mass"] / m0 - 1).max() <= 1e-6
    ref = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    ref.set_option(gpu.OPT_POISSON_KERNEL, 0)
    ref.step(22)
    for name in ("g", "pot", "pot_lo"):
        assert np.array_equal(sim.array(name), ref.array(name)), name


def test_long_transport_two_switches(gpu):
    """The 384x128x96 long-transport workload through two electrode switches of its
    schedule (electrode k live during steps [2000 k, 2000 (k + 1))), 4500 steps: every
    component's mass within 1e-6 and no error status."""
    w = W.transport_3d_384x128x96()
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    sim.step(1)
    sim.autotune(reps=2)
    m0 = sim.observe()["mass"]
    done = 1
    for k, V in sorted(w.schedule)[:3]:
        if k > done:
            sim.step(k - done)
            done = k
        sim.set_electrodes(V)
    sim.step(4500 - done)
    o = sim.observe()
    assert o["status"] == 0
    assert np.abs(o["mass"] / m0 - 1).max() <= 1e-6, o["mass"] / m0 - 1
    assert np.isfinite(o["centroid"]).all() and np.isfinite(o["f_drag"]).all()


def test_error_paths(gpu):
    """Non-finite state is reported (not a fault); a Poisson cap of one sweep is reported."""
    w = W.small_2d()
    w.phi_init = w.phi_init.copy()
    w.phi_init[0, 0, 10, 10] = np.nan
    sim = gpu.Simulation(w)
    sim.step(2)
    with pytest.raises(gpu.LBEHDError) as e:
        sim.observe()
    assert e.value.code == -4

    w = W.small_2d()
    w.params = dict(w.params, poisson_max_iter=1, poisson_tol=1e-12)
    sim = gpu.Simulation(w, poisson_check_every=1)
    assert sim.step(3) == -3


def test_zero_copy_views(gpu):
    w = W.small_3d()
    sim = gpu.Simulation(w)
    sim.step(3)
    t = sim.tensor("phi").cpu().numpy()
    assert np.array_equal(t, sim.array("phi"))
    assert sim.launch_count() > 0


def test_handles_with_different_tails_coexist(gpu):
    """Kernel attributes (shared-memory limits) are per kernel, not per handle: a handle
    created after another with a smaller multigrid tail must not break the first one."""
    big = gpu.Simulation(W.small_2d(nx=64, ny=40, seed=7, R=9.0, V=0.03))
    small = gpu.Simulation(W.small_2d())
    small.step(3)
    big.step(3)
    assert big.observe()["status"] == 0 and small.observe()["status"] == 0

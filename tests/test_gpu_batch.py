"""Batched form: many uneven instances advanced by one graph launch per step.

Every instance of a batch must compute what the same instance computes alone: the state
arrays (populations, fields, potential) are compared bit for bit with single-instance
runs in graph mode using the same collide kernel and the same multigrid smoother (a batch's
default, whole-level red-black sweeps, and once the block-local smoother), after enough
steps to include a
multigrid rebuild (every 16 steps). One instance is also compared with the FP64 oracle
at the parity bars of the single-instance tests. The collide-kernel autotuner must leave
the state untouched.
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

pytestmark = pytest.mark.gpu

STATE = ("g", "fphi", "frho", "phi", "rho", "u", "qsrc", "pot", "pot_lo", "eps")


@pytest.fixture(scope="module")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_12868_b300 import build, lbehd
    build.build()
    return lbehd


def uneven_3d():
    """Four uneven 3D instances: sizes, viscosity ratio, contact angle and potential differ;
    nx = 36 and 44 leave ragged tiles for every staged tile width."""
    return [
        W.droplet_3d(32, 16, 16, R=5.0, pillar_h=3, electrodes=[(20, 28, 4, 12)], V=[0.05],
                     seed=21),
        W.droplet_3d(36, 24, 16, R=6.0, pillar_h=3, electrodes=[(22, 30, 6, 18)], V=[0.03],
                     visc_ratio=0.2, theta12=100.0, seed=22),
        W.droplet_3d(44, 16, 20, R=5.0, pillar_h=4, electrodes=[(28, 38, 4, 12)], V=[0.07],
                     visc_ratio=5.0, theta12=140.0, seed=23),
        W.droplet_3d(64, 32, 18, R=7.0, pillar_h=3, electrodes=[(40, 52, 8, 24)], V=[0.04],
                     visc_ratio=1.0, theta12=75.0, seed=24),
    ]


def plain(gpu, w, smoother=0, warm=0):
    """A single handle in graph mode with the given multigrid smoother and warm start (0 for
    both: a batch's defaults)."""
    sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
    sim.set_option(gpu.OPT_MG_SMOOTHER, smoother)
    sim.set_option(gpu.OPT_WARM_START, warm)
    return sim


def single_run(gpu, w, variant, steps):
    sim = plain(gpu, w)
    sim.set_option(gpu.OPT_COLLIDE, variant)
    sim.step(steps)
    return sim


def assert_same_state(a, b, what):
    for name in STATE:
        x, y = a.array(name), b.array(name)
        assert np.array_equal(x, y), (what, name, float(np.abs(x - y).max()))


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_batch_bitwise_equals_single_instances(gpu, variant):
    ws = uneven_3d()
    batch = gpu.Batch(ws)
    batch.set_option(gpu.OPT_COLLIDE, variant)
    steps = 20
    batch.step(steps)
    obs = batch.observe()
    st = batch.stats()
    assert st["steps"] == steps and st["graph_launches"] == steps - 1
    for i, w in enumerate(ws):
        sim = single_run(gpu, w, variant, steps)
        assert_same_state(batch[i], sim, f"instance {i}")
        o = sim.observe()
        # the staged kernels use the same tiles alone and batched (bitwise observables);
        # the global-load kernel's batched launch packs sites into warps differently, so
        # its FP32 warp partial sums differ in rounding
        rtol = 1e-6 if variant == 1 else 0.0
        for k in ("centroid", "velocity", "f_ele", "f_ele_total", "mass"):
            scale = np.abs(o[k]).max()
            assert np.abs(obs[i][k] - o[k]).max() <= rtol * scale, (i, k, obs[i][k], o[k])
        assert obs[i]["status"] == 0 and obs[i]["step"] == o["step"]
        sim.close()
    batch.close()


def test_batch_least_residual_start_bitwise_equals_single_instances(gpu):
    """The same comparison with every solve started from the least-residual combination of
    the last two increments (LBEHD_OPT_WARM_START = 1, a handle's default) on both sides."""
    ws = uneven_3d()
    batch = gpu.Batch(ws)
    batch.set_option(gpu.OPT_WARM_START, 1)
    steps = 20
    batch.step(steps)
    for i, w in enumerate(ws):
        sim = plain(gpu, w, warm=1)
        sim.step(steps)
        assert_same_state(batch[i], sim, f"instance {i}")
        assert batch.observe()[i]["status"] == 0
        sim.close()
    batch.close()


def test_batch_block_smoother_bitwise_equals_single_instances(gpu):
    """The same comparison with the block-local smoother (LBEHD_OPT_MG_SMOOTHER = 1) on both
    sides."""
    ws = uneven_3d()
    batch = gpu.Batch(ws)
    batch.set_option(gpu.OPT_MG_SMOOTHER, 1)
    steps = 20
    batch.step(steps)
    for i, w in enumerate(ws):
        sim = plain(gpu, w, 1)
        sim.step(steps)
        assert_same_state(batch[i], sim, f"instance {i}")
        sim.close()
    batch.close()


def test_batch_mixing_the_two_smoothers(gpu):
    """A 44^3 lattice coarsens once (22 is not a multiple of 4) to 22^3 = 10648 cells, too many
    for the shared-memory tail, so it has no tail and keeps whole-level sweeps with the
    block-local option set, while the other instances smooth block by block: one batched
    V-cycle runs both on level 0. Every instance equals its single-handle run bit for bit."""
    ws = uneven_3d()[:2] + [W.droplet_3d(44, 44, 44, R=8.0, pillar_h=4,
                                         electrodes=[(28, 36, 16, 28)], V=[0.05], seed=25)]
    batch = gpu.Batch(ws)
    batch.set_option(gpu.OPT_MG_SMOOTHER, 1)
    steps = 20
    batch.step(steps)
    for i, w in enumerate(ws):
        sim = gpu.Simulation(w, poisson_mode=gpu.POISSON_GRAPH)
        sim.set_option(gpu.OPT_WARM_START, 0)
        assert sim.get_option(gpu.OPT_MG_SMOOTHER) == (0 if i == 2 else 1)
        sim.step(steps)
        assert_same_state(batch[i], sim, f"instance {i}")
        assert batch.observe()[i]["status"] == 0
        sim.close()
    batch.close()


def test_batch_2d_bitwise_equals_single_instances(gpu):
    ws = [W.small_2d(), W.small_2d(nx=64, ny=40, seed=7, R=9.0, V=0.03),
          W.small_2d(nx=52, ny=32, seed=8, R=7.0, V=0.06)]
    batch = gpu.Batch(ws)
    batch.step(18)
    for i, w in enumerate(ws):
        sim = single_run(gpu, w, gpu.COLLIDE_AUTO, 18)
        assert_same_state(batch[i], sim, f"2D instance {i}")


def test_batch_instance_matches_oracle(gpu, oracle_mod):
    """Instance 2 of the batch (ragged nx = 44) against the FP64 oracle after 30 steps."""
    from test_gpu_parity import compare_fields, compare_populations
    ws = uneven_3d()
    batch = gpu.Batch(ws)
    batch.step(30)
    w = ws[2]
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    orc.step(30)
    compare_populations(batch[2], orc)
    compare_fields(batch[2], orc)


def test_batch_autotune_mixed_groups(gpu):
    """The autotuner's per-instance choices (whatever they are) give the same states as
    single-instance runs with those choices; the tuning itself leaves the state alone."""
    ws = uneven_3d()
    batch = gpu.Batch(ws)
    batch.step(3)
    before = [{n: batch[i].array(n) for n in STATE} for i in range(len(ws))]
    variants, ms = batch.autotune(reps=5)
    assert len(variants) == len(ws) and all(1 <= v <= 4 for v in variants)
    for i in range(len(ws)):
        assert set(ms[i]) == {1, 2, 3, 4} and all(t > 0 for t in ms[i].values())
        assert ms[i][variants[i]] == min(ms[i].values())
        for n in STATE:
            assert np.array_equal(before[i][n], batch[i].array(n)), (i, n)
    batch.step(17)
    for i, w in enumerate(ws):
        sim = plain(gpu, w)
        sim.step(3)
        sim.set_option(gpu.OPT_COLLIDE, variants[i])
        sim.step(17)
        assert_same_state(batch[i], sim, f"tuned instance {i}")


def test_single_autotune_keeps_state(gpu):
    w = W.small_3d()
    sim = plain(gpu, w)
    ref = plain(gpu, w)
    sim.step(5)
    ref.step(5)
    o0 = sim.observe()
    v, ms = sim.autotune(reps=3)
    assert 1 <= v <= 4 and ms[v] == min(ms.values())
    o1 = sim.observe()
    for k in ("centroid", "velocity", "f_ele", "mass"):
        assert np.array_equal(o0[k], o1[k])
    ref.set_option(gpu.OPT_COLLIDE, v)
    sim.step(10)
    ref.step(10)
    assert_same_state(sim, ref, "after autotune")


def test_batch_instance_calls_refused(gpu):
    ws = uneven_3d()[:2]
    batch = gpu.Batch(ws)
    inst = batch[0]
    lib = gpu.load()
    assert lib.lbehd_step(inst._h, 1) == -1
    assert b"lbehd_batch_step" in lib.lbehd_last_error(inst._h)
    assert lib.lbehd_set_option(inst._h, gpu.OPT_COLLIDE, 1) == -1
    assert lib.lbehd_autotune(inst._h, 1, None) == -1
    assert lib.lbehd_profile_enable(inst._h, 1) == -1
    lib.lbehd_destroy(inst._h)   # a no-op on a batch instance
    batch.step(2)
    assert batch.observe()[0]["status"] == 0
    inst.set_electrodes([0.0])   # electrode switching works per instance
    batch.step(1)
    assert lib.lbehd_batch_instance(batch._b, 2) is None


def test_batched_sweep_64_instances(gpu):
    """The 64-instance sweep (sizes 48^3 to 128x64x64, viscosity ratio, contact angle and
    potential drawn per instance) at full size: 20 batched steps, every instance bitwise
    equal to its own single-instance run, every component mass conserved to 1e-6."""
    ws = W.batched_sweep()
    batch = gpu.Batch(ws)
    variants, _ = batch.autotune(reps=3)
    batch.step(1)
    m0 = [o["mass"] for o in batch.observe()]
    batch.step(19)
    obs = batch.observe()
    for i, w in enumerate(ws):
        assert obs[i]["status"] == 0
        assert np.abs(obs[i]["mass"] / m0[i] - 1).max() <= 1e-6, i
    for i, w in enumerate(ws):
        sim = plain(gpu, w)
        sim.set_option(gpu.OPT_COLLIDE, variants[i])
        sim.step(20)
        for name in ("g", "fphi", "frho", "pot"):
            assert np.array_equal(batch[i].array(name), sim.array(name)), (i, name)
        sim.close()
    batch.close()


def test_batch_eager_profile_steps_match_graph_steps(gpu):
    """Profiling runs the batch step as eager launches with host-checked loops: the same
    states as the graph replays, and every kernel class is timed."""
    ws = uneven_3d()
    a, b = gpu.Batch(ws), gpu.Batch(ws)
    a.step(20)
    b.step(5)
    b.profile(True)
    b.step(12)   # includes the multigrid rebuild at step 16
    prof = b.profile_read()
    b.profile(False)
    b.step(3)
    for i in range(len(ws)):
        assert_same_state(a[i], b[i], f"eager instance {i}")
    for k in ("fields", "mg", "cg", "collide", "obs"):
        assert prof[k][1] > 0 and prof[k][0] > 0, k

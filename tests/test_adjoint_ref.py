"""Pins of the FP64 discrete-adjoint reference (oracle/adjoint_ref.py), CPU only.

The reference restates the oracle step in differentiable PyTorch. It must (1) be the same
map as the C oracle, and (2) have gradients equal to finite differences of itself, for the
whole schedule loss and for the Gauss-law solve alone (whose backward pass is an
implicit-function adjoint solve, not autograd).
"""
import numpy as np
import pytest
import torch

from paper_2608_12868_b300 import workloads as W

T = torch.float64


@pytest.fixture(scope="module")
def ref(oracle_mod):
    from oracle import adjoint_ref as AR
    return AR


def tiny_3d():
    return W.droplet_3d(16, 8, 12, R=3.5, pillar_h=3, electrodes=[(4, 8, 2, 6), (8, 12, 2, 6)],
                        V=[0.03, 0.05], seed=5)


def model_for(oracle_mod, ref, w):
    orc = oracle_mod.OracleSim(w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    return orc, ref.RefModel(w.dim, w.shape, w.solid, w.elec, w.params, orc.normal)


@pytest.mark.parametrize("case", ["3d", "2d"])
def test_reference_step_is_the_oracle_step(oracle_mod, ref, case):
    w = tiny_3d() if case == "3d" else W.small_2d(nx=24, ny=16, R=5.0)
    orc, m = model_for(oracle_mod, ref, w)
    st = m.initial_state(w.phi_init)
    V = torch.tensor(w.params["V"], dtype=T)
    for _ in range(6):
        orc.step(1)
        st, Phi = m.step(st, V)
    for name in ("g", "fphi", "frho"):
        a = st[name].numpy().reshape(getattr(orc, name).shape)
        assert np.abs(a - getattr(orc, name)).max() <= 1e-12, name
    assert np.abs(Phi.numpy().reshape(orc.Phi.shape) - orc.Phi).max() <= 1e-12
    assert abs(float(m.centroid_x(Phi)) - orc.observables()["centroid"][0]) <= 1e-11


def test_reference_schedule_gradient_matches_finite_differences(oracle_mod, ref):
    """dL/dV for a 2-electrode, 2-segment schedule over 12 steps; L = droplet x centroid."""
    w = tiny_3d()
    _, m = model_for(oracle_mod, ref, w)
    Vs = torch.tensor([[0.03, 0.05], [0.06, 0.01]], dtype=T, requires_grad=True)
    L = ref.schedule_loss(m, w.phi_init, Vs, 6)
    L.backward()
    h = 1e-5
    for k in range(2):
        for e in range(2):
            Vp, Vm = Vs.detach().clone(), Vs.detach().clone()
            Vp[k, e] += h
            Vm[k, e] -= h
            fd = (float(ref.schedule_loss(m, w.phi_init, Vp, 6)) -
                  float(ref.schedule_loss(m, w.phi_init, Vm, 6))) / (2 * h)
            assert abs(fd - float(Vs.grad[k, e])) <= 1e-5 * abs(fd), (k, e, fd, Vs.grad[k, e])


def test_poisson_adjoint_solve_matches_finite_differences(oracle_mod, ref):
    """The Gauss-law solve's backward (one adjoint solve with the same operator) against
    finite differences in eps, rho and V for a random linear functional of phi."""
    w = tiny_3d()
    _, m = model_for(oracle_mod, ref, w)
    rng = np.random.default_rng(7)
    N = m.N
    fl = m.fluid.numpy() > 0
    eps = torch.tensor(np.where(fl, rng.uniform(1.0, 10.0, N), 0.0), dtype=T, requires_grad=True)
    rho = torch.tensor(np.where(fl, rng.normal(0, 1e-4, N), 0.0), dtype=T, requires_grad=True)
    V = torch.tensor([0.03, 0.05], dtype=T, requires_grad=True)
    wts = torch.tensor(rng.normal(size=N), dtype=T)
    L = (wts * ref.PoissonSolve.apply(eps, rho, V, m)).sum()
    L.backward()

    def f(e, r, v):
        return float((wts * ref.PoissonSolve.apply(e, r, v, m)).sum())

    h = 1e-6
    for e_ in range(2):
        Vp, Vm = V.detach().clone(), V.detach().clone()
        Vp[e_] += h
        Vm[e_] -= h
        fd = (f(eps.detach(), rho.detach(), Vp) - f(eps.detach(), rho.detach(), Vm)) / (2 * h)
        assert abs(fd - float(V.grad[e_])) <= 1e-5 * abs(fd) + 1e-12
    for i in rng.choice(np.nonzero(fl)[0], 4, replace=False):
        for which, t, g in (("rho", rho, rho.grad), ("eps", eps, eps.grad)):
            tp, tm = t.detach().clone(), t.detach().clone()
            tp[i] += h
            tm[i] -= h
            args_p = (tp, rho.detach(), V.detach()) if which == "eps" else (eps.detach(), tp, V.detach())
            args_m = (tm, rho.detach(), V.detach()) if which == "eps" else (eps.detach(), tm, V.detach())
            fd = (f(*args_p) - f(*args_m)) / (2 * h)
            assert abs(fd - float(g[i])) <= 1e-5 * abs(fd) + 1e-12, (which, i, fd, float(g[i]))


def test_reference_taylor_remainder_is_second_order(oracle_mod, ref):
    """Along a random direction d, the Taylor remainder |L(V + h d) - L(V) - h g.d| of the
    schedule loss falls as h^2 (about 4x per halving of h): the reference gradient g is the
    derivative of L, not just close to a difference quotient."""
    w = tiny_3d()
    _, m = model_for(oracle_mod, ref, w)
    Vs = torch.tensor([[0.03, 0.05], [0.06, 0.01]], dtype=T, requires_grad=True)
    L = ref.schedule_loss(m, w.phi_init, Vs, 6)
    L.backward()
    d = torch.tensor(np.random.default_rng(5).normal(size=(2, 2)), dtype=T)
    gd = float((Vs.grad * d).sum())
    L0 = float(L.detach())
    # small enough that a gradient error of 1 % would pull the ratios towards 2 (first order),
    # large enough that the remainders stay far above FP64 rounding of L (~1e-14)
    hs = [1e-3, 5e-4, 2.5e-4]
    rem = [abs(float(ref.schedule_loss(m, w.phi_init, Vs.detach() + h * d, 6)) - L0 - h * gd)
           for h in hs]
    for a, b in zip(rem, rem[1:]):
        assert 3.6 < a / b < 4.4, rem
    assert rem[-1] < 0.1 * abs(hs[-1] * gd), (rem, gd)

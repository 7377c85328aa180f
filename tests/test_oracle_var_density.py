"""Pins of the oracle's variable-density momentum scheme (large density ratios: Table 1's
densities in Eq. 9 with a variable rho; the pressure-based populations described in
oracle/lbehd_oracle.c), against what the mathematics fixes:

* Young-Laplace at Table 1's water/air density ratio (830) -> the capillary force, the
  pressure recovery and the density-gradient term together
* hydrostatic balance of a heavy layer under a body force on it -> the pressure gradient
  term and the density-gradient force (u stays at rest, dp/dy = -rho g)
* equal densities: plane Poiseuille -> the equilibrium, the force term and one relaxation
  time
* two layers of different density and viscosity in a force-driven channel -> the viscous
  stress div(rho nu (grad u + grad u^T)) with rho nu from the phase fields (the steady
  profile solves d/dy(mu du/dy) = -f for the run's own mu(y))
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W

RATIO_AIR = 998.0 / 1.2
RHO_TABLE1 = (1.0, 970.0 / 998.0, 1.2 / 998.0)   # water (droplet), oil, air
NU_TABLE1 = (0.1, 0.1, 0.1 * (0.0179 / 1.2) / (1.0 / 998.0))   # air's kinematic viscosity


def _params(**kw):
    p = dict(W.make_params(V=()))
    p.update(density_model=1, rho_phase=RHO_TABLE1, nu=NU_TABLE1)
    p.update(kw)
    return p


def _channel(ny, nx=2):
    shape = (1, ny, nx)
    yy = np.arange(ny)[None, :, None] * np.ones(shape)
    solid = np.zeros(shape, np.uint8)
    solid[(yy == 0) | (yy == ny - 1)] = 2
    return shape, yy, solid, np.full(shape, -1, np.int16)


def test_laplace_at_the_water_air_density_ratio(oracle_mod):
    """A water drop (R = 12) in air at rest: the pressure jump is gamma_13 / R (2D) within
    the diffuse interface's few per cent, and the spurious currents stay small."""
    n, R = 48, 12.0
    shape = (1, n, n)
    yy, xx = np.mgrid[0:n, 0:n]
    c = (n - 1) / 2
    pd = (0.5 * (1 - np.tanh(2 * (np.sqrt((xx - c) ** 2 + (yy - c) ** 2) - R) / 5)))[None]
    phi = np.zeros((3,) + shape)
    phi[0], phi[2] = pd, 1 - pd
    p = _params()
    s = oracle_mod.OracleSim(2, shape, np.zeros(shape, np.uint8), np.full(shape, -1, np.int16),
                             phi, p)
    s.step(1)
    m0 = s.Phi[0].sum()
    s.step(2999)
    Rm = np.sqrt(s.Phi[0][0].sum() / np.pi)
    dp = s.pstar[0][int(c), int(c)] - s.pstar[0][0, 0]
    assert abs(dp / (p["gamma13"] / Rm) - 1) < 0.06, dp / (p["gamma13"] / Rm)
    assert np.abs(s.u).max() < 1e-4
    assert abs(s.Phi[0].sum() / m0 - 1) < 1e-12


def test_hydrostatic_heavy_layer(oracle_mod):
    """Water below air between two walls, a body force -g y on the water phase alone (its
    weight, rho_1 = 1): at rest, dp/dy = -g inside the water and 0 inside the air."""
    ny, g = 42, 2e-6
    shape, yy, solid, elec = _channel(ny)
    h = 18.5
    P1 = 0.5 * (1 - np.tanh(2 * (yy - h) / 5)) * (solid == 0)
    phi = np.stack([P1, 0 * P1, (1 - P1) * (solid == 0)])
    s = oracle_mod.OracleSim(2, shape, solid, elec, phi, _params(body_droplet=(0.0, -g, 0.0)))
    s.step(16000)   # the pressure waves between the walls die out slowly
    p = s.pstar[0][:, 0]
    dpdy_water = np.polyfit(np.arange(3, 12), p[3:12], 1)[0]
    dpdy_air = np.polyfit(np.arange(27, 38), p[27:38], 1)[0]
    assert abs(dpdy_water / -g - 1) < 0.005, dpdy_water / -g
    assert abs(dpdy_air) < 0.005 * g, dpdy_air / g
    assert np.abs(s.u).max() < 1e-6


def test_equal_densities_plane_poiseuille(oracle_mod):
    """All densities 1: the body-force-driven channel between halfway bounce-back walls
    has the parabola u(y) = f/(2 nu) (y - y0)(y1 - y)."""
    ny, f, nu = 34, 1e-6, 0.1
    shape, yy, solid, elec = _channel(ny)
    one = (solid == 0).astype(float)
    phi = np.stack([one, 0 * one, 0 * one])
    s = oracle_mod.OracleSim(2, shape, solid, elec, phi,
                             _params(rho_phase=(1.0, 1.0, 1.0), nu=(nu, nu, nu),
                                     body=(f, 0.0, 0.0)))
    s.step(int(8 * (ny - 2) ** 2 / nu))
    y = np.arange(1, ny - 1)
    ex = f / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    num = s.u[0][0, 1:ny - 1, 0]
    assert np.sqrt(((num - ex) ** 2).sum() / (ex ** 2).sum()) < 2e-3


def test_two_layer_channel_viscous_stress(oracle_mod):
    """Water (rho 1, nu 0.1) below a lighter, more viscous layer (rho 0.3, nu 0.4) in a
    channel driven by a uniform force density f: the steady u(y) solves d/dy(mu du/dy) = -f
    with mu = rho nu of the run's own phase fields and no slip at both walls. Using nu in
    place of rho nu (or dropping the density-gradient term) changes the profile by tens of
    per cent."""
    ny, f = 42, 1e-6
    shape, yy, solid, elec = _channel(ny)
    h = 20.5
    P1 = 0.5 * (1 - np.tanh(2 * (yy - h) / 5)) * (solid == 0)
    phi = np.stack([P1, (1 - P1) * (solid == 0), 0 * P1])
    rho_ph, nu_ph = (1.0, 0.3, 1.0), (0.1, 0.4, 0.1)
    s = oracle_mod.OracleSim(2, shape, solid, elec, phi,
                             _params(rho_phase=rho_ph, nu=nu_ph, body=(f, 0.0, 0.0),
                                     gamma12=0.0006))
    s.step(30000)
    P = s.Phi[:, 0, :, 0]
    rho = sum(P[c] * rho_ph[c] for c in range(3))
    nu = sum(P[c] * nu_ph[c] for c in range(3))
    mu = (rho * nu)[1:ny - 1]
    # cell-centred fluid rows 1..ny-2, walls half a cell outside them; integrate
    # du/dy = (A - f y)/mu from the lower wall with A fixed by u = 0 at the upper wall
    y = np.arange(1, ny - 1, dtype=float)
    yf = np.concatenate([[0.5], 0.5 * (y[1:] + y[:-1]), [ny - 1.5]])   # faces
    muf = np.interp(yf, y, mu)
    dyf = np.diff(yf)

    def profile(A):
        dudy = (A - f * yf) / muf
        u_f = np.concatenate([[0.0], np.cumsum(0.5 * (dudy[1:] + dudy[:-1]) * dyf)])
        return np.interp(y, yf, u_f), u_f[-1]

    A0, A1 = 0.0, f * ny
    for _ in range(200):
        Am = 0.5 * (A0 + A1)
        if profile(Am)[1] > 0:
            A1 = Am
        else:
            A0 = Am
    ex, _ = profile(0.5 * (A0 + A1))
    num = s.u[0][0, 1:ny - 1, 0]
    err = np.sqrt(((num - ex) ** 2).sum() / (ex ** 2).sum())
    assert err < 0.02, err

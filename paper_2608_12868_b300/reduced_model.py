"""Reduced-order model of the electrically driven droplet (Results, Eqs. 1-7), fed by the
droplet observables the CUDA step reports (``lbehd_observe``: centroid, velocity, electric
force, drag).

The paper closes its control loop with a one-degree-of-freedom equation of motion for the
droplet's displacement S towards the live electrode (Eq. 5):

    m S'' = -C_drag 2 R0 mu_bar S' + Lambda K_e C_ele exp(-2 alpha0 (S0 - S)),

a linear viscous drag (Eq. 1 in the droplet-dissipation regime, effective viscosity mu_bar
the geometric mean of the three phases' viscosities) against a dielectrophoretic pull that
grows exponentially as the droplet-electrode distance S_e = S0 - S shrinks (Eqs. 2-4, the
lowest mode of the field in a strip of height h_e + l_e, decay rate alpha0). Eq. 7 integrates
the slowly varying (overdamped) form of Eq. 5, with an inertial correction, into the time
needed to travel a distance S_t, and the switching times of an electrode protocol follow
from it (Results, programmable transport, Fig. 5b/c).

Here the two lumped coefficients of Eq. 5 are fitted to simulated runs, as the paper fits
C_drag and Lambda to its LB runs:

* ``c = C_drag 2 R0 mu_bar`` from the drag the step reports against the droplet velocity
  (``fit_drag``), or from the stopping distance of a decelerating droplet
  (``drag_coefficient_deceleration``, the paper's C_drag,sim = m V0 / (2 R0 mu_bar S_max));
* ``A = Lambda K_e C_ele`` and ``alpha0`` from the electric force against the
  droplet-electrode distance (``fit_force_law``: ln F_ele is linear in S_e).

``ReducedModel`` then integrates Eq. 5 (classical fourth-order Runge-Kutta), evaluates
Eq. 7, and derives electrode switching times. Everything is host-side numpy; nothing here
runs the method's step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------- Eqs. 1-4

def effective_viscosity(mu):
    """mu_bar = (mu_o mu_w mu_g)^(1/3): the geometric mean of the three phases' dynamic
    viscosities that replaces the lubricant viscosity in the drag model (Eq. 1)."""
    mu = np.asarray(mu, dtype=np.float64)
    if mu.shape != (3,) or np.any(mu <= 0):
        raise ValueError("three positive viscosities expected")
    return float(np.prod(mu) ** (1.0 / 3.0))


def drag_coefficient(f_drag, velocity, R0, mu_bar):
    """C_drag of the linear drag law F_drag = C_drag 2 R0 mu_bar V (Eq. 5's drag term)."""
    return float(f_drag) / (2.0 * R0 * mu_bar * float(velocity))


def drag_coefficient_deceleration(m, V0, S_max, R0, mu_bar):
    """C_drag,sim = m V0 / (2 R0 mu_bar S_max): a droplet released at V0 with no drive stops
    after S_max = m V0 / (C_drag 2 R0 mu_bar) under the linear drag of Eq. 5."""
    return m * V0 / (2.0 * R0 * mu_bar * S_max)


def dep_prefactor(eps_w, R0, sigma_w, sigma_o):
    """K_e = 2 pi eps_w R0^3 (sigma_w - sigma_o) / (sigma_w - 2 sigma_o) of the
    point-dipole dielectrophoretic force (Eq. 2)."""
    return 2.0 * math.pi * eps_w * R0 ** 3 * (sigma_w - sigma_o) / (sigma_w - 2.0 * sigma_o)


def strip_alpha0(h_e, l_e):
    """alpha0 = pi / (2 (h_e + l_e)): decay rate of the lowest mode of the potential in the
    strip between the grounded surface and the top of the electrode (Eq. 4)."""
    return math.pi / (2.0 * (h_e + l_e))


def strip_C_ele(phi0, h_e, l_e):
    """C_ele of Eq. 4 for an electrode of height l_e at distance h_e above the surface,
    held at phi0: 2 alpha0 phi0^2 cos^2(alpha0 l_e) / (J_D + alpha0 J_N)^2 with
    J_N = l_e / 2 - sin(2 alpha0 l_e) / (4 alpha0), J_D = h_e / 2 + sin(2 alpha0 l_e) / (4 alpha0).
    The printed combination J_D + alpha0 J_N adds a length and a pure number, so it is taken
    as printed, in lattice units."""
    a0 = strip_alpha0(h_e, l_e)
    s = math.sin(2.0 * a0 * l_e) / (4.0 * a0)
    J_N = l_e / 2.0 - s
    J_D = h_e / 2.0 + s
    return 2.0 * a0 * phi0 ** 2 * math.cos(a0 * l_e) ** 2 / (J_D + a0 * J_N) ** 2


def electric_force(S_e, K_e, C_ele, alpha0, Lam=1.0):
    """Lambda K_e C_ele exp(-2 alpha0 S_e): Eq. 3 (Lambda = 1), scaled by Eq. 5's Lambda."""
    return Lam * K_e * C_ele * np.exp(-2.0 * alpha0 * np.asarray(S_e, dtype=np.float64))


# --------------------------------------------------------------------- fits

def fit_drag(velocity, f_drag):
    """Least-squares slope c of f_drag = c V through the origin (the linear drag of the
    droplet-dissipation regime). Returns (c, relative RMS residual)."""
    V = np.asarray(velocity, dtype=np.float64).ravel()
    F = np.asarray(f_drag, dtype=np.float64).ravel()
    if V.size != F.size or V.size < 2 or not np.any(V != 0):
        raise ValueError("need at least two samples with nonzero velocity")
    c = float(V @ F / (V @ V))
    resid = float(np.sqrt(np.mean((F - c * V) ** 2)) / max(np.sqrt(np.mean(F ** 2)), 1e-300))
    return c, resid


def fit_force_law(S_e, f_ele):
    """Fit f_ele = B exp(-2 alpha0 S_e) (Eqs. 3 and 5) by linear least squares on ln f_ele.
    Returns (B, alpha0, relative RMS residual of the fitted force)."""
    S = np.asarray(S_e, dtype=np.float64).ravel()
    F = np.asarray(f_ele, dtype=np.float64).ravel()
    if S.size != F.size or S.size < 2 or np.any(F <= 0):
        raise ValueError("need at least two samples of a positive force")
    X = np.stack([np.ones_like(S), S], axis=1)
    (lnB, slope), *_ = np.linalg.lstsq(X, np.log(F), rcond=None)
    B, a0 = float(np.exp(lnB)), float(-slope / 2.0)
    fit = B * np.exp(-2.0 * a0 * S)
    resid = float(np.sqrt(np.mean((F - fit) ** 2)) / np.sqrt(np.mean(F ** 2)))
    return B, a0, resid


# --------------------------------------------------------------------- Eq. 5

@dataclass
class ReducedModel:
    """Eq. 5 with lumped coefficients: m S'' = -c S' + A exp(-2 alpha0 (S0 - S)).

    m: droplet mass (unit density: its volume); c = C_drag 2 R0 mu_bar; A = Lambda K_e C_ele,
    the electric force at the electrode (S_e = 0); alpha0: decay rate; S0: initial
    droplet-electrode distance. S is measured from the start towards the electrode."""
    m: float
    c: float
    A: float
    alpha0: float
    S0: float

    @classmethod
    def from_paper(cls, m, C_drag, R0, mu_bar, Lam, K_e, C_ele, alpha0, S0):
        """The coefficients as Eq. 5 writes them."""
        return cls(m=m, c=C_drag * 2.0 * R0 * mu_bar, A=Lam * K_e * C_ele, alpha0=alpha0, S0=S0)

    def force(self, S):
        return self.A * np.exp(-2.0 * self.alpha0 * (self.S0 - np.asarray(S, dtype=np.float64)))

    def _accel(self, S, V):
        return (-self.c * V + self.A * math.exp(-2.0 * self.alpha0 * (self.S0 - S))) / self.m

    def _rk4(self, S, V, h):
        """One classical fourth-order Runge-Kutta step of (S, V)."""
        k1s, k1v = V, self._accel(S, V)
        k2s, k2v = V + 0.5 * h * k1v, self._accel(S + 0.5 * h * k1s, V + 0.5 * h * k1v)
        k3s, k3v = V + 0.5 * h * k2v, self._accel(S + 0.5 * h * k2s, V + 0.5 * h * k2v)
        k4s, k4v = V + h * k3v, self._accel(S + h * k3s, V + h * k3v)
        return (S + h / 6.0 * (k1s + 2.0 * k2s + 2.0 * k3s + k4s),
                V + h / 6.0 * (k1v + 2.0 * k2v + 2.0 * k3v + k4v))

    def trajectory(self, times, S_init=0.0, V_init=0.0, substeps=64):
        """S(t) and V(t) at the increasing `times` (from t = 0, S(0) = S_init,
        V(0) = V_init; the paper's start is 0, 0), by fourth-order Runge-Kutta with
        `substeps` steps per output interval."""
        t = np.asarray(times, dtype=np.float64)
        if t.ndim != 1 or np.any(np.diff(t) < 0) or (t.size and t[0] < 0):
            raise ValueError("times must be increasing and non-negative")
        S, V, tc = float(S_init), float(V_init), 0.0
        outS, outV = np.empty_like(t), np.empty_like(t)
        for k, tk in enumerate(t):
            h = (float(tk) - tc) / substeps
            for _ in range(substeps if tk > tc else 0):
                S, V = self._rk4(S, V, h)
            tc = float(tk)
            outS[k], outV[k] = S, V
        return outS, outV

    def time_to_reach(self, S_target, S_init=0.0, V_init=0.0, dt=None, t_max=None):
        """First time S reaches S_target under Eq. 5 (fourth-order Runge-Kutta, linear
        interpolation inside the crossing step). Returns (t, V at that time). The step is at
        most a quarter of the viscous time m / c (the explicit scheme's stability)."""
        tau = self.m / self.c
        dt = min(dt or tau / 20.0, tau / 4.0)
        t_max = t_max or 1e3 * max(self.transport_time(S_target - S_init), tau)
        S, V, t = float(S_init), float(V_init), 0.0
        while t < t_max:
            Sn, Vn = self._rk4(S, V, dt)
            if Sn >= S_target:
                f = (S_target - S) / (Sn - S)
                return t + f * dt, V + f * (Vn - V)
            S, V, t = Sn, Vn, t + dt
        raise RuntimeError("the droplet does not reach the target within t_max")

    def transport_time(self, S_t):
        """Eq. 7: t = c / (2 alpha0 A) (e^{2 alpha0 S0} - e^{2 alpha0 (S0 - S_t)})
        + 2 alpha0 m S_t / c, written with the lumped coefficients (c = C_drag 2 R0 mu_bar,
        A = Lambda K_e C_ele): the overdamped transit time (the first term, exact for m -> 0)
        plus the inertial correction of Eq. 6."""
        a0 = self.alpha0
        return (self.c / (2.0 * a0 * self.A) *
                (math.exp(2.0 * a0 * self.S0) - math.exp(2.0 * a0 * (self.S0 - S_t))) +
                2.0 * a0 * self.m * S_t / self.c)


def switching_schedule(model, electrode_positions, x_start, switch_distance, t_max=None):
    """Switching times of a sequential-electrode protocol (Results, long-distance transport):
    electrode k is live until the droplet comes within `switch_distance` of it, then
    electrode k + 1 is switched on. The droplet's state (position, velocity) carries over at
    each switch; each stage runs Eq. 5 with S0 the distance to the live electrode at the
    stage's start. Returns the switching times (one per electrode but the last) and the
    droplet positions at them."""
    x, V, t = float(x_start), 0.0, 0.0
    times, where = [], []
    for xe in electrode_positions[:-1]:
        S0 = xe - x
        if S0 <= switch_distance:
            raise ValueError("the droplet already sits within the switching distance")
        stage = ReducedModel(model.m, model.c, model.A, model.alpha0, S0)
        dt, V = stage.time_to_reach(S0 - switch_distance, V_init=V, t_max=t_max)
        t += dt
        x = xe - switch_distance
        times.append(t)
        where.append(x)
    return np.array(times), np.array(where)

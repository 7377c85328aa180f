"""Seeded synthetic inputs for the coupled LB-EHD step.

This module only builds inputs: geometry (solid flags, electrode ids), the initial
phase indicators and the lattice-unit parameters. It holds none of the method's
arithmetic, and both the CUDA path and the FP64 oracle consume what it returns.

Geometry conventions (lattice units, site index i = x + nx (y + ny z)):

* the vertical axis is y in 2D (nz = 1) and z in 3D;
* vertical index 0 is the substrate floor (solid class 1), the last vertical index is a
  grounded top wall (solid class 2, neutral wetting, phi = 0);
* micropillars are solid class 1 standing on the floor;
* electrode patches are floor and pillar nodes inside an x (and y) range, with
  electrode id k >= 0; every other solid node is zero-flux for the potential.

Initial state (the droplet resting on the lubricant film, as in the paper's Fig. 1 and
problem statement): Phi_1 (droplet) = (1 - tanh(2 (r - R) / W)) / 2, Phi_2 (lubricant)
fills from the floor to the pillar tops outside the droplet with the same tanh profile,
Phi_3 (ambient) = 1 - Phi_1 - Phi_2. The seed jitters the droplet interface by uniform
noise of amplitude 1e-6.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Fluid property ratios shared by every workload (droplet, lubricant, ambient).
SURFACE_TENSION = {"gamma12": 6e-4, "gamma13": 1e-3, "gamma23": 8e-4}
PERMITTIVITY = (10.0, 2.0, 1.0)
CONDUCTIVITY = (1e-2, 1e-4, 1e-6)
NU_DROPLET = 0.1
NU_AMBIENT = 0.01
MOBILITY = 0.0025
WIDTH = 5.0
THETA23 = 45.0


@dataclass
class Workload:
    """Everything one run needs. Arrays have shape (nz, ny, nx) (Phi: (3, nz, ny, nx))."""
    name: str
    dim: int
    shape: tuple
    solid: np.ndarray
    elec: np.ndarray
    phi_init: np.ndarray
    params: dict
    steps: int = 0
    schedule: list = field(default_factory=list)   # [(step, [V_0, V_1, ...]), ...]

    @property
    def sites(self):
        return int(np.prod(self.shape))


def theta13_from_young(theta12, theta23=THETA23, g=SURFACE_TENSION):
    """Droplet/ambient angle consistent with gamma13 cos t13 = gamma12 cos t12 + gamma23 cos t23."""
    c = (g["gamma12"] * math.cos(math.radians(theta12)) +
         g["gamma23"] * math.cos(math.radians(theta23))) / g["gamma13"]
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def make_params(*, visc_ratio=1.0, theta12=120.0, V=(0.05,), R=16.0, height=64, alpha=None,
                body=(0.0, 0.0, 0.0), poisson_tol=1e-7, poisson_max_iter=100):
    """Lattice-unit parameters. alpha follows alpha* = alpha mu_w / (eps_w R0^2 E0^2) = 1e-4
    with E0 = phi0 / (fluid height)."""
    nu = (NU_DROPLET, NU_DROPLET * visc_ratio, NU_AMBIENT)
    if alpha is None:
        E0 = max(abs(v) for v in V) / max(height - 2, 1) if len(V) else 0.0
        alpha = 1e-4 * PERMITTIVITY[0] * R * R * E0 * E0 / (1.0 * NU_DROPLET)
    return {
        "nu": nu, "eps": PERMITTIVITY, "sig": CONDUCTIVITY, **SURFACE_TENSION,
        "theta12": theta12, "theta23": THETA23, "theta13": theta13_from_young(theta12),
        "mobility": MOBILITY, "W": WIDTH, "alpha": alpha, "body": tuple(body), "s_bulk": 1.0,
        "V": list(V), "poisson_tol": poisson_tol, "poisson_max_iter": poisson_max_iter,
    }


# Table 1 (Results): densities 998 (water, the droplet), 970 (silicone oil, the
# lubricant) and 1.2 kg/m^3 (air); dynamic viscosities 1, 0.5-5 and 0.0179 cP. In lattice
# units the water density is 1 and its kinematic viscosity NU_DROPLET.
RHO_TABLE1 = (1.0, 970.0 / 998.0, 1.2 / 998.0)


def table1_viscosities(visc_ratio=1.0):
    """Kinematic viscosities of Table 1 (nu_i = mu_i / rho_i) scaled to nu_water =
    NU_DROPLET; visc_ratio = mu_oil / mu_water."""
    return (NU_DROPLET, NU_DROPLET * visc_ratio * 998.0 / 970.0,
            NU_DROPLET * 0.0179 * 998.0 / 1.2)


def with_table1_densities(w, visc_ratio=1.0):
    """The same workload with Table 1's densities and viscosities (the variable-density
    momentum scheme, density_model 1)."""
    params = dict(w.params, density_model=1, rho_phase=RHO_TABLE1,
                  nu=table1_viscosities(visc_ratio))
    return Workload(w.name + "_table1_densities", w.dim, w.shape, w.solid, w.elec, w.phi_init,
                    params, steps=w.steps, schedule=list(w.schedule))


def _coords(shape):
    nz, ny, nx = shape
    return np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")


def _tanh_profile(d, W=WIDTH):
    """(1 - tanh(2 d / W)) / 2: 1 inside (d < 0), 0 outside."""
    return 0.5 * (1.0 - np.tanh(2.0 * d / W))


def pillar_geometry(dim, shape, *, pillar_w, pillar_gap, pillar_h, x_range=None,
                    electrodes=(), top_ground=True):
    """Solid flags and electrode ids for a floor with micropillars and a top wall.

    electrodes: list of (x0, x1, y0, y1) ranges (y ignored in 2D); nodes of the floor
    and of pillars inside a range get that electrode's index.
    """
    nz, ny, nx = shape
    zz, yy, xx = _coords(shape)
    vert = yy if dim == 2 else zz
    nv = ny if dim == 2 else nz
    solid = np.zeros(shape, dtype=np.uint8)
    elec = np.full(shape, -1, dtype=np.int16)
    solid[vert == 0] = 1
    pitch = pillar_w + pillar_gap
    in_x = (xx % pitch) < pillar_w
    if x_range is not None:
        in_x &= (xx >= x_range[0]) & (xx < x_range[1])
    in_p = in_x if dim == 2 else in_x & ((yy % pitch) < pillar_w)
    solid[in_p & (vert >= 1) & (vert <= pillar_h)] = 1
    if top_ground:
        solid[vert == nv - 1] = 2
        elec[vert == nv - 1] = -2
    for k, (x0, x1, y0, y1) in enumerate(electrodes):
        m = (xx >= x0) & (xx < x1) & (solid == 1)
        if dim == 3:
            m &= (yy >= y0) & (yy < y1)
        elec[m] = k
    return solid, elec


def droplet_on_film(dim, shape, solid, *, center, R, film_top, seed, W=WIDTH):
    """Initial (Phi_1, Phi_2, Phi_3): droplet of radius R at `center` (x, y[, z]) over a
    lubricant film whose surface sits at vertical coordinate film_top."""
    zz, yy, xx = _coords(shape)
    if dim == 2:
        r = np.sqrt((xx - center[0]) ** 2 + (yy - center[1]) ** 2)
        vert = yy
    else:
        r = np.sqrt((xx - center[0]) ** 2 + (yy - center[1]) ** 2 + (zz - center[2]) ** 2)
        vert = zz
    p1 = _tanh_profile(r - R, W)
    film = _tanh_profile(vert - film_top, W)
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1e-6, 1e-6, size=shape) * 4.0 * p1 * (1.0 - p1)
    p1 = p1 + noise
    p2 = (1.0 - p1) * film
    p3 = 1.0 - p1 - p2
    phi = np.stack([p1, p2, p3])
    phi[:, solid != 0] = 0.0
    return phi


# --------------------------------------------------------------------- named workloads

def droplet_2d_128x64(seed=0):
    """2D D2Q9: 128x64, row of 8 pillars (width 4, gap 4, height 6) infused to the pillar
    tops, droplet R = 16 at x = 40, bottom electrode x in [70, 90) at 0.05, top grounded.
    2000 steps."""
    shape = (1, 64, 128)
    solid, elec = pillar_geometry(2, shape, pillar_w=4, pillar_gap=4, pillar_h=6,
                                  x_range=(24, 88), electrodes=[(70, 90, 0, 0)])
    film = 6.5
    phi = droplet_on_film(2, shape, solid, center=(40.0, film + 16 - 2), R=16.0,
                          film_top=film, seed=seed)
    params = make_params(V=(0.05,), R=16.0, height=64)
    return Workload("droplet_2d_128x64", 2, shape, solid, elec, phi, params, steps=2000,
                    schedule=[(0, [0.05])])


def droplet_3d(nx=128, ny=64, nz=64, *, R=20.0, xc=None, pillar_h=8, electrodes=None,
               visc_ratio=1.0, theta12=120.0, V=None, seed=1, name=None, steps=10000):
    """3D D3Q19 square micropillar array (4x4 lu pillars, pitch 8, height pillar_h) with a
    lubricant film at the pillar tops and a droplet of radius R resting on it."""
    shape = (nz, ny, nx)
    if electrodes is None:
        electrodes = [(int(round(0.625 * nx)), int(round(0.78125 * nx)),
                       int(round(0.34375 * ny)), int(round(0.65625 * ny)))]
    if V is None:
        V = [0.05] * len(electrodes)
    solid, elec = pillar_geometry(3, shape, pillar_w=4, pillar_gap=4, pillar_h=pillar_h,
                                  electrodes=electrodes)
    film = pillar_h + 0.5
    if xc is None:
        xc = 0.3 * nx
    phi = droplet_on_film(3, shape, solid, center=(xc, ny / 2.0, film + R - 2), R=R,
                          film_top=film, seed=seed)
    params = make_params(visc_ratio=visc_ratio, theta12=theta12, V=V, R=R, height=nz)
    return Workload(name or f"droplet_3d_{nx}x{ny}x{nz}", 3, shape, solid, elec, phi, params,
                    steps=steps, schedule=[(0, list(V))])


def droplet_3d_128x64x64(seed=1):
    """3D D3Q19: 128x64x64, 4x4 pillars pitch 8 height 8 with film, droplet R = 20 at
    x = 0.3 Lx, one electrode patch x in [80, 100), y in [22, 42) at 0.05."""
    return droplet_3d(128, 64, 64, R=20.0, electrodes=[(80, 100, 22, 42)], seed=seed,
                      name="droplet_3d_128x64x64", steps=10000)


def transport_3d_384x128x96(seed=2, visc_ratio=1.0, theta12=120.0):
    """3D long transport: 384x128x96, pillar pitch 8, droplet R = 28, 12 bottom electrodes
    (width 16, pitch 24 from x = 64) switched in sequence every 2000 steps at 0.05."""
    electrodes = [(64 + 24 * k, 80 + 24 * k, 0, 128) for k in range(12)]
    V0 = [0.05] + [0.0] * 11
    w = droplet_3d(384, 128, 96, R=28.0, xc=40.0, electrodes=electrodes, V=V0,
                   visc_ratio=visc_ratio, theta12=theta12, seed=seed,
                   name="transport_3d_384x128x96", steps=50000)
    w.schedule = [(2000 * k, [0.05 if j == k else 0.0 for j in range(12)]) for k in range(12)]
    return w


def batched_sweep(n=64, seed=0):
    """64 uneven 3D instances, sizes between 48x48x48 and 128x64x64, lubricant viscosity
    ratio log-uniform in [0.1, 10], contact angle uniform in [60, 150] degrees, electrode
    potential uniform in [0.01, 0.08], droplet radius 10-20 lu."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(6, 17)) * 8
        ny = int(rng.integers(6, 9)) * 8
        nz = int(rng.integers(48, 65))
        R = float(rng.uniform(10.0, 20.0))
        R = min(R, (nz - 12) / 2.0 - 2.0, ny / 2.0 - 3.0)
        ratio = float(10.0 ** rng.uniform(-1.0, 1.0))
        theta = float(rng.uniform(60.0, 150.0))
        V = float(rng.uniform(0.01, 0.08))
        ex0 = int(0.625 * nx)
        ex1 = int(0.78125 * nx)
        w = droplet_3d(nx, ny, nz, R=R, xc=0.3 * nx, electrodes=[(ex0, ex1, ny // 3, 2 * ny // 3)],
                       visc_ratio=ratio, theta12=theta, V=[V], seed=1000 + k,
                       name=f"batch{k}_{nx}x{ny}x{nz}", steps=5000)
        out.append(w)
    return out


def control_3d_96x64x64(seed=4):
    """Differentiable-control case: 96x64x64, 16 bottom electrodes (width 6 lu, pitch 6
    from x = 0) each driven by 20 piecewise-constant segments seeded uniform in
    [0, 0.06]; 4000 steps."""
    electrodes = [(6 * k, 6 * k + 6, 16, 48) for k in range(16)]
    rng = np.random.default_rng(seed)
    sched = rng.uniform(0.0, 0.06, size=(20, 16))
    w = droplet_3d(96, 64, 64, R=14.0, xc=30.0, electrodes=electrodes, V=list(sched[0]),
                   seed=seed, name="control_3d_96x64x64", steps=4000)
    w.schedule = [(200 * s, list(sched[s])) for s in range(20)]
    return w


def control_3d_24x16x16(seed=4, segments=4, seg_steps=5):
    """A 24x16x16 copy of the differentiable-control case, small enough for the FP64
    discrete-adjoint reference: 4 bottom electrodes (width 6 lu, pitch 6 from x = 0,
    y in [4, 12)), pillars of height 3, droplet R = 4 at x = 8, `segments` piecewise-constant
    segments of `seg_steps` steps seeded uniform in [0, 0.06]."""
    electrodes = [(6 * k, 6 * k + 6, 4, 12) for k in range(4)]
    rng = np.random.default_rng(seed)
    sched = rng.uniform(0.0, 0.06, size=(segments, 4))
    w = droplet_3d(24, 16, 16, R=4.0, xc=8.0, pillar_h=3, electrodes=electrodes,
                   V=list(sched[0]), seed=seed, name="control_3d_24x16x16",
                   steps=segments * seg_steps)
    w.schedule = [(seg_steps * s, list(sched[s])) for s in range(segments)]
    return w


def small_3d(nx=24, ny=16, nz=16, seed=3, R=5.0, V=0.05):
    """Small 3D case for full-field parity: a few pillars, a droplet and one electrode."""
    return droplet_3d(nx, ny, nz, R=R, xc=0.35 * nx, pillar_h=3,
                      electrodes=[(int(0.6 * nx), int(0.85 * nx), ny // 4, 3 * ny // 4)],
                      V=[V], seed=seed, name=f"small_3d_{nx}x{ny}x{nz}", steps=100)


def small_2d(nx=48, ny=32, seed=5, R=8.0, V=0.05):
    """Small 2D case: pillar row, droplet, one electrode."""
    shape = (1, ny, nx)
    solid, elec = pillar_geometry(2, shape, pillar_w=4, pillar_gap=4, pillar_h=4,
                                  electrodes=[(int(0.6 * nx), int(0.8 * nx), 0, 0)])
    film = 4.5
    phi = droplet_on_film(2, shape, solid, center=(0.35 * nx, film + R - 2), R=R,
                          film_top=film, seed=seed)
    params = make_params(V=(V,), R=R, height=ny)
    return Workload(f"small_2d_{nx}x{ny}", 2, shape, solid, elec, phi, params, steps=100,
                    schedule=[(0, [V])])


def electrode_above(dim=2, nx=256, ny=24, nz=1, *, l_e=8, x_e=240, w_e=8, V=0.05, wall=True,
                    droplet=None, pillar_h=0, seed=6, name=None):
    """The electrode geometry of the paper's Fig. 1: an electrode block held at V above a
    grounded substrate, every other wall zero-flux (Results, the problem set-up: the pillar
    surface at zero potential, the electrode at phi0, Neumann elsewhere).

    Vertical axis v (y in 2D, z in 3D) with nv nodes: the substrate floor v = 0 (and any
    micropillars of height pillar_h, width 4, gap 4) is grounded (solid class 1, id -2); the
    top wall v = nv - 1 is zero-flux (class 2, id -1); the electrode (class 2, id 0) hangs
    from the top wall, l_e nodes high (v in [nv - 1 - l_e, nv - 1)), at x in [x_e, x_e + w_e),
    across all of y. With `wall` a zero-flux column at x = 0 ends the x-periodicity. The
    potential lives in the strip between the ground nodes (v = 0) and the zero-flux face of
    the top wall (v = nv - 1.5): height H = nv - 1.5 = h_e + l_e, the electrode-surface
    distance h_e = H - l_e. `droplet` = (xc, R) puts a droplet resting on the floor (or the
    pillar tops); without it the box holds the ambient phase alone."""
    shape = (nz, ny, nx)
    zz, yy, xx = _coords(shape)
    vert = yy if dim == 2 else zz
    nv = ny if dim == 2 else nz
    solid = np.zeros(shape, dtype=np.uint8)
    elec = np.full(shape, -1, dtype=np.int16)
    solid[vert == 0] = 1
    elec[vert == 0] = -2
    if pillar_h > 0:
        in_p = (xx % 8) < 4
        if dim == 3:
            in_p &= (yy % 8) < 4
        m = in_p & (vert >= 1) & (vert <= pillar_h) & (xx >= 8) & (xx < x_e - 8)
        solid[m] = 1
        elec[m] = -2
    solid[vert == nv - 1] = 2
    m = (xx >= x_e) & (xx < x_e + w_e) & (vert >= nv - 1 - l_e) & (vert < nv - 1)
    solid[m] = 2
    elec[m] = 0
    if wall:
        solid[xx == 0] = 2
        elec[(xx == 0) & (vert > 0)] = -1
    if droplet is not None:
        xc, R = droplet
        base = pillar_h + 0.5 if pillar_h > 0 else 0.5
        center = (xc, base + R - 2) if dim == 2 else (xc, ny / 2.0, base + R - 2)
        phi = droplet_on_film(dim, shape, solid, center=center, R=R, film_top=base, seed=seed)
    else:
        phi = np.zeros((3,) + shape)
        phi[2] = 1.0
        phi[:, solid != 0] = 0.0
    params = make_params(V=(V,), R=droplet[1] if droplet else 8.0, height=nv)
    return Workload(name or f"electrode_above_{dim}d_{nx}x{ny}x{nz}", dim, shape, solid, elec,
                    phi, params, steps=1, schedule=[(0, [V])])


def droplet_3d_128x64x64_table1_densities(seed=1):
    """The 128x64x64 droplet workload with Table 1's densities (water : oil : air =
    998 : 970 : 1.2) and viscosities, run by the variable-density momentum scheme."""
    return with_table1_densities(droplet_3d_128x64x64(seed))


WORKLOADS = {
    "droplet_2d_128x64": droplet_2d_128x64,
    "droplet_3d_128x64x64": droplet_3d_128x64x64,
    "droplet_3d_128x64x64_table1_densities": droplet_3d_128x64x64_table1_densities,
    "transport_3d_384x128x96": transport_3d_384x128x96,
    "control_3d_96x64x64": control_3d_96x64x64,
}

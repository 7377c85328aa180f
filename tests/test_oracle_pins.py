"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets one part of the oracle so that a plausible mistake there (a dropped
term, a wrong sign, a missing c_s^2, a transposed index) fails it:

* lattice weights / moment matrices  -> isotropy identities, M M^-1 = I
* AC source scale and sharpening (Eqs. 8, 17, 18) -> flat-interface tanh width W
* chemical potential / Upsilons (Eqs. 10-11) -> Young-Laplace per phase pair, 2D and 3D
* wetting ghosts (Eq. 20a) -> equilibrium contact angle, sum rule of the three RHS
* momentum MRT + forcing -> plane Poiseuille (second-order), momentum budget
* Gauss law (Eq. 13) -> layered capacitor closed form, dense-LU brute force,
  superposition
* electric force (Eq. 12) -> F_e(lambda V) = lambda^2 F_e(V) at zero charge
* charge transport (Eq. 14) -> exp(-sigma t / eps) relaxation, exact charge conservation
* streaming / bounce-back -> exact per-component mass conservation, translation and
  mirror invariance
"""
import numpy as np
import pytest

from paper_2608_12868_b300 import workloads as W


def _grid(shape):
    return np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")


def _sim(O, dim, shape, solid, elec, phi, params):
    return O.OracleSim(dim, shape, solid, elec, phi, params)


def _periodic(shape):
    return np.zeros(shape, np.uint8), np.full(shape, -1, np.int16)


# --------------------------------------------------------------------- lattices

@pytest.mark.parametrize("name", ["D2Q9", "D3Q19", "D2Q5", "D3Q7"])
def test_lattice_isotropy_and_moment_matrix(oracle_mod, name):
    L = oracle_mod.LATTICES[name]
    e, w, cs2 = L.e.astype(float), L.w, L.cs2
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("n,na->a", w, e)).max() < 1e-15
    dims = 2 if name.startswith("D2") else 3
    second = np.einsum("n,na,nb->ab", w, e, e)[:dims, :dims]
    assert np.allclose(second, cs2 * np.eye(dims), atol=1e-15)
    if name in ("D2Q9", "D3Q19"):
        fourth = np.einsum("n,na,nb,nc,nd->abcd", w, e, e, e, e)[:dims, :dims, :dims, :dims]
        d = np.eye(dims)
        iso = cs2 * cs2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) +
                           np.einsum("ad,bc->abcd", d, d))
        assert np.allclose(fourth, iso, atol=1e-15)
    assert np.allclose(L.M @ L.Minv, np.eye(L.Q), atol=1e-13)
    assert all(L.e[L.opp[n]].tolist() == (-L.e[n]).tolist() for n in range(L.Q))
    # the printed D3Q19 weights: omega(0) = 1/3, omega(1) = 1/18, omega(2) = 1/36
    if name == "D3Q19":
        sq = (L.e ** 2).sum(1)
        assert np.allclose(w[sq == 0], 1 / 3) and np.allclose(w[sq == 1], 1 / 18)
        assert np.allclose(w[sq == 2], 1 / 36)


# --------------------------------------------------------------------- phase field

def test_flat_interface_relaxes_to_tanh_of_width_W(oracle_mod):
    """Conservative AC equilibrium (Eq. 8): Phi = (1 + tanh(2x/W))/2 with W = 5. A factor
    c_s^2 missing in the source (Eq. 17) would give width W/3 or 3W."""
    ny, nx = 64, 2
    shape = (1, ny, nx)
    _, yy, _ = _grid(shape)
    band = lambda Wd, a, b: 0.5 * (np.tanh(2 * (yy - a) / Wd) - np.tanh(2 * (yy - b) / Wd))
    p1 = band(9.0, 20.3, 44.3)
    s = _sim(oracle_mod, 2, shape, *_periodic(shape), np.stack([p1, 0 * p1, 1 - p1]),
             W.make_params(V=()))
    s.step(15000)
    prof = s.Phi[0][0, :, 0]
    best = None
    for Wd in np.arange(4.0, 6.01, 0.02):
        for a in np.arange(19.5, 21.0, 0.02):
            b = a + 24.0
            err = np.abs(prof - band(Wd, a, b)[0, :, 0]).max()
            if best is None or err < best[0]:
                best = (err, Wd, a)
    err, Wfit, _ = best
    assert abs(Wfit - 5.0) < 0.25, best
    assert err < 0.01, best


@pytest.mark.parametrize("inner,outer", [(0, 2), (0, 1), (1, 2)])
def test_young_laplace_2d_each_pair(oracle_mod, inner, outer):
    """Delta p = gamma_ij / R in 2D for a binary drop of phase i in phase j (Eqs. 10-11)."""
    n, R = 48, 12.0
    shape = (1, n, n)
    _, yy, xx = _grid(shape)
    c = (n - 1) / 2
    pd = 0.5 * (1 - np.tanh(2 * (np.sqrt((xx - c) ** 2 + (yy - c) ** 2) - R) / 5))
    phi = np.zeros((3,) + shape)
    phi[inner], phi[outer] = pd, 1 - pd
    p = W.make_params(V=())
    s = _sim(oracle_mod, 2, shape, *_periodic(shape), phi, p)
    s.step(3000)
    Rm = np.sqrt(s.Phi[inner][0].sum() / np.pi)
    cs2 = 1 / 3
    dp = cs2 * (s.pstar[0][int(c), int(c)] - s.pstar[0][0, 0])
    gamma = {(0, 2): p["gamma13"], (0, 1): p["gamma12"], (1, 2): p["gamma23"]}[(inner, outer)]
    assert abs(dp / (gamma / Rm) - 1) < 0.05


@pytest.mark.slow
def test_young_laplace_3d(oracle_mod):
    """Delta p = 2 gamma_13 / R in 3D (D3Q19)."""
    n, R = 28, 9.0
    shape = (n, n, n)
    zz, yy, xx = _grid(shape)
    c = (n - 1) / 2
    r = np.sqrt((xx - c) ** 2 + (yy - c) ** 2 + (zz - c) ** 2)
    pd = 0.5 * (1 - np.tanh(2 * (r - R) / 5))
    p = W.make_params(V=())
    s = _sim(oracle_mod, 3, shape, *_periodic(shape), np.stack([pd, 0 * pd, 1 - pd]), p)
    s.step(1000)
    Rm = (3 * s.Phi[0].sum() / (4 * np.pi)) ** (1 / 3)
    dp = (s.pstar[r < Rm - 4].mean() - s.pstar[r > Rm + 5].mean()) / 3
    assert abs(dp / (2 * p["gamma13"] / Rm) - 1) < 0.06


def _cap(theta, nx, R, yy, xx):
    """Binary circular cap of contact angle theta on a wall at y = 0.5 (2D)."""
    t = np.radians(theta)
    yc = 0.5 - R * np.cos(t)
    d = np.sqrt((xx - nx / 2) ** 2 + (yy - yc) ** 2) - R
    return 0.5 * (1 - np.tanh(2 * d / 5))


def _measure_angle(P, c):
    col = P[:, int(c)]
    j = np.where((col[:-1] >= 0.5) & (col[1:] < 0.5))[0][-1]
    h = j + (col[j] - 0.5) / (col[j] - col[j + 1]) - 0.5
    row = P[1]
    idx = np.where(row >= 0.5)[0]
    a, b = idx[0], idx[-1]
    xl = a - (row[a] - 0.5) / (row[a] - row[a - 1])
    xr = b + (row[b] - 0.5) / (row[b] - row[b + 1])
    half = (xr - xl) / 2
    yc = (h * h - 0.25 - half * half) / (2 * (h - 0.5))
    return np.degrees(np.arccos(-yc / (h - yc)))


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_contact_angle(oracle_mod, theta):
    """Eq. 20a: a binary drop of phase 1 in phase 3 on a flat substrate keeps the prescribed
    theta_13 (measured through phase 1); with the sign of the wetting term flipped it drifts
    towards 180 - theta by more than 15 degrees over the same run."""
    nx, ny, R = 64, 32, 10.0
    shape = (1, ny, nx)
    _, yy, xx = _grid(shape)
    solid = np.zeros(shape, np.uint8)
    solid[yy == 0] = 1
    solid[yy == ny - 1] = 2
    elec = np.full(shape, -1, np.int16)
    pd = _cap(theta, nx, R, yy, xx)
    phi = np.stack([pd, 0 * pd, 1 - pd])
    phi[:, solid != 0] = 0
    p = W.make_params(V=())
    p.update(theta13=theta, theta12=90.0, theta23=90.0)
    s = _sim(oracle_mod, 2, shape, solid, elec, phi, p)
    s.step(10000)
    assert abs(_measure_angle(s.Phi[0][0], nx / 2) - theta) < 3.0


def test_wetting_ghosts_keep_sum_one(oracle_mod):
    """The three right-hand sides of Eq. 20a sum to zero, so ghost values on boundary solid
    nodes sum to the fluid sum (1) whatever the angles."""
    w = W.small_2d()
    p = dict(w.params)
    p.update(theta12=130.0, theta13=70.0, theta23=40.0)
    s = _sim(oracle_mod, 2, w.shape, w.solid, w.elec, w.phi_init, p)
    s.step(3)
    bnd = np.argwhere(s.normal > 0)
    assert len(bnd) > 10
    total = s.Phi.sum(0)
    nz, ny, nx = s.shape
    for z, y, x in bnd:
        e = s.Lf.e[s.normal[z, y, x]]
        f = ((z + e[2]) % nz, (y + e[1]) % ny, (x + e[0]) % nx)
        assert s.solid[f] == 0
        assert abs(total[z, y, x] - total[f]) < 1e-13
    bnd = s.normal > 0
    # a ghost differs from its fluid neighbour where two phases meet the wall
    assert np.abs(s.Phi[0][bnd]).max() > 0


# --------------------------------------------------------------------- momentum

@pytest.mark.slow
def test_plane_poiseuille_second_order(oracle_mod):
    """Body-force-driven channel between halfway bounce-back walls: u(y) = g/(2 nu)
    (y - y0)(y1 - y), error falling ~4x when the resolution doubles."""
    errs = []
    for ny in (18, 34):
        shape = (1, ny, 2)
        _, yy, _ = _grid(shape)
        solid = np.zeros(shape, np.uint8)
        solid[(yy == 0) | (yy == ny - 1)] = 2
        elec = np.full(shape, -1, np.int16)
        one = np.ones(shape)
        phi = np.stack([one, 0 * one, 0 * one])
        phi[:, solid != 0] = 0
        gx = 1e-6
        s = _sim(oracle_mod, 2, shape, solid, elec, phi, W.make_params(V=(), body=(gx, 0, 0)))
        s.step(int(8 * (ny - 2) ** 2 / 0.1))
        y = np.arange(1, ny - 1)
        ex = gx / (2 * 0.1) * (y - 0.5) * (ny - 1.5 - y)
        num = s.u[0][0, 1:ny - 1, 0]
        errs.append(np.sqrt(((num - ex) ** 2).sum() / (ex ** 2).sum()))
    assert errs[0] < 2e-3 and errs[1] < 5e-4
    assert errs[0] / errs[1] > 3.0


def test_momentum_budget_equals_total_force(oracle_mod):
    """Periodic box: sum_x j(t+1) - sum_x j(t) = sum_x F(t) (the forcing term adds F to the
    momentum moment, streaming moves it)."""
    w = W.small_2d()
    shape = w.shape
    phi = w.phi_init.copy()
    phi[2] = 1 - phi[0] - phi[1]
    s = _sim(oracle_mod, 2, shape, *_periodic(shape), phi,
             dict(w.params, body=(3e-6, -2e-6, 0.0), V=[]))
    s.step(5)
    e = s.Lf.e
    j0 = np.einsum("na,nk->a", e.astype(float), s.g.reshape(s.Lf.Q, -1))
    s.step(1)
    F = s.F.reshape(3, -1).sum(1)
    j1 = np.einsum("na,nk->a", e.astype(float), s.g.reshape(s.Lf.Q, -1))
    assert np.allclose(j1 - j0, F, rtol=1e-9, atol=1e-15)


# --------------------------------------------------------------------- electric

def _column(O, eps_phase, V):
    ny = 20
    shape = (1, ny, 1)
    _, yy, _ = _grid(shape)
    solid = np.zeros(shape, np.uint8)
    solid[yy == 0] = 1
    solid[yy == ny - 1] = 2
    elec = np.full(shape, -1, np.int16)
    elec[yy == 0] = 0
    elec[yy == ny - 1] = -2
    phi = np.stack([eps_phase, 0 * eps_phase, 1 - eps_phase])
    phi[:, solid != 0] = 0
    return O.OracleSim(2, shape, solid, elec, phi, W.make_params(V=(V,))), ny


def test_layered_capacitor_closed_form(oracle_mod):
    """Gauss law (Eq. 13) in a 1D column of random layers: the discrete solution is the
    series-resistor formula phi_k = V (1 - sum_{j<k} 1/eps_j+1/2 / sum_j 1/eps_j+1/2)."""
    rng = np.random.default_rng(0)
    layers = (rng.uniform(size=(1, 20, 1)) > 0.5).astype(float)
    s, ny = _column(oracle_mod, layers, 0.7)
    s.step(1)
    eps = s.eps[0, :, 0]
    faces = [eps[1]] + [0.5 * (eps[j] + eps[j + 1]) for j in range(1, ny - 2)] + [eps[ny - 2]]
    rinv = 1 / np.array(faces)
    exact = np.array([0.7 * (1 - rinv[:k].sum() / rinv.sum()) for k in range(1, ny - 1)])
    assert np.abs(s.pot[0, 1:ny - 1, 0] - exact).max() < 1e-12


def _assemble_dense(s):
    """Dense matrix of div(eps grad .) on fluid nodes, written from the operator's
    definition independently of the oracle's CG code."""
    nz, ny, nx = s.shape
    idx = -np.ones(s.shape, int)
    fl = np.argwhere(s.solid == 0)
    for k, (z, y, x) in enumerate(fl):
        idx[z, y, x] = k
    n = len(fl)
    A = np.zeros((n, n))
    b = np.zeros(n)
    V = s.params["V"]
    for k, (z, y, x) in enumerate(fl):
        b[k] = s.rho[z, y, x]
        for ev in s.Ls.e[1:]:
            zz, yy, xx = (z + ev[2]) % nz, (y + ev[1]) % ny, (x + ev[0]) % nx
            if s.solid[zz, yy, xx] == 0:
                kf = 0.5 * (s.eps[z, y, x] + s.eps[zz, yy, xx])
                A[k, k] += kf
                A[k, idx[zz, yy, xx]] -= kf
            elif s.elec[zz, yy, xx] >= 0 or s.elec[zz, yy, xx] == -2:
                kf = s.eps[z, y, x]
                A[k, k] += kf
                b[k] += kf * (V[s.elec[zz, yy, xx]] if s.elec[zz, yy, xx] >= 0 else 0.0)
    return A, b, fl


def test_poisson_matches_dense_lu_3d(oracle_mod):
    """Brute force on a tiny 3D grid with pillars, two electrodes, random charge."""
    w = W.droplet_3d(12, 8, 10, R=3.0, pillar_h=2, electrodes=[(6, 10, 0, 4), (0, 3, 4, 8)],
                     V=[0.05, -0.02], seed=7, steps=1)
    s = _sim(oracle_mod, 3, w.shape, w.solid, w.elec, w.phi_init, w.params)
    rng = np.random.default_rng(1)
    rho0 = rng.normal(scale=1e-4, size=w.shape) * (w.solid == 0)
    for q in range(s.Ls.Q):
        s.frho[q] = s.Ls.w[q] * rho0
    s.step(1)
    A, b, fl = _assemble_dense(s)
    x = np.linalg.solve(A, b)
    got = np.array([s.pot[z, y, x_] for z, y, x_ in fl])
    assert np.abs(got - x).max() < 1e-11 * np.abs(x).max()


def test_potential_superposition(oracle_mod):
    """With rho_e = 0 and fixed Phi the potential is linear in the electrode voltages."""
    def pot(V):
        w = W.droplet_3d(12, 8, 10, R=3.0, pillar_h=2, electrodes=[(6, 10, 0, 4), (0, 3, 4, 8)],
                         V=V, seed=7, steps=1)
        s = _sim(oracle_mod, 3, w.shape, w.solid, w.elec, w.phi_init, w.params)
        s.step(1)
        return s.pot.copy()
    a, b, ab = pot([0.05, 0.0]), pot([0.0, -0.03]), pot([0.05, -0.03])
    assert np.abs(ab - a - b).max() < 1e-12


def test_electric_force_scales_with_voltage_squared(oracle_mod):
    """Eq. 12 at zero charge: F_e = -|E|^2 grad(eps)/2, so F_e(2V) = 4 F_e(V)."""
    def fe(V):
        w = W.small_3d(V=V)
        s = _sim(oracle_mod, 3, w.shape, w.solid, w.elec, w.phi_init, w.params)
        s.step(1)
        return s.Fe.copy()
    f1, f2 = fe(0.05), fe(0.1)
    assert np.abs(f1).max() > 0
    assert np.abs(f2 - 4 * f1).max() < 1e-9 * np.abs(f2).max()


@pytest.mark.parametrize("sigma,steps,tol", [(1e-2, 300, 2e-3), (0.5, 40, 5e-3)])
def test_charge_relaxation_rate(oracle_mod, sigma, steps, tol):
    """Eq. 14 in a uniform conductor: d rho_e/dt = div(sigma grad phi) = -(sigma/eps) rho_e,
    so the charge inside a disk around a blob decays as exp(-sigma t / eps). At the fast
    rate (sigma/eps = 0.05 per step) the 0.5 dC/dt term of the charge collision matters:
    without it the decay is off by ~5%."""
    n = 40
    shape = (1, n, n)
    _, yy, xx = _grid(shape)
    solid = np.zeros(shape, np.uint8)
    solid[(yy == 0) | (yy == n - 1)] = 2
    elec = np.full(shape, -1, np.int16)
    elec[(yy == 0) | (yy == n - 1)] = -2
    one = np.ones(shape)
    phi = np.stack([one, 0 * one, 0 * one])
    phi[:, solid != 0] = 0
    p = W.make_params(V=(), alpha=1e-6)
    p["sig"] = (sigma,) + tuple(p["sig"][1:])
    s = _sim(oracle_mod, 2, shape, solid, elec, phi, p)
    c = n / 2
    rho0 = 1e-3 * np.exp(-((xx - c) ** 2 + (yy - c) ** 2) / 32.0) * (solid == 0)
    for q in range(s.Ls.Q):
        s.frho[q] = s.Ls.w[q] * rho0
    disk = ((xx - c) ** 2 + (yy - c) ** 2) <= 14 ** 2
    k = p["sig"][0] / p["eps"][0]
    s.step(steps)
    t = s.step_count - 1
    ratio = (s.rho * disk).sum() / (rho0 * disk).sum()
    assert abs(ratio / np.exp(-k * t) - 1) < tol
    assert abs(s.rho.sum() / rho0.sum() - 1) < 1e-12


# --------------------------------------------------------------------- conservation

def test_mass_and_charge_conservation_2d(oracle_mod):
    """Bounce-back + periodic boundaries conserve sum Phi_i for each component and the total
    charge to rounding, with pillars, wetting, flow and a live electrode."""
    w = W.small_2d()
    s = _sim(oracle_mod, 2, w.shape, w.solid, w.elec, w.phi_init, w.params)
    s.step(1)
    m0 = s.observables()["mass"]
    s.step(150)
    m1 = s.observables()["mass"]
    assert np.abs(m1 / m0 - 1).max() < 1e-12
    assert abs(s.observables()["charge"]) < 1e-15
    assert np.abs(s.u).max() > 0


def test_translation_invariance(oracle_mod):
    """Shifting the whole periodic setup by dx shifts the result by dx."""
    w = W.small_2d()
    s1 = _sim(oracle_mod, 2, w.shape, w.solid, w.elec, w.phi_init, w.params)
    sh = lambda a: np.roll(a, 8, axis=-1)
    s2 = _sim(oracle_mod, 2, w.shape, sh(w.solid), sh(w.elec), sh(w.phi_init), w.params)
    s1.step(20)
    s2.step(20)
    assert np.abs(sh(s1.fphi) - s2.fphi).max() < 1e-12
    assert np.abs(sh(s1.g) - s2.g).max() < 1e-12


def test_mirror_symmetry(oracle_mod):
    """A setup symmetric under x -> -x stays symmetric (u_x antisymmetric)."""
    nx, ny = 40, 28
    shape = (1, ny, nx)
    _, yy, xx = _grid(shape)
    solid = np.zeros(shape, np.uint8)
    solid[yy == 0] = 1
    solid[yy == ny - 1] = 2
    xs = xx - (nx - 1) / 2
    solid[(np.abs(xs) % 8 < 2) & (yy >= 1) & (yy <= 4)] = 1
    elec = np.full(shape, -1, np.int16)
    elec[yy == ny - 1] = -2
    elec[(np.abs(xs) > 14) & (solid == 1)] = 0
    phi = W.droplet_on_film(2, shape, solid, center=((nx - 1) / 2, 4.5 + 6), R=8.0,
                            film_top=4.5, seed=None)
    phi = 0.5 * (phi + phi[..., ::-1])
    s = _sim(oracle_mod, 2, shape, solid, elec, phi, W.make_params(V=(0.05,)))
    s.step(60)
    assert np.abs(s.Phi - s.Phi[..., ::-1]).max() < 1e-11
    assert np.abs(s.u[0] + s.u[0][..., ::-1]).max() < 1e-13


def test_dielectrophoretic_force_points_to_the_electrode(oracle_mod):
    """Eq. 12 at zero charge: the high-permittivity droplet is pulled towards the live
    electrode (it migrates in the electrode direction, Results, Fig. 2a)."""
    for w in (W.small_2d(), W.small_3d()):
        s = _sim(oracle_mod, w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
        s.step(1)
        assert s.observables()["f_ele"][0] > 0


def test_coulomb_force_follows_field_and_charge_sign(oracle_mod):
    """rho_e E term of Eq. 12: in a uniform medium between a live bottom plate and a
    grounded top plate, E points up, so a positive charge blob feels an upward force and a
    negative one a downward force."""
    n = 24
    shape = (1, n, n)
    _, yy, xx = _grid(shape)
    solid = np.zeros(shape, np.uint8)
    solid[yy == 0] = 1
    solid[yy == n - 1] = 2
    elec = np.full(shape, -1, np.int16)
    elec[yy == 0] = 0
    elec[yy == n - 1] = -2
    one = np.ones(shape)
    phi = np.stack([0 * one, 0 * one, one])
    phi[:, solid != 0] = 0
    for sign in (1.0, -1.0):
        s = _sim(oracle_mod, 2, shape, solid, elec, phi, W.make_params(V=(0.05,)))
        blob = sign * 1e-5 * np.exp(-((xx - 12) ** 2 + (yy - 12) ** 2) / 8.0) * (solid == 0)
        for q in range(s.Ls.Q):
            s.frho[q] = s.Ls.w[q] * blob
        s.step(1)
        assert s.E[1][solid == 0].min() > 0
        assert sign * s.observables()["f_ele_total"][1] > 0


def test_uniform_accelerated_flow_invariants(oracle_mod):
    """Periodic box, uniform Phi, body force F. Exact discrete facts of the scheme:
    u^n = (n + 1/2) F (the half-force velocity shift), sum p* stays constant (the force term
    carries no mass), and each phase field's first moment equals Phi (u - F/2), which holds
    only with the d(Phi u)/dt term of Eq. 17 and its (I - S/2) factor."""
    shape = (1, 6, 5)
    one = np.ones(shape)
    phi = np.stack([0.3 * one, 0.2 * one, 0.5 * one])
    F = np.array([2e-5, -1e-5, 0.0])
    s = _sim(oracle_mod, 2, shape, *_periodic(shape), phi, W.make_params(V=(), body=tuple(F)))
    p0 = s.g.sum()
    s.step(12)
    n = s.step_count - 1          # fields are those of the last computed step
    for a in range(2):
        assert np.abs(s.u[a] - (n + 0.5) * F[a]).max() < 1e-15
    assert abs(s.g.sum() - p0) < 1e-12
    e = s.Lf.e.astype(float)
    # j^{n+1} = (1 - s) j^n + s Phi u^n + (1 - s/2) Phi (u^n - u^{n-1}); the first step has
    # no time difference, so j^N = Phi N F + (1 - s)^(N-1) (s/2 - 1) Phi F.
    N = s.step_count
    rate = 1.0 / (0.5 + 0.0025 / (1 / 3))
    for c, P in enumerate((0.3, 0.2, 0.5)):
        j = np.einsum("na,n...->a...", e, s.fphi[c])
        for a in range(2):
            exact = P * N * F[a] + (1 - rate) ** (N - 1) * (rate / 2 - 1) * P * F[a]
            assert np.abs(j[a] - exact).max() < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_charge_diffusion_variance(oracle_mod, dim):
    """Eq. 14 with sigma = 0: a charge blob spreads by pure diffusion, its variance along x
    growing as var0 + 2 alpha t, with alpha = c_s^2 (tau_rho - 1/2) on D2Q5 / D3Q7."""
    n = 40 if dim == 2 else 20
    shape = (1, n, n) if dim == 2 else (n, n, 40)
    zz, yy, xx = _grid(shape)
    vert = yy if dim == 2 else zz
    nv = shape[1] if dim == 2 else shape[0]
    solid = np.zeros(shape, np.uint8)
    solid[(vert == 0) | (vert == nv - 1)] = 2
    elec = np.full(shape, -1, np.int16)
    elec[solid != 0] = -2
    one = np.ones(shape)
    phi = np.stack([0 * one, 0 * one, one])
    phi[:, solid != 0] = 0
    p = W.make_params(V=(), alpha=0.05)
    p["sig"] = (0.0, 0.0, 0.0)
    s = _sim(oracle_mod, dim, shape, solid, elec, phi, p)
    cx = shape[-1] / 2
    r2 = (xx - cx) ** 2 + (yy - shape[1] / 2) ** 2 + ((zz - shape[0] / 2) ** 2 if dim == 3 else 0)
    rho0 = 1e-7 * np.exp(-r2 / 18.0) * (solid == 0)
    for q in range(s.Ls.Q):
        s.frho[q] = s.Ls.w[q] * rho0
    var = lambda r: (r * (xx - cx) ** 2).sum() / r.sum()
    v0 = var(rho0)
    s.step(101)
    t = s.step_count - 1
    assert abs((var(s.rho) - v0) / (2 * 0.05 * t) - 1) < 0.02


def _charge_in_uniform_flow(O, dim, U, alpha, steps):
    """A small charge blob (sigma = 0, so no conduction; amplitude 1e-7, so its own field
    exerts a negligible force) in a fully periodic box whose fluid moves uniformly at
    u = (U, 0, 0). A uniform background of opposite charge makes the box neutral, so the
    Gauss-law problem without Dirichlet nodes is consistent; it is translation invariant and
    drops out of the blob's moments. Momentum and charge populations start at their
    equilibria with that velocity. Returns the blob's centroid shift along x and its
    variance growth along x and along y."""
    shape = (1, 40, 96) if dim == 2 else (24, 24, 64)
    zz, yy, xx = _grid(shape)
    solid, elec = _periodic(shape)
    one = np.ones(shape)
    phi = np.stack([0 * one, 0 * one, one])
    p = W.make_params(V=(), alpha=alpha)
    p["sig"] = (0.0, 0.0, 0.0)
    s = _sim(O, dim, shape, solid, elec, phi, p)
    u = np.array([U, 0.0, 0.0])
    ef, cs2 = s.Lf.e.astype(float), s.Lf.cs2
    for n in range(s.Lf.Q):
        eu = ef[n] @ u
        s.g[n] = s.Lf.w[n] * (1 + eu / cs2 + eu * eu / (2 * cs2 * cs2) - u @ u / (2 * cs2))
    x0, yc, zc = 20.0, shape[1] / 2 - 0.5, shape[0] / 2 - 0.5
    r2 = (xx - x0) ** 2 + (yy - yc) ** 2 + ((zz - zc) ** 2 if dim == 3 else 0)
    blob = 1e-7 * np.exp(-r2 / 8.0)
    Q = blob.sum()
    bg = -Q / blob.size
    es, cs2s = s.Ls.e.astype(float), s.Ls.cs2
    for q in range(s.Ls.Q):
        s.frho[q] = s.Ls.w[q] * (blob + bg) * (1 + (es[q] @ u) / cs2s)

    def stats(b):
        c = (b * xx).sum() / Q
        return c, (b * (xx - c) ** 2).sum() / Q, (b * (yy - yc) ** 2).sum() / Q

    c0, vx0, vy0 = stats(blob)
    s.step(steps)
    # frho holds the populations after `steps` collide + stream passes
    b1 = s.frho.sum(0) - bg
    assert abs(b1.sum() / Q - 1) < 1e-9
    c1, vx1, vy1 = stats(b1)
    return c1 - c0, vx1 - vx0, vy1 - vy0


@pytest.mark.parametrize("dim", [2, 3])
def test_charge_advection_in_uniform_flow(oracle_mod, dim):
    """Eq. 14 with u: the rho_e u flux of the charge equation (the e.u / c_s^2 term of the
    charge equilibrium, Eq. 20b's collision) carries a blob at exactly the fluid velocity,
    so its centroid moves by U per step; and with the R = w e.d(rho_e u)/dt / c_s^2 term of
    the charge collision the blob still spreads isotropically, by 2 alpha t along and
    across the flow. Without R (or with its sign flipped) the scheme's O(dt) error reduces
    the along-flow diffusivity by about (tau - 1/2) U^2 (twice that): 3 % (6 %) of alpha in
    2D and 3.4 % (7.4 %) in 3D at U = 0.1, which the 1 % bar catches. A dropped or
    sign-flipped e.u term fails the centroid check."""
    U, alpha, steps = (0.1, 0.05, 160) if dim == 2 else (0.1, 0.05, 100)
    shift, dvx, dvy = _charge_in_uniform_flow(oracle_mod, dim, U, alpha, steps)
    assert abs(shift / (U * steps) - 1) < 1e-6, shift
    assert abs(dvy / (2 * alpha * steps) - 1) < 0.02, dvy
    assert abs(dvx / dvy - 1) < 0.01, (dvx, dvy)


@pytest.mark.parametrize("which", ["droplet", "uniform"])
def test_drag_force_balance_in_a_uniform_mixture(oracle_mod, which):
    """Drag as the force balance of the Results (driving force minus the droplet's inertia
    m dV/dt; -m dV/dt with no drive). In a periodic box filled with a uniform mixture
    Phi_1 = Phi_2 = 1/2 every site accelerates as a whole: u^n = (n + 1/2) F. A uniform
    body force b moves the droplet phase with everything else, so it meets no drag. A body
    force b1 on the droplet phase alone (force density Phi_1 b1) drives M1 b1 into the
    droplet but accelerates only at b1 / 2 per step, because every site carries as much
    lubricant: the drag is M1 b1 / 2, the force handed to the lubricant. A mistake in the
    inertia term (a sign, the M1 factor, a lag other than one step) or in the body forces'
    share changes these values."""
    shape = (1, 6, 5)
    one = np.ones(shape)
    phi = np.stack([0.5 * one, 0.5 * one, 0 * one])
    b = np.array([3e-6, -2e-6, 0.0])
    kw = {"body": tuple(b)} if which == "uniform" else {}
    p = W.make_params(V=(), **kw)
    if which == "droplet":
        p["body_droplet"] = tuple(b)
    s = _sim(oracle_mod, 2, shape, *_periodic(shape), phi, p)
    s.step(1)
    assert np.all(s.observables()["f_drag"] == 0.0)   # no V^{n-1} yet
    s.step(9)
    o = s.observables()
    n = s.step_count - 1
    acc = b if which == "uniform" else 0.5 * b
    assert np.abs(o["velocity"] - (n + 0.5) * acc).max() < 1e-15
    assert np.all(o["f_ele"] == 0.0)
    expect = np.zeros(3) if which == "uniform" else 0.5 * o["M1"] * b
    assert np.abs(o["f_drag"] - expect).max() < 1e-9 * o["M1"] * np.abs(b).max()
    # switched off: the mixture coasts, dV/dt = 0 and nothing drives it, so no drag
    s.set_body_force(body=(0, 0, 0), body_droplet=(0, 0, 0))
    s.step(3)
    o = s.observables()
    assert np.abs(o["f_drag"]).max() < 1e-9 * o["M1"] * np.abs(b).max()


def _strip_far_field(O, ny, l_e):
    """Potential of the paper's Fig. 1 electrode geometry (2D, no droplet, no charge): the
    oracle's Gauss-law solution, the strip height H = ny - 1.5 from the grounded floor
    nodes to the zero-flux face of the top wall, and the row in the middle."""
    w = W.electrode_above(2, 256, ny, 1, l_e=l_e, x_e=240, w_e=8, V=0.05)
    s = _sim(O, w.dim, w.shape, w.solid, w.elec, w.phi_init, w.params)
    s.params["oracle_poisson_tol"] = 1e-14
    s._prm.poisson_tol = 1e-14
    s.step(1)
    return s.pot[0], ny - 1.5, ny // 2


@pytest.mark.parametrize("ny,l_e", [(24, 8), (34, 12)])
def test_strip_lowest_mode_far_from_the_electrode(oracle_mod, ny, l_e):
    """Eqs. 3-4 rest on the lowest mode of Laplace's equation in the strip between the
    grounded surface and the zero-flux top: phi ~ sin(k v) e^{-alpha S_e}, k = pi / (2 H).
    For the discrete operator of Eq. 13 that mode is exact, with the x decay rate fixed by
    cosh(alpha) = 2 - cos(k): far from the electrode every three consecutive values along a
    row satisfy phi(x - 1) + phi(x + 1) = 2 cosh(alpha) phi(x), and every column is
    proportional to sin(k v). A Dirichlet face coefficient of eps/2 instead of eps (or a
    ground held one node off) moves the effective strip height and fails both."""
    pot, H, v = _strip_far_field(oracle_mod, ny, l_e)
    k = np.pi / (2 * H)
    alpha = np.arccosh(2 - np.cos(k))
    row = pot[v, 30:101]   # 140 or more nodes from the electrode: higher modes < 2e-6
    est = np.arccosh((row[2:] + row[:-2]) / row[1:-1] / 2)
    assert np.abs(est / alpha - 1).max() < 1e-4, (est.min(), est.max(), alpha)
    vv = np.arange(1, pot.shape[0] - 1)
    col = pot[vv, 120] / pot[v, 120]
    assert np.abs(col - np.sin(k * vv) / np.sin(k * v)).max() < 1e-5

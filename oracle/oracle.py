"""FP64 CPU oracle of the coupled ternary phase-field / leaky-dielectric LB step.

TEST INFRASTRUCTURE ONLY: this module is for the tests, the package smoke check and
the benchmark's CPU-baseline leg. The product (the CUDA library and its binding) never
imports it, and it imports nothing from the product.

The step itself is plain C (``lbehd_oracle.c``, built into ``liboracle.so`` next to
this file). This wrapper holds what is easier to read in numpy:

* the velocity sets and their weights (D2Q9 / D3Q19 for momentum and the three phase
  fields, D2Q5 / D3Q7 for charge and the Poisson faces; Methods, "Unified Lattice
  Boltzmann Model", D3Q19 weights printed after Eq. 16),
* the moment matrices M of the raw-moment collision (Eq. 15) from their monomial
  definitions, inverted with ``numpy.linalg.inv``,
* the equilibrium initial populations, and
* the droplet observables (centroid, velocity, electric force, drag; the force
  balance around Eq. 1 and Eq. 5) as plain FP64 sums over the fields.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbehd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
QMAX = 19

# --------------------------------------------------------------------- lattices

# Velocity sets: index 0 is the rest velocity; each moving velocity is followed by its
# opposite.
_E = {
    "D2Q9": [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
             (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0)],
    "D3Q19": [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
              (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
              (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
              (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)],
    "D2Q5": [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)],
    "D3Q7": [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
}


def _weights(name):
    e = np.array(_E[name])
    sq = (e * e).sum(1)
    table = {
        "D2Q9": {0: 4 / 9, 1: 1 / 9, 2: 1 / 36},
        "D3Q19": {0: 1 / 3, 1: 1 / 18, 2: 1 / 36},   # omega(0), omega(1), omega(2) after Eq. 16
        "D2Q5": {0: 1 / 3, 1: 1 / 6},
        "D3Q7": {0: 1 / 4, 1: 1 / 8},
    }[name]
    return np.array([table[int(s)] for s in sq])


_CS2 = {"D2Q9": 1 / 3, "D3Q19": 1 / 3, "D2Q5": 1 / 3, "D3Q7": 1 / 4}

# Moment basis: (row class, monomial). Classes: 0 zeroth, 1 first, 2 trace of the
# second-order block, 3 its deviatoric / off-diagonal part, 4 order >= 3.
_BASIS = {
    "D2Q9": [
        (0, lambda x, y, z: 1), (1, lambda x, y, z: x), (1, lambda x, y, z: y),
        (2, lambda x, y, z: x * x + y * y), (3, lambda x, y, z: x * x - y * y),
        (3, lambda x, y, z: x * y),
        (4, lambda x, y, z: x * x * y), (4, lambda x, y, z: x * y * y),
        (4, lambda x, y, z: x * x * y * y)],
    "D3Q19": [
        (0, lambda x, y, z: 1), (1, lambda x, y, z: x), (1, lambda x, y, z: y),
        (1, lambda x, y, z: z),
        (2, lambda x, y, z: x * x + y * y + z * z),
        (3, lambda x, y, z: x * x - y * y), (3, lambda x, y, z: x * x - z * z),
        (3, lambda x, y, z: x * y), (3, lambda x, y, z: x * z), (3, lambda x, y, z: y * z),
        (4, lambda x, y, z: x * x * y), (4, lambda x, y, z: x * x * z),
        (4, lambda x, y, z: x * y * y), (4, lambda x, y, z: x * z * z),
        (4, lambda x, y, z: y * y * z), (4, lambda x, y, z: y * z * z),
        (4, lambda x, y, z: x * x * y * y), (4, lambda x, y, z: x * x * z * z),
        (4, lambda x, y, z: y * y * z * z)],
    "D2Q5": [
        (0, lambda x, y, z: 1), (1, lambda x, y, z: x), (1, lambda x, y, z: y),
        (2, lambda x, y, z: x * x + y * y), (3, lambda x, y, z: x * x - y * y)],
    "D3Q7": [
        (0, lambda x, y, z: 1), (1, lambda x, y, z: x), (1, lambda x, y, z: y),
        (1, lambda x, y, z: z), (2, lambda x, y, z: x * x + y * y + z * z),
        (3, lambda x, y, z: x * x - y * y), (3, lambda x, y, z: x * x - z * z)],
}


class Lattice:
    """A velocity set, its weights, c_s^2 and the moment matrix M (rows = moments)."""

    def __init__(self, name):
        self.name = name
        self.e = np.array(_E[name], dtype=np.int64)
        self.Q = len(self.e)
        self.w = _weights(name)
        self.cs2 = _CS2[name]
        self.opp = np.array([next(m for m in range(self.Q) if (self.e[m] == -self.e[n]).all())
                             for n in range(self.Q)])
        basis = _BASIS[name]
        self.rowclass = np.array([c for c, _ in basis])
        self.M = np.array([[float(f(*ev)) for ev in self.e] for _, f in basis])
        self.Minv = np.linalg.inv(self.M)


LATTICES = {name: Lattice(name) for name in _E}


def lattices_for(dim):
    """(flow/phase lattice, charge/Poisson lattice) for a 2D or 3D run."""
    return (LATTICES["D2Q9"], LATTICES["D2Q5"]) if dim == 2 else (LATTICES["D3Q19"],
                                                                   LATTICES["D3Q7"])


# --------------------------------------------------------------------- ctypes

class _OLat(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_int), ("e", (ctypes.c_int * 3) * QMAX),
                ("w", ctypes.c_double * QMAX), ("opp", ctypes.c_int * QMAX),
                ("cs2", ctypes.c_double), ("M", ctypes.c_double * (QMAX * QMAX)),
                ("Minv", ctypes.c_double * (QMAX * QMAX)), ("rowclass", ctypes.c_int * QMAX)]


class _OPrm(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int),
                ("nu", ctypes.c_double * 3), ("eps", ctypes.c_double * 3),
                ("sig", ctypes.c_double * 3),
                ("gamma12", ctypes.c_double), ("gamma13", ctypes.c_double),
                ("gamma23", ctypes.c_double),
                ("cos12", ctypes.c_double), ("cos13", ctypes.c_double),
                ("cos23", ctypes.c_double),
                ("mobility", ctypes.c_double), ("W", ctypes.c_double),
                ("alpha", ctypes.c_double), ("body", ctypes.c_double * 3),
                ("body1", ctypes.c_double * 3), ("s_bulk", ctypes.c_double),
                ("poisson_tol", ctypes.c_double),
                ("poisson_max_iter", ctypes.c_int), ("n_electrodes", ctypes.c_int),
                ("V", ctypes.c_double * 64),
                ("var_density", ctypes.c_int), ("rhoph", ctypes.c_double * 3)]


_P = ctypes.POINTER(ctypes.c_double)


class _OSt(ctypes.Structure):
    _fields_ = [("solid", ctypes.POINTER(ctypes.c_uint8)),
                ("elec", ctypes.POINTER(ctypes.c_int16)),
                ("normal", ctypes.POINTER(ctypes.c_int32)),
                ("g", _P), ("fphi", _P), ("frho", _P),
                ("phiu_prev", _P), ("rhou_prev", _P), ("q_prev", _P),
                ("have_prev", ctypes.c_int),
                ("Phi", _P), ("rho", _P), ("pstar", _P), ("pot", _P), ("eps", _P), ("sig", _P),
                ("u", _P), ("F", _P), ("Fe", _P), ("Fs", _P), ("E", _P),
                ("gradPhi", _P), ("lapPhi", _P), ("mu", _P), ("FPhi", _P), ("qsrc", _P),
                ("post", _P), ("cg_r", _P), ("cg_z", _P), ("cg_p", _P), ("cg_Ap", _P),
                ("poisson_iters", ctypes.c_int), ("poisson_resid", ctypes.c_double)]


def build(force=False):
    """Compile liboracle.so with gcc (plain C99 + OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", _LIB + ".tmp",
           _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_step.restype = ctypes.c_int
        _lib.oracle_poisson.restype = ctypes.c_int
        _lib.oracle_get_threads.restype = ctypes.c_int
    return _lib


def set_threads(n):
    lib().oracle_set_threads(int(n))


def upsilon(gamma12, gamma13, gamma23):
    """Eq. 11: (Upsilon_1, Upsilon_2, Upsilon_3) and Upsilon_T of the ternary free energy
    from the pairwise surface tensions (the coefficients the oracle's step uses)."""
    Y = (ctypes.c_double * 3)()
    YT = ctypes.c_double()
    lib().oracle_upsilon(ctypes.c_double(gamma12), ctypes.c_double(gamma13),
                         ctypes.c_double(gamma23), Y, ctypes.byref(YT))
    return np.array(Y[:]), YT.value


def get_threads():
    return int(lib().oracle_get_threads())


def _olat(L):
    s = _OLat()
    s.Q = L.Q
    for n in range(L.Q):
        for a in range(3):
            s.e[n][a] = int(L.e[n][a])
        s.w[n] = L.w[n]
        s.opp[n] = int(L.opp[n])
        s.rowclass[n] = int(L.rowclass[n])
    s.cs2 = L.cs2
    for k in range(L.Q):
        for n in range(L.Q):
            s.M[k * L.Q + n] = L.M[k, n]
            s.Minv[k * L.Q + n] = L.Minv[k, n]
    return s


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# --------------------------------------------------------------------- simulation

class OracleSim:
    """One coupled LB-EHD run on the CPU in FP64.

    Arrays are numpy with shape (..., nz, ny, nx); site index i = x + nx (y + ny z).
    ``solid``: 0 fluid, 1 substrate solid (wetting angles apply), 2 neutral solid
    (90 degrees). ``elec``: -1 zero-flux, -2 ground (phi = 0), k >= 0 electrode k.
    ``phi_init``: (3, nz, ny, nx) initial Phi_1..3 (droplet, lubricant, ambient).
    ``params``: dict of lattice-unit parameters (see ``workloads``).
    """

    def __init__(self, dim, shape, solid, elec, phi_init, params):
        nz, ny, nx = shape
        self.dim, self.shape = dim, (nz, ny, nx)
        self.N = N = nx * ny * nz
        self.Lf, self.Ls = lattices_for(dim)
        Q, QS = self.Lf.Q, self.Ls.Q
        self.params = dict(params)
        self.solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.shape)
        self.elec = np.ascontiguousarray(elec, dtype=np.int16).reshape(self.shape)
        self.normal = np.zeros(self.shape, dtype=np.int32)
        z = lambda *s: np.zeros(s + self.shape)
        self.g, self.fphi, self.frho = z(Q), z(3, Q), z(QS)
        self.phiu_prev, self.rhou_prev, self.q_prev = z(3, 3), z(3), z(1)[0]
        self.Phi, self.rho, self.pstar, self.pot = z(3), z(1)[0], z(1)[0], z(1)[0]
        self.eps, self.sig = z(1)[0], z(1)[0]
        self.u, self.F, self.Fe, self.Fs, self.E = z(3), z(3), z(3), z(3), z(3)
        self.gradPhi, self.lapPhi, self.mu, self.FPhi = z(3, 3), z(3), z(3), z(3, 3)
        self.qsrc = z(1)[0]
        self.post = z(max(Q, QS))
        self.cg = [z(1)[0] for _ in range(4)]
        self.step_count = 0
        self._drop_prev = self._drop_cur = None   # (M1, sum Phi_1 u) of the last two steps
        self.poisson_iters = 0
        self.poisson_resid = 0.0
        self._prm = self._make_prm()
        self._lf, self._ls = _olat(self.Lf), _olat(self.Ls)
        lib().oracle_normals(ctypes.byref(self._prm), ctypes.byref(self._lf),
                             _ptr(self.solid, ctypes.c_uint8), _ptr(self.normal, ctypes.c_int32))
        # Initial populations at equilibrium with u = 0, rho_e = 0 (Eq. 16) and p* = 1
        # (the incompressible momentum equilibrium) or, with the variable-density scheme,
        # the gauge pressure p = 0 (every momentum population 0).
        fluid = (self.solid == 0)
        phi0 = np.asarray(phi_init, dtype=np.float64).reshape((3,) + self.shape) * fluid
        g0 = 0.0 if self._prm.var_density else 1.0
        for n in range(Q):
            self.g[n] = g0 * self.Lf.w[n] * fluid
            for c in range(3):
                self.fphi[c, n] = phi0[c] * self.Lf.w[n]
        self._st = self._make_state()

    def _make_prm(self):
        p = self.params
        s = _OPrm()
        s.dim = self.dim
        s.nz, s.ny, s.nx = self.shape
        for c in range(3):
            s.nu[c], s.eps[c], s.sig[c] = p["nu"][c], p["eps"][c], p["sig"][c]
        s.gamma12, s.gamma13, s.gamma23 = p["gamma12"], p["gamma13"], p["gamma23"]
        s.cos12 = np.cos(np.radians(p["theta12"]))
        s.cos13 = np.cos(np.radians(p["theta13"]))
        s.cos23 = np.cos(np.radians(p["theta23"]))
        s.mobility, s.W, s.alpha = p["mobility"], p["W"], p["alpha"]
        for a in range(3):
            s.body[a] = p.get("body", (0, 0, 0))[a]
            s.body1[a] = p.get("body_droplet", (0, 0, 0))[a]
        s.s_bulk = p.get("s_bulk", 1.0)
        s.poisson_tol = p.get("oracle_poisson_tol", 1e-12)
        s.poisson_max_iter = p.get("oracle_poisson_max_iter", 200000)
        V = list(p.get("V", []))
        s.n_electrodes = len(V)
        for k, v in enumerate(V):
            s.V[k] = v
        s.var_density = 1 if p.get("density_model", 0) == 1 else 0
        for c in range(3):
            s.rhoph[c] = p.get("rho_phase", (1.0, 1.0, 1.0))[c]
        return s

    def _make_state(self):
        st = _OSt()
        st.solid = _ptr(self.solid, ctypes.c_uint8)
        st.elec = _ptr(self.elec, ctypes.c_int16)
        st.normal = _ptr(self.normal, ctypes.c_int32)
        for name in ("g", "fphi", "frho", "phiu_prev", "rhou_prev", "q_prev", "Phi", "rho",
                     "pstar", "pot", "eps", "sig", "u", "F", "Fe", "Fs", "E", "gradPhi",
                     "lapPhi", "mu", "FPhi", "qsrc", "post"):
            setattr(st, name, _ptr(getattr(self, name)))
        st.cg_r, st.cg_z, st.cg_p, st.cg_Ap = (_ptr(a) for a in self.cg)
        st.have_prev = 0
        return st

    def set_electrodes(self, V):
        V = list(V)
        self._prm.n_electrodes = len(V)
        for k, v in enumerate(V):
            self._prm.V[k] = v
        self.params["V"] = V

    def step(self, n=1):
        """Advance n coupled steps. Returns the number of Poisson solves that hit the cap."""
        bad = 0
        for _ in range(n):
            rc = lib().oracle_step(ctypes.byref(self._prm), ctypes.byref(self._lf),
                                   ctypes.byref(self._ls), ctypes.byref(self._st))
            bad += rc != 0
            self.step_count += 1
            self._drop_prev, self._drop_cur = self._drop_cur, self._droplet_momentum()
            self.poisson_iters = self._st.poisson_iters
            self.poisson_resid = self._st.poisson_resid
        return bad

    # ----------------------------------------------------------------- observables

    def _droplet_momentum(self):
        """(M1, sum Phi_1 u) over fluid nodes, of the fields of the step just taken."""
        P1 = self.Phi[0] * (self.solid == 0)
        return P1.sum(), np.array([(P1 * self.u[a]).sum() for a in range(3)])

    def set_body_force(self, body=None, body_droplet=None):
        """Change the uniform and the droplet-phase body force from the next step on."""
        if body is not None:
            self.params["body"] = tuple(body)
        if body_droplet is not None:
            self.params["body_droplet"] = tuple(body_droplet)
        for a in range(3):
            self._prm.body[a] = self.params.get("body", (0, 0, 0))[a]
            self._prm.body1[a] = self.params.get("body_droplet", (0, 0, 0))[a]

    def observables(self):
        """Droplet observables of the fields computed in the last step (FP64 sums over
        fluid nodes): mass M1 = sum Phi_1, centroid sum Phi_1 x / M1, velocity
        V = sum Phi_1 u / M1, electric force on the droplet sum Phi_1 F_e, total electric
        force sum F_e, per-component mass sum Phi_i and total charge sum rho_e.

        Drag (Results, the force balance of the migrating droplet, Eqs. 1 and 5: the
        driving force minus the droplet's inertia m dV/dt, which is -m dV/dt when nothing
        drives it): f_drag = f_ele + M1 (body + body_droplet) - M1 (V^n - V^{n-1}), with
        unit density so that m = M1, dV/dt the difference of the last two steps'
        velocities, and the body forces' share on the droplet M1 (body + body_droplet).
        Zero until two steps have been taken."""
        fluid = (self.solid == 0)
        nz, ny, nx = self.shape
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        P1 = self.Phi[0] * fluid
        M1 = P1.sum()
        inv = 1.0 / M1 if M1 != 0.0 else 0.0
        out = {
            "M1": M1,
            "centroid": np.array([(P1 * xx).sum(), (P1 * yy).sum(), (P1 * zz).sum()]) * inv,
            "velocity": np.array([(P1 * self.u[a]).sum() for a in range(3)]) * inv,
            "f_ele": np.array([(P1 * self.Fe[a]).sum() for a in range(3)]),
            "f_ele_total": np.array([(self.Fe[a] * fluid).sum() for a in range(3)]),
            "mass": np.array([(self.Phi[c] * fluid).sum() for c in range(3)]),
            "charge": (self.rho * fluid).sum(),
        }
        drag = np.zeros(3)
        if self._drop_prev is not None:
            M1p, Pp = self._drop_prev
            Vp = Pp / M1p if M1p != 0.0 else np.zeros(3)
            push = (np.asarray(self.params.get("body", (0, 0, 0)), dtype=np.float64) +
                    np.asarray(self.params.get("body_droplet", (0, 0, 0)), dtype=np.float64))
            drag = out["f_ele"] + M1 * push - M1 * (out["velocity"] - Vp)
        out["f_drag"] = drag
        return out

    def poisson(self):
        """Solve Eq. 13 alone on the current eps / rho / geometry (used by the pins)."""
        self._st.cg_r = _ptr(self.cg[0])
        return lib().oracle_poisson(ctypes.byref(self._prm), ctypes.byref(self._ls),
                                    ctypes.byref(self._st))

"""FP64 discrete-adjoint reference of the coupled LB-EHD step (differentiable PyTorch, CPU).

TEST INFRASTRUCTURE ONLY: the tests use this module to check the gradients of the CUDA
adjoint. The product never imports it.

``RefModel.step`` restates one coupled step n -> n+1 in vectorised PyTorch FP64. It follows
the stages and their order of ``oracle_step`` in ``lbehd_oracle.c``, the oracle of the
Method section:
moments (Eq. 19); wetting ghosts (Eq. 20a); eps, sigma linear in Phi (Table 1); isotropic
gradients and Laplacians; chemical potential (Eqs. 10-11), capillary force and sharpening
flux (Eq. 18); the Gauss law (Eq. 13); electric force (Eq. 12); u = j + F/2 and the
conduction source of Eq. 14; the three raw-moment MRT collisions (momentum, Eqs. 15-17,
Eqs. 14 and 20b) with pull streaming and halfway bounce-back; and the products kept for the
next step's backward differences. A test checks it against the C oracle.

Its gradient by ``torch.autograd`` is the exact gradient of the discrete step map (the
discrete adjoint). Every operation is differentiable. The only non-smooth one is |Phi
(1 - Phi)| in Eq. 18, whose derivative is taken as sign(.). The Gauss-law solve is a direct
sparse solve (scipy's SuperLU) wrapped in an autograd function. Its backward pass is the
implicit-function theorem: one adjoint solve with the same symmetric operator, mu = A^-1
(dL/dphi), then dL/d(eps, rho, V) = -mu^T dR/d(eps, rho, V) for the residual R = A phi - b.
The loss of the control problem is the x centroid of the droplet (Phi_1) after the last step,
as a function of the per-electrode potential schedule.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

from . import oracle as O

T = torch.float64


def _site_index(shape):
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)


def _neighbours(shape, e):
    """Flat index of site i + e_n (periodic) for every velocity of e: (Q, N) int64."""
    nz, ny, nx = shape
    x, y, z = _site_index(shape)
    out = []
    for ev in e:
        X = (x + ev[0]) % nx
        Y = (y + ev[1]) % ny
        Z = (z + ev[2]) % nz
        out.append(X + nx * (Y + ny * Z))
    return np.array(out, dtype=np.int64)


class RefModel:
    """The discrete step map of one geometry and parameter set."""

    def __init__(self, dim, shape, solid, elec, params, normal):
        self.dim, self.shape = dim, tuple(shape)
        nz, ny, nx = self.shape
        self.N = N = nx * ny * nz
        self.Lf, self.Ls = O.lattices_for(dim)
        p = dict(params)
        self.p = p
        solid = np.asarray(solid, dtype=np.int64).reshape(-1)
        elec = np.asarray(elec, dtype=np.int64).reshape(-1)
        normal = np.asarray(normal, dtype=np.int64).reshape(-1)
        self.solid_np = solid
        self.fluid_np = solid == 0
        self.fluid = torch.tensor(self.fluid_np, dtype=T)
        self.dirichlet_np = (solid != 0) & ((elec >= 0) | (elec == -2))
        self.elec_np = elec
        self.n_elec = len(p.get("V", []))
        self.nbf = _neighbours(self.shape, self.Lf.e)     # flow lattice
        self.nbs = _neighbours(self.shape, self.Ls.e)     # charge / Poisson faces
        # wetting ghosts: boundary solid nodes, their fluid source along the lattice normal
        gi = np.nonzero((solid != 0) & (normal > 0))[0]
        self.g_site = torch.tensor(gi)
        self.g_src = torch.tensor(self.nbf[normal[gi], gi])
        ek = self.Lf.e[normal[gi]]
        self.g_len = torch.tensor(np.sqrt((ek * ek).sum(1).astype(np.float64)), dtype=T)
        c12 = np.cos(np.radians(p["theta12"]))
        c13 = np.cos(np.radians(p["theta13"]))
        c23 = np.cos(np.radians(p["theta23"]))
        wet = (solid[gi] == 1).astype(np.float64)
        self.g_c12 = torch.tensor(wet * c12, dtype=T)
        self.g_c13 = torch.tensor(wet * c13, dtype=T)
        self.g_c23 = torch.tensor(wet * c23, dtype=T)
        # pull-streaming gathers with halfway bounce-back (solid nodes hold 0)
        self.pull_f = self._pull(self.Lf, self.nbf)
        self.pull_s = self._pull(self.Ls, self.nbs)
        # lattice tables as tensors
        self.ef = torch.tensor(self.Lf.e, dtype=T)
        self.wf = torch.tensor(self.Lf.w, dtype=T)
        self.es = torch.tensor(self.Ls.e, dtype=T)
        self.ws = torch.tensor(self.Ls.w, dtype=T)
        self.Mf, self.Mfi = torch.tensor(self.Lf.M, dtype=T), torch.tensor(self.Lf.Minv, dtype=T)
        self.Ms, self.Msi = torch.tensor(self.Ls.M, dtype=T), torch.tensor(self.Ls.Minv, dtype=T)
        self.rcf = torch.tensor(self.Lf.rowclass)
        self.rcs = torch.tensor(self.Ls.rowclass)
        # Poisson faces: neighbour class of every (face, fluid site)
        self._poisson_setup()

    def _pull(self, L, nb):
        Q, N = L.Q, self.N
        pop = np.zeros((Q, N), dtype=np.int64)
        site = np.zeros((Q, N), dtype=np.int64)
        for n in range(Q):
            src = nb[L.opp[n]]   # i - e_n
            bounce = ~self.fluid_np[src]
            pop[n] = np.where(bounce, L.opp[n], n)
            site[n] = np.where(bounce, np.arange(N), src)
        return torch.tensor(pop * N + site)

    def _poisson_setup(self):
        fl = self.fluid_np
        self.fidx = np.nonzero(fl)[0]
        self.fpos = -np.ones(self.N, dtype=np.int64)
        self.fpos[self.fidx] = np.arange(len(self.fidx))
        faces = []
        for n in range(1, self.Ls.Q):
            j = self.nbs[n][self.fidx]
            kind = np.where(fl[j], 1, np.where(self.dirichlet_np[j], 2, 0))
            faces.append((j, kind))
        self.pfaces = faces
        self.dir_sites = np.nonzero(self.dirichlet_np)[0]
        # Dirichlet value of every site as a linear map of V: value = V[elec] (ground: 0)
        sel = np.zeros((self.N, max(self.n_elec, 1)))
        for s_ in self.dir_sites:
            if self.elec_np[s_] >= 0:
                sel[s_, self.elec_np[s_]] = 1.0
        self.dir_map = torch.tensor(sel, dtype=T)

    # ---------------------------------------------------------------- pieces

    def dirichlet_field(self, V):
        """Potential held at Dirichlet solid nodes (V of the electrode, 0 on ground)."""
        if self.n_elec == 0:
            return torch.zeros(self.N, dtype=T)
        return self.dir_map @ V

    def poisson_residual(self, phi_f, eps, rho, V):
        """R = A(eps) phi - b(eps, rho, V) on the fluid nodes (Eq. 13)."""
        full = torch.zeros(self.N, dtype=T).index_put((torch.tensor(self.fidx),), phi_f)
        full = full + self.dirichlet_field(V)
        fi = torch.tensor(self.fidx)
        R = -rho[fi]
        for j, kind in self.pfaces:
            jt = torch.tensor(j)
            kf = torch.where(torch.tensor(kind == 1), 0.5 * (eps[fi] + eps[jt]),
                             torch.where(torch.tensor(kind == 2), eps[fi], torch.zeros_like(eps[fi])))
            R = R + kf * (full[fi] - full[jt])
        return R

    def poisson_matrix(self, eps, rho, V):
        fl_n = len(self.fidx)
        e = eps.detach().numpy()
        r = rho.detach().numpy()
        dvals = self.dirichlet_field(V.detach()).numpy()
        rows, cols, vals = [], [], []
        diag = np.zeros(fl_n)
        b = r[self.fidx].copy()
        for j, kind in self.pfaces:
            ei = e[self.fidx]
            k = np.where(kind == 1, 0.5 * (ei + e[j]), np.where(kind == 2, ei, 0.0))
            diag += k
            m = kind == 1
            rows.append(np.arange(fl_n)[m])
            cols.append(self.fpos[j[m]])
            vals.append(-k[m])
            b += np.where(kind == 2, k * dvals[j], 0.0)
        rows.append(np.arange(fl_n))
        cols.append(np.arange(fl_n))
        vals.append(diag)
        A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(fl_n, fl_n))
        return A, b

    # ---------------------------------------------------------------- the step

    def initial_state(self, phi_init):
        fl = self.fluid
        phi0 = torch.tensor(np.asarray(phi_init, dtype=np.float64).reshape(3, -1)) * fl
        g = self.wf[:, None] * fl[None, :]
        fphi = phi0[:, None, :] * self.wf[None, :, None]
        frho = torch.zeros(self.Ls.Q, self.N, dtype=T)
        return {"g": g, "fphi": fphi, "frho": frho, "phiu_prev": None, "rhou_prev": None,
                "q_prev": None}

    def _mrt(self, M, Mi, f, feq, rate, R=None, C=None, Cp=None):
        m, meq = M @ f, M @ feq
        ms = m - rate * (m - meq)
        if R is not None:
            ms = ms + (1.0 - 0.5 * rate) * (M @ R)
        if C is not None:
            mC = M @ C
            ms = ms + mC + 0.5 * (mC - (M @ Cp))
        return Mi @ ms

    def step(self, st, V):
        """One coupled step; returns (new state, Phi of this step (3, N))."""
        p, N = self.p, self.N
        Lf, Ls = self.Lf, self.Ls
        fl = self.fluid
        cs2, cs2s, W = Lf.cs2, Ls.cs2, p["W"]
        ef, wf = self.ef, self.wf
        # 1. moments
        Phi = st["fphi"].sum(1) * fl
        rho = st["frho"].sum(0) * fl
        pstar = st["g"].sum(0) * fl
        j = (ef.T @ st["g"]) * fl
        # 2. wetting ghosts (Eq. 20a), explicit in the fluid values along the normal
        if len(self.g_site):
            P1, P2, P3 = Phi[0, self.g_src], Phi[1, self.g_src], Phi[2, self.g_src]
            s4 = 4.0 / W
            H1 = s4 * (-self.g_c13 * P1 * P3 - self.g_c12 * P1 * P2)
            H2 = s4 * (self.g_c12 * P1 * P2 - self.g_c23 * P2 * P3)
            H3 = s4 * (self.g_c23 * P2 * P3 + self.g_c13 * P1 * P3)
            ghost = torch.stack([P1 - self.g_len * H1, P2 - self.g_len * H2,
                                 P3 - self.g_len * H3])
            Phi = Phi.index_put((torch.arange(3)[:, None], self.g_site[None, :]), ghost)
        # 3. properties
        epsv = torch.tensor(p["eps"], dtype=T)
        sigv = torch.tensor(p["sig"], dtype=T)
        eps = epsv @ Phi
        sig = sigv @ Phi
        # 4. isotropic stencils at fluid nodes
        nb = torch.tensor(self.nbf[1:])                   # (Q-1, N)
        w1, e1 = wf[1:], ef[1:]
        Pn = Phi[:, nb]                                   # (3, Q-1, N)
        grad = torch.einsum("q,qa,cqn->can", w1, e1, Pn) / cs2 * fl
        lap = 2.0 / cs2 * torch.einsum("q,cqn->cn", w1, Pn - Phi[:, None, :]) * fl
        # 5. chemical potential, capillary force, sharpening flux
        g12, g13, g23 = p["gamma12"], p["gamma13"], p["gamma23"]
        Y = [g12 + g13 - g23, g12 + g23 - g13, g13 + g23 - g12]
        YT = 3.0 / (1.0 / Y[0] + 1.0 / Y[1] + 1.0 / Y[2])
        tri = 24.0 * YT / W * Phi[0] * Phi[1] * Phi[2]
        mu = torch.stack([24.0 * Y[c] / W * Phi[c] * (Phi[c] - 1.0) * (Phi[c] - 0.5) - tri -
                          0.75 * Y[c] * W * lap[c] for c in range(3)]) * fl
        Fs = torch.einsum("cn,can->an", mu, grad)
        gn = torch.sqrt((grad * grad).sum(1) + 1e-10)                     # (3, N)
        lam = 4.0 / W * torch.abs(Phi * (1.0 - Phi))
        lam_n = lam[:, None, :] * grad / gn[:, None, :]                    # (3, 3, N)
        J = lam_n.sum(0)
        sumsq = (Phi * Phi).sum(0)
        safe = torch.where(fl > 0, sumsq, torch.ones_like(sumsq))
        FPhi = (lam_n - (Phi * Phi / safe)[:, None, :] * J[None, :, :]) * fl
        # 6. Gauss law
        Vt = V if self.n_elec else torch.zeros(1, dtype=T)
        pot = PoissonSolve.apply(eps, rho, Vt, self)
        # 7. electric force; zero-flux solid neighbours mirror the node's own value
        neum = torch.tensor((~self.fluid_np) & (~self.dirichlet_np))
        ph = torch.where(neum[nb], pot[None, :].expand(nb.shape), pot[nb])
        gp = torch.einsum("q,qa,qn->an", w1, e1, ph) / cs2
        ge = torch.einsum("q,qa,qn->an", w1, e1, eps[nb]) / cs2
        E2 = (gp * gp).sum(0)
        Fe = (rho * (-gp) - 0.5 * E2 * ge) * fl
        body = torch.tensor(p.get("body", (0.0, 0.0, 0.0)), dtype=T)[:, None]
        F = (Fs + Fe + body) * fl
        # 8. velocity, conduction source
        u = (j + 0.5 * F) * fl
        q = torch.zeros(N, dtype=T)
        for n in range(1, Ls.Q):
            jn = torch.tensor(self.nbs[n])
            fj = fl[jn]
            q = q + fj * 0.5 * (sig + sig[jn]) * (pot[jn] - pot)
        q = q * fl
        phiu = Phi[:, None, :] * u[None, :, :]
        rhou = rho[None, :] * u
        phiu_prev = phiu if st["phiu_prev"] is None else st["phiu_prev"]
        rhou_prev = rhou if st["rhou_prev"] is None else st["rhou_prev"]
        q_prev = q if st["q_prev"] is None else st["q_prev"]
        # 9a. momentum collision + stream
        uu = (u * u).sum(0)
        nu = torch.tensor(p["nu"], dtype=T) @ Phi
        s_nu = 1.0 / (nu / cs2 + 0.5)
        eu = ef @ u                                                          # (Q, N)
        eF = ef @ F
        uF = (u * F).sum(0)
        feq = wf[:, None] * (pstar + eu / cs2 + eu * eu / (2 * cs2 * cs2) - uu / (2 * cs2))
        R = wf[:, None] * ((eF - uF) / cs2 + eu * eF / (cs2 * cs2))
        rc = self.rcf[:, None]
        rate = torch.where(rc <= 1, torch.zeros(1, dtype=T),
                           torch.where(rc == 2, torch.full((1,), p.get("s_bulk", 1.0), dtype=T),
                                       torch.where(rc == 3, s_nu[None, :],
                                                   torch.ones(1, dtype=T))))
        post = self._mrt(self.Mf, self.Mfi, st["g"], feq, rate, R=R) * fl
        g_new = post.reshape(-1)[self.pull_f] * fl
        # 9b. phase fields
        tau_phi = 0.5 + p["mobility"] / cs2
        rate_p = torch.where(rc == 0, torch.zeros(1, dtype=T),
                             torch.where(rc == 1, torch.full((1,), 1.0 / tau_phi, dtype=T),
                                         torch.ones(1, dtype=T)))
        fphi_new = []
        for c in range(3):
            A = cs2 * FPhi[c] + (phiu[c] - phiu_prev[c])
            eA = ef @ A
            feq_c = Phi[c] * wf[:, None] * (1.0 + eu / cs2)
            C = wf[:, None] / cs2 * eA
            post_c = self._mrt(self.Mf, self.Mfi, st["fphi"][c], feq_c, rate_p, R=C) * fl
            fphi_new.append(post_c.reshape(-1)[self.pull_f] * fl)
        fphi_new = torch.stack(fphi_new)
        # 9c. charge
        es, ws = self.es, self.ws
        tau_rho = 0.5 + p["alpha"] / cs2s
        rcs = self.rcs[:, None]
        rate_s = torch.where(rcs == 0, torch.zeros(1, dtype=T),
                             torch.where(rcs == 1, torch.full((1,), 1.0 / tau_rho, dtype=T),
                                         torch.ones(1, dtype=T)))
        D = rhou - rhou_prev
        eus = es @ u
        feq_s = rho * ws[:, None] * (1.0 + eus / cs2s)
        Rs = ws[:, None] / cs2s * (es @ D)
        Cs = ws[:, None] * q
        Cps = ws[:, None] * q_prev
        post_s = self._mrt(self.Ms, self.Msi, st["frho"], feq_s, rate_s, R=Rs, C=Cs, Cp=Cps) * fl
        frho_new = post_s.reshape(-1)[self.pull_s] * fl
        # 10. products for the next step's backward differences
        new = {"g": g_new, "fphi": fphi_new, "frho": frho_new, "phiu_prev": phiu,
               "rhou_prev": rhou, "q_prev": q}
        return new, Phi

    def centroid_x(self, Phi):
        x = torch.tensor(_site_index(self.shape)[0], dtype=T)
        P1 = Phi[0] * self.fluid
        return (P1 * x).sum() / P1.sum()


class PoissonSolve(torch.autograd.Function):
    """phi = A(eps)^-1 b(eps, rho, V) on the fluid nodes, the Dirichlet values on the
    Dirichlet nodes, 0 elsewhere. Backward: implicit-function theorem (adjoint solve)."""

    @staticmethod
    def forward(ctx, eps, rho, V, model):
        A, b = model.poisson_matrix(eps, rho, V)
        fl_n = len(model.fidx)
        phi_f = spla.spsolve(A, b) if fl_n else np.zeros(0)
        out = model.dirichlet_field(V).clone()
        out[torch.tensor(model.fidx)] = torch.tensor(phi_f, dtype=T)
        ctx.model = model
        ctx.A = A
        ctx.save_for_backward(eps, rho, V, torch.tensor(phi_f, dtype=T))
        return out

    @staticmethod
    def backward(ctx, gout):
        model = ctx.model
        eps, rho, V, phi_f = ctx.saved_tensors
        fi = torch.tensor(model.fidx)
        g_f = gout[fi].numpy()
        mu = torch.tensor(spla.spsolve(ctx.A, g_f), dtype=T)   # A is symmetric
        with torch.enable_grad():
            e = eps.detach().requires_grad_(True)
            r = rho.detach().requires_grad_(True)
            v = V.detach().requires_grad_(True)
            R = model.poisson_residual(phi_f, e, r, v)
            ge, gr, gv = torch.autograd.grad(R, (e, r, v), grad_outputs=-mu, allow_unused=True)
        ge = torch.zeros_like(eps) if ge is None else ge
        gr = torch.zeros_like(rho) if gr is None else gr
        gv = torch.zeros_like(V) if gv is None else gv
        # the Dirichlet nodes hold V directly
        if model.n_elec:
            gv = gv + model.dir_map.T @ gout
        return ge, gr, gv, None


def schedule_loss(model, phi_init, Vsched, seg_steps, checkpoint=True):
    """x centroid of the droplet after len(Vsched) * seg_steps steps, with electrode
    potentials Vsched[k] (tensor (S, n_electrodes)) during segment k."""
    st = model.initial_state(phi_init)
    Phi = None
    for k in range(Vsched.shape[0]):
        for _ in range(seg_steps):
            if checkpoint and Vsched.requires_grad:
                st, Phi = _ckpt_step(model, st, Vsched[k])
            else:
                st, Phi = model.step(st, Vsched[k])
    return model.centroid_x(Phi)


def _ckpt_step(model, st, V):
    keys = ("g", "fphi", "frho", "phiu_prev", "rhou_prev", "q_prev")
    first = st["phiu_prev"] is None

    def fn(*args):
        s = dict(zip(keys, args[:-1]))
        if first:
            s["phiu_prev"] = s["rhou_prev"] = s["q_prev"] = None
        new, Phi = model.step(s, args[-1])
        return tuple(new[k] for k in keys) + (Phi,)

    z = torch.zeros(1, dtype=T)
    args = [st[k] if st[k] is not None else z for k in keys] + [V]
    out = torch.utils.checkpoint.checkpoint(fn, *args, use_reentrant=False)
    return dict(zip(keys, out[:-1])), out[-1]

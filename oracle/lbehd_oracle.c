/*
 * lbehd_oracle.c -- FP64 CPU oracle for one time step of the coupled ternary
 * phase-field / leaky-dielectric lattice Boltzmann (LB-EHD) method of
 * "Controlling the dynamics of an electric-field-driven droplet on a
 * lubricant-infused micropillar surface" (Methods, Eqs. 8-21).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path loads this file: only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg do. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Style: plain loops over lattice sites, FP64 throughout, one stage per equation,
 * executed in the order of oracle_step(). Collisions use the dense moment matrix M
 * and its inverse (computed by the Python wrapper with numpy.linalg.inv) exactly as
 * Eq. 15 and the momentum/charge collision equations are written: m = M f,
 * m* = (I - S) m + S m_eq + (I - S/2) M C, f* = M^-1 m*.
 *
 * Readings of points the paper leaves open:
 *  - Phase field and momentum use D2Q9 / D3Q19; charge uses D2Q5 / D3Q7.
 *  - Moment basis: raw monomials with the second-order block split into trace and
 *    deviatoric parts; all moments of order >= 3 relax at rate 1.
 *  - AC source (Eq. 17): first moment = c_s^2 F_Phi + d(Phi u)/dt so that the
 *    recovered equation is Eq. 8 with M = c_s^2 (tau_Phi - 1/2).
 *  - Normal of Eq. 18: n = grad Phi / sqrt(|grad Phi|^2 + 1e-10) (continuous where
 *    grad Phi = 0).
 *  - Time derivatives are backward differences, zero on the first step.
 *  - Wetting (Eq. 20a): ghost Phi on boundary solid nodes from the fluid node along
 *    the lattice normal, normal pointing into the fluid.
 *  - Poisson (Eq. 13): 5/7-point finite-volume operator with arithmetic-mean face
 *    permittivity, Dirichlet values held at electrode/ground solid nodes, zero flux
 *    at every other solid face; solved to the fixed point by Jacobi-preconditioned CG.
 *  - Charge (Eq. 14): conduction source Q = div(sigma grad phi) with the same
 *    face discretisation and zero flux at every solid face.
 *  - Large density ratios (Table 1's densities; Eq. 9 with a variable rho), when
 *    var_density is set: the momentum populations carry the pressure and rho u,
 *    g_eq,n = w_n p/c_s^2 + rho s_n(u) (n > 0), g_eq,0 = (w_0 - 1) p/c_s^2 + rho s_0(u),
 *    s_n(u) = w_n [e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)], with rho = sum_i
 *    Phi_i rho_i; the force term G_n = (e_n - u).[Gamma_n F + s_n c_s^2 grad rho]/c_s^2,
 *    Gamma_n = w_n + s_n, carries the body forces and the density gradient; rho u =
 *    sum e g + F/2 and p = c_s^2/(1 - w_0) [sum_{n>0} g_n + u.grad(rho)/2 + rho s_0(u)];
 *    one relaxation time, tau = 1/2 + nu/c_s^2, for every moment (BGK).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

/* One velocity set with its moment transform. */
typedef struct {
    int Q;
    int e[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
    double cs2;
    double M[QMAX * QMAX];    /* M[k*Q + n] = moment k of velocity n */
    double Minv[QMAX * QMAX];
    int rowclass[QMAX];       /* 0 zeroth, 1 first, 2 trace, 3 deviatoric, 4 order>=3 */
} olat_t;

/* Physical and numerical parameters in lattice units. */
typedef struct {
    int dim, nx, ny, nz;
    double nu[3], eps[3], sig[3];
    double gamma12, gamma13, gamma23;
    double cos12, cos13, cos23;   /* wetting angles on substrate solid (class 1) */
    double mobility, W, alpha;
    double body[3];
    double body1[3];              /* force density on the droplet phase: Phi_1 body1 */
    double s_bulk;
    double poisson_tol;
    int poisson_max_iter;
    int n_electrodes;
    double V[64];
    int var_density;              /* 1: the pressure-based variable-density momentum scheme */
    double rhoph[3];              /* phase densities rho_i (var_density) */
} oprm_t;

/* State and per-step fields. Every array is owned by the caller. */
typedef struct {
    const uint8_t *solid;   /* 0 fluid, 1 substrate solid, 2 neutral solid */
    const int16_t *elec;    /* -1 none (zero flux), -2 ground, k>=0 electrode k */
    const int32_t *normal;  /* lattice normal of boundary solids, 0 elsewhere */
    double *g, *fphi, *frho;            /* pre-collision populations at time n */
    double *phiu_prev, *rhou_prev, *q_prev;
    int have_prev;
    double *Phi, *rho, *pstar, *pot, *eps, *sig;
    double *u, *F, *Fe, *Fs, *E;
    double *gradPhi, *lapPhi, *mu, *FPhi, *qsrc;
    double *post;                        /* Q*N scratch */
    double *cg_r, *cg_z, *cg_p, *cg_Ap;  /* N scratch each */
    int poisson_iters;
    double poisson_resid;
} ost_t;

/* ------------------------------------------------------------------ geometry */

static long site_nbr(const oprm_t *p, long i, const int *e)
{
    long nxy = (long)p->nx * p->ny;
    int x = (int)(i % p->nx), y = (int)((i / p->nx) % p->ny), z = (int)(i / nxy);
    x = (x + e[0] + p->nx) % p->nx;
    y = (y + e[1] + p->ny) % p->ny;
    z = (z + e[2] + p->nz) % p->nz;
    return x + (long)p->nx * (y + (long)p->ny * z);
}

static int is_dirichlet(const ost_t *s, long i)
{
    return s->solid[i] != 0 && (s->elec[i] >= 0 || s->elec[i] == -2);
}

static double dirichlet_value(const oprm_t *p, const ost_t *s, long i)
{
    return s->elec[i] >= 0 ? p->V[s->elec[i]] : 0.0;
}

/*
 * Lattice normal of every boundary solid node (a solid node with at least one fluid
 * neighbour in the flow lattice): among the fluid neighbours, the direction e_k with
 * the largest e_k . v / |e_k|, where v = sum_n w_n e_n [neighbour n is fluid].
 * Integer arithmetic (weights scaled by 36), ties to the lowest index.
 * Needed by the wetting condition, Eq. 20a.
 */
void oracle_normals(const oprm_t *p, const olat_t *L, const uint8_t *solid, int32_t *normal)
{
    long N = (long)p->nx * p->ny * p->nz;
    for (long i = 0; i < N; i++) {
        normal[i] = 0;
        if (!solid[i])
            continue;
        long v[3] = {0, 0, 0};
        int any = 0;
        for (int n = 1; n < L->Q; n++) {
            long j = site_nbr(p, i, L->e[n]);
            if (!solid[j]) {
                long iw = lround(36.0 * L->w[n]);
                for (int a = 0; a < 3; a++)
                    v[a] += iw * L->e[n][a];
                any = 1;
            }
        }
        if (!any)
            continue;
        int best = 0;
        long bs = 0, bn2 = 1;
        for (int n = 1; n < L->Q; n++) {
            long j = site_nbr(p, i, L->e[n]);
            if (solid[j])
                continue;
            long s = 0, n2 = 0;
            for (int a = 0; a < 3; a++) {
                s += L->e[n][a] * v[a];
                n2 += L->e[n][a] * L->e[n][a];
            }
            /* compare s/sqrt(n2) > bs/sqrt(bn2) through sign-preserving squares */
            long lhs = s * (s < 0 ? -s : s) * bn2;
            long rhs = bs * (bs < 0 ? -bs : bs) * n2;
            if (best == 0 || lhs > rhs) {
                best = n;
                bs = s;
                bn2 = n2;
            }
        }
        normal[i] = best;
    }
}

/* ------------------------------------------------------------------ Poisson */

/* Eq. 11: the coefficients Upsilon_i of the ternary free energy from the pairwise surface
 * tensions, Upsilon_i = gamma_ij + gamma_ik - gamma_jk ({i, j, k} = {1, 2, 3}), and
 * Upsilon_T = 3 / sum_i (1 / Upsilon_i). */
void oracle_upsilon(double g12, double g13, double g23, double Y[3], double *YT)
{
    Y[0] = g12 + g13 - g23;
    Y[1] = g12 + g23 - g13;
    Y[2] = g13 + g23 - g12;
    *YT = 3.0 / (1.0 / Y[0] + 1.0 / Y[1] + 1.0 / Y[2]);
}

/* Face coefficient between fluid node i and neighbour j for the operator of Eq. 13. */
static double eps_face(const ost_t *s, long i, long j)
{
    if (!s->solid[j])
        return 0.5 * (s->eps[i] + s->eps[j]);
    if (is_dirichlet(s, j))
        return s->eps[i];
    return 0.0;
}

/* (A x)_i = sum_faces k (x_i - x_j) over fluid j, + k x_i over Dirichlet j. */
static void poisson_apply(const oprm_t *p, const olat_t *S, const ost_t *s,
                          const double *x, double *Ax)
{
    long N = (long)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) {
            Ax[i] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int n = 1; n < S->Q; n++) {
            long j = site_nbr(p, i, S->e[n]);
            double k = eps_face(s, i, j);
            if (k == 0.0)
                continue;
            acc += k * x[i];
            if (!s->solid[j])
                acc -= k * x[j];
        }
        Ax[i] = acc;
    }
}

static double dot_fluid(const ost_t *s, long N, const double *a, const double *b)
{
    double acc = 0.0;
#pragma omp parallel for reduction(+ : acc) schedule(static)
    for (long i = 0; i < N; i++)
        if (!s->solid[i])
            acc += a[i] * b[i];
    return acc;
}

/*
 * Solve div(eps grad phi) = -rho_e (Eq. 13) on the fluid nodes, written as the SPD
 * system A phi = b with b_i = rho_e,i + sum over Dirichlet faces of eps_i V.
 * Jacobi-preconditioned conjugate gradients from the warm start in s->pot, stopped
 * at ||r||_2 <= tol ||b||_2. Dirichlet solid nodes receive their value, other
 * solid nodes 0. Returns 0, or -1 when the iteration cap is reached.
 */
int oracle_poisson(const oprm_t *p, const olat_t *S, ost_t *s)
{
    long N = (long)p->nx * p->ny * p->nz;
    double *r = s->cg_r, *z = s->cg_z, *d = s->cg_p, *Ad = s->cg_Ap;
    double *b = s->qsrc; /* borrowed as the right-hand side; rewritten later */
    double *diag = s->post;

#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) {
            s->pot[i] = is_dirichlet(s, i) ? dirichlet_value(p, s, i) : 0.0;
            b[i] = 0.0;
            diag[i] = 1.0;
            continue;
        }
        double bi = s->rho[i], di = 0.0;
        for (int n = 1; n < S->Q; n++) {
            long j = site_nbr(p, i, S->e[n]);
            double k = eps_face(s, i, j);
            di += k;
            if (s->solid[j] && k != 0.0)
                bi += k * dirichlet_value(p, s, j);
        }
        b[i] = bi;
        diag[i] = di > 0.0 ? di : 1.0;
    }
    double bnorm = sqrt(dot_fluid(s, N, b, b));
    if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++)
            if (!s->solid[i])
                s->pot[i] = 0.0;
        s->poisson_iters = 0;
        s->poisson_resid = 0.0;
        return 0;
    }
    poisson_apply(p, S, s, s->pot, Ad);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        r[i] = s->solid[i] ? 0.0 : b[i] - Ad[i];
        z[i] = r[i] / diag[i];
        d[i] = z[i];
    }
    double rz = dot_fluid(s, N, r, z);
    double rn = sqrt(dot_fluid(s, N, r, r));
    int it = 0;
    while (rn > p->poisson_tol * bnorm && it < p->poisson_max_iter) {
        poisson_apply(p, S, s, d, Ad);
        double alpha = rz / dot_fluid(s, N, d, Ad);
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++) {
            if (s->solid[i])
                continue;
            s->pot[i] += alpha * d[i];
            r[i] -= alpha * Ad[i];
            z[i] = r[i] / diag[i];
        }
        double rz_new = dot_fluid(s, N, r, z);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++)
            if (!s->solid[i])
                d[i] = z[i] + beta * d[i];
        rn = sqrt(dot_fluid(s, N, r, r));
        it++;
    }
    s->poisson_iters = it;
    s->poisson_resid = rn / bnorm;
    return rn <= p->poisson_tol * bnorm ? 0 : -1;
}

/* ------------------------------------------------------------------ collision */

/* m* = m - S (m - m_eq) + (I - S/2) M R + M C + 1/2 M (C - C_prev); f* = M^-1 m*.
 * R, C, Cp may be NULL. rate[k] is the relaxation rate of moment k. */
static void mrt_collide(const olat_t *L, const double *f, const double *feq,
                        const double *R, const double *C, const double *Cp,
                        const double *rate, double *fout)
{
    int Q = L->Q;
    double m[QMAX], meq[QMAX], mR[QMAX], mC[QMAX], mCp[QMAX], ms[QMAX];
    for (int k = 0; k < Q; k++) {
        m[k] = meq[k] = mR[k] = mC[k] = mCp[k] = 0.0;
        for (int n = 0; n < Q; n++) {
            double Mkn = L->M[k * Q + n];
            m[k] += Mkn * f[n];
            meq[k] += Mkn * feq[n];
            if (R)
                mR[k] += Mkn * R[n];
            if (C)
                mC[k] += Mkn * C[n];
            if (Cp)
                mCp[k] += Mkn * Cp[n];
        }
    }
    for (int k = 0; k < Q; k++)
        ms[k] = m[k] - rate[k] * (m[k] - meq[k]) + (1.0 - 0.5 * rate[k]) * mR[k] + mC[k] +
                0.5 * (mC[k] - mCp[k]);
    for (int n = 0; n < Q; n++) {
        double acc = 0.0;
        for (int k = 0; k < Q; k++)
            acc += L->Minv[n * Q + k] * ms[k];
        fout[n] = acc;
    }
}

/* Pull streaming with halfway bounce-back at solid links; solid nodes hold 0. */
static void stream_pull(const oprm_t *p, const olat_t *L, const ost_t *s,
                        const double *post, double *fnew)
{
    long N = (long)p->nx * p->ny * p->nz;
    int Q = L->Q;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int n = 0; n < Q; n++) {
            if (s->solid[i]) {
                fnew[n * N + i] = 0.0;
                continue;
            }
            int back[3] = {-L->e[n][0], -L->e[n][1], -L->e[n][2]};
            long src = site_nbr(p, i, back);
            fnew[n * N + i] = s->solid[src] ? post[L->opp[n] * N + i] : post[n * N + src];
        }
    }
}

/* ------------------------------------------------------------------ one step */

/*
 * One coupled step n -> n+1. Lf: D2Q9/D3Q19 (g and the three phase fields),
 * Ls: D2Q5/D3Q7 (charge and the Poisson faces). Returns 0, or -1 if the Poisson
 * solve hit its iteration cap (the step is still completed).
 */
int oracle_step(const oprm_t *p, const olat_t *Lf, const olat_t *Ls, ost_t *s)
{
    long N = (long)p->nx * p->ny * p->nz;
    int Q = Lf->Q, QS = Ls->Q;
    double cs2 = Lf->cs2, cs2s = Ls->cs2, W = p->W;

    /* 1. Moments: Phi_i = sum_n f_Phi_i,n (Eq. 19); rho_e = sum_n f_rho,n;
     *    p* = sum_n g_n; j = sum_n g_n e_n (kept in u until the force is known). */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int c = 0; c < 3; c++)
            s->Phi[c * N + i] = 0.0;
        s->rho[i] = s->pstar[i] = 0.0;
        for (int a = 0; a < 3; a++)
            s->u[a * N + i] = 0.0;
        if (s->solid[i])
            continue;
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int n = 0; n < Q; n++)
                acc += s->fphi[((long)c * Q + n) * N + i];
            s->Phi[c * N + i] = acc;
        }
        double acc = 0.0;
        for (int n = 0; n < QS; n++)
            acc += s->frho[n * N + i];
        s->rho[i] = acc;
        double ps = 0.0, j[3] = {0, 0, 0};
        for (int n = 0; n < Q; n++) {
            double gn = s->g[n * N + i];
            ps += gn;
            for (int a = 0; a < 3; a++)
                j[a] += gn * Lf->e[n][a];
        }
        s->pstar[i] = ps;
        for (int a = 0; a < 3; a++)
            s->u[a * N + i] = j[a];
    }

    /* 2. Wetting ghosts (Eq. 20a) on boundary solid nodes, explicit in the fluid
     *    values at f = s + e_k: Phi_i(s) = Phi_i(f) - |e_k| * RHS_i(Phi(f)). */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        if (!s->solid[i] || s->normal[i] == 0)
            continue;
        const int *ek = Lf->e[s->normal[i]];
        long f = site_nbr(p, i, ek);
        double len = sqrt((double)(ek[0] * ek[0] + ek[1] * ek[1] + ek[2] * ek[2]));
        double P1 = s->Phi[f], P2 = s->Phi[N + f], P3 = s->Phi[2 * N + f];
        double c12 = 0.0, c13 = 0.0, c23 = 0.0;
        if (s->solid[i] == 1) {
            c12 = p->cos12;
            c13 = p->cos13;
            c23 = p->cos23;
        }
        double H1 = 4.0 / W * (-c13 * P1 * P3 - c12 * P1 * P2);
        double H2 = 4.0 / W * (c12 * P1 * P2 - c23 * P2 * P3);
        double H3 = 4.0 / W * (c23 * P2 * P3 + c13 * P1 * P3);
        s->Phi[i] = P1 - len * H1;
        s->Phi[N + i] = P2 - len * H2;
        s->Phi[2 * N + i] = P3 - len * H3;
    }

    /* 3. Phase-dependent properties, linear in Phi_i (Table 1 values per phase). */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        double e = 0.0, sg = 0.0;
        for (int c = 0; c < 3; c++) {
            e += s->Phi[c * N + i] * p->eps[c];
            sg += s->Phi[c * N + i] * p->sig[c];
        }
        s->eps[i] = e;
        s->sig[i] = sg;
    }

    /* 4. Isotropic gradient and Laplacian of Phi_i at fluid nodes:
     *    grad X = (1/cs2) sum w_n e_n X(x+e_n), lap X = (2/cs2) sum w_n (X(x+e_n)-X(x)). */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int c = 0; c < 3; c++) {
            s->lapPhi[c * N + i] = 0.0;
            for (int a = 0; a < 3; a++)
                s->gradPhi[(c * 3 + a) * N + i] = 0.0;
        }
        if (s->solid[i])
            continue;
        for (int n = 1; n < Q; n++) {
            long j = site_nbr(p, i, Lf->e[n]);
            for (int c = 0; c < 3; c++) {
                double X = s->Phi[c * N + j];
                for (int a = 0; a < 3; a++)
                    s->gradPhi[(c * 3 + a) * N + i] += Lf->w[n] * Lf->e[n][a] * X / cs2;
                s->lapPhi[c * N + i] += 2.0 / cs2 * Lf->w[n] * (X - s->Phi[c * N + i]);
            }
        }
    }

    /* 5. Chemical potential (Eq. 10, Upsilons from Eq. 11), capillary force
     *    F_s = sum_i mu_i grad Phi_i, and the AC sharpening flux F_Phi,i (Eq. 18). */
    double Y[3], YT;
    oracle_upsilon(p->gamma12, p->gamma13, p->gamma23, Y, &YT);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++)
            s->Fs[a * N + i] = 0.0;
        for (int c = 0; c < 3; c++) {
            s->mu[c * N + i] = 0.0;
            for (int a = 0; a < 3; a++)
                s->FPhi[(c * 3 + a) * N + i] = 0.0;
        }
        if (s->solid[i])
            continue;
        double P[3] = {s->Phi[i], s->Phi[N + i], s->Phi[2 * N + i]};
        double lam_n[3][3], sumsq = 0.0, J[3] = {0, 0, 0};
        for (int c = 0; c < 3; c++) {
            double mu = 24.0 * Y[c] / W * P[c] * (P[c] - 1.0) * (P[c] - 0.5) -
                        24.0 * YT / W * P[0] * P[1] * P[2] -
                        0.75 * Y[c] * W * s->lapPhi[c * N + i];
            s->mu[c * N + i] = mu;
            double gx = s->gradPhi[(c * 3 + 0) * N + i], gy = s->gradPhi[(c * 3 + 1) * N + i],
                   gz = s->gradPhi[(c * 3 + 2) * N + i];
            s->Fs[i] += mu * gx;
            s->Fs[N + i] += mu * gy;
            s->Fs[2 * N + i] += mu * gz;
            /* n = grad Phi / |grad Phi|, regularised as grad / sqrt(|grad|^2 + 1e-10) so
             * that it stays continuous where grad Phi vanishes (critical points of Phi) */
            double gn = sqrt(gx * gx + gy * gy + gz * gz + 1e-10);
            double lam = 4.0 / W * fabs(P[c] * (1.0 - P[c]));
            lam_n[c][0] = lam * gx / gn;
            lam_n[c][1] = lam * gy / gn;
            lam_n[c][2] = lam * gz / gn;
            for (int a = 0; a < 3; a++)
                J[a] += lam_n[c][a];
            sumsq += P[c] * P[c];
        }
        for (int c = 0; c < 3; c++)
            for (int a = 0; a < 3; a++)
                s->FPhi[(c * 3 + a) * N + i] = lam_n[c][a] - P[c] * P[c] / sumsq * J[a];
    }

    /* 6. Electric potential, Gauss law (Eq. 13). */
    int rc = oracle_poisson(p, Ls, s);

    /* 7. E = -grad phi (isotropic stencil; zero-flux solid neighbours mirror the
     *    node's own value, Dirichlet neighbours hold their value), grad eps from the
     *    eps field, electric force F_e = rho_e E - |E|^2 grad(eps) / 2 (Eq. 12).
     *    Total force F = F_s + F_e + body + Phi_1 body1: a uniform body force and one
     *    acting on the droplet phase alone (gravity on a droplet much denser than its
     *    surroundings, the sliding-droplet validation of the Methods). */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int a = 0; a < 3; a++)
            s->E[a * N + i] = s->Fe[a * N + i] = s->F[a * N + i] = 0.0;
        if (s->solid[i])
            continue;
        double gp[3] = {0, 0, 0}, ge[3] = {0, 0, 0};
        for (int n = 1; n < Q; n++) {
            long j = site_nbr(p, i, Lf->e[n]);
            double ph = s->pot[j];
            if (s->solid[j] && !is_dirichlet(s, j))
                ph = s->pot[i];
            for (int a = 0; a < 3; a++) {
                gp[a] += Lf->w[n] * Lf->e[n][a] * ph / cs2;
                ge[a] += Lf->w[n] * Lf->e[n][a] * s->eps[j] / cs2;
            }
        }
        double E2 = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
        for (int a = 0; a < 3; a++) {
            s->E[a * N + i] = -gp[a];
            s->Fe[a * N + i] = s->rho[i] * (-gp[a]) - 0.5 * E2 * ge[a];
            s->F[a * N + i] = s->Fs[a * N + i] + s->Fe[a * N + i] + p->body[a] +
                              s->Phi[i] * p->body1[a];
        }
    }

    /* 8. Velocity u = j + F/2 (unit reference density; with var_density,
     *    u = (j + F/2) / rho), and the conduction source Q = div(sigma grad phi) of
     *    Eq. 14 with zero flux through every solid face. */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        s->qsrc[i] = 0.0;
        if (s->solid[i])
            continue;
        double dens = 1.0;
        if (p->var_density)
            dens = s->Phi[i] * p->rhoph[0] + s->Phi[N + i] * p->rhoph[1] +
                   s->Phi[2 * N + i] * p->rhoph[2];
        for (int a = 0; a < 3; a++)
            s->u[a * N + i] = (s->u[a * N + i] + 0.5 * s->F[a * N + i]) / dens;
        double q = 0.0;
        for (int n = 1; n < QS; n++) {
            long j = site_nbr(p, i, Ls->e[n]);
            if (s->solid[j])
                continue;
            q += 0.5 * (s->sig[i] + s->sig[j]) * (s->pot[j] - s->pot[i]);
        }
        s->qsrc[i] = q;
    }

    /* Backward differences are zero on the first step. */
    if (!s->have_prev) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++) {
            for (int c = 0; c < 3; c++)
                for (int a = 0; a < 3; a++)
                    s->phiu_prev[(c * 3 + a) * N + i] = s->Phi[c * N + i] * s->u[a * N + i];
            for (int a = 0; a < 3; a++)
                s->rhou_prev[a * N + i] = s->rho[i] * s->u[a * N + i];
            s->q_prev[i] = s->qsrc[i];
        }
        s->have_prev = 1;
    }

    /* 9a. Momentum populations: incompressible equilibrium, Guo-type force term
     *     R_g, raw-moment MRT (second momentum-collision equation of the Methods); or,
     *     with var_density, the pressure-based scheme (header) with one relaxation time. */
    double tau_phi = 0.5 + p->mobility / cs2;
    double tau_rho = 0.5 + p->alpha / cs2s;
    if (p->var_density) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++) {
            if (s->solid[i]) {
                for (int n = 0; n < Q; n++)
                    s->post[n * N + i] = 0.0;
                continue;
            }
            double u[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
            double F[3] = {s->F[i], s->F[N + i], s->F[2 * N + i]};
            double dens = 0.0, nu = 0.0, gr[3] = {0, 0, 0};
            for (int c = 0; c < 3; c++) {
                dens += s->Phi[c * N + i] * p->rhoph[c];
                nu += s->Phi[c * N + i] * p->nu[c];
                for (int a = 0; a < 3; a++)
                    gr[a] += p->rhoph[c] * s->gradPhi[(c * 3 + a) * N + i];
            }
            double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            double sn[QMAX];
            for (int n = 0; n < Q; n++) {
                const int *e = Lf->e[n];
                double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
                sn[n] = Lf->w[n] * (eu / cs2 + eu * eu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
            }
            double gsum = 0.0;
            for (int n = 1; n < Q; n++)
                gsum += s->g[n * N + i];
            double ugr = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
            double pr = cs2 / (1.0 - Lf->w[0]) * (gsum + 0.5 * ugr + dens * sn[0]);
            s->pstar[i] = pr;
            double tau = 0.5 + nu / cs2;
            for (int n = 0; n < Q; n++) {
                const int *e = Lf->e[n];
                double geq = (n == 0 ? Lf->w[0] - 1.0 : Lf->w[n]) * pr / cs2 + dens * sn[n];
                double G = 0.0;
                for (int a = 0; a < 3; a++)
                    G += (e[a] - u[a]) * ((Lf->w[n] + sn[n]) * F[a] + sn[n] * cs2 * gr[a]);
                G /= cs2;
                double gn = s->g[n * N + i];
                s->post[n * N + i] = gn - (gn - geq) / tau + (1.0 - 0.5 / tau) * G;
            }
        }
        stream_pull(p, Lf, s, s->post, s->g);
    }
    if (!p->var_density) {
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) {
            for (int n = 0; n < Q; n++)
                s->post[n * N + i] = 0.0;
            continue;
        }
        double u[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
        double F[3] = {s->F[i], s->F[N + i], s->F[2 * N + i]};
        double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        double nu = 0.0;
        for (int c = 0; c < 3; c++)
            nu += s->Phi[c * N + i] * p->nu[c];
        double s_nu = 1.0 / (nu / cs2 + 0.5);
        double f[QMAX], feq[QMAX], R[QMAX], rate[QMAX], out[QMAX];
        for (int n = 0; n < Q; n++) {
            const int *e = Lf->e[n];
            double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
            double eF = e[0] * F[0] + e[1] * F[1] + e[2] * F[2];
            double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
            f[n] = s->g[n * N + i];
            feq[n] = Lf->w[n] * (s->pstar[i] + eu / cs2 + eu * eu / (2.0 * cs2 * cs2) -
                                 uu / (2.0 * cs2));
            R[n] = Lf->w[n] * ((eF - uF) / cs2 + eu * eF / (cs2 * cs2));
        }
        for (int k = 0; k < Q; k++) {
            int rcl = Lf->rowclass[k];
            rate[k] = rcl <= 1 ? 0.0 : rcl == 2 ? p->s_bulk : rcl == 3 ? s_nu : 1.0;
        }
        mrt_collide(Lf, f, feq, R, NULL, NULL, rate, out);
        for (int n = 0; n < Q; n++)
            s->post[n * N + i] = out[n];
    }
    /* Streaming writes into the population array itself (post is a copy). */
    stream_pull(p, Lf, s, s->post, s->g);
    }

    /* 9b. Phase-field populations (Eqs. 15-17) for the three components. */
    for (int c = 0; c < 3; c++) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < N; i++) {
            if (s->solid[i]) {
                for (int n = 0; n < Q; n++)
                    s->post[n * N + i] = 0.0;
                continue;
            }
            double P = s->Phi[c * N + i];
            double u[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
            double A[3];
            for (int a = 0; a < 3; a++)
                A[a] = cs2 * s->FPhi[(c * 3 + a) * N + i] +
                       (P * u[a] - s->phiu_prev[(c * 3 + a) * N + i]);
            double f[QMAX], feq[QMAX], C[QMAX], rate[QMAX], out[QMAX];
            for (int n = 0; n < Q; n++) {
                const int *e = Lf->e[n];
                double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
                double eA = e[0] * A[0] + e[1] * A[1] + e[2] * A[2];
                f[n] = s->fphi[((long)c * Q + n) * N + i];
                feq[n] = P * Lf->w[n] * (1.0 + eu / cs2);
                C[n] = Lf->w[n] / cs2 * eA;
            }
            for (int k = 0; k < Q; k++) {
                int rcl = Lf->rowclass[k];
                rate[k] = rcl == 0 ? 0.0 : rcl == 1 ? 1.0 / tau_phi : 1.0;
            }
            /* Eq. 15 applies (I - S/2) to M C. */
            mrt_collide(Lf, f, feq, C, NULL, NULL, rate, out);
            for (int n = 0; n < Q; n++)
                s->post[n * N + i] = out[n];
        }
        stream_pull(p, Lf, s, s->post, s->fphi + (long)c * Q * N);
    }

    /* 9c. Charge populations (charge-collision equation of the Methods, Eq. 20b):
     *     advection-diffusion with diffusivity alpha, force-like term R for d(rho u)/dt
     *     and conduction source C with its 0.5 dC/dt correction. */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        if (s->solid[i]) {
            for (int n = 0; n < QS; n++)
                s->post[n * N + i] = 0.0;
            continue;
        }
        double r = s->rho[i];
        double u[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
        double D[3];
        for (int a = 0; a < 3; a++)
            D[a] = r * u[a] - s->rhou_prev[a * N + i];
        double f[QMAX], feq[QMAX], R[QMAX], C[QMAX], Cp[QMAX], rate[QMAX], out[QMAX];
        for (int n = 0; n < QS; n++) {
            const int *e = Ls->e[n];
            double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
            double eD = e[0] * D[0] + e[1] * D[1] + e[2] * D[2];
            f[n] = s->frho[n * N + i];
            feq[n] = r * Ls->w[n] * (1.0 + eu / cs2s);
            R[n] = Ls->w[n] / cs2s * eD;
            C[n] = Ls->w[n] * s->qsrc[i];
            Cp[n] = Ls->w[n] * s->q_prev[i];
        }
        for (int k = 0; k < QS; k++) {
            int rcl = Ls->rowclass[k];
            rate[k] = rcl == 0 ? 0.0 : rcl == 1 ? 1.0 / tau_rho : 1.0;
        }
        mrt_collide(Ls, f, feq, R, C, Cp, rate, out);
        for (int n = 0; n < QS; n++)
            s->post[n * N + i] = out[n];
    }
    stream_pull(p, Ls, s, s->post, s->frho);

    /* 10. Products kept for the next step's backward differences. */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; i++) {
        for (int c = 0; c < 3; c++)
            for (int a = 0; a < 3; a++)
                s->phiu_prev[(c * 3 + a) * N + i] = s->Phi[c * N + i] * s->u[a * N + i];
        for (int a = 0; a < 3; a++)
            s->rhou_prev[a * N + i] = s->rho[i] * s->u[a * N + i];
        s->q_prev[i] = s->qsrc[i];
    }
    return rc;
}

/* ------------------------------------------------------------------ threads */
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

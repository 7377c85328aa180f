// adjoint.cuh -- discrete adjoint of the coupled step: the vector-Jacobian product of one
// step n -> n+1, in FP32, for gradients of a droplet observable with respect to the
// electrode potentials (the programmable switching of the Results).
//
// The forward state of step n is S^n = (g, f_Phi, f_rho at time n; Phi^{n-1}, rho^{n-1},
// u^{n-1}, Q^{n-1}), the fields the step reads besides its populations. The adjoint state
// lambda^n has the same layout. One reversed step takes lambda^{n+1} (and, for the last step,
// the loss seed on Phi^n) and produces lambda^n and this step's dL/dV, in five kernels:
//
//   k_adj_collide   at each fluid site: the reverse of collide_site. Reverse push-streaming
//                   gathers the adjoints of the 83 post-collision populations. The three
//                   collisions, the velocity, the forces (Eqs. 10-12), the sharpening flux
//                   (Eq. 18) and the chemical potential are then differentiated back to the
//                   site's populations, its own fields and the previous-step fields. The
//                   adjoints of the stencil sums (grad Phi, the Laplacian sums, grad phi,
//                   the conduction source) are written as a 16-float record per site.
//   k_adj_gather    at each site: the adjoints of Phi_i and phi from the records of the
//                   sites whose stencils read it (a gather, so no atomics).
//   (Poisson)       the adjoint Gauss-law solve A mu = phi_bar with the same symmetric
//                   operator (the forward's preconditioned CG).
//   k_adj_fields    at each fluid site: phi_bar -> rho_bar (mu) and eps_bar (the operator's
//                   dependence on eps), the wetting ghosts' Jacobians (Eq. 20a) back to their
//                   fluid sources, the next step's adjoints of Phi^n and rho^n, and the loss
//                   seed; then the moments (Eq. 19) give lambda of f_Phi and f_rho.
//   k_adj_vgrad     dL/dV of this step: the Dirichlet nodes' own phi_bar plus the operator's
//                   dependence on the Dirichlet values.
//
// Every formula is the derivative of the corresponding forward formula in kernels.cuh,
// term by term; the first step, where the backward differences are zero by definition,
// contributes no derivative through them.
#pragma once

#include "kernels.cuh"
#include "poisson.cuh"

namespace lbehd {

constexpr int ADJ_REC = 16;   // per-site record: gP_bar[9], sP_bar[3], gpot_bar[3], q_bar

// Forward arrays of step n (as stored by the forward replay) and the fields recomputed
// from them by k_fields.
struct AdjFwd {
    const float *g, *fphi, *frho;              // populations at time n
    const float *phi_prev, *rho_prev;          // Phi^{n-1}, rho^{n-1}
    const float *u_prev, *q_prev;              // u^{n-1}, Q^{n-1}
    const float *phi, *rho, *eps;              // Phi^n (with ghosts), rho^n, eps^n
    const float *pot, *pot_lo;                 // phi^n as hi + lo
    const uint8_t *info, *normal;
};

// Adjoint arrays.
struct AdjBuf {
    const float *lg_in, *lf_in, *lr_in;        // lambda of the populations at n + 1
    const float *lup_in, *lqp_in;              // lambda of u^n, Q^n (prev fields of n + 1)
    const float *lPp_in, *lrp_in;              // lambda of Phi^n, rho^n (prev fields of n + 1)
    float *lg_out, *lf_out, *lr_out;           // lambda of the populations at n
    float *lPp_out, *lrp_out, *lup_out, *lqp_out;   // lambda of Phi^{n-1}, rho^{n-1}, u^{n-1}, Q^{n-1}
    float *rec;                                // [ADJ_REC][N]
    float *jb;                                 // [12][N]: adjoints of the first moments of
                                               // f_Phi_1..3 (3 x 3) and f_rho (3)
    float *loc;                                // [5][N]: Phi_bar (3), rho_bar, phi_bar (site's own)
    float *phibar;                             // [3][N] gathered Phi_bar
    float *potbar;                             // [N] gathered phi_bar
    const float *mu;                           // [N] adjoint potential
    const float *seed;                         // [3][N] dL/dPhi^n of the loss (or null)
};

template <class L>
__device__ __forceinline__ float edot(int n, const float (&v)[3])
{
    return (L::ex(n) ? (L::ex(n) > 0 ? v[0] : -v[0]) : 0.f) +
           (L::ey(n) ? (L::ey(n) > 0 ? v[1] : -v[1]) : 0.f) +
           (L::ez(n) ? (L::ez(n) > 0 ? v[2] : -v[2]) : 0.f);
}

template <class L>
__device__ __forceinline__ void eacc(int n, float s, float (&v)[3])
{
    if (L::ex(n))
        v[0] += L::ex(n) > 0 ? s : -s;
    if (L::ey(n))
        v[1] += L::ey(n) > 0 ? s : -s;
    if (L::ez(n))
        v[2] += L::ez(n) > 0 ? s : -s;
}

// ---------------------------------------------------------------- reverse collide

template <int D>
__device__ void adj_collide_site(const Params &P, const AdjFwd &Fw, const AdjBuf &A, int first,
                                 int x, int y, int z)
{
    using L = Lat<D>;
    constexpr int Q = L::Q, QS = L::QS;
    const int N = (int)P.N;
    const int i = x + P.nx * (y + P.ny * z);
    const int nx = P.nx, nxy = P.nx * P.ny;
    const int oxp = x + 1 == P.nx ? 1 - P.nx : 1, oxm = x == 0 ? P.nx - 1 : -1;
    const int oyp = (y + 1 == P.ny ? 1 - P.ny : 1) * nx, oym = (y == 0 ? P.ny - 1 : -1) * nx;
    const int ozp = (z + 1 == P.nz ? 1 - P.nz : 1) * nxy, ozm = (z == 0 ? P.nz - 1 : -1) * nxy;
    auto off = [&](int n) -> int {
        return (L::ex(n) > 0 ? oxp : (L::ex(n) < 0 ? oxm : 0)) +
               (L::ey(n) > 0 ? oyp : (L::ey(n) < 0 ? oym : 0)) +
               (L::ez(n) > 0 ? ozp : (L::ez(n) < 0 ? ozm : 0));
    };
    constexpr float inv_cs2 = 3.0f;
    constexpr float wmov = 1.0f - L::w(0);

    // ================= forward recomputation (as in collide_site)
    float Pc[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        Pc[c] = Fw.phi[c * N + i];
    const float pot_i = Fw.pot[i], lo_i = Fw.pot_lo[i];
    const float sig_i = Pc[0] * P.sig[0] + Pc[1] * P.sig[1] + Pc[2] * P.sig[2];
    float gP[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float sP[3] = {0.f, 0.f, 0.f}, gpot[3] = {0.f, 0.f, 0.f};
    float qsrc = 0.0f, Sg_self[3] = {0.f, 0.f, 0.f}, Sq_self = 0.0f, Sq_dph = 0.0f;
    unsigned fluid_nb = 1u;
#pragma unroll
    for (int n = 1; n < Q; n++) {
        const int j = i + off(n);
        const float wn = L::w(n);
        const int pt = Fw.info[j] & 3;
        float Pn[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            Pn[c] = Fw.phi[c * N + j];
            sP[c] += wn * Pn[c];
            if (L::ex(n))
                gP[c][0] += (L::ex(n) > 0 ? wn : -wn) * Pn[c];
            if (L::ey(n))
                gP[c][1] += (L::ey(n) > 0 ? wn : -wn) * Pn[c];
            if (L::ez(n))
                gP[c][2] += (L::ez(n) > 0 ? wn : -wn) * Pn[c];
        }
        const float dph = pt == PT_NEUMANN ? 0.0f : (Fw.pot[j] - pot_i) + (Fw.pot_lo[j] - lo_i);
        if (pt != PT_NEUMANN)
            eacc<L>(n, wn, Sg_self);
        eacc<L>(n, wn * dph, gpot);
        if (pt == PT_FLUID) {
            fluid_nb |= 1u << n;
            if (n <= 2 * D) {
                const float sig_j = Pn[0] * P.sig[0] + Pn[1] * P.sig[1] + Pn[2] * P.sig[2];
                qsrc += 0.5f * (sig_i + sig_j) * dph;
                Sq_self += 0.5f * (sig_i + sig_j);
                Sq_dph += 0.5f * dph;
            }
        }
    }
    float lP[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        lP[c] = 2.0f * inv_cs2 * (sP[c] - wmov * Pc[c]);
#pragma unroll
        for (int a = 0; a < 3; a++)
            gP[c][a] *= inv_cs2;
    }
    const float W = P.W;
    const float ktri = 24.0f * P.YT / W;
    const float tri = ktri * Pc[0] * Pc[1] * Pc[2];
    float mu[3], Fs[3] = {0.f, 0.f, 0.f}, geps[3], E[3], E2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        mu[c] = 24.0f * P.Y[c] / W * Pc[c] * (Pc[c] - 1.0f) * (Pc[c] - 0.5f) - tri -
                0.75f * P.Y[c] * W * lP[c];
#pragma unroll
        for (int a = 0; a < 3; a++)
            Fs[a] += mu[c] * gP[c][a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        geps[a] = P.eps[0] * gP[0][a] + P.eps[1] * gP[1][a] + P.eps[2] * gP[2][a];
        E[a] = -inv_cs2 * gpot[a];
        E2 += E[a] * E[a];
    }
    const float rho = Fw.rho[i];
    float Fe[3], F[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        Fe[a] = rho * E[a] - 0.5f * E2 * geps[a];
        F[a] = Fs[a] + Fe[a] + P.body[a] + Pc[0] * P.body1[a];
    }
    float gn[3], lam[3], ln[3][3], J[3] = {0.f, 0.f, 0.f}, sumsq = 0.0f, FPhi[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        gn[c] = sqrtf(gP[c][0] * gP[c][0] + gP[c][1] * gP[c][1] + gP[c][2] * gP[c][2] + 1e-10f);
        lam[c] = 4.0f / W * fabsf(Pc[c] * (1.0f - Pc[c])) / gn[c];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ln[c][a] = lam[c] * gP[c][a];
            J[a] += ln[c][a];
        }
        sumsq += Pc[c] * Pc[c];
    }
    const float inv_sumsq = 1.0f / sumsq;
    float rr[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        rr[c] = Pc[c] * Pc[c] * inv_sumsq;
#pragma unroll
        for (int a = 0; a < 3; a++)
            FPhi[c][a] = ln[c][a] - rr[c] * J[a];
    }
    float gs[Q], dp = 0.0f, jm[3] = {0.f, 0.f, 0.f};
    float m2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int n = 0; n < Q; n++) {
        const float v = Fw.g[n * N + i];
        gs[n] = v;
        dp += v;
        eacc<L>(n, v, jm);
        if (L::ex(n))
            m2[0] += v;
        if (L::ey(n))
            m2[1] += v;
        if (L::ez(n))
            m2[2] += v;
        if (L::ex(n) && L::ey(n))
            m2[3] += L::ex(n) * L::ey(n) > 0 ? v : -v;
        if (L::ex(n) && L::ez(n))
            m2[4] += L::ex(n) * L::ez(n) > 0 ? v : -v;
        if (L::ey(n) && L::ez(n))
            m2[5] += L::ey(n) * L::ez(n) > 0 ? v : -v;
    }
    float u[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        u[a] = jm[a] + 0.5f * F[a];
    float uo[3], Po[3], rho_o = 0.0f, q_o = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        uo[a] = first ? 0.0f : Fw.u_prev[a * N + i];
        Po[a] = first ? 0.0f : Fw.phi_prev[a * N + i];
    }
    if (!first) {
        rho_o = Fw.rho_prev[i];
        q_o = Fw.q_prev[i];
    }
    (void)q_o;

    // ================= adjoints of the outputs (reverse push streaming)
    auto post_bar = [&](const float *lam_in, int n) -> float {
        const bool fl = (fluid_nb >> n) & 1u;
        const int slot = fl ? n : opposite(n);
        const int site = fl ? i + off(n) : i;
        return lam_in[(size_t)slot * N + site];
    };
    float ub[3], Fb[3] = {0.f, 0.f, 0.f}, Pcb[3] = {0.f, 0.f, 0.f};
    float rhob = 0.0f, qb = A.lqp_in[i];
#pragma unroll
    for (int a = 0; a < 3; a++)
        ub[a] = A.lup_in[a * N + i];
    float Pob[3] = {0.f, 0.f, 0.f}, uob[3] = {0.f, 0.f, 0.f}, rhoob = 0.0f, qob = 0.0f;
    float FPhib[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};

    // ---- momentum collision
    float gsb[Q];
    {
        const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const float nu = Pc[0] * P.nu[0] + Pc[1] * P.nu[1] + Pc[2] * P.nu[2];
        const float den = inv_cs2 * nu + 0.5f;
        const float c_nu = 1.0f - 1.0f / den;
        const float c_b = 1.0f - P.s_bulk;
        const float b0 = post_bar(A.lg_in, 0);   // rest: dp - sum_{n>=1} v_n
        float C0b = 0.0f, Vb[3] = {0.f, 0.f, 0.f}, c_nub = 0.0f;
        float d1b = 0.f, d2b = 0.f, dxyb = 0.f, dxzb = 0.f, dyzb = 0.f, dTb = 0.f, dpb = b0;
        const float d1 = (m2[0] - m2[1]) - (u[0] * u[0] - u[1] * u[1]) + (u[0] * F[0] - u[1] * F[1]);
        const float d2 = (m2[0] - m2[2]) - (u[0] * u[0] - u[2] * u[2]) + (u[0] * F[0] - u[2] * F[2]);
        const float dxy = m2[3] - u[0] * u[1] + 0.5f * (u[0] * F[1] + u[1] * F[0]);
        const float dxz = m2[4] - u[0] * u[2] + 0.5f * (u[0] * F[2] + u[2] * F[0]);
        const float dyz = m2[5] - u[1] * u[2] + 0.5f * (u[1] * F[2] + u[2] * F[1]);
#pragma unroll
        for (int n = 1; n < Q; n++) {
            const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
            const int e2 = cx * cx + cy * cy + cz * cz;
            const float an = post_bar(A.lg_in, n) - b0;
            const float eu = edot<L>(n, u), eF = edot<L>(n, F);
            const float wn = L::w(n);
            C0b += wn * an;
            eacc<L>(n, wn * an, Vb);
            eacc<L>(n, an * wn * (9.0f * eu + 4.5f * eF), ub);
            eacc<L>(n, an * wn * 4.5f * eu, Fb);
            float corr = 0.0f;
            if (D == 3) {
                if (e2 == 1) {
                    float k1, k2;
                    if (cx) {
                        k1 = 1.0f / 6.0f;
                        k2 = 1.0f / 6.0f;
                    } else if (cy) {
                        k1 = -1.0f / 3.0f;
                        k2 = 1.0f / 6.0f;
                    } else {
                        k1 = 1.0f / 6.0f;
                        k2 = -1.0f / 3.0f;
                    }
                    corr = k1 * d1 + k2 * d2;
                    d1b += c_nu * an * k1;
                    d2b += c_nu * an * k2;
                    dTb += c_b * an * (1.0f / 6.0f);
                } else {
                    corr = 0.25f * (cx * cy * dxy + cx * cz * dxz + cy * cz * dyz);
                    dxyb += c_nu * an * 0.25f * cx * cy;
                    dxzb += c_nu * an * 0.25f * cx * cz;
                    dyzb += c_nu * an * 0.25f * cy * cz;
                }
            } else {
                if (e2 == 1) {
                    const float k1 = cx ? 0.25f : -0.25f;
                    corr = k1 * d1;
                    d1b += c_nu * an * k1;
                    dTb += c_b * an * 0.25f;
                } else {
                    corr = 0.25f * cx * cy * dxy;
                    dxyb += c_nu * an * 0.25f * cx * cy;
                }
            }
            c_nub += an * corr;
        }
        // d's -> m2, u, F, dp
        float m2b[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        m2b[0] += d1b + d2b + dTb;
        m2b[1] += -d1b + dTb;
        m2b[2] += -d2b + (D == 3 ? dTb : 0.0f);
        m2b[3] += dxyb;
        m2b[4] += dxzb;
        m2b[5] += dyzb;
        ub[0] += (d1b + d2b) * (F[0] - 2.0f * u[0]);
        ub[1] += d1b * (2.0f * u[1] - F[1]);
        ub[2] += d2b * (2.0f * u[2] - F[2]);
        Fb[0] += (d1b + d2b) * u[0];
        Fb[1] += -d1b * u[1];
        Fb[2] += -d2b * u[2];
        ub[0] += -dxyb * (u[1] - 0.5f * F[1]) - dxzb * (u[2] - 0.5f * F[2]);
        ub[1] += -dxyb * (u[0] - 0.5f * F[0]) - dyzb * (u[2] - 0.5f * F[2]);
        ub[2] += -dxzb * (u[0] - 0.5f * F[0]) - dyzb * (u[1] - 0.5f * F[1]);
        Fb[0] += 0.5f * (dxyb * u[1] + dxzb * u[2]);
        Fb[1] += 0.5f * (dxyb * u[0] + dyzb * u[2]);
        Fb[2] += 0.5f * (dxzb * u[0] + dyzb * u[1]);
        dpb += -(float)D * (1.0f / 3.0f) * dTb;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ub[a] += dTb * (F[a] - 2.0f * u[a]);
            Fb[a] += dTb * u[a];
        }
        // c_nu = 1 - 1/(3 nu + 0.5)
        const float nub = c_nub * inv_cs2 / (den * den);
#pragma unroll
        for (int c = 0; c < 3; c++)
            Pcb[c] += nub * P.nu[c];
        // C0 = dp - 1.5 uu - 1.5 uF; V = 3u + 1.5F
        dpb += C0b;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ub[a] += -C0b * (3.0f * u[a] + 1.5f * F[a]) + 3.0f * Vb[a];
            Fb[a] += -1.5f * C0b * u[a] + 1.5f * Vb[a];
        }
        (void)uu;
        // moments of gs: dp, jm (= u - F/2, back-propagated below with the full u_bar), m2
#pragma unroll
        for (int n = 0; n < Q; n++) {
            float v = dpb;
            if (L::ex(n))
                v += m2b[0];
            if (L::ey(n))
                v += m2b[1];
            if (L::ez(n))
                v += m2b[2];
            if (L::ex(n) && L::ey(n))
                v += L::ex(n) * L::ey(n) > 0 ? m2b[3] : -m2b[3];
            if (L::ex(n) && L::ez(n))
                v += L::ex(n) * L::ez(n) > 0 ? m2b[4] : -m2b[4];
            if (L::ey(n) && L::ez(n))
                v += L::ey(n) * L::ez(n) > 0 ? m2b[5] : -m2b[5];
            gsb[n] = v;
        }
    }

    // ---- phase-field collisions
    const float c_phi = 1.0f - P.inv_tau_phi;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float *lin = A.lf_in + (size_t)c * Q * N;
        const float b0 = post_bar(lin, 0);   // rest: Pc - sum_{n>=1} v_n
        float Ppb = b0, Bb[3] = {0.f, 0.f, 0.f}, delb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int n = 1; n < Q; n++) {
            const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
            const float an = post_bar(lin, n) - b0;
            Ppb += L::w(n) * an;
            eacc<L>(n, L::w(n) * an, Bb);
            if (cx * cx + cy * cy + cz * cz == 1)
                eacc<L>(n, an, delb);
        }
        const float Pp = Pc[c];
        float jfb[3], Ab[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            // del = c_phi/2 (jf - Pp u + A/2), B = 3 Pp u + 1.5 A
            jfb[a] = 0.5f * c_phi * delb[a];
            Ppb += -0.5f * c_phi * delb[a] * u[a] + 3.0f * Bb[a] * u[a];
            ub[a] += -0.5f * c_phi * delb[a] * Pp + 3.0f * Bb[a] * Pp;
            Ab[a] = 0.25f * c_phi * delb[a] + 1.5f * Bb[a];
            // A = cs2 FPhi + (Pp u - Po uo); zero difference on the first step
            FPhib[c][a] += L::cs2 * Ab[a];
            if (!first) {
                Ppb += Ab[a] * u[a];
                ub[a] += Ab[a] * Pp;
                Pob[c] += -Ab[a] * uo[a];
                uob[a] += -Ab[a] * Po[c];
            }
        }
        Pcb[c] += Ppb;
        // jf = sum e_n f_n: lambda of f_Phi_c,n gets e_n . jfb (written by k_adj_fields)
#pragma unroll
        for (int a = 0; a < 3; a++)
            A.jb[(size_t)(3 * c + a) * N + i] = jfb[a];
    }

    // ---- charge collision
    {
        constexpr float inv_cs2s = 1.0f / L::cs2s;
        const float c_rho = 1.0f - P.inv_tau_rho;
        const float b0 = post_bar(A.lr_in, 0);   // rest: C0 - sum_{n>=1} v_n
        float C0b = b0, Bb[3] = {0.f, 0.f, 0.f}, delb[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int n = 1; n < QS; n++) {
            const float an = post_bar(A.lr_in, n) - b0;
            C0b += L::ws(n) * an;
            eacc<L>(n, L::ws(n) * an, Bb);
            eacc<L>(n, an, delb);
        }
        // C0 = rho + qsrc + (qsrc - q_o) / 2
        rhob += C0b;
        if (first) {
            qb += C0b;
        } else {
            qb += 1.5f * C0b;
            qob += -0.5f * C0b;
        }
        float jrb[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            // del = c_rho/2 (jr - rho u + Dm/2), B = inv_cs2s (rho u + Dm/2)
            jrb[a] = 0.5f * c_rho * delb[a];
            rhob += -0.5f * c_rho * delb[a] * u[a] + inv_cs2s * Bb[a] * u[a];
            ub[a] += -0.5f * c_rho * delb[a] * rho + inv_cs2s * Bb[a] * rho;
            const float Dmb = 0.25f * c_rho * delb[a] + 0.5f * inv_cs2s * Bb[a];
            if (!first) {
                // Dm = rho u - rho_o uo
                rhob += Dmb * u[a];
                ub[a] += Dmb * rho;
                rhoob += -Dmb * uo[a];
                uob[a] += -Dmb * rho_o;
            }
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
            A.jb[(size_t)(9 + a) * N + i] = jrb[a];
    }

    // ---- u = jm + F/2 (ub is now complete)
#pragma unroll
    for (int a = 0; a < 3; a++)
        Fb[a] += 0.5f * ub[a];
#pragma unroll
    for (int n = 0; n < Q; n++)
        A.lg_out[(size_t)n * N + i] = gsb[n] + edot<L>(n, ub);

    // ---- forces: F = Fs + Fe + body + Phi_1 body1; Fe = rho E - E2 geps / 2;
    //      Fs = sum mu_c gP_c
    float gPb[3][3], gpotb[3], gepsb[3], Eb[3], E2b = 0.0f, mub[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        Pcb[0] += Fb[a] * P.body1[a];
        rhob += Fb[a] * E[a];
        Eb[a] = Fb[a] * rho;
        E2b += -0.5f * Fb[a] * geps[a];
        gepsb[a] = -0.5f * E2 * Fb[a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        Eb[a] += 2.0f * E[a] * E2b;
        gpotb[a] = -inv_cs2 * Eb[a];
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
        mub[c] = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            mub[c] += Fb[a] * gP[c][a];
            gPb[c][a] = mu[c] * Fb[a] + P.eps[c] * gepsb[a];
        }
    }
    // mu_c = 24 Y_c/W Pc (Pc - 1)(Pc - 1/2) - tri - 3/4 Y_c W lP_c
    float trib = 0.0f, lPb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        Pcb[c] += mub[c] * 24.0f * P.Y[c] / W * (3.0f * Pc[c] * Pc[c] - 3.0f * Pc[c] + 0.5f);
        trib += -mub[c];
        lPb[c] = -0.75f * P.Y[c] * W * mub[c];
    }
    Pcb[0] += trib * ktri * Pc[1] * Pc[2];
    Pcb[1] += trib * ktri * Pc[0] * Pc[2];
    Pcb[2] += trib * ktri * Pc[0] * Pc[1];
    float sPb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        sPb[c] = 2.0f * inv_cs2 * lPb[c];
        Pcb[c] += -2.0f * inv_cs2 * wmov * lPb[c];
    }
    // ---- sharpening flux: FPhi_c = ln_c - r_c J, ln_c = lam_c gP_c, J = sum ln_c
    {
        float Jb[3] = {0.f, 0.f, 0.f}, lnb[3][3], rb[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            rb[c] = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                rb[c] += -FPhib[c][a] * J[a];
                Jb[a] += -rr[c] * FPhib[c][a];
            }
        }
        float sumsqb = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
#pragma unroll
            for (int a = 0; a < 3; a++)
                lnb[c][a] = FPhib[c][a] + Jb[a];
            // r_c = Pc^2 / sumsq
            Pcb[c] += rb[c] * 2.0f * Pc[c] * inv_sumsq;
            sumsqb += -rb[c] * Pc[c] * Pc[c] * inv_sumsq * inv_sumsq;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            Pcb[c] += 2.0f * Pc[c] * sumsqb;
            float lamb = 0.0f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                lamb += lnb[c][a] * gP[c][a];
                gPb[c][a] += lam[c] * lnb[c][a];
            }
            // lam = 4/W |s| / gn with s = Pc (1 - Pc)
            const float s = Pc[c] * (1.0f - Pc[c]);
            const float sg = s > 0.0f ? 1.0f : (s < 0.0f ? -1.0f : 0.0f);
            Pcb[c] += lamb * 4.0f / W * sg * (1.0f - 2.0f * Pc[c]) / gn[c];
            const float gnb = -lamb * lam[c] / gn[c];
#pragma unroll
            for (int a = 0; a < 3; a++)
                gPb[c][a] += gnb * gP[c][a] / gn[c];
        }
    }
    // ---- the conduction source's own-site terms: sig_i and -phi_i
#pragma unroll
    for (int c = 0; c < 3; c++)
        Pcb[c] += qb * Sq_dph * P.sig[c];
    float potb = -qb * Sq_self;
#pragma unroll
    for (int a = 0; a < 3; a++)
        potb += -gpotb[a] * Sg_self[a];

    // ---- records for the neighbours (gather pass) and the site's own adjoints
    float *rec = A.rec;
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int a = 0; a < 3; a++)
            rec[(size_t)(3 * c + a) * N + i] = gPb[c][a] * inv_cs2;   // d/d(raw weighted sum)
#pragma unroll
    for (int c = 0; c < 3; c++)
        rec[(size_t)(9 + c) * N + i] = sPb[c];
#pragma unroll
    for (int a = 0; a < 3; a++)
        rec[(size_t)(12 + a) * N + i] = gpotb[a];
    rec[(size_t)15 * N + i] = qb;
#pragma unroll
    for (int c = 0; c < 3; c++)
        A.loc[(size_t)c * N + i] = Pcb[c];
    A.loc[(size_t)3 * N + i] = rhob;
    A.loc[(size_t)4 * N + i] = potb;
#pragma unroll
    for (int c = 0; c < 3; c++)
        A.lPp_out[(size_t)c * N + i] = Pob[c];
    A.lrp_out[i] = rhoob;
#pragma unroll
    for (int a = 0; a < 3; a++)
        A.lup_out[(size_t)a * N + i] = uob[a];
    A.lqp_out[i] = qob;
}

template <int D>
__global__ void __launch_bounds__(BX) k_adj_collide(Params P, AdjFwd Fw, AdjBuf A, int first)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx)
        return;
    const int i = x + P.nx * (y + P.ny * z);
    const int N = (int)P.N;
    if ((Fw.info[i] & 3) == PT_FLUID) {
        adj_collide_site<D>(P, Fw, A, first, x, y, z);
        return;
    }
    // solid site: no populations, no stencil of its own (k_adj_fields zeroes f_Phi, f_rho)
    using L = Lat<D>;
#pragma unroll
    for (int n = 0; n < L::Q; n++)
        A.lg_out[(size_t)n * N + i] = 0.0f;
#pragma unroll
    for (int k = 0; k < ADJ_REC; k++)
        A.rec[(size_t)k * N + i] = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; k++)
        A.loc[(size_t)k * N + i] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        A.lPp_out[(size_t)c * N + i] = 0.0f;
        A.lup_out[(size_t)c * N + i] = 0.0f;
    }
    A.lrp_out[i] = 0.0f;
    A.lqp_out[i] = 0.0f;
}

// ---------------------------------------------------------------- gather

// Phi_bar and phi_bar at site y: its own terms plus, for every fluid site x = y - e_n, the
// terms of x's stencil sums that read y.
template <int D>
__global__ void __launch_bounds__(BX) k_adj_gather(Params P, AdjFwd Fw, AdjBuf A)
{
    using L = Lat<D>;
    const int x0 = blockIdx.x * blockDim.x + threadIdx.x, y0 = blockIdx.y, z0 = blockIdx.z;
    if (x0 >= P.nx)
        return;
    const int N = (int)P.N, nx = P.nx, ny = P.ny, nz = P.nz;
    const int i = x0 + nx * (y0 + ny * z0);
    const int pt_y = Fw.info[i] & 3;
    float Pb[3], potb;
#pragma unroll
    for (int c = 0; c < 3; c++)
        Pb[c] = A.loc[(size_t)c * N + i];
    potb = A.loc[(size_t)4 * N + i];
    float sig_y = 0.0f, phi_y = Fw.pot[i] + Fw.pot_lo[i];
#pragma unroll
    for (int c = 0; c < 3; c++)
        sig_y += Fw.phi[c * N + i] * P.sig[c];
#pragma unroll
    for (int n = 1; n < L::Q; n++) {
        // x = y - e_n reads y as its neighbour n
        int X = x0 - L::ex(n), Y = y0 - L::ey(n), Z = z0 - L::ez(n);
        X += X < 0 ? nx : (X >= nx ? -nx : 0);
        Y += Y < 0 ? ny : (Y >= ny ? -ny : 0);
        Z += Z < 0 ? nz : (Z >= nz ? -nz : 0);
        const int xs = X + nx * (Y + ny * Z);
        if ((Fw.info[xs] & 3) != PT_FLUID)
            continue;
        const float wn = L::w(n);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            float v = wn * A.rec[(size_t)(9 + c) * N + xs];
            if (L::ex(n))
                v += (L::ex(n) > 0 ? wn : -wn) * A.rec[(size_t)(3 * c + 0) * N + xs];
            if (L::ey(n))
                v += (L::ey(n) > 0 ? wn : -wn) * A.rec[(size_t)(3 * c + 1) * N + xs];
            if (L::ez(n))
                v += (L::ez(n) > 0 ? wn : -wn) * A.rec[(size_t)(3 * c + 2) * N + xs];
            Pb[c] += v;
        }
        if (pt_y != PT_NEUMANN) {
            float g = 0.0f;
            if (L::ex(n))
                g += (L::ex(n) > 0 ? wn : -wn) * A.rec[(size_t)12 * N + xs];
            if (L::ey(n))
                g += (L::ey(n) > 0 ? wn : -wn) * A.rec[(size_t)13 * N + xs];
            if (L::ez(n))
                g += (L::ez(n) > 0 ? wn : -wn) * A.rec[(size_t)14 * N + xs];
            potb += g;
        }
        if (pt_y == PT_FLUID && n <= 2 * D) {
            const float qb = A.rec[(size_t)15 * N + xs];
            float sig_x = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; c++)
                sig_x += Fw.phi[c * N + xs] * P.sig[c];
            const float dph = phi_y - (Fw.pot[xs] + Fw.pot_lo[xs]);
            potb += qb * 0.5f * (sig_x + sig_y);
#pragma unroll
            for (int c = 0; c < 3; c++)
                Pb[c] += qb * 0.5f * dph * P.sig[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
        A.phibar[(size_t)c * N + i] = Pb[c];
    A.potbar[i] = potb;
}

// ---------------------------------------------------------------- fields

struct AdjFieldsArgs {
    float cos12, cos13, cos23, s4;   // wetting coefficients, 4 / W
    float *rhs;                      // [N] Poisson adjoint right-hand side (fluid phi_bar)
};

// Right-hand side of the adjoint Gauss-law solve: phi_bar on the fluid nodes.
__global__ void __launch_bounds__(BX) k_adj_rhs(long long N, const uint8_t *__restrict__ info,
                                                const float *__restrict__ potbar,
                                                float *__restrict__ rhs)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        rhs[i] = (info[i] & 3) == PT_FLUID ? potbar[i] : 0.0f;
}

// lambda of the populations at n for every fluid site y.
template <int D>
__global__ void __launch_bounds__(BX) k_adj_fields(Params P, AdjFwd Fw, AdjBuf A,
                                                   AdjFieldsArgs W)
{
    using L = Lat<D>;
    using LS = Lat<D>;
    const int x0 = blockIdx.x * blockDim.x + threadIdx.x, y0 = blockIdx.y, z0 = blockIdx.z;
    if (x0 >= P.nx)
        return;
    const int N = (int)P.N, nx = P.nx, ny = P.ny, nz = P.nz;
    const int i = x0 + nx * (y0 + ny * z0);
    if ((Fw.info[i] & 3) != PT_FLUID) {
#pragma unroll
        for (int m = 0; m < 3 * L::Q; m++)
            A.lf_out[(size_t)m * N + i] = 0.0f;
#pragma unroll
        for (int n = 0; n < L::QS; n++)
            A.lr_out[(size_t)n * N + i] = 0.0f;
        return;
    }
    auto site = [&](int n, int sgn) {
        int X = x0 + sgn * L::ex(n), Y = y0 + sgn * L::ey(n), Z = z0 + sgn * L::ez(n);
        X += X < 0 ? nx : (X >= nx ? -nx : 0);
        Y += Y < 0 ? ny : (Y >= ny ? -ny : 0);
        Z += Z < 0 ? nz : (Z >= nz ? -nz : 0);
        return X + nx * (Y + ny * Z);
    };
    float Pb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        Pb[c] = A.phibar[(size_t)c * N + i] + A.lPp_in[(size_t)c * N + i];
        if (A.seed)
            Pb[c] += A.seed[(size_t)c * N + i];
    }
    // eps_bar: the operator of Eq. 13 depends on eps at the fluid nodes through the face
    // coefficients (eps_i + eps_j)/2 (fluid j) and eps_i (Dirichlet j)
    const float mu_i = A.mu[i], phi_i = Fw.pot[i] + Fw.pot_lo[i];
    float epsb = 0.0f, rhob = A.loc[(size_t)3 * N + i] + mu_i + A.lrp_in[i];
#pragma unroll
    for (int n = 1; n < LS::QS; n++) {
        const int j = site(n, 1);
        const int pt = Fw.info[j] & 3;
        const float dphi = phi_i - (Fw.pot[j] + Fw.pot_lo[j]);
        if (pt == PT_FLUID)
            epsb += -0.5f * dphi * (mu_i - A.mu[j]);
        else if (pt == PT_DIRICHLET)
            epsb += -mu_i * dphi;
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
        Pb[c] += epsb * P.eps[c];
    // wetting ghosts whose fluid source is this site: ghost s = y - e_k with normal k
    const float P1 = Fw.phi[i], P2 = Fw.phi[N + i], P3 = Fw.phi[2 * N + i];
#pragma unroll
    for (int k = 1; k < L::Q; k++) {
        const int s = site(k, -1);
        if ((Fw.info[s] & 3) == PT_FLUID || Fw.normal[s] != k)
            continue;
        float c12 = 0.0f, c13 = 0.0f, c23 = 0.0f;
        if (((Fw.info[s] >> 2) & 3) == 1) {
            c12 = W.cos12;
            c13 = W.cos13;
            c23 = W.cos23;
        }
        const int kx = L::ex(k), ky = L::ey(k), kz = L::ez(k);
        const float len = (kx * kx + ky * ky + kz * kz) == 2 ? 1.41421356237f : 1.0f;
        const float q = len * W.s4;
        const float g1 = A.phibar[s], g2 = A.phibar[(size_t)N + s], g3 = A.phibar[(size_t)2 * N + s];
        // ghost_c = P_c - len H_c(P); H as in k_fields
        Pb[0] += g1 - q * (g1 * (-c13 * P3 - c12 * P2) + g2 * (c12 * P2) + g3 * (c13 * P3));
        Pb[1] += g2 - q * (g1 * (-c12 * P1) + g2 * (c12 * P1 - c23 * P3) + g3 * (c23 * P3));
        Pb[2] += g3 - q * (g1 * (-c13 * P1) + g2 * (-c23 * P2) + g3 * (c23 * P2 + c13 * P1));
    }
    // moments: Phi_c = sum_n f_Phi_c,n, rho = sum_n f_rho,n; plus the collisions' first-moment
    // terms e_n . jb
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float jf[3] = {A.jb[(size_t)(3 * c) * N + i], A.jb[(size_t)(3 * c + 1) * N + i],
                             A.jb[(size_t)(3 * c + 2) * N + i]};
#pragma unroll
        for (int n = 0; n < L::Q; n++)
            A.lf_out[((size_t)c * L::Q + n) * N + i] = edot<L>(n, jf) + Pb[c];
    }
    {
        const float jr[3] = {A.jb[(size_t)9 * N + i], A.jb[(size_t)10 * N + i],
                             A.jb[(size_t)11 * N + i]};
#pragma unroll
        for (int n = 0; n < L::QS; n++)
            A.lr_out[(size_t)n * N + i] = edot<L>(n, jr) + rhob;
    }
}

// dL/dV of one step: sum over each electrode's Dirichlet nodes of their phi_bar, and of
// mu_i eps_i over the fluid faces touching them. grad[e] += (FP64).
constexpr int VGRAD_THREADS = 256;
template <int D>
__global__ void __launch_bounds__(VGRAD_THREADS) k_adj_vgrad(Params P, AdjFwd Fw, AdjBuf A,
                                                             const int16_t *__restrict__ elec,
                                                             int n_e, double *__restrict__ grad)
{
    using L = Lat<D>;
    __shared__ double acc[LBEHD_MAX_ELECTRODES];
    for (int e = threadIdx.x; e < n_e; e += blockDim.x)
        acc[e] = 0.0;
    __syncthreads();
    const int N = (int)P.N, nx = P.nx, ny = P.ny, nz = P.nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const int pt = Fw.info[i] & 3;
        if (pt == PT_DIRICHLET) {
            const int e = elec[i];
            if (e >= 0 && e < n_e)
                atomicAdd(&acc[e], (double)A.potbar[i]);
        } else if (pt == PT_FLUID) {
            const int x0 = i % nx, y0 = (i / nx) % ny, z0 = i / (nx * ny);
            const float t = A.mu[i] * Fw.eps[i];
#pragma unroll
            for (int n = 1; n < L::QS; n++) {
                int X = x0 + L::ex(n), Y = y0 + L::ey(n), Z = z0 + L::ez(n);
                X += X < 0 ? nx : (X >= nx ? -nx : 0);
                Y += Y < 0 ? ny : (Y >= ny ? -ny : 0);
                Z += Z < 0 ? nz : (Z >= nz ? -nz : 0);
                const int j = X + nx * (Y + ny * Z);
                if ((Fw.info[j] & 3) == PT_DIRICHLET) {
                    const int e = elec[j];
                    if (e >= 0 && e < n_e)
                        atomicAdd(&acc[e], (double)t);
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n_e; e += blockDim.x)
        if (acc[e] != 0.0)
            atomicAdd(&grad[e], acc[e]);
}

// Loss seed: L = x centroid of Phi_1 over the fluid nodes; dL/dPhi_1 = (x - x_c) / M1.
__global__ void __launch_bounds__(BX) k_adj_seed(Params P, const uint8_t *__restrict__ info,
                                                 double xc, double M1, float *__restrict__ seed)
{
    const int N = (int)P.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const bool fl = (info[i] & 3) == PT_FLUID;
        seed[i] = fl ? (float)(((double)(i % P.nx) - xc) / M1) : 0.0f;
        seed[N + i] = 0.0f;
        seed[2 * N + i] = 0.0f;
    }
}

constexpr double ADJ_POISSON_TOL = 1e-4;   // relative residual of the adjoint solves

// Start of the adjoint Gauss-law solve A mu = rhs from the warm start mu: r = rhs - A mu on
// the active cells, partials of ||r||^2 and ||rhs||^2 over blocks of BX consecutive sites.
template <int D>
__device__ __forceinline__ void adj_pcg_init_site(const MgDims &d, const float *eps,
                                                  const uint8_t *info, const float *Dg,
                                                  const float *mu, const float *rhs, float *r,
                                                  int i, float (&v)[2])
{
    int x, y, z;
    cell_xyz(d, i, x, y, z);
    float dummy[1] = {0.f};
    pcg_Ap_site<D>(d, eps, info, Dg, mu, r, x, y, z, dummy);   // r = A mu
    const float b = Dg[i] > 0.0f ? rhs[i] : 0.0f;
    const float ri = Dg[i] > 0.0f ? __fsub_rn(b, r[i]) : 0.0f;
    r[i] = ri;
    v[0] = __fmul_rn(ri, ri);
    v[1] = __fmul_rn(b, b);
}

template <int D>
__global__ void __launch_bounds__(BX) k_adj_pcg_init(MgDims d, const float *__restrict__ eps,
                                                     const uint8_t *__restrict__ info,
                                                     const float *__restrict__ Dg,
                                                     const float *__restrict__ mu,
                                                     const float *__restrict__ rhs,
                                                     float *__restrict__ r,
                                                     double *__restrict__ partials,
                                                     unsigned *zero = nullptr)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    if (zero && i == 0)   // the grid-barrier counter of the persistent solve that follows
        *zero = 0u;
    float v[2] = {0.f, 0.f};
    if (i < d.nx * d.ny * d.nz)
        adj_pcg_init_site<D>(d, eps, info, Dg, mu, rhs, r, i, v);
    block_partials<2>(v, partials);
}

// Warm start of the adjoint solve: mu = 2 mu1 - mu2 (linear extrapolation in time).
__global__ void __launch_bounds__(BX) k_adj_extrapolate(long long n, const float *__restrict__ mu1,
                                                        const float *__restrict__ mu2,
                                                        float *__restrict__ mu)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        mu[i] = __fmaf_rn(2.0f, mu1[i], -mu2[i]);
}

}  // namespace lbehd

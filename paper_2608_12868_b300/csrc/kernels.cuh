// kernels.cuh -- device kernels of the coupled LB-EHD step (sm_103a, FP32 state).
//
// One step n -> n+1 runs:
//   k_fields    Phi_i = sum_n f_Phi_i,n (Eq. 19), rho_e = sum f_rho, permittivity, wetting
//               ghosts on boundary solid nodes (Eq. 20a), Dirichlet potentials;
//   (poisson.cuh) the Gauss law solve, div(eps grad phi) = -rho_e (Eq. 13);
//   k_collide   per fluid site, everything else fused: isotropic stencils of Phi_i and phi,
//               chemical potential (Eqs. 10-11), capillary and electric forces (Eq. 12),
//               sharpening flux (Eq. 18), conduction source of Eq. 14, then collide and
//               push-stream the momentum, three phase-field (Eqs. 15-17) and charge
//               populations with halfway bounce-back, and block partial sums (FP64) of the
//               droplet observables;
//   k_obs_final_split  the deterministic FP64 sum of those partials (when they are read).
//
// The raw-moment MRT collisions are evaluated in closed form. With every moment of order
// >= 3 relaxing at rate 1 (and the trace of the momentum flux at s_bulk), M^-1 m* reduces
// to  f* = f_eq + C/2 + sum_k (1 - s_k) delta_k col_k,  where delta_k is moment k of
// f - f_eq + C/2 and col_k is column k of M^-1 (only the moments with s_k != 1 appear).
// The columns used, for the raw monomial basis with a trace / deviatoric second-order
// block:
//   first order e_a          : +1/2 on +a, -1/2 on -a
//   3D  ex^2 - ey^2          : 1/6 on +-x, -1/3 on +-y, 1/6 on +-z
//   3D  ex^2 - ez^2          : 1/6 on +-x, 1/6 on +-y, -1/3 on +-z
//   3D  trace e^2            : 1/6 on every axis velocity, -1 on rest
//   2D  ex^2 - ey^2          : 1/4 on +-x, -1/4 on +-y;  trace: 1/4 on axes, -1 on rest
//   ea eb (a != b)           : ea eb / 4 on the four diagonals of the (a, b) plane
// Momentum populations are stored shifted, g_n - w_n, so FP32 keeps the small pressure
// and velocity deviations.
#pragma once

#include <type_traits>

#include <cuda.h>

#include <cstdint>

#include "lattice.cuh"
#include "tma.cuh"

namespace lbehd {

constexpr int NOBS = 16;      // observable accumulators per block
constexpr int BX = 128;       // threads per block along x

// info byte: bits 0-1 potential type, bits 2-3 wetting class.
enum : uint8_t { PT_FLUID = 0, PT_DIRICHLET = 1, PT_NEUMANN = 2 };

struct Params {
    int nx, ny, nz;
    long long N;
    float nu[3], eps[3], sig[3];
    float Y[3], YT;
    float cos12, cos13, cos23;
    float W;
    float inv_tau_phi, inv_tau_rho;
    float s_bulk;
    float body[3];
    float body1[3];   // force density on the droplet phase alone: Phi_1 body1
};

// The variable-density scheme's parameters: only its kernels receive them (a larger
// parameter block made the compiler emit 9 % more instructions in the equal-density
// collide kernel, so that kernel keeps Params as it is).
struct ParamsVD : Params {
    float rho_ph[3];   // phase densities
};

template <bool VD>
using CollideParams = typename std::conditional<VD, ParamsVD, Params>::type;

struct State {
    const float *g, *fphi, *frho;     // pre-collision populations at time n
    float *g_out, *fphi_out, *frho_out;
    const float *phi, *phi_prev;      // [3][N] Phi at n and n-1
    const float *rho, *rho_prev;      // rho_e at n and n-1
    float *u, *q;                     // u and conduction source: read as n-1, written as n
    const float *pot, *pot_lo;        // potential as a compensated pair hi + lo
    const uint8_t *info;
    double *obs_partials;             // [NOBS][nblocks]
    int *flag;                        // bit 0: non-finite value seen; bit 1: staging timed out
};

// Rest-population bookkeeping of a conserved zeroth moment. The post-collision rest
// population is f*_0 = f_0 + sum_{n>0} (f_n - f*_n), the incoming rest population plus what
// the moving populations hand over, so that the populations' total is carried from step to
// step without a rounding bias. Near equilibrium f_n and f*_n are within a factor two of each
// other, so each difference is exact in FP32 (Sterbenz), and their sum is small, so adding
// the differences up rounds only far below the populations' own ulp. Summing the incoming
// populations into Phi and subtracting the outgoing sum instead rounds twice per site at the
// populations' ulp; on near-uniform regions those roundings repeat with the same sign from
// step to step, and the component masses of the 128x64x64 droplet drifted by up to 1e-9 per
// step (2e-5 over 20 000 steps). With this bookkeeping they stay within 1.1e-7 over 30 000
// steps. The explicit _rn operations keep the compiler from fusing f_n - f*_n with the
// product that formed f*_n, which would subtract the unrounded product rather than the
// stored population.
__device__ __forceinline__ float rest_acc(float acc, float f_in, float f_out)
{
    return __fadd_rn(acc, __fsub_rn(f_in, f_out));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- initial state

template <int D>
__global__ void __launch_bounds__(BX) k_init(Params P, const float *__restrict__ phi0,
                                             float *__restrict__ g, float *__restrict__ fphi,
                                             float *__restrict__ frho,
                                             const uint8_t *__restrict__ info)
{
    using L = Lat<D>;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx)
        return;
    const size_t N = P.N, i = x + (size_t)P.nx * (y + (size_t)P.ny * z);
    const bool fluid = (info[i] & 3) == PT_FLUID;
#pragma unroll
    for (int n = 0; n < L::Q; n++) {
        g[n * N + i] = 0.0f;   // shifted: g_n - w_n with p* = 1, u = 0
#pragma unroll
        for (int c = 0; c < 3; c++)
            fphi[(c * L::Q + n) * N + i] = fluid ? phi0[c * N + i] * L::w(n) : 0.0f;
    }
#pragma unroll
    for (int n = 0; n < L::QS; n++)
        frho[n * N + i] = 0.0f;
}

// ---------------------------------------------------------------- moments + ghosts

// Pointers one moments + ghosts pass reads and writes (buffers of the step's parity).
struct FieldPtrs {
    const float *fphi, *frho;
    float *phi_out, *rho_out, *eps_out, *pot, *pot_lo;
    const uint8_t *info, *normal;
    const int16_t *elec;
    const double *V;
};

template <int D>
__device__ __forceinline__ void fields_site(const Params &P, const FieldPtrs &F, int x, int y, int z)
{
    using L = Lat<D>;
    constexpr int Q = L::Q;
    const float *__restrict__ fphi = F.fphi;
    const float *__restrict__ frho = F.frho;
    float *__restrict__ phi_out = F.phi_out;
    float *__restrict__ rho_out = F.rho_out;
    float *__restrict__ pot = F.pot;
    float *__restrict__ pot_lo = F.pot_lo;
    const uint8_t *__restrict__ info = F.info;
    const uint8_t *__restrict__ normal = F.normal;
    const int16_t *__restrict__ elec = F.elec;
    const double *__restrict__ V = F.V;
    // 32-bit indices below 19 N < 2^31 (checked at init), from one base pointer per set
    const int N = (int)P.N, i = x + P.nx * (y + P.ny * z);
    const uint8_t inf = info[i];
    float Ph[3] = {0.0f, 0.0f, 0.0f};
    if ((inf & 3) == PT_FLUID) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float *fc = fphi + (size_t)c * Q * N;
            float acc = 0.0f;
#pragma unroll
            for (int n = 0; n < Q; n++)
                acc += fc[n * N + i];
            Ph[c] = acc;
        }
        float r = 0.0f;
#pragma unroll
        for (int n = 0; n < L::QS; n++)
            r += frho[n * N + i];
        rho_out[i] = r;
    } else {
        rho_out[i] = 0.0f;
        const int k = normal[i];
        if (k > 0) {
            // Eq. 20a, explicit in the fluid node f = s + e_k along the lattice normal.
            const int kx = L::ex(k), ky = L::ey(k), kz = L::ez(k);
            const int X = (x + kx + P.nx) % P.nx, Y = (y + ky + P.ny) % P.ny,
                      Z = (z + kz + P.nz) % P.nz;
            const int f = X + P.nx * (Y + P.ny * Z);
            float Pf[3];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float *fc = fphi + (size_t)c * Q * N;
                float acc = 0.0f;
#pragma unroll
                for (int n = 0; n < Q; n++)
                    acc += fc[n * N + f];
                Pf[c] = acc;
            }
            float c12 = 0.0f, c13 = 0.0f, c23 = 0.0f;
            if (((inf >> 2) & 3) == 1) {
                c12 = P.cos12;
                c13 = P.cos13;
                c23 = P.cos23;
            }
            const float len = (kx * kx + ky * ky + kz * kz) == 2 ? 1.41421356237f : 1.0f;
            const float s = 4.0f / P.W;
            const float H1 = s * (-c13 * Pf[0] * Pf[2] - c12 * Pf[0] * Pf[1]);
            const float H2 = s * (c12 * Pf[0] * Pf[1] - c23 * Pf[1] * Pf[2]);
            const float H3 = s * (c23 * Pf[1] * Pf[2] + c13 * Pf[0] * Pf[2]);
            Ph[0] = Pf[0] - len * H1;
            Ph[1] = Pf[1] - len * H2;
            Ph[2] = Pf[2] - len * H3;
        }
        if ((inf & 3) == PT_DIRICHLET) {
            const int id = elec[i];
            const double v = id >= 0 ? V[id] : 0.0;
            const float hi = (float)v;
            pot[i] = hi;
            pot_lo[i] = (float)(v - (double)hi);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++)
        phi_out[c * N + i] = Ph[c];
    F.eps_out[i] = Ph[0] * P.eps[0] + Ph[1] * P.eps[1] + Ph[2] * P.eps[2];
}

template <int D>
__global__ void __launch_bounds__(BX) k_fields(Params P, FieldPtrs F)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x < P.nx)
        fields_site<D>(P, F, x, y, z);
}

// ---------------------------------------------------------------- fused collide + stream

// Population sources for collide_site: straight from global memory, or from a
// shared-memory tile staged by bulk copies.
// Indices n N + i are 32-bit (19 N < 2^31 is checked at init); the 3 Q phase-field arrays
// need 64 bits.
struct GlobalPops {
    const float *__restrict__ gp, *__restrict__ fp, *__restrict__ rp;
    int N, i, Q;
    __device__ __forceinline__ float g(int n) const { return gp[n * N + i]; }
    __device__ __forceinline__ float phi(int c, int n) const
    {
        return fp[(size_t)(c * Q + n) * N + i];
    }
    __device__ __forceinline__ float rho(int n) const { return rp[n * N + i]; }
};

// The staged kernel's populations: the phase-field sets (57 / 27 arrays) from the tile staged
// in shared memory; the momentum and charge sets (one coalesced read per array and site) read
// into registers at the start of the tile, so that their latency overlaps the halo loads.
// Measured on 128x64x64: 82.0 us per launch (64x2 tiles) against 85.9 us with all 83 arrays
// staged.
template <int D>
struct StagedPops {
    float gr[Lat<D>::Q], rr[Lat<D>::QS];
    const float *s;   // [phase array][tile site], stride BX
    int t;
    __device__ __forceinline__ float g(int n) const { return gr[n]; }
    __device__ __forceinline__ float phi(int c, int n) const
    {
        return s[(c * Lat<D>::Q + n) * BX + t];
    }
    __device__ __forceinline__ float rho(int n) const { return rr[n]; }
};

// Stencil-field sources for collide_site: Phi_1..3, the compensated potential and the node
// class at the site and at its lattice neighbours, from global memory or from a halo tile
// in shared memory.
struct GlobalStencil {
    const float *__restrict__ p0, *__restrict__ p1, *__restrict__ p2, *__restrict__ pot,
        *__restrict__ plo;
    const uint8_t *__restrict__ info;
    int i;
    int oxp, oxm, oyp, oym, ozp, ozm;
    template <class L>
    __device__ __forceinline__ int idx(int n) const
    {
        return i + (L::ex(n) > 0 ? oxp : (L::ex(n) < 0 ? oxm : 0)) +
               (L::ey(n) > 0 ? oyp : (L::ey(n) < 0 ? oym : 0)) +
               (L::ez(n) > 0 ? ozp : (L::ez(n) < 0 ? ozm : 0));
    }
    template <class L>
    __device__ __forceinline__ void at(int n, float (&P)[3], float &ph, float &lo, int &pt) const
    {
        const int j = n ? idx<L>(n) : i;
        P[0] = p0[j];
        P[1] = p1[j];
        P[2] = p2[j];
        ph = pot[j];
        lo = plo[j];
        pt = info[j] & 3;
    }
};

// Tiles of the staged collide kernel: TX x TY sites (TX * TY = BX), TY in {2, 4, 8}.
// Halo tile layout: HX x HY x HZ sites, each as a float4 (Phi_1, Phi_2, Phi_3, pot) and a
// float2 (pot_lo, node class as the bits of a float), so that a neighbour's six fields come
// in two shared-memory loads.
template <int D, int TY>
struct Halo {
    static constexpr int TX = BX / TY;
    static constexpr int HX = TX + 2, HY = TY + 2, HZ = D == 3 ? 3 : 1;
    static constexpr int N = HX * HY * HZ;
};

template <int D, int TY>
struct SmemStencil {
    const float4 *a;   // Halo::N of (Phi_1, Phi_2, Phi_3, pot)
    const float2 *b;   // Halo::N of (pot_lo, info bits)
    int h;             // halo index of the site
    template <class L>
    __device__ __forceinline__ void at(int n, float (&P)[3], float &ph, float &lo, int &pt) const
    {
        using H = Halo<D, TY>;
        constexpr int HX = H::HX, HXY = H::HX * H::HY;
        const int j = h + L::ex(n) + HX * L::ey(n) + HXY * L::ez(n);
        const float4 v = a[j];
        const float2 w = b[j];
        P[0] = v.x;
        P[1] = v.y;
        P[2] = v.z;
        ph = v.w;
        lo = w.x;
        pt = __float_as_int(w.y) & 3;
    }
};

// The site's own scalar fields read by collide_site (charge now and before, the previous
// velocity, Phi and conduction source), loaded early so their latency overlaps other work.
struct SitePre {
    float rho, rho_o, q_o, uo[3], Po[3];
};

__device__ __forceinline__ SitePre load_site_pre(const State &S, size_t N, int i)
{
    SitePre p;
    p.rho = S.rho[i];
    p.rho_o = S.rho_prev[i];
    p.q_o = S.q[i];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        p.uo[a] = S.u[a * N + i];
        p.Po[a] = S.phi_prev[a * N + i];
    }
    return p;
}

// Push streaming of one site's post-collision populations: f*_n goes to x + e_n, or into the
// opposite slot at x when x + e_n is solid (halfway bounce-back).
template <class L>
struct Pusher {
    unsigned fluid_nb;   // bit n: x + e_n is fluid
    int i, N;
    int oxp, oxm, oyp, oym, ozp, ozm;   // periodic neighbour offsets
    __device__ __forceinline__ int off(int n) const
    {
        return (L::ex(n) > 0 ? oxp : (L::ex(n) < 0 ? oxm : 0)) +
               (L::ey(n) > 0 ? oyp : (L::ey(n) < 0 ? oym : 0)) +
               (L::ez(n) > 0 ? ozp : (L::ez(n) < 0 ? ozm : 0));
    }
    __device__ __forceinline__ void operator()(float *out, int n, float v) const
    {
        const bool fl = (fluid_nb >> n) & 1u;
        out[fl ? n * N + (i + off(n)) : opposite(n) * N + i] = v;   // < 19 N < 2^31
    }
};

template <class L>
__device__ __forceinline__ Pusher<L> make_pusher(const Params &P, int x, int y, int z, int i,
                                                 unsigned fluid_nb)
{
    const int nx = P.nx, nxy = P.nx * P.ny;
    return Pusher<L>{fluid_nb, i, (int)P.N,
                     x + 1 == P.nx ? 1 - P.nx : 1, x == 0 ? P.nx - 1 : -1,
                     (y + 1 == P.ny ? 1 - P.ny : 1) * nx, (y == 0 ? P.ny - 1 : -1) * nx,
                     (z + 1 == P.nz ? 1 - P.nz : 1) * nxy, (z == 0 ? P.nz - 1 : -1) * nxy};
}

// Moments of the (shifted, gs = g - w) momentum populations: dp = sum gs, jm = sum e gs,
// m2 = (sum ex^2 gs, sum ey^2 gs, sum ez^2 gs, sum ex ey gs, sum ex ez gs, sum ey ez gs).
template <int D, class Pops>
__device__ __forceinline__ void momentum_moments(const Pops &pops, float &dp, float (&jm)[3],
                                                 float (&m2)[6])
{
    using L = Lat<D>;
    dp = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++)
        jm[a] = 0.0f;
#pragma unroll
    for (int k = 0; k < 6; k++)
        m2[k] = 0.0f;
#pragma unroll
    for (int n = 0; n < L::Q; n++) {
        const float v = pops.g(n);
        dp += v;
        if (L::ex(n))
            jm[0] += L::ex(n) > 0 ? v : -v;
        if (L::ey(n))
            jm[1] += L::ey(n) > 0 ? v : -v;
        if (L::ez(n))
            jm[2] += L::ez(n) > 0 ? v : -v;
        if (L::ex(n))
            m2[0] += v;   // sum ex^2 gs
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
}

// Momentum collision (incompressible equilibrium, Guo forcing, MRT) and its push.
template <int D, class Push>
__device__ __forceinline__ void momentum_collide(const Params &P, const State &S, const Push &push,
                                                 const float (&Pc)[3],
                                                 float dp, const float (&m2)[6],
                                                 const float (&u)[3], const float (&F)[3])
{
    using L = Lat<D>;
    constexpr int Q = L::Q;
    constexpr float inv_cs2 = 3.0f;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float nu = Pc[0] * P.nu[0] + Pc[1] * P.nu[1] + Pc[2] * P.nu[2];
    const float c_nu = 1.0f - 1.0f / (inv_cs2 * nu + 0.5f);
    const float c_b = 1.0f - P.s_bulk;
    // non-equilibrium moments of g - g_eq + R/2 (deviatoric / off-diagonal / trace):
    // second moments of the populations less those of the equilibrium (c_s^2 p* I + u u)
    // plus half those of the force term (u F + F u)
    const float uFd[3] = {u[0] * F[0], u[1] * F[1], u[2] * F[2]};
    const float d1 = (m2[0] - m2[1]) - (u[0] * u[0] - u[1] * u[1]) + (uFd[0] - uFd[1]);
    const float d2 = (m2[0] - m2[2]) - (u[0] * u[0] - u[2] * u[2]) + (uFd[0] - uFd[2]);
    const float dxy = m2[3] - u[0] * u[1] + 0.5f * (u[0] * F[1] + u[1] * F[0]);
    const float dxz = m2[4] - u[0] * u[2] + 0.5f * (u[0] * F[2] + u[2] * F[0]);
    const float dyz = m2[5] - u[1] * u[2] + 0.5f * (u[1] * F[2] + u[2] * F[1]);
    const float dT = (m2[0] + m2[1] + m2[2]) - (float)D * (1.0f / 3.0f) * dp - uu + uF;
    // w_n [C0 + e.V + (e.u)(4.5 e.u + 4.5 e.F)] = g_eq,n - w_n + R_n / 2
    const float C0 = dp - 1.5f * uu - 1.5f * uF;
    const float V[3] = {3.0f * u[0] + 1.5f * F[0], 3.0f * u[1] + 1.5f * F[1],
                        3.0f * u[2] + 1.5f * F[2]};
    float sum = 0.0f;
#pragma unroll
    for (int n = 1; n < Q; n++) {
        const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
        const int e2 = cx * cx + cy * cy + cz * cz;
        const float eu = (cx ? (cx > 0 ? u[0] : -u[0]) : 0.f) + (cy ? (cy > 0 ? u[1] : -u[1]) : 0.f) +
                         (cz ? (cz > 0 ? u[2] : -u[2]) : 0.f);
        const float eF = (cx ? (cx > 0 ? F[0] : -F[0]) : 0.f) + (cy ? (cy > 0 ? F[1] : -F[1]) : 0.f) +
                         (cz ? (cz > 0 ? F[2] : -F[2]) : 0.f);
        const float eV = (cx ? (cx > 0 ? V[0] : -V[0]) : 0.f) + (cy ? (cy > 0 ? V[1] : -V[1]) : 0.f) +
                         (cz ? (cz > 0 ? V[2] : -V[2]) : 0.f);
        float v = L::w(n) * (C0 + eV + eu * (4.5f * eu + 4.5f * eF));
        float corr = 0.0f, corrT = 0.0f;
        if (D == 3) {
            if (e2 == 1) {
                corr = cx ? (d1 + d2) * (1.0f / 6.0f)
                          : (cy ? d2 * (1.0f / 6.0f) - d1 * (1.0f / 3.0f)
                                : d1 * (1.0f / 6.0f) - d2 * (1.0f / 3.0f));
                corrT = dT * (1.0f / 6.0f);
            } else {
                corr = 0.25f * (cx * cy * dxy + cx * cz * dxz + cy * cz * dyz);
            }
        } else {
            if (e2 == 1) {
                corr = cx ? 0.25f * d1 : -0.25f * d1;
                corrT = 0.25f * dT;
            } else {
                corr = 0.25f * cx * cy * dxy;
            }
        }
        v += c_nu * corr + c_b * corrT;
        sum += v;
        push(S.g_out, n, v);
    }
    // rest population: exact remainder of the conserved zeroth moment (the FP32
    // weights do not sum to 1 exactly, which would otherwise create mass every step).
    // The shifted populations are small, so the sums' rounding is far below the
    // phase fields' (whose rest populations use rest_acc).
    push(S.g_out, 0, dp - sum);
    if (!isfinite(dp + u[0] + u[1] + u[2]))
        atomicOr(S.flag, 1);
}

// Momentum collision of the variable-density scheme (Table 1's densities in Eq. 9): the
// populations carry the gauge pressure and rho u (g_eq,n = w_n p/c_s^2 + rho s_n(u), n > 0;
// g_eq,0 = (w_0 - 1) p/c_s^2 + rho s_0(u); s_n(u) = w_n [e.u/c_s^2 + (e.u)^2/(2 c_s^4) -
// u^2/(2 c_s^2)]), the force term G_n = (e_n - u).[(w_n + s_n) F + s_n c_s^2 grad rho]/c_s^2
// carries the force density and the density gradient, p = c_s^2/(1 - w_0) [sum_{n>0} g_n +
// u.grad(rho)/2 + rho s_0(u)], and every moment relaxes with tau = 1/2 + nu/c_s^2. The
// populations are stored as g itself. gsum = sum_n g_n, g0 = g_0.
template <int D, class Push, class Pops>
__device__ __forceinline__ void momentum_collide_vd(const Params &P, const State &S,
                                                    const Push &push, const Pops &pops,
                                                    const float (&Pc)[3], float gsum,
                                                    float dens, const float (&gr)[3],
                                                    const float (&u)[3], const float (&F)[3])
{
    using L = Lat<D>;
    constexpr int Q = L::Q;
    constexpr float inv_cs2 = 3.0f;
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const float uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
    const float ug = u[0] * gr[0] + u[1] * gr[1] + u[2] * gr[2];
    const float nu = Pc[0] * P.nu[0] + Pc[1] * P.nu[1] + Pc[2] * P.nu[2];
    const float itau = 1.0f / (inv_cs2 * nu + 0.5f);
    const float cf = 1.0f - 0.5f * itau;
    const float s0 = L::w(0) * (-1.5f * uu);
    const float pc = ((gsum - pops.g(0)) + 0.5f * ug + dens * s0) *
                     (1.0f / (1.0f - L::w(0)));   // p / c_s^2
#pragma unroll
    for (int n = 0; n < Q; n++) {
        const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
        const float eu = (cx ? (cx > 0 ? u[0] : -u[0]) : 0.f) + (cy ? (cy > 0 ? u[1] : -u[1]) : 0.f) +
                         (cz ? (cz > 0 ? u[2] : -u[2]) : 0.f);
        const float eF = (cx ? (cx > 0 ? F[0] : -F[0]) : 0.f) + (cy ? (cy > 0 ? F[1] : -F[1]) : 0.f) +
                         (cz ? (cz > 0 ? F[2] : -F[2]) : 0.f);
        const float eg = (cx ? (cx > 0 ? gr[0] : -gr[0]) : 0.f) +
                         (cy ? (cy > 0 ? gr[1] : -gr[1]) : 0.f) +
                         (cz ? (cz > 0 ? gr[2] : -gr[2]) : 0.f);
        const float sn = L::w(n) * (inv_cs2 * eu + 4.5f * eu * eu - 1.5f * uu);
        const float geq = (n == 0 ? L::w(0) - 1.0f : L::w(n)) * pc + dens * sn;
        const float G = inv_cs2 * (L::w(n) + sn) * (eF - uF) + sn * (eg - ug);
        const float g = pops.g(n);
        push(S.g_out, n, g - (g - geq) * itau + cf * G);
    }
    if (!isfinite(pc + u[0] + u[1] + u[2]))
        atomicOr(S.flag, 1);
}

// Collision of phase field c (Eqs. 15-17) and its push.
template <int D, class Push, class Pops>
__device__ __forceinline__ void phase_collide(const Params &P, const State &S, const Push &push,
                                              const Pops &pops, int c,
                                              float Pp, float Po, const float (&FP)[3],
                                              const float (&u)[3], const float (&uo)[3])
{
    using L = Lat<D>;
    constexpr int Q = L::Q;
    constexpr float inv_cs2 = 3.0f;
    const float c_phi = 1.0f - P.inv_tau_phi;
    float jf[3] = {0.f, 0.f, 0.f}, fin[Q];
#pragma unroll
    for (int n = 1; n < Q; n++) {
        const float v = pops.phi(c, n);
        fin[n] = v;
        if (L::ex(n))
            jf[0] += L::ex(n) > 0 ? v : -v;
        if (L::ey(n))
            jf[1] += L::ey(n) > 0 ? v : -v;
        if (L::ez(n))
            jf[2] += L::ez(n) > 0 ? v : -v;
    }
    float B[3], del[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float A = L::cs2 * FP[a] + (Pp * u[a] - Po * uo[a]);
        del[a] = c_phi * 0.5f * (jf[a] - Pp * u[a] + 0.5f * A);
        B[a] = inv_cs2 * Pp * u[a] + 0.5f * inv_cs2 * A;   // w_n (P + e.B) = f_eq + C/2
    }
    float *out = S.fphi_out + (size_t)c * Q * (size_t)P.N;
    float dsum = 0.0f;
#pragma unroll
    for (int n = 1; n < Q; n++) {
        const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
        const float eB = (cx ? (cx > 0 ? B[0] : -B[0]) : 0.f) + (cy ? (cy > 0 ? B[1] : -B[1]) : 0.f) +
                         (cz ? (cz > 0 ? B[2] : -B[2]) : 0.f);
        float v = L::w(n) * (Pp + eB);
        if (cx * cx + cy * cy + cz * cz == 1)
            v += (cx ? (cx > 0 ? del[0] : -del[0]) : 0.f) + (cy ? (cy > 0 ? del[1] : -del[1]) : 0.f) +
                 (cz ? (cz > 0 ? del[2] : -del[2]) : 0.f);
        dsum = rest_acc(dsum, fin[n], v);
        push(out, n, v);
    }
    push(out, 0, __fadd_rn(pops.phi(c, 0), dsum));   // Phi is conserved
}

// Charge collision (Eq. 20b: advection-diffusion, d(rho u)/dt, conduction) and its push.
template <int D, class Push, class Pops>
__device__ __forceinline__ void charge_collide(const Params &P, const State &S, const Push &push,
                                               const Pops &pops,
                                               float rho, float rho_o, float qsrc, float q_o,
                                               const float (&u)[3], const float (&uo)[3])
{
    using L = Lat<D>;
    constexpr int QS = L::QS;
    constexpr float inv_cs2s = 1.0f / L::cs2s;
    float jr[3] = {0.f, 0.f, 0.f}, fr[QS];
#pragma unroll
    for (int n = 1; n < QS; n++) {
        const float v = pops.rho(n);
        fr[n] = v;
        if (L::ex(n))
            jr[0] += L::ex(n) > 0 ? v : -v;
        if (L::ey(n))
            jr[1] += L::ey(n) > 0 ? v : -v;
        if (L::ez(n))
            jr[2] += L::ez(n) > 0 ? v : -v;
    }
    const float c_rho = 1.0f - P.inv_tau_rho;
    const float Qt = qsrc + 0.5f * (qsrc - q_o);
    float B[3], del[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float Dm = rho * u[a] - rho_o * uo[a];
        del[a] = c_rho * 0.5f * (jr[a] - rho * u[a] + 0.5f * Dm);
        B[a] = inv_cs2s * (rho * u[a] + 0.5f * Dm);
    }
    const float C0 = rho + Qt;
    float dsum = 0.0f;
#pragma unroll
    for (int n = 1; n < QS; n++) {
        const int cx = L::ex(n), cy = L::ey(n), cz = L::ez(n);
        const float eB = (cx ? (cx > 0 ? B[0] : -B[0]) : 0.f) + (cy ? (cy > 0 ? B[1] : -B[1]) : 0.f) +
                         (cz ? (cz > 0 ? B[2] : -B[2]) : 0.f);
        const float ed = (cx ? (cx > 0 ? del[0] : -del[0]) : 0.f) + (cy ? (cy > 0 ? del[1] : -del[1]) : 0.f) +
                         (cz ? (cz > 0 ? del[2] : -del[2]) : 0.f);
        const float v = L::ws(n) * (C0 + eB) + ed;
        dsum = rest_acc(dsum, fr[n], v);
        push(S.frho_out, n, v);
    }
    // zeroth moment: rho_e + source
    push(S.frho_out, 0, __fadd_rn(__fadd_rn(pops.rho(0), Qt), dsum));
}

// Sharpening flux F_Phi,i of Eq. 18 from the site's Phi_i and their gradients.
__device__ __forceinline__ void sharpening_flux(float W, const float (&Pc)[3],
                                                const float (&gP)[3][3], float (&FPhi)[3][3])
{
    float ln[3][3], J[3] = {0.f, 0.f, 0.f}, sumsq = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        // n = grad / sqrt(|grad|^2 + 1e-10): continuous where grad Phi vanishes
        const float gn = sqrtf(gP[c][0] * gP[c][0] + gP[c][1] * gP[c][1] +
                               gP[c][2] * gP[c][2] + 1e-10f);
        const float lam = 4.0f / W * fabsf(Pc[c] * (1.0f - Pc[c])) / gn;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ln[c][a] = lam * gP[c][a];
            J[a] += ln[c][a];
        }
        sumsq += Pc[c] * Pc[c];
    }
    const float inv_sumsq = 1.0f / sumsq;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float r = Pc[c] * Pc[c] * inv_sumsq;
#pragma unroll
        for (int a = 0; a < 3; a++)
            FPhi[c][a] = ln[c][a] - r * J[a];
    }
}

// Everything the step does at one fluid site after the moments and the Poisson solve:
// stencils, forces, the three collisions, push streaming, observable contributions.
// Written for a low instruction count: 32-bit neighbour offsets computed once, the
// equilibrium + half-source terms folded into one scalar and one vector per population set
// (f*_n = w_n (C + e_n . B) + ...), and the non-equilibrium second moments of the momentum
// populations formed from their raw moments and the closed-form moments of g_eq and R:
//   Pi(g_eq) = c_s^2 p* I + u u,   Pi(R) = u F + F u.
template <int D, class Pops, class Stencil, bool VD = false>
__device__ __forceinline__ void collide_site(const CollideParams<VD> &P, const State &S, int x,
                                             int y, int z,
                                             int i, int first, const Pops &pops,
                                             const Stencil &st, const SitePre &pre,
                                             float (&ob)[NOBS])
{
    using L = Lat<D>;
    constexpr int Q = L::Q;
    const int N = (int)P.N;
    // ---- momentum moments (shifted populations gs = g - w), first: the site's momentum
    // populations are then dead before the stencils, and ten moments stay live instead
    float dp, jm[3], m2[6];
    momentum_moments<D>(pops, dp, jm, m2);

    // ---- stencils of Phi_i and phi over the flow lattice
    float Pc[3], pot_i, lo_i;
    int pt_i;
    st.template at<L>(0, Pc, pot_i, lo_i, pt_i);
    const float sig_i = Pc[0] * P.sig[0] + Pc[1] * P.sig[1] + Pc[2] * P.sig[2];
    float gP[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float sP[3] = {0.f, 0.f, 0.f}, gpot[3] = {0.f, 0.f, 0.f};
    float qsrc = 0.0f;
    unsigned fluid_nb = 1u;   // bit n: x + e_n is fluid (bit 0: the site itself)
#pragma unroll
    for (int n = 1; n < Q; n++) {
        float Pn[3], potj, loj;
        int pt;
        st.template at<L>(n, Pn, potj, loj, pt);
        const float wn = L::w(n);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            sP[c] += wn * Pn[c];
            if (L::ex(n))
                gP[c][0] += (L::ex(n) > 0 ? wn : -wn) * Pn[c];
            if (L::ey(n))
                gP[c][1] += (L::ey(n) > 0 ? wn : -wn) * Pn[c];
            if (L::ez(n))
                gP[c][2] += (L::ez(n) > 0 ? wn : -wn) * Pn[c];
        }
        // phi(x + e_n) - phi(x) from the compensated pairs (zero-flux solid: mirror)
        const float dph = pt == PT_NEUMANN ? 0.0f : (potj - pot_i) + (loj - lo_i);
        if (L::ex(n))
            gpot[0] += (L::ex(n) > 0 ? wn : -wn) * dph;
        if (L::ey(n))
            gpot[1] += (L::ey(n) > 0 ? wn : -wn) * dph;
        if (L::ez(n))
            gpot[2] += (L::ez(n) > 0 ? wn : -wn) * dph;
        if (pt == PT_FLUID) {
            fluid_nb |= 1u << n;
            if (n <= 2 * D) {
                const float sig_j = Pn[0] * P.sig[0] + Pn[1] * P.sig[1] + Pn[2] * P.sig[2];
                qsrc += 0.5f * (sig_i + sig_j) * dph;
            }
        }
    }
    constexpr float inv_cs2 = 3.0f;
    constexpr float wmov = 1.0f - L::w(0);   // sum of the moving weights
    float lP[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        lP[c] = 2.0f * inv_cs2 * (sP[c] - wmov * Pc[c]);
#pragma unroll
        for (int a = 0; a < 3; a++)
            gP[c][a] *= inv_cs2;
    }

    // ---- chemical potential (Eqs. 10-11), capillary and electric forces (Eq. 12)
    const float W = P.W;
    const float tri = 24.0f * P.YT / W * Pc[0] * Pc[1] * Pc[2];
    float Fs[3] = {0.f, 0.f, 0.f}, geps[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float mu = 24.0f * P.Y[c] / W * Pc[c] * (Pc[c] - 1.0f) * (Pc[c] - 0.5f) - tri -
                         0.75f * P.Y[c] * W * lP[c];
#pragma unroll
        for (int a = 0; a < 3; a++)
            Fs[a] += mu * gP[c][a];
    }
    float E[3], E2 = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        geps[a] = P.eps[0] * gP[0][a] + P.eps[1] * gP[1][a] + P.eps[2] * gP[2][a];
        E[a] = -inv_cs2 * gpot[a];
        E2 += E[a] * E[a];
    }
    const float rho = pre.rho;
    float Fe[3], F[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        Fe[a] = rho * E[a] - 0.5f * E2 * geps[a];
        F[a] = Fs[a] + Fe[a] + P.body[a] + Pc[0] * P.body1[a];
    }

    // ---- sharpening flux F_Phi,i (Eq. 18)
    float FPhi[3][3];
    sharpening_flux(P.W, Pc, gP, FPhi);

    // ---- velocity from the momentum moments (formed above) and the force; with variable
    // density, rho u = j + F/2 with rho = sum Phi_i rho_i
    float u[3], dens = 1.0f, gr[3] = {0.f, 0.f, 0.f};
    if constexpr (VD) {
        dens = Pc[0] * P.rho_ph[0] + Pc[1] * P.rho_ph[1] + Pc[2] * P.rho_ph[2];
#pragma unroll
        for (int a = 0; a < 3; a++)
            gr[a] = P.rho_ph[0] * gP[0][a] + P.rho_ph[1] * gP[1][a] + P.rho_ph[2] * gP[2][a];
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
        u[a] = VD ? (jm[a] + 0.5f * F[a]) / dens : jm[a] + 0.5f * F[a];
    float uo[3], Po[3], rho_o, q_o;
    if (first) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            uo[a] = u[a];
            Po[a] = Pc[a];
        }
        rho_o = rho;
        q_o = qsrc;
    } else {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            uo[a] = pre.uo[a];
            Po[a] = pre.Po[a];
        }
        rho_o = pre.rho_o;
        q_o = pre.q_o;
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
        S.u[a * (size_t)N + i] = u[a];
    S.q[i] = qsrc;

    const Pusher<L> push = make_pusher<L>(P, x, y, z, i, fluid_nb);
    if (VD)
        momentum_collide_vd<D>(P, S, push, pops, Pc, dp, dens, gr, u, F);
    else
        momentum_collide<D>(P, S, push, Pc, dp, m2, u, F);
#pragma unroll
    for (int c = 0; c < 3; c++)
        phase_collide<D>(P, S, push, pops, c, Pc[c], Po[c], FPhi[c], u, uo);
    charge_collide<D>(P, S, push, pops, rho, rho_o, qsrc, q_o, u, uo);

    // ---- observable contributions
    ob[0] = Pc[0];
    ob[1] = Pc[0] * (float)x;
    ob[2] = Pc[0] * (float)y;
    ob[3] = Pc[0] * (float)z;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ob[4 + a] = Pc[0] * u[a];
        ob[7 + a] = Pc[0] * Fe[a];
        ob[10 + a] = Fe[a];
    }
    ob[13] = Pc[1];
    ob[14] = Pc[2];
    ob[15] = rho;
    if (!isfinite(Pc[0] + Pc[1] + Pc[2] + rho + qsrc))
        atomicOr(S.flag, 1);
}

// Block partial sums of the observables: FP32 within the block (warp butterflies, then the
// block's warps in order), one conversion to FP64 per observable; the sum over blocks is FP64
// (k_obs_final_split). The FP64 pipe of this part is narrow: converting and adding every
// warp's sums in FP64 at the end of each block kept it 18 % busy over the whole collide
// kernel (ncu). A block's FP32 partial carries ~1e-7 relative rounding, which the FP64 sum
// over thousands of blocks does not accumulate into a bias.
// Warp sums of the 16 observables, transposed: afterwards lane l holds the sum of
// observable (l >> 1) & 15. Each round halves what a lane carries: it keeps the half its lane
// bit selects, sends the other half to its partner and adds the partner's. The partners and
// the operands of every addition are those of warp_sum's butterfly (offsets 16, 8, 4, 2, 1),
// so each sum has warp_sum's bits; 16 shuffles and 16 adds instead of 80 and 80.
__device__ __forceinline__ float warp_sum16_transposed(const float (&ob)[16])
{
    const int lane = threadIdx.x & 31;
    float a8[8], a4[4], a2[2];
    const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4, b2 = lane & 2;
#pragma unroll
    for (int j = 0; j < 8; j++)
        a8[j] = (b16 ? ob[j + 8] : ob[j]) +
                __shfl_xor_sync(0xffffffffu, b16 ? ob[j] : ob[j + 8], 16);
#pragma unroll
    for (int j = 0; j < 4; j++)
        a4[j] = (b8 ? a8[j + 4] : a8[j]) + __shfl_xor_sync(0xffffffffu, b8 ? a8[j] : a8[j + 4], 8);
#pragma unroll
    for (int j = 0; j < 2; j++)
        a2[j] = (b4 ? a4[j + 2] : a4[j]) + __shfl_xor_sync(0xffffffffu, b4 ? a4[j] : a4[j + 2], 4);
    float a = (b2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, b2 ? a2[0] : a2[1], 2);
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    return a;
}

__device__ __forceinline__ void block_obs_partials(const float (&ob)[NOBS], double *partials,
                                                   size_t blk, size_t nblk)
{
    static_assert(NOBS == 16, "the transposed warp sum carries 16 observables");
    __shared__ float sm[NOBS][BX / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float v = warp_sum16_transposed(ob);
    if ((lane & 1) == 0)
        sm[(lane >> 1) & 15][wid] = v;
    __syncthreads();
    if (threadIdx.x < NOBS) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < BX / 32; w++)
            acc += sm[threadIdx.x][w];
        partials[threadIdx.x * nblk + blk] = (double)acc;
    }
}

// One site of the global-load variant (no-op for x >= nx or a non-fluid site).
template <int D, bool VD = false>
__device__ __forceinline__ void collide_global_site(const CollideParams<VD> &P, const State &S,
                                                    int first,
                                                    int x, int y, int z, float (&ob)[NOBS])
{
    const int i = x + P.nx * (y + P.ny * z);
    if (x < P.nx && (S.info[i] & 3) == PT_FLUID) {
        const GlobalPops pops{S.g, S.fphi, S.frho, (int)P.N, i, Lat<D>::Q};
        const int nx = P.nx, nxy = P.nx * P.ny;
        const GlobalStencil st{S.phi, S.phi + P.N, S.phi + 2 * P.N, S.pot, S.pot_lo, S.info, i,
                               x + 1 == P.nx ? 1 - P.nx : 1, x == 0 ? P.nx - 1 : -1,
                               (y + 1 == P.ny ? 1 - P.ny : 1) * nx, (y == 0 ? P.ny - 1 : -1) * nx,
                               (z + 1 == P.nz ? 1 - P.nz : 1) * nxy, (z == 0 ? P.nz - 1 : -1) * nxy};
        const SitePre pre = load_site_pre(S, (size_t)P.N, i);
        collide_site<D, GlobalPops, GlobalStencil, VD>(P, S, x, y, z, i, first, pops, st, pre,
                                                       ob);
    }
}

__device__ __forceinline__ size_t grid_block_index()
{
    return blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
}

__device__ __forceinline__ size_t grid_block_count()
{
    return (size_t)gridDim.x * gridDim.y * gridDim.z;
}

// 4 resident blocks per SM (128 registers per thread; a few bytes of L1-cached spill):
// the kernel is memory-latency bound and needs the warps.
template <int D, bool VD = false>
__global__ void __launch_bounds__(BX, 4) k_collide(CollideParams<VD> P, State S, int first)
{
    float ob[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; k++)
        ob[k] = 0.0f;
    collide_global_site<D, VD>(P, S, first, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y,
                               blockIdx.z, ob);
    block_obs_partials(ob, S.obs_partials, grid_block_index(), grid_block_count());
}

// Tensor maps of the three population sets of one buffer, each a 4D tensor
// (x, y, z, population array), box TX x TY x 1 x (all arrays of the set).
struct PopMaps {
    CUtensorMap g, fphi, frho;
};

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

template <int D>
constexpr int staged_pop_floats()
{
    return 3 * Lat<D>::Q * BX;   // the phase-field sets
}

template <int D, int TY>
constexpr size_t staged_smem_bytes()
{
    return (size_t)staged_pop_floats<D>() * 4 + (size_t)Halo<D, TY>::N * (16 + 8);
}

// The step on a TX x TY tile: thread 0 issues a 4D TMA tensor copy of the tile's phase-field
// populations (completing on an mbarrier) while the block loads the stencil fields of the
// tile and its one-site halo (periodic wrap) cooperatively; the momentum and charge
// populations are read from global memory by their own site's thread. Needs nx % 4 == 0 (16-byte row strides for the tensor
// maps). A barrier wait that never completes sets flag bit 1, waits once more for the copies
// in flight and leaves the block (its partials zeroed).
constexpr int STAGE_MAX_POLLS = 1 << 22;
template <int D, int TY, bool VD = false>
__device__ __forceinline__ void collide_staged_tile(const CollideParams<VD> &P, const State &S,
                                                    int first,
                                                    const PopMaps *maps, int x0, int y0, int z,
                                                    size_t blk, size_t nblk)
{
    using L = Lat<D>;
    using H = Halo<D, TY>;
    constexpr int Q = L::Q, HN = H::N, HX = H::HX, HY = H::HY, TX = H::TX;
    extern __shared__ __align__(128) float spop[];   // populations, then halo fields
    float4 *sha = reinterpret_cast<float4 *>(spop + staged_pop_floats<D>());
    float2 *shb = reinterpret_cast<float2 *>(sha + HN);
    __shared__ __align__(8) uint64_t bar;
    const int t = threadIdx.x, tx = t & (TX - 1), ty = t / TX;
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (t == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)staged_pop_floats<D>() * 4u);
        tma_load_4d(spop, &maps->fphi, x0, y0, z, 0, &bar);
    }
    const size_t N = P.N;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < P.nx && y < P.ny;
    const int i = active ? x + P.nx * (y + P.ny * z) : 0;
    const SitePre pre = load_site_pre(S, N, i);   // issued now, used after the staging
    // the momentum and charge populations, issued now into registers (their DRAM latency
    // overlaps the halo loads; the momentum ones become ten moments first thing)
    StagedPops<D> pops;
#pragma unroll
    for (int n = 0; n < Q; n++)
        pops.gr[n] = S.g[n * (int)N + i];
#pragma unroll
    for (int n = 0; n < L::QS; n++)
        pops.rr[n] = S.frho[n * (int)N + i];
    // stencil fields of the tile and its halo, periodic in every direction: every load of
    // this thread is issued before the first shared-memory store
    constexpr int HIT = (HN + BX - 1) / BX;
    const float *phi0 = S.phi, *phi1 = S.phi + N, *phi2 = S.phi + 2 * N;
    float hv[HIT][5];
    uint8_t hinf[HIT];
#pragma unroll
    for (int k = 0; k < HIT; k++) {
        const int e = t + k * BX;
        if (e < HN) {
            const int hx = e % HX, hy = (e / HX) % HY, hz = e / (HX * HY);
            int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = D == 3 ? z - 1 + hz : z;
            gx += gx < 0 ? P.nx : (gx >= P.nx ? -P.nx : 0);
            gy += gy < 0 ? P.ny : (gy >= P.ny ? -P.ny : 0);
            gz += gz < 0 ? P.nz : (gz >= P.nz ? -P.nz : 0);
            const int g = gx + P.nx * (gy + P.ny * gz);
            hv[k][0] = phi0[g];
            hv[k][1] = phi1[g];
            hv[k][2] = phi2[g];
            hv[k][3] = S.pot[g];
            hv[k][4] = S.pot_lo[g];
            hinf[k] = S.info[g];
        }
    }
#pragma unroll
    for (int k = 0; k < HIT; k++) {
        const int e = t + k * BX;
        if (e < HN) {
            sha[e] = make_float4(hv[k][0], hv[k][1], hv[k][2], hv[k][3]);
            shb[e] = make_float2(hv[k][4], __int_as_float((int)hinf[k]));
        }
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, STAGE_MAX_POLLS);
    float ob[NOBS];
#pragma unroll
    for (int k = 0; k < NOBS; k++)
        ob[k] = 0.0f;
    if (__syncthreads_or(!ok)) {
        if (t == 0)
            atomicOr(S.flag, 2);
        mbar_wait_bounded(&bar, 0, STAGE_MAX_POLLS);
        block_obs_partials(ob, S.obs_partials, blk, nblk);
        return;
    }
    const int h = (tx + 1) + HX * ((ty + 1) + HY * (D == 3 ? 1 : 0));
    if (active && (__float_as_int(shb[h].y) & 3) == PT_FLUID) {
        pops.s = spop;
        pops.t = t;
        const SmemStencil<D, TY> st{sha, shb, h};
        collide_site<D, StagedPops<D>, SmemStencil<D, TY>, VD>(P, S, x, y, z, i, first, pops, st,
                                                               pre, ob);
    }
    block_obs_partials(ob, S.obs_partials, blk, nblk);
}

template <int D, int TY, bool VD = false>
__global__ void __launch_bounds__(BX, 4) k_collide_staged(CollideParams<VD> P, State S, int first,
                                                          const __grid_constant__ PopMaps maps)
{
    collide_staged_tile<D, TY, VD>(P, S, first, &maps, blockIdx.x * Halo<D, TY>::TX,
                                   blockIdx.y * TY, blockIdx.z, grid_block_index(),
                                   grid_block_count());
}

// Fixed-order FP64 sum of the observable partials: block k reduces observable k.
// obs[0..NOBS) receives this step's sums and obs[NOBS..2 NOBS) the previous step's (for the
// drag force balance).
constexpr int OBS_THREADS = 256;
__device__ __forceinline__ void obs_final_block(const double *__restrict__ partials,
                                                long long nblocks, double *__restrict__ obs, int k)
{
    const double *p = partials + k * nblocks;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long b = threadIdx.x;
    for (; b + 3 * OBS_THREADS < nblocks; b += 4 * OBS_THREADS) {
        a0 += p[b];
        a1 += p[b + OBS_THREADS];
        a2 += p[b + 2 * OBS_THREADS];
        a3 += p[b + 3 * OBS_THREADS];
    }
    for (; b < nblocks; b += OBS_THREADS)
        a0 += p[b];
    double a = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        a += __shfl_xor_sync(0xffffffffu, a, o);
    __shared__ double sm[OBS_THREADS / 32];
    if ((threadIdx.x & 31) == 0)
        sm[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < OBS_THREADS / 32; w++)
            t += sm[w];
        obs[NOBS + k] = obs[k];
        obs[k] = t;
    }
}

// The same sums split over NOBS x (OBS_THREADS / 32) one-warp CTAs (FP64 adds are slow on
// this part, so one CTA per observable is latency-bound): CTA (k, w) forms warp w's sum of
// obs_final_block's order and the last CTA of observable k to finish adds the warp sums in
// order. Same bits as obs_final_block (one CTA per observable, as the batched form sums).
// cnt[NOBS] must be zero before the first launch; the last
// CTA resets it.
__global__ void __launch_bounds__(32) k_obs_final_split(const double *__restrict__ partials,
                                                        long long nblocks, double *wsum,
                                                        unsigned *cnt, double *obs)
{
    constexpr int NW = OBS_THREADS / 32;
    const int k = blockIdx.x / NW, w = blockIdx.x % NW;
    const double *p = partials + k * nblocks;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long b = 32 * w + threadIdx.x;
    for (; b + 3 * OBS_THREADS < nblocks; b += 4 * OBS_THREADS) {
        a0 += p[b];
        a1 += p[b + OBS_THREADS];
        a2 += p[b + 2 * OBS_THREADS];
        a3 += p[b + 3 * OBS_THREADS];
    }
    for (; b < nblocks; b += OBS_THREADS)
        a0 += p[b];
    double a = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        a += __shfl_xor_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) {
        wsum[blockIdx.x] = a;
        __threadfence();
        if (atomicAdd(&cnt[k], 1u) == (unsigned)(NW - 1)) {
            __threadfence();
            double t = 0.0;
            for (int j = 0; j < NW; j++)
                t += __ldcg(wsum + k * NW + j);
            obs[NOBS + k] = obs[k];
            obs[k] = t;
            cnt[k] = 0u;
        }
    }
}

}  // namespace lbehd

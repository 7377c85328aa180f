// poisson.cuh -- Gauss law (Eq. 13) on the GPU: multigrid-preconditioned conjugate
// gradients on the per-step increment of the potential.
//
// Each step solves A delta = r0 with r0 = b - A phi^{n-1}, where A is the 7/5-point
// finite-volume operator of div(eps grad .) (face eps = (eps_i + eps_j)/2, Dirichlet value
// on the solid node with face eps = eps_fluid, zero flux elsewhere) and b = rho_e + Dirichlet
// terms. The potential is stored as a compensated pair of floats (hi + lo); r0 is formed
// from compensated differences of it, so the FP32 iteration on the small increment is not
// limited by the rounding of phi itself, and differences of phi (E, the conduction source
// of Eq. 14) keep ~FP64 accuracy. The warm
// start is the increment of two steps back (consecutive increments alternate in sign
// because the charge collision relaxes its first moments with 1 - 1/tau_rho ~ -1).
//
// Preconditioner: one symmetric V-cycle of cell-centred geometric multigrid. Coarse cells
// aggregate 2x2(x2) fine cells; coarse face coefficients are the sums of the fine faces
// they cover and the coarse diagonal is the sum of the children's diagonals minus twice
// their internal faces (Galerkin operator for piecewise-constant prolongation), both scaled
// by mg_scale (< 1 over-corrects, which compensates the weak constant interpolation).
// Smoother: red-black Gauss-Seidel, (red, black)^nu before and (black, red)^nu after the
// coarse correction; the coarsest level runs symmetric sweeps. A cell is active when its
// diagonal is positive.
//
// CG scalars (alpha, beta, r.z, ...) stay in device memory, so an iteration needs no host
// round trip; reductions are FP32 within a warp and FP64 across warps and blocks.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace lbehd {

struct MgDims {
    int nx, ny, nz;
};

struct CgScalars {
    double rz;        // r . z of the current iteration
    double rz_old;
    double pq;        // p . A p
    double rr;        // ||r||^2 (current residual)
    double bb;        // ||b||^2
    double alpha, beta;
    double tol2;      // tol^2 (set by the host)
    int iters;        // iterations of the current pass
    int max_iter;
    int done;         // 1 once rr <= tol2 * bb or iters >= max_iter
    int converged;
    int step_iters;   // iterations of the current step, all passes
    int nonconv;      // sticky: some pass stopped at max_iter without converging
    long long total_iters;
};

__device__ __forceinline__ size_t cell(const MgDims &d, int x, int y, int z)
{
    return (size_t)x + (size_t)d.nx * ((size_t)y + (size_t)d.ny * (size_t)z);
}

__device__ __forceinline__ int wrapp(int v, int n) { return v + 1 == n ? 0 : v + 1; }
__device__ __forceinline__ int wrapm(int v, int n) { return v == 0 ? n - 1 : v - 1; }

// Block reduction of up to 4 FP32 values into FP64 partials[k * nblk + blk].
template <int NV>
__device__ __forceinline__ void block_partials(float (&v)[NV], double *partials)
{
    __shared__ double sm[NV][BX / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const float s = warp_sum(v[k]);
        if (lane == 0)
            sm[k][wid] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < BX / 32; w++)
            acc += sm[threadIdx.x][w];
        const size_t nblk = (size_t)gridDim.x * gridDim.y * gridDim.z;
        const size_t blk = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
        partials[threadIdx.x * nblk + blk] = acc;
    }
}

// ---------------------------------------------------------------- level-0 operator

// Face coefficients to the +x/+y/+z neighbours and the diagonal (all faces, Dirichlet
// faces included) from eps and the node classes.
template <int D>
__global__ void __launch_bounds__(BX) k_mg_setup0(Params P, const float *__restrict__ eps,
                                                  const uint8_t *__restrict__ info,
                                                  float *__restrict__ Dg, float *__restrict__ kx,
                                                  float *__restrict__ ky, float *__restrict__ kz)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx)
        return;
    const MgDims d{P.nx, P.ny, P.nz};
    const size_t i = cell(d, x, y, z);
    float kp[3] = {0.f, 0.f, 0.f}, diag = 0.0f;
    if ((info[i] & 3) == PT_FLUID) {
        const float ei = eps[i];
        const size_t nb[6] = {cell(d, wrapp(x, d.nx), y, z), cell(d, wrapm(x, d.nx), y, z),
                              cell(d, x, wrapp(y, d.ny), z), cell(d, x, wrapm(y, d.ny), z),
                              cell(d, x, y, wrapp(z, d.nz)), cell(d, x, y, wrapm(z, d.nz))};
#pragma unroll
        for (int f = 0; f < 2 * D; f++) {
            const int pt = info[nb[f]] & 3;
            float k = 0.0f;
            if (pt == PT_FLUID)
                k = 0.5f * (ei + eps[nb[f]]);
            else if (pt == PT_DIRICHLET)
                k = ei;
            diag += k;
            if ((f & 1) == 0)
                kp[f >> 1] = pt == PT_FLUID ? k : 0.0f;
        }
    }
    Dg[i] = diag;
    kx[i] = kp[0];
    ky[i] = kp[1];
    kz[i] = kp[2];
}

// Galerkin coarsening (scaled) of one level.
__global__ void __launch_bounds__(BX) k_mg_coarsen(MgDims f, MgDims c, int cz2, float scale,
                                                   const float *__restrict__ Df,
                                                   const float *__restrict__ kxf,
                                                   const float *__restrict__ kyf,
                                                   const float *__restrict__ kzf,
                                                   float *__restrict__ Dc, float *__restrict__ kxc,
                                                   float *__restrict__ kyc, float *__restrict__ kzc)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y, Z = blockIdx.z;
    if (X >= c.nx)
        return;
    const int nzc = cz2 ? 2 : 1;
    float dsum = 0.f, internal = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int g = 0; g < nzc; g++) {
                const int x = 2 * X + a, y = 2 * Y + b, z = nzc * Z + g;
                if (x >= f.nx || y >= f.ny || z >= f.nz)
                    continue;
                const size_t i = cell(f, x, y, z);
                dsum += Df[i];
                // +x face: internal if the +x child exists in this coarse cell
                if (a == 0 && x + 1 < f.nx)
                    internal += kxf[i];
                else
                    fx += kxf[i];
                if (b == 0 && y + 1 < f.ny)
                    internal += kyf[i];
                else
                    fy += kyf[i];
                if (cz2) {
                    if (g == 0 && z + 1 < f.nz)
                        internal += kzf[i];
                    else
                        fz += kzf[i];
                }
            }
    const size_t I = cell(c, X, Y, Z);
    const float dc = dsum - 2.0f * internal;
    Dc[I] = dc > 0.0f ? scale * dc : 0.0f;
    kxc[I] = scale * fx;
    kyc[I] = scale * fy;
    kzc[I] = scale * fz;
}

// ---------------------------------------------------------------- smoother / transfers

__device__ __forceinline__ float offdiag_sum(const MgDims &d, size_t i, int x, int y, int z,
                                             const float *__restrict__ kx,
                                             const float *__restrict__ ky,
                                             const float *__restrict__ kz,
                                             const float *__restrict__ v)
{
    const int xp = wrapp(x, d.nx), xm = wrapm(x, d.nx);
    const int yp = wrapp(y, d.ny), ym = wrapm(y, d.ny);
    float s = kx[i] * v[cell(d, xp, y, z)] + kx[cell(d, xm, y, z)] * v[cell(d, xm, y, z)] +
              ky[i] * v[cell(d, x, yp, z)] + ky[cell(d, x, ym, z)] * v[cell(d, x, ym, z)];
    if (d.nz > 1) {
        const int zp = wrapp(z, d.nz), zm = wrapm(z, d.nz);
        s += kz[i] * v[cell(d, x, y, zp)] + kz[cell(d, x, y, zm)] * v[cell(d, x, y, zm)];
    }
    return s;
}

// One red-black Gauss-Seidel half sweep of A x = b on one level.
__global__ void __launch_bounds__(BX) k_mg_gs(MgDims d, const float *__restrict__ Dg,
                                              const float *__restrict__ kx,
                                              const float *__restrict__ ky,
                                              const float *__restrict__ kz,
                                              const float *__restrict__ b, float *__restrict__ xv,
                                              int color)
{
    const int y = blockIdx.y, z = blockIdx.z;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((y + z + color) & 1);
    if (x >= d.nx)
        return;
    const size_t i = cell(d, x, y, z);
    const float di = Dg[i];
    if (di <= 0.0f)
        return;
    xv[i] = (b[i] + offdiag_sum(d, i, x, y, z, kx, ky, kz, xv)) / di;
}

// b_c = restriction (sum over children) of the fine residual b_f - A_f x_f.
__global__ void __launch_bounds__(BX) k_mg_restrict(MgDims f, MgDims c, int cz2,
                                                    const float *__restrict__ Df,
                                                    const float *__restrict__ kx,
                                                    const float *__restrict__ ky,
                                                    const float *__restrict__ kz,
                                                    const float *__restrict__ bf,
                                                    const float *__restrict__ xf,
                                                    float *__restrict__ bc)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y, Z = blockIdx.z;
    if (X >= c.nx)
        return;
    const int nzc = cz2 ? 2 : 1;
    float acc = 0.0f;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int g = 0; g < nzc; g++) {
                const int x = 2 * X + a, y = 2 * Y + b, z = nzc * Z + g;
                if (x >= f.nx || y >= f.ny || z >= f.nz)
                    continue;
                const size_t i = cell(f, x, y, z);
                const float di = Df[i];
                if (di <= 0.0f)
                    continue;
                acc += bf[i] - (di * xf[i] - offdiag_sum(f, i, x, y, z, kx, ky, kz, xf));
            }
    bc[cell(c, X, Y, Z)] = acc;
}

// x_f += x_c(parent) on active fine cells.
__global__ void __launch_bounds__(BX) k_mg_prolong(MgDims f, MgDims c, int cz2,
                                                   const float *__restrict__ Df,
                                                   const float *__restrict__ xc,
                                                   float *__restrict__ xf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= f.nx)
        return;
    const size_t i = cell(f, x, y, z);
    if (Df[i] <= 0.0f)
        return;
    xf[i] += xc[cell(c, x >> 1, y >> 1, cz2 ? (z >> 1) : z)];
}

// ---------------------------------------------------------------- small-level tail

constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_MAX_CELLS = 1024;   // cells of the finest tail level
constexpr int TAIL_THREADS = 1024;

struct TailLevels {
    int nl;                            // levels in the tail (the last is the coarsest)
    int nu, coarse;
    MgDims d[TAIL_MAX_LEVELS];
    int cz2[TAIL_MAX_LEVELS];
    int off[TAIL_MAX_LEVELS];          // offset of each level in the shared arrays
    const float *D[TAIL_MAX_LEVELS], *kx[TAIL_MAX_LEVELS], *ky[TAIL_MAX_LEVELS],
        *kz[TAIL_MAX_LEVELS];
    const float *b0;                   // right-hand side of the finest tail level (global)
    float *x0;                         // its solution (global)
    int total;                         // cells of all tail levels
};

// The V-cycle on every level from the tail's finest down, in shared memory, one CTA. Thread t
// owns cell t of every tail level (levels have <= TAIL_THREADS cells), so its coordinates are
// computed once. Same arithmetic, cell by cell, as the multi-launch levels above it.
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(TailLevels T)
{
    extern __shared__ float sm[];
    const int tot = T.total, t = threadIdx.x;
    float *sD = sm, *skx = sm + tot, *sky = sm + 2 * tot, *skz = sm + 3 * tot, *sx = sm + 4 * tot,
          *sb = sm + 5 * tot;
    int cx[TAIL_MAX_LEVELS], cy[TAIL_MAX_LEVELS], cz[TAIL_MAX_LEVELS];
    bool own[TAIL_MAX_LEVELS];
#pragma unroll
    for (int l = 0; l < TAIL_MAX_LEVELS; l++) {
        own[l] = false;
        cx[l] = cy[l] = cz[l] = 0;
        if (l < T.nl) {
            const MgDims d = T.d[l];
            const int n = d.nx * d.ny * d.nz, o = T.off[l];
            own[l] = t < n;
            if (own[l]) {
                cx[l] = t % d.nx;
                cy[l] = (t / d.nx) % d.ny;
                cz[l] = t / (d.nx * d.ny);
                sD[o + t] = T.D[l][t];
                skx[o + t] = T.kx[l][t];
                sky[o + t] = T.ky[l][t];
                skz[o + t] = T.kz[l][t];
                sx[o + t] = 0.0f;
                if (l == 0)
                    sb[t] = T.b0[t];
            }
        }
    }
    __syncthreads();
    auto gs = [&](int l, int color) {
        if (own[l] && ((cx[l] + cy[l] + cz[l]) & 1) == color) {
            const int o = T.off[l];
            const float di = sD[o + t];
            if (di > 0.0f)
                sx[o + t] = (sb[o + t] + offdiag_sum(T.d[l], t, cx[l], cy[l], cz[l], skx + o, sky + o,
                                                     skz + o, sx + o)) / di;
        }
        __syncthreads();
    };
    // down: smooth, restrict
#pragma unroll 1
    for (int l = 0; l + 1 < T.nl; l++) {
        for (int s = 0; s < T.nu; s++) {
            gs(l, 0);
            gs(l, 1);
        }
        if (own[l + 1]) {
            const MgDims f = T.d[l];
            const int fo = T.off[l], nzc = T.cz2[l] ? 2 : 1;
            float acc = 0.0f;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int g = 0; g < nzc; g++) {
                        const int x = 2 * cx[l + 1] + a, y = 2 * cy[l + 1] + b,
                                  z = nzc * cz[l + 1] + g;
                        if (x >= f.nx || y >= f.ny || z >= f.nz)
                            continue;
                        const int i = (int)cell(f, x, y, z);
                        const float di = sD[fo + i];
                        if (di <= 0.0f)
                            continue;
                        acc += sb[fo + i] - (di * sx[fo + i] - offdiag_sum(f, i, x, y, z, skx + fo,
                                                                           sky + fo, skz + fo, sx + fo));
                    }
            sb[T.off[l + 1] + t] = acc;
        }
        __syncthreads();
    }
    // coarsest: symmetric sweeps
    const int lc = T.nl - 1;
#pragma unroll 1
    for (int s = 0; s < T.coarse; s++) {
        gs(lc, 0);
        gs(lc, 1);
        gs(lc, 1);
        gs(lc, 0);
    }
    // up: prolong, smooth
#pragma unroll 1
    for (int l = T.nl - 2; l >= 0; l--) {
        if (own[l]) {
            const int fo = T.off[l];
            if (sD[fo + t] > 0.0f)
                sx[fo + t] += sx[T.off[l + 1] + (int)cell(T.d[l + 1], cx[l] >> 1, cy[l] >> 1,
                                                           T.cz2[l] ? (cz[l] >> 1) : cz[l])];
        }
        __syncthreads();
        for (int s = 0; s < T.nu; s++) {
            gs(l, 1);
            gs(l, 0);
        }
    }
    if (own[0])
        T.x0[t] = sx[t];
}

// ---------------------------------------------------------------- CG on level 0

// r = b - A (phi + delta) from the compensated potential; partials of ||r||^2 and ||b||^2.
// Only differences of the potential enter: r_i = rho_i + sum_faces k_f (phi_j - phi_i), with
// phi_j - phi_i = (hi_j - hi_i) + (lo_j - lo_i) + (delta_j - delta_i). Neighbouring hi parts
// are close, so their difference is exact in FP32, and r keeps the accuracy an FP64
// evaluation of b - A phi would have, in FP32 arithmetic.
template <int D>
__global__ void __launch_bounds__(BX) k_pcg_init(Params P, const float *__restrict__ pot,
                                                 const float *__restrict__ pot_lo,
                                                 const float *__restrict__ delta,
                                                 const float *__restrict__ eps,
                                                 const float *__restrict__ rho,
                                                 const uint8_t *__restrict__ info,
                                                 const float *__restrict__ Dg,
                                                 float *__restrict__ r, double *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    float v[2] = {0.f, 0.f};
    if (x < P.nx) {
        const MgDims d{P.nx, P.ny, P.nz};
        const size_t i = cell(d, x, y, z);
        float ri = 0.0f;
        if (Dg[i] > 0.0f) {
            const float ei = eps[i], hi = pot[i], lo = pot_lo[i], di = delta[i];
            float b = rho[i];
            ri = b;
            const size_t nb[6] = {cell(d, wrapp(x, d.nx), y, z), cell(d, wrapm(x, d.nx), y, z),
                                  cell(d, x, wrapp(y, d.ny), z), cell(d, x, wrapm(y, d.ny), z),
                                  cell(d, x, y, wrapp(z, d.nz)), cell(d, x, y, wrapm(z, d.nz))};
#pragma unroll
            for (int f = 0; f < 2 * D; f++) {
                const size_t j = nb[f];
                const int pt = info[j] & 3;
                if (pt == PT_FLUID) {
                    const float dphi = (pot[j] - hi) + (pot_lo[j] - lo) + (delta[j] - di);
                    ri += 0.5f * (ei + eps[j]) * dphi;
                } else if (pt == PT_DIRICHLET) {
                    const float dphi = (pot[j] - hi) + (pot_lo[j] - lo) - di;
                    ri += ei * dphi;
                    b += ei * (pot[j] + pot_lo[j]);
                }
            }
            v[0] = ri * ri;
            v[1] = b * b;
        }
        r[i] = ri;
    }
    block_partials<2>(v, partials);
}

// p = z + beta p (beta = 0 on the first iteration).
__global__ void __launch_bounds__(BX) k_pcg_p(size_t n, const float *__restrict__ zv,
                                              float *__restrict__ p, const CgScalars *__restrict__ s)
{
    const float beta = s->iters == 0 ? 0.0f : (float)s->beta;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = zv[i] + (beta != 0.0f ? beta * p[i] : 0.0f);
}

// q = A p with the operator of this step (from eps and the node classes; the multigrid
// hierarchy may be a few steps old, which only changes the preconditioner) and partials of
// p . q. Dirichlet neighbours hold no correction (p = 0 there).
template <int D>
__global__ void __launch_bounds__(BX) k_pcg_Ap(Params P, const float *__restrict__ eps,
                                               const uint8_t *__restrict__ info,
                                               const float *__restrict__ Dg,
                                               const float *__restrict__ p, float *__restrict__ q,
                                               double *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    float v[1] = {0.f};
    if (x < P.nx) {
        const MgDims d{P.nx, P.ny, P.nz};
        const size_t i = cell(d, x, y, z);
        float qi = 0.0f;
        if (Dg[i] > 0.0f) {
            const float ei = eps[i], pi = p[i];
            const size_t nb[6] = {cell(d, wrapp(x, d.nx), y, z), cell(d, wrapm(x, d.nx), y, z),
                                  cell(d, x, wrapp(y, d.ny), z), cell(d, x, wrapm(y, d.ny), z),
                                  cell(d, x, y, wrapp(z, d.nz)), cell(d, x, y, wrapm(z, d.nz))};
#pragma unroll
            for (int f = 0; f < 2 * D; f++) {
                const size_t j = nb[f];
                const int pt = info[j] & 3;
                if (pt == PT_FLUID)
                    qi += 0.5f * (ei + eps[j]) * (pi - p[j]);
                else if (pt == PT_DIRICHLET)
                    qi += ei * pi;
            }
            v[0] = pi * qi;
        }
        q[i] = qi;
    }
    block_partials<1>(v, partials);
}

// delta += alpha p, r -= alpha q, partials of ||r||^2.
__global__ void __launch_bounds__(BX) k_pcg_update(size_t n, const float *__restrict__ p,
                                                   const float *__restrict__ q,
                                                   float *__restrict__ delta, float *__restrict__ r,
                                                   const CgScalars *__restrict__ s,
                                                   double *__restrict__ partials)
{
    const float a = (float)s->alpha;
    float v[1] = {0.f};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        delta[i] += a * p[i];
        const float ri = r[i] - a * q[i];
        r[i] = ri;
        v[0] += ri * ri;
    }
    // 1D grid: reuse the generic block reduction (gridDim.y = gridDim.z = 1)
    block_partials<1>(v, partials);
}

// partials of r . z
__global__ void __launch_bounds__(BX) k_pcg_dot(size_t n, const float *__restrict__ a,
                                                const float *__restrict__ b,
                                                double *__restrict__ partials)
{
    float v[1] = {0.0f};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        v[0] += a[i] * b[i];
    block_partials<1>(v, partials);
}

// Fixed-order FP64 sum of nv partial arrays and the CG scalar update that follows.
//   op 0: start     rr, bb            -> done if rr <= tol2 bb (resets the step counter)
//   op 4: restart   as op 0 for a refinement pass (keeps the step counter)
//   op 1: r.z       rz                -> beta = rz / rz_old, rz_old = rz
//   op 2: p.Ap      pq                -> alpha = rz / pq
//   op 3: ||r||^2   rr                -> iters++, done / converged
// With use_cond, ops 0, 4 and 3 also set the graph's while-loop condition to !done; with
// use_ref, op 0 clears and op 3 sets the condition of the refinement block.
constexpr int SCALAR_THREADS = 1024;
__global__ void __launch_bounds__(SCALAR_THREADS) k_pcg_scalar(const double *__restrict__ partials,
                                                               long long nblocks, int nv, int op,
                                                               CgScalars *__restrict__ s,
                                                               cudaGraphConditionalHandle cond,
                                                               int use_cond,
                                                               cudaGraphConditionalHandle cond_ref,
                                                               int use_ref)
{
    __shared__ double sm[2][SCALAR_THREADS / 32];
    double tot[2] = {0.0, 0.0};
    for (int k = 0; k < nv; k++) {
        const double *p = partials + k * nblocks;
        double a0 = 0.0, a1 = 0.0;
        long long b = threadIdx.x;
        for (; b + SCALAR_THREADS < nblocks; b += 2 * SCALAR_THREADS) {
            a0 += p[b];
            a1 += p[b + SCALAR_THREADS];
        }
        if (b < nblocks)
            a0 += p[b];
        double a = a0 + a1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0)
            sm[k][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        for (int k = 0; k < nv; k++) {
            double a = sm[k][threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                a += __shfl_xor_sync(0xffffffffu, a, o);
            tot[k] = a;
        }
    }
    if (threadIdx.x != 0)
        return;
    if (op == 0 || op == 4) {
        s->rr = tot[0];
        s->bb = tot[1];
        s->iters = 0;
        if (op == 0)
            s->step_iters = 0;
        s->converged = s->rr <= s->tol2 * s->bb || s->rr < 1e-60;
        s->done = s->converged || s->max_iter <= 0;
    } else if (op == 1) {
        s->rz = tot[0];
        s->beta = s->iters == 0 || s->rz_old == 0.0 ? 0.0 : s->rz / s->rz_old;
        s->rz_old = s->rz;
    } else if (op == 2) {
        s->pq = tot[0];
        s->alpha = (!s->done && s->pq > 0.0) ? s->rz / s->pq : 0.0;
    } else if (!s->done) {
        s->rr = tot[0];
        s->iters += 1;
        s->step_iters += 1;
        s->total_iters += 1;
        s->converged = s->rr <= s->tol2 * s->bb || s->rr < 1e-60;
        s->done = s->converged || s->iters >= s->max_iter;
        if (s->done && !s->converged)
            s->nonconv = 1;
    }
    if (use_cond && op != 1 && op != 2)
        cudaGraphSetConditional(cond, s->done ? 0u : 1u);
    // refinement check runs only when the main pass iterated
    if (use_ref && op == 0)
        cudaGraphSetConditional(cond_ref, 0u);
    if (use_ref && op == 3)
        cudaGraphSetConditional(cond_ref, 1u);
}

// phi += delta on active cells, phi kept as the compensated pair hi + lo (two-sum in FP32:
// the rounding error of hi + delta is carried into lo); acc += delta when acc is given
// (accumulates a refinement correction into the step's increment).
__global__ void __launch_bounds__(BX) k_pcg_apply(size_t n, const float *__restrict__ Dg,
                                                  const float *__restrict__ delta,
                                                  float *__restrict__ acc,
                                                  float *__restrict__ pot,
                                                  float *__restrict__ pot_lo)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        if (Dg[i] <= 0.0f)
            continue;
        const float d = delta[i];
        if (acc)
            acc[i] += d;
        const float hi = pot[i];
        const float t = hi + d;                       // two-sum: t + err = hi + d exactly
        const float bv = t - hi;
        const float err = (hi - (t - bv)) + (d - bv);
        const float lo = pot_lo[i] + err;
        const float s = t + lo;                       // renormalise the pair
        pot[i] = s;
        pot_lo[i] = lo - (s - t);
    }
}

}  // namespace lbehd

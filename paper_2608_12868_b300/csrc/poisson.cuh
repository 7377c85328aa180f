// poisson.cuh -- Gauss law (Eq. 13) on the GPU: multigrid-preconditioned conjugate
// gradients on the per-step increment of the potential.
//
// Each step solves A delta = r0 with r0 = b - A phi^{n-1}, where A is the 7/5-point
// finite-volume operator of div(eps grad .) (face eps = (eps_i + eps_j)/2, Dirichlet value
// on the solid node with face eps = eps_fluid, zero flux elsewhere) and b = rho_e + Dirichlet
// terms. The potential is stored as a compensated pair of floats (hi + lo); r0 is formed
// from compensated differences of it, so the FP32 iteration on the small increment is not
// limited by the rounding of phi itself, and differences of phi (E, the conduction source
// of Eq. 14) keep ~FP64 accuracy. The warm start is the combination of the last two
// steps' increments with the least residual (k_pcg_init_mr), or the increment of two steps
// back alone (consecutive increments alternate in sign because the charge collision relaxes
// its first moments with 1 - 1/tau_rho ~ -1).
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
//
// Every multiply-add of these kernels is written out with the rounding intrinsics (fmul /
// fadd / fma), so the compiler cannot fuse or split operations differently from one kernel to
// the next: the single-instance and the batched kernels, which inline the same bodies,
// produce the same bits. The stencil bodies issue all their loads before testing the node
// classes (every index is in range), so a thread waits for one memory round trip, not a
// chain of dependent ones.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace lbehd {

// Lattice extents of one level, with the constants of a multiply-high division by nx, ny and
// nx / 2 (cell coordinates from a flat index without a hardware divide).
struct MgDims {
    int nx, ny, nz;
    uint32_t mx, my, mh;         // multipliers
    uint32_t sx, sy, sh;         // shifts
};

// n / d for 0 <= n < 2^31 as (hi32(n m) + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1 (round-up method; the sum fits 32 bits for n < 2^31).
inline void fastdiv_constants(uint32_t d, uint32_t &m, uint32_t &s)
{
    s = 0;
    while ((1ull << s) < d)
        s++;
    m = (uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1);
}

inline MgDims mg_dims(int nx, int ny, int nz)
{
    MgDims d{nx, ny, nz, 0, 0, 0, 0, 0, 0};
    fastdiv_constants((uint32_t)nx, d.mx, d.sx);
    fastdiv_constants((uint32_t)ny, d.my, d.sy);
    fastdiv_constants((uint32_t)(nx / 2 > 0 ? nx / 2 : 1), d.mh, d.sh);
    return d;
}

__device__ __forceinline__ int fdiv(int n, uint32_t m, uint32_t s)
{
    return (int)((__umulhi((uint32_t)n, m) + (uint32_t)n) >> s);
}

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
    int refine;       // the step's first pass iterated (a refinement check follows)
    long long total_iters;
};

// Site indices fit 32 bits (19 N < 2^31 is checked at init).
__device__ __forceinline__ int cell(const MgDims &d, int x, int y, int z)
{
    return x + d.nx * (y + d.ny * z);
}

__device__ __forceinline__ void cell_xyz(const MgDims &d, int c, int &x, int &y, int &z)
{
    const int r = fdiv(c, d.mx, d.sx);
    x = c - r * d.nx;
    z = fdiv(r, d.my, d.sy);
    y = r - z * d.ny;
}

// Indices of the six neighbours of cell i = (x, y, z), periodic in every direction
// (+x, -x, +y, -y, +z, -z; in 2D the z neighbours are the cell itself).
struct Nb6 {
    int n[6];
};

__device__ __forceinline__ Nb6 nb6(const MgDims &d, int i, int x, int y, int z)
{
    const int sy = d.nx, sz = d.nx * d.ny, sn = sz * d.nz;
    Nb6 r;
    r.n[0] = i + (x + 1 == d.nx ? 1 - d.nx : 1);
    r.n[1] = i + (x == 0 ? d.nx - 1 : -1);
    r.n[2] = i + (y + 1 == d.ny ? sy - sz : sy);
    r.n[3] = i + (y == 0 ? sz - sy : -sy);
    r.n[4] = i + (z + 1 == d.nz ? sz - sn : sz);
    r.n[5] = i + (z == 0 ? sn - sz : -sz);
    return r;
}

// Block reduction of up to 4 FP32 values into FP64 partials[k * nblk + blk].
template <int NV>
__device__ __forceinline__ void block_partials(float (&v)[NV], double *partials, size_t blk,
                                               size_t nblk)
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
        partials[threadIdx.x * nblk + blk] = acc;
    }
}

template <int NV>
__device__ __forceinline__ void block_partials(float (&v)[NV], double *partials)
{
    block_partials<NV>(v, partials, grid_block_index(), grid_block_count());
}

// ---------------------------------------------------------------- level-0 operator

// Face coefficients to the +x/+y/+z neighbours and the diagonal (all faces, Dirichlet
// faces included) from eps and the node classes.
template <int D>
__device__ __forceinline__ void mg_setup0_cell(const MgDims &d, const float *eps,
                                               const uint8_t *info,
                                               float *Dg, float *kx,
                                               float *ky, float *kz,
                                               int x, int y, int z)
{
    const int i = cell(d, x, y, z);
    float kp[3] = {0.f, 0.f, 0.f}, diag = 0.0f;
    const Nb6 nb = nb6(d, i, x, y, z);
    const int pti = info[i] & 3;
    const float ei = eps[i];
    int pt[2 * D];
    float ej[2 * D];
#pragma unroll
    for (int f = 0; f < 2 * D; f++) {
        pt[f] = info[nb.n[f]] & 3;
        ej[f] = eps[nb.n[f]];
    }
    if (pti == PT_FLUID) {
#pragma unroll
        for (int f = 0; f < 2 * D; f++) {
            float k = 0.0f;
            if (pt[f] == PT_FLUID)
                k = __fmul_rn(0.5f, __fadd_rn(ei, ej[f]));
            else if (pt[f] == PT_DIRICHLET)
                k = ei;
            diag = __fadd_rn(diag, k);
            if ((f & 1) == 0)
                kp[f >> 1] = pt[f] == PT_FLUID ? k : 0.0f;
        }
    }
    Dg[i] = diag;
    kx[i] = kp[0];
    ky[i] = kp[1];
    kz[i] = kp[2];
}

template <int D>
__global__ void __launch_bounds__(BX) k_mg_setup0(MgDims d, const float *__restrict__ eps,
                                                  const uint8_t *__restrict__ info,
                                                  float *__restrict__ Dg, float *__restrict__ kx,
                                                  float *__restrict__ ky, float *__restrict__ kz)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < d.nx)
        mg_setup0_cell<D>(d, eps, info, Dg, kx, ky, kz, x, blockIdx.y, blockIdx.z);
}

// Galerkin coarsening (scaled) of one level.
__device__ __forceinline__ void mg_coarsen_cell(const MgDims &f, const MgDims &c, int cz2,
                                                float scale, const float *Df,
                                                const float *kxf,
                                                const float *kyf,
                                                const float *kzf,
                                                float *Dc, float *kxc,
                                                float *kyc, float *kzc,
                                                int X, int Y, int Z)
{
    const int nzc = cz2 ? 2 : 1;
    float dsum = 0.f, internal = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int g = 0; g < nzc; g++) {
                const int x = 2 * X + a, y = 2 * Y + b, z = nzc * Z + g;
                if (x >= f.nx || y >= f.ny || z >= f.nz)
                    continue;
                const int i = cell(f, x, y, z);
                dsum = __fadd_rn(dsum, Df[i]);
                // +x face: internal if the +x child exists in this coarse cell
                if (a == 0 && x + 1 < f.nx)
                    internal = __fadd_rn(internal, kxf[i]);
                else
                    fx = __fadd_rn(fx, kxf[i]);
                if (b == 0 && y + 1 < f.ny)
                    internal = __fadd_rn(internal, kyf[i]);
                else
                    fy = __fadd_rn(fy, kyf[i]);
                if (cz2) {
                    if (g == 0 && z + 1 < f.nz)
                        internal = __fadd_rn(internal, kzf[i]);
                    else
                        fz = __fadd_rn(fz, kzf[i]);
                }
            }
    const int I = cell(c, X, Y, Z);
    const float dc = __fmaf_rn(-2.0f, internal, dsum);
    Dc[I] = dc > 0.0f ? __fmul_rn(scale, dc) : 0.0f;
    kxc[I] = __fmul_rn(scale, fx);
    kyc[I] = __fmul_rn(scale, fy);
    kzc[I] = __fmul_rn(scale, fz);
}

__global__ void __launch_bounds__(BX) k_mg_coarsen(MgDims f, MgDims c, int cz2, float scale,
                                                   const float *__restrict__ Df,
                                                   const float *__restrict__ kxf,
                                                   const float *__restrict__ kyf,
                                                   const float *__restrict__ kzf,
                                                   float *__restrict__ Dc, float *__restrict__ kxc,
                                                   float *__restrict__ kyc, float *__restrict__ kzc)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X < c.nx)
        mg_coarsen_cell(f, c, cz2, scale, Df, kxf, kyf, kzf, Dc, kxc, kyc, kzc, X, blockIdx.y,
                        blockIdx.z);
}

// ---------------------------------------------------------------- smoother / transfers

__device__ __forceinline__ float offdiag_sum(const MgDims &d, int i, int x, int y, int z,
                                             const float *kx,
                                             const float *ky,
                                             const float *kz,
                                             const float *v)
{
    const Nb6 nb = nb6(d, i, x, y, z);
    float s = __fmul_rn(kx[i], v[nb.n[0]]);
    s = __fmaf_rn(kx[nb.n[1]], v[nb.n[1]], s);
    s = __fmaf_rn(ky[i], v[nb.n[2]], s);
    s = __fmaf_rn(ky[nb.n[3]], v[nb.n[3]], s);
    if (d.nz > 1) {
        s = __fmaf_rn(kz[i], v[nb.n[4]], s);
        s = __fmaf_rn(kz[nb.n[5]], v[nb.n[5]], s);
    }
    return s;
}

// Gauss-Seidel update of one cell of A x = b.
__device__ __forceinline__ void mg_gs_cell(const MgDims &d, const float *Dg,
                                           const float *kx,
                                           const float *ky,
                                           const float *kz,
                                           const float *b, float *xv,
                                           int x, int y, int z)
{
    const int i = cell(d, x, y, z);
    const float di = Dg[i], bi = b[i];
    const float off = offdiag_sum(d, i, x, y, z, kx, ky, kz, xv);
    if (di > 0.0f)
        xv[i] = __fdiv_rn(__fadd_rn(bi, off), di);
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
    if (x < d.nx)
        mg_gs_cell(d, Dg, kx, ky, kz, b, xv, x, y, z);
}

// Restriction, b_c = sum over the children of the fine residual b_f - A_f x_f, in two
// passes: the residual of every fine cell (0 on inactive cells), then the sum over each
// coarse cell's children in the order (x, y, z) = (2X + a, 2Y + b, 2Z + g), a outermost
// (the shared-memory tail sums in the same order).
__device__ __forceinline__ void mg_resid_cell(const MgDims &f, const float *Df,
                                              const float *kx,
                                              const float *ky,
                                              const float *kz,
                                              const float *bf,
                                              const float *xf, float *rf,
                                              int x, int y, int z)
{
    const int i = cell(f, x, y, z);
    const float di = Df[i], xi = xf[i], bi = bf[i];
    const float Ax = __fmaf_rn(di, xi, -offdiag_sum(f, i, x, y, z, kx, ky, kz, xf));
    rf[i] = di > 0.0f ? __fsub_rn(bi, Ax) : 0.0f;
}

__device__ __forceinline__ void mg_restrict_sum_cell(const MgDims &f, const MgDims &c, int cz2,
                                                     const float *rf,
                                                     float *bc, int X, int Y, int Z)
{
    // fine nx, ny are twice the coarse ones; only z may end on a single child
    const int z0 = cz2 ? 2 * Z : Z;
    const bool z1 = cz2 && z0 + 1 < f.nz;
    const int i = cell(f, 2 * X, 2 * Y, z0), sy = f.nx, sz = f.nx * f.ny;
    const float r000 = rf[i], r001 = z1 ? rf[i + sz] : 0.0f;
    const float r010 = rf[i + sy], r011 = z1 ? rf[i + sy + sz] : 0.0f;
    const float r100 = rf[i + 1], r101 = z1 ? rf[i + 1 + sz] : 0.0f;
    const float r110 = rf[i + 1 + sy], r111 = z1 ? rf[i + 1 + sy + sz] : 0.0f;
    float acc = 0.0f;
    acc = __fadd_rn(acc, r000);
    if (z1)
        acc = __fadd_rn(acc, r001);
    acc = __fadd_rn(acc, r010);
    if (z1)
        acc = __fadd_rn(acc, r011);
    acc = __fadd_rn(acc, r100);
    if (z1)
        acc = __fadd_rn(acc, r101);
    acc = __fadd_rn(acc, r110);
    if (z1)
        acc = __fadd_rn(acc, r111);
    bc[cell(c, X, Y, Z)] = acc;
}

__global__ void __launch_bounds__(BX) k_mg_resid(MgDims f, const float *__restrict__ Df,
                                                 const float *__restrict__ kx,
                                                 const float *__restrict__ ky,
                                                 const float *__restrict__ kz,
                                                 const float *__restrict__ bf,
                                                 const float *__restrict__ xf,
                                                 float *__restrict__ rf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < f.nx)
        mg_resid_cell(f, Df, kx, ky, kz, bf, xf, rf, x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(BX) k_mg_restrict_sum(MgDims f, MgDims c, int cz2,
                                                        const float *__restrict__ rf,
                                                        float *__restrict__ bc)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X < c.nx)
        mg_restrict_sum_cell(f, c, cz2, rf, bc, X, blockIdx.y, blockIdx.z);
}

// x_f += x_c(parent) on active fine cells.
__device__ __forceinline__ void mg_prolong_cell(const MgDims &f, const MgDims &c, int cz2,
                                                const float *Df,
                                                const float *xc,
                                                float *xf, int x, int y, int z)
{
    const int i = cell(f, x, y, z);
    const float di = Df[i], xi = xf[i], xp = xc[cell(c, x >> 1, y >> 1, cz2 ? (z >> 1) : z)];
    if (di > 0.0f)
        xf[i] = __fadd_rn(xi, xp);
}

__global__ void __launch_bounds__(BX) k_mg_prolong(MgDims f, MgDims c, int cz2,
                                                   const float *__restrict__ Df,
                                                   const float *__restrict__ xc,
                                                   float *__restrict__ xf)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < f.nx)
        mg_prolong_cell(f, c, cz2, Df, xc, xf, x, blockIdx.y, blockIdx.z);
}

// ---------------------------------------------------------------- block-local smoother
//
// The alternative smoother (LBEHD_OPT_MG_SMOOTHER = 1): block-Jacobi between blocks of a level,
// red-black Gauss-Seidel within each block. A level is tiled into blocks of BjShape cells
// (1024: one per thread of a 1024-thread CTA; ragged at the high ends). A block copies x on
// its cells and a one-cell halo (periodic) into shared memory, runs `nu` red-black sweep pairs
// there with the halo held at its value at the start, and writes its own cells to the output
// array. Each block's result depends only on the input arrays, so the blocks may run in any
// order and on any CTA:
//  * on the way down the level starts from x = 0 (nothing is read) and the pairs run
//    (red, black); the output is the level's x;
//  * on the way up every copied cell first takes the coarse correction, x + x_c(parent) on
//    active cells (the arithmetic of mg_prolong_cell), and the pairs run (black, red), the
//    transpose of the way down, so the V-cycle stays symmetric; the output goes to a second
//    array (the level's restriction scratch), since other blocks still read x as their halo.
// A cell's update has the arithmetic of mg_gs_cell, with its neighbours read from the copy.
// With r given (level 0 on the way up), the block also forms its partial of r . z over its
// cells (z = the smoothed x): FP32 within each warp, then FP64 over the warps by a butterfly.
// Against whole-level red-black sweeps, one V-cycle of this smoother costs one grid-wide
// dependency per level and direction instead of one per half sweep.
constexpr int BJ_THREADS = 1024;

template <int D>
struct BjShape;
template <>
struct BjShape<3> {
    static constexpr int X = 16, Y = 8, Z = 8;
};
template <>
struct BjShape<2> {
    static constexpr int X = 32, Y = 32, Z = 1;
};

template <int D>
__host__ __device__ inline int bj_blocks(const MgDims &d)
{
    using S = BjShape<D>;
    return ((d.nx + S::X - 1) / S::X) * ((d.ny + S::Y - 1) / S::Y) * ((d.nz + S::Z - 1) / S::Z);
}

// v in [-1, n + block extent] folded into [0, n) (a level can be smaller than a block).
__device__ __forceinline__ int bj_wrap(int v, int n)
{
    v = v < 0 ? v + n : v;
    return v >= n ? v % n : v;
}

template <int D>
__device__ __forceinline__ void mg_bj_block(const MgDims &d, const float *Dg, const float *kx,
                                            const float *ky, const float *kz, const float *b,
                                            const float *xin, float *xout, int blk, int nu,
                                            bool up, const MgDims &c, int cz2, const float *xc,
                                            const float *r, double *partials)
{
    using S = BjShape<D>;
    constexpr int HX = S::X + 2, HY = S::Y + 2, HZ = D == 3 ? S::Z + 2 : 1;
    constexpr int NH = HX * HY * HZ, SZ = HX * HY;
    static_assert(S::X * S::Y * S::Z == BJ_THREADS, "one cell per thread");
    __shared__ float xs[NH];
    __shared__ double wsm[BJ_THREADS / 32];
    const int nbx = (d.nx + S::X - 1) / S::X, nby = (d.ny + S::Y - 1) / S::Y;
    const int bx = blk % nbx, rest = blk / nbx;
    const int x0 = bx * S::X, y0 = (rest % nby) * S::Y, z0 = (rest / nby) * S::Z;
    const int t = threadIdx.x;
    const int lx = t % S::X, ly = (t / S::X) % S::Y, lz = t / (S::X * S::Y);
    const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
    const bool own = x < d.nx && y < d.ny && z < d.nz;
    const bool zterms = D == 3 && d.nz > 1;
    float di = 0.0f, bi = 0.0f, ri = 0.0f, k[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int i = 0;
    if (own) {
        i = cell(d, x, y, z);
        const Nb6 nb = nb6(d, i, x, y, z);
        di = Dg[i];
        bi = b[i];
        k[0] = kx[i];
        k[1] = kx[nb.n[1]];
        k[2] = ky[i];
        k[3] = ky[nb.n[3]];
        if (zterms) {
            k[4] = kz[i];
            k[5] = kz[nb.n[5]];
        }
        if (r)
            ri = r[i];
    }
    // the copy of x: every load of this thread issued before the first shared store (the
    // parent's value is read whether or not the cell is active, so that the loads are
    // independent)
    constexpr int HIT = (NH + BJ_THREADS - 1) / BJ_THREADS;
    float hxg[HIT], hdg[HIT], hxp[HIT];
#pragma unroll
    for (int k = 0; k < HIT; k++) {
        const int e = t + k * BJ_THREADS;
        hxg[k] = hdg[k] = hxp[k] = 0.0f;
        if (up && e < NH) {
            const int hx = e % HX, hy = (e / HX) % HY, hz = e / SZ;
            const int gx = bj_wrap(x0 - 1 + hx, d.nx), gy = bj_wrap(y0 - 1 + hy, d.ny);
            const int gz = D == 3 ? bj_wrap(z0 - 1 + hz, d.nz) : 0;
            const int g = cell(d, gx, gy, gz);
            hxg[k] = xin[g];
            hdg[k] = Dg[g];
            hxp[k] = xc[cell(c, gx >> 1, gy >> 1, cz2 ? (gz >> 1) : gz)];
        }
    }
#pragma unroll
    for (int k = 0; k < HIT; k++) {
        const int e = t + k * BJ_THREADS;
        if (e < NH)
            xs[e] = up ? (hdg[k] > 0.0f ? __fadd_rn(hxg[k], hxp[k]) : hxg[k]) : 0.0f;
    }
    __syncthreads();
    const int h = (lx + 1) + HX * (ly + 1) + (D == 3 ? SZ * (lz + 1) : 0);
    const int col = (x + y + z) & 1;
    const bool act = own && di > 0.0f;
    for (int s = 0; s < nu; s++) {
        for (int half = 0; half < 2; half++) {
            if (act && col == (up ? 1 - half : half)) {
                float sum = __fmul_rn(k[0], xs[h + 1]);
                sum = __fmaf_rn(k[1], xs[h - 1], sum);
                sum = __fmaf_rn(k[2], xs[h + HX], sum);
                sum = __fmaf_rn(k[3], xs[h - HX], sum);
                if (zterms) {
                    sum = __fmaf_rn(k[4], xs[h + SZ], sum);
                    sum = __fmaf_rn(k[5], xs[h - SZ], sum);
                }
                xs[h] = __fdiv_rn(__fadd_rn(bi, sum), di);
            }
            __syncthreads();
        }
    }
    if (own)
        xout[i] = xs[h];
    if (r) {
        const float v = warp_sum(own ? __fmaf_rn(ri, xs[h], 0.0f) : 0.0f);
        if ((t & 31) == 0)
            wsm[t >> 5] = (double)v;
        __syncthreads();
        if (t < 32) {   // FP64 over the 32 warp sums by a butterfly (FP64 adds are slow here)
            double acc = wsm[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (t == 0)
                partials[blk] = acc;
        }
    }
    __syncthreads();   // the shared copies are rewritten by this CTA's next block
}

// One block-local smoothing pass of a level, one CTA per block.
template <int D>
__global__ void __launch_bounds__(BJ_THREADS, 1) k_mg_bj(MgDims d, const float *Dg,
                                                         const float *kx, const float *ky,
                                                         const float *kz, const float *b,
                                                         const float *xin, float *xout, int nu,
                                                         int up, MgDims c, int cz2,
                                                         const float *xc, const float *r,
                                                         double *partials)
{
    mg_bj_block<D>(d, Dg, kx, ky, kz, b, xin, xout, (int)blockIdx.x, nu, up != 0, c, cz2, xc, r,
                   partials);
}

// ---------------------------------------------------------------- small-level tail

constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_MAX_TOTAL = 8192;   // cells of all tail levels (6 floats each: 192 KB)
constexpr int TAIL_THREADS = 1024;
constexpr size_t TAIL_SMEM_MAX = 6 * sizeof(float) * TAIL_MAX_TOTAL;   // dynamic shared memory

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

// The V-cycle on every level from the tail's finest down, in shared memory, one CTA; the
// threads stride over the cells of each level. Same arithmetic, cell by cell, as the
// multi-launch levels above it (and the same for any assignment of cells to threads: a
// red-black half sweep reads only cells of the other colour).
// ops_loaded: the levels' operators (D, kx, ky, kz) are already in `sm` from an earlier call
// of the same CTA (a persistent solve keeps them across its V-cycles).
__device__ __forceinline__ void mg_tail_block(const TailLevels &T, float *sm, bool ops_loaded = false)
{
    const int tot = T.total, t = threadIdx.x;
    float *sD = sm, *skx = sm + tot, *sky = sm + 2 * tot, *skz = sm + 3 * tot, *sx = sm + 4 * tot,
          *sb = sm + 5 * tot;
    auto ncell = [&](int l) { return T.d[l].nx * T.d[l].ny * T.d[l].nz; };
#pragma unroll 1
    for (int l = 0; l < T.nl; l++) {
        const int n = ncell(l), o = T.off[l];
        for (int c = t; c < n; c += TAIL_THREADS) {
            if (!ops_loaded) {
                sD[o + c] = T.D[l][c];
                skx[o + c] = T.kx[l][c];
                sky[o + c] = T.ky[l][c];
                skz[o + c] = T.kz[l][c];
            }
            sx[o + c] = 0.0f;
            if (l == 0)
                sb[c] = T.b0[c];
        }
    }
    __syncthreads();
    auto gs = [&](int l, int color) {
        const MgDims d = T.d[l];
        const int n = ncell(l), o = T.off[l];
        for (int c = t; c < n; c += TAIL_THREADS) {
            int x, y, z;
            cell_xyz(d, c, x, y, z);
            if (((x + y + z) & 1) != color)
                continue;
            const float di = sD[o + c];
            if (di > 0.0f)
                sx[o + c] = __fdiv_rn(__fadd_rn(sb[o + c], offdiag_sum(d, c, x, y, z, skx + o,
                                                                       sky + o, skz + o, sx + o)),
                                      di);
        }
        __syncthreads();
    };
    // nsw red-black half sweeps of level l (colour color_of(k) for sweep k) when the level has
    // at most TAIL_THREADS cells: thread t owns cell t, whose coordinates, neighbours,
    // coefficients and right-hand side stay in registers across the sweeps (b is fixed while
    // a level is smoothed). Same arithmetic as gs, in offdiag_sum's order.
    // A level of at most 32 cells is swept by warp 0 alone, with warp barriers.
    auto owned = [&](int l, int nsw, auto color_of) {
        const MgDims d = T.d[l];
        const int n = ncell(l), o = T.off[l];
        const bool warp_only = n <= 32;
        if (warp_only && t >= 32) {
            __syncthreads();
            return;
        }
        const bool own = t < n;
        int col = -1, n0 = 0, n1 = 0, n2 = 0, n3 = 0, n4 = 0, n5 = 0;
        float di = 0.f, bi = 0.f, kxi = 0.f, kxm = 0.f, kyi = 0.f, kym = 0.f, kzi = 0.f, kzm = 0.f;
        if (own) {
            int x, y, z;
            cell_xyz(d, t, x, y, z);
            const Nb6 nb = nb6(d, t, x, y, z);
            n0 = nb.n[0];
            n1 = nb.n[1];
            n2 = nb.n[2];
            n3 = nb.n[3];
            n4 = nb.n[4];
            n5 = nb.n[5];
            di = sD[o + t];
            bi = sb[o + t];
            kxi = skx[o + t];
            kxm = skx[o + n1];
            kyi = sky[o + t];
            kym = sky[o + n3];
            kzi = skz[o + t];
            kzm = skz[o + n5];
            col = di > 0.0f ? ((x + y + z) & 1) : -1;
        }
        const float *v = sx + o;
#pragma unroll 1
        for (int k = 0; k < nsw; k++) {
            if (col == color_of(k)) {
                float s = __fmul_rn(kxi, v[n0]);
                s = __fmaf_rn(kxm, v[n1], s);
                s = __fmaf_rn(kyi, v[n2], s);
                s = __fmaf_rn(kym, v[n3], s);
                if (d.nz > 1) {
                    s = __fmaf_rn(kzi, v[n4], s);
                    s = __fmaf_rn(kzm, v[n5], s);
                }
                sx[o + t] = __fdiv_rn(__fadd_rn(bi, s), di);
            }
            if (warp_only)
                __syncwarp();
            else
                __syncthreads();
        }
        if (warp_only)
            __syncthreads();
    };
    // down: smooth, restrict
#pragma unroll 1
    for (int l = 0; l + 1 < T.nl; l++) {
        if (ncell(l) <= TAIL_THREADS) {
            owned(l, 2 * T.nu, [](int k) { return k & 1; });
        } else {
            for (int s = 0; s < T.nu; s++) {
                gs(l, 0);
                gs(l, 1);
            }
        }
        const MgDims f = T.d[l], cd = T.d[l + 1];
        const int fo = T.off[l], co = T.off[l + 1], nzc = T.cz2[l] ? 2 : 1, nc = ncell(l + 1);
        for (int C = t; C < nc; C += TAIL_THREADS) {
            int X, Y, Z;
            cell_xyz(cd, C, X, Y, Z);
            float acc = 0.0f;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++)
                    for (int g = 0; g < nzc; g++) {
                        const int x = 2 * X + a, y = 2 * Y + b, z = nzc * Z + g;
                        if (x >= f.nx || y >= f.ny || z >= f.nz)
                            continue;
                        const int i = (int)cell(f, x, y, z);
                        const float di = sD[fo + i];
                        if (di <= 0.0f)
                            continue;
                        const float Ax = __fmaf_rn(di, sx[fo + i],
                                                   -offdiag_sum(f, i, x, y, z, skx + fo, sky + fo,
                                                                skz + fo, sx + fo));
                        acc = __fadd_rn(acc, __fsub_rn(sb[fo + i], Ax));
                    }
            sb[co + C] = acc;
        }
        __syncthreads();
    }
    // coarsest: symmetric sweeps
    const int lc = T.nl - 1;
    if (ncell(lc) <= TAIL_THREADS) {
        owned(lc, 4 * T.coarse, [](int k) { return ((k & 3) == 1 || (k & 3) == 2) ? 1 : 0; });
    } else {
#pragma unroll 1
        for (int s = 0; s < T.coarse; s++) {
            gs(lc, 0);
            gs(lc, 1);
            gs(lc, 1);
            gs(lc, 0);
        }
    }
    // up: prolong, smooth
#pragma unroll 1
    for (int l = T.nl - 2; l >= 0; l--) {
        const MgDims f = T.d[l], cd = T.d[l + 1];
        const int fo = T.off[l], co = T.off[l + 1], n = ncell(l);
        for (int c = t; c < n; c += TAIL_THREADS) {
            if (sD[fo + c] <= 0.0f)
                continue;
            int x, y, z;
            cell_xyz(f, c, x, y, z);
            sx[fo + c] = __fadd_rn(sx[fo + c],
                                   sx[co + (int)cell(cd, x >> 1, y >> 1, T.cz2[l] ? (z >> 1) : z)]);
        }
        __syncthreads();
        if (n <= TAIL_THREADS) {
            owned(l, 2 * T.nu, [](int k) { return (k & 1) ? 0 : 1; });
        } else {
            for (int s = 0; s < T.nu; s++) {
                gs(l, 1);
                gs(l, 0);
            }
        }
    }
    const int n0 = ncell(0);
    for (int c = t; c < n0; c += TAIL_THREADS)
        T.x0[c] = sx[c];
}

__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail(TailLevels T)
{
    extern __shared__ float sm[];
    mg_tail_block(T, sm);
}

// ---------------------------------------------------------------- CG on level 0

// r = b - A (phi + delta) from the compensated potential; partials of ||r||^2 and ||b||^2.
// Only differences of the potential enter: r_i = rho_i + sum_faces k_f (phi_j - phi_i), with
// phi_j - phi_i = (hi_j - hi_i) + (lo_j - lo_i) + (delta_j - delta_i). Neighbouring hi parts
// are close, so their difference is exact in FP32, and r keeps the accuracy an FP64
// evaluation of b - A phi would have, in FP32 arithmetic.
// pcg_init_value returns r_i without storing it (so that several sites' loads can be in
// flight together); pcg_init_site stores it. zero_delta: delta is all zeros (read as such
// without loading it; same arithmetic).
template <int D>
__device__ __forceinline__ float pcg_init_value(const MgDims &d, const float *pot,
                                                const float *pot_lo, const float *delta,
                                                const float *eps, const float *rho,
                                                const uint8_t *info, const float *Dg, int x,
                                                int y, int z, float (&v)[2],
                                                bool zero_delta = false)
{
    {
        const int i = cell(d, x, y, z);
        const Nb6 nb = nb6(d, i, x, y, z);
        const float Di = Dg[i], ei = eps[i], hi = pot[i], lo = pot_lo[i];
        const float di = zero_delta ? 0.0f : delta[i];
        const float rh = rho[i];
        int pt[2 * D];
        float ph[2 * D], pl[2 * D], dl[2 * D], ej[2 * D];
#pragma unroll
        for (int f = 0; f < 2 * D; f++) {
            const int j = nb.n[f];
            pt[f] = info[j] & 3;
            ph[f] = pot[j];
            pl[f] = pot_lo[j];
            dl[f] = zero_delta ? 0.0f : delta[j];
            ej[f] = eps[j];
        }
        float ri = 0.0f;
        if (Di > 0.0f) {
            float b = rh;
            ri = b;
#pragma unroll
            for (int f = 0; f < 2 * D; f++) {
                if (pt[f] == PT_FLUID) {
                    const float dphi = __fadd_rn(__fadd_rn(__fsub_rn(ph[f], hi), __fsub_rn(pl[f], lo)),
                                                 __fsub_rn(dl[f], di));
                    ri = __fmaf_rn(__fmul_rn(0.5f, __fadd_rn(ei, ej[f])), dphi, ri);
                } else if (pt[f] == PT_DIRICHLET) {
                    const float dphi =
                        __fsub_rn(__fadd_rn(__fsub_rn(ph[f], hi), __fsub_rn(pl[f], lo)), di);
                    ri = __fmaf_rn(ei, dphi, ri);
                    b = __fmaf_rn(ei, __fadd_rn(ph[f], pl[f]), b);
                }
            }
            v[0] = __fmul_rn(ri, ri);
            v[1] = __fmul_rn(b, b);
        }
        return ri;
    }
}

template <int D>
__device__ __forceinline__ void pcg_init_site(const MgDims &d, const float *pot,
                                              const float *pot_lo,
                                              const float *delta,
                                              const float *eps,
                                              const float *rho,
                                              const uint8_t *info,
                                              const float *Dg, float *r,
                                              int x, int y, int z, float (&v)[2])
{
    r[cell(d, x, y, z)] = pcg_init_value<D>(d, pot, pot_lo, delta, eps, rho, info, Dg, x, y, z, v);
}

template <int D>
__global__ void __launch_bounds__(BX) k_pcg_init(MgDims d, const float *__restrict__ pot,
                                                 const float *__restrict__ pot_lo,
                                                 const float *__restrict__ delta,
                                                 const float *__restrict__ eps,
                                                 const float *__restrict__ rho,
                                                 const uint8_t *__restrict__ info,
                                                 const float *__restrict__ Dg,
                                                 float *__restrict__ r, double *__restrict__ partials,
                                                 unsigned *zero = nullptr)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    if (zero && i == 0)   // the grid-barrier counter of the persistent solve that follows
        *zero = 0u;
    float v[2] = {0.f, 0.f};
    if (i < d.nx * d.ny * d.nz) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        pcg_init_site<D>(d, pot, pot_lo, delta, eps, rho, info, Dg, r, x, y, z, v);
    }
    block_partials<2>(v, partials);
}

// p = z + beta p (beta = 0 on the first iteration).
// The 1D CG kernels walk the sites with a grid stride: block b of nb covers sites
// b BX + t, (b + nb) BX + t, ... (the partition fixes each partial sum). The _t forms take
// the thread's index t within its BX-thread block explicitly.
__device__ __forceinline__ float pcg_beta(const CgScalars *s)
{
    return s->iters == 0 ? 0.0f : (float)s->beta;
}

__device__ __forceinline__ void pcg_p_site(int i, float beta, const float *zv, float *p)
{
    p[i] = beta != 0.0f ? __fmaf_rn(beta, p[i], zv[i]) : zv[i];
}

__device__ __forceinline__ void pcg_p_range(int n, const float *zv,
                                            float *p, const CgScalars *s,
                                            int b, int nb)
{
    const float beta = pcg_beta(s);
    for (int i = b * BX + threadIdx.x; i < n; i += nb * BX)
        pcg_p_site(i, beta, zv, p);
}

__global__ void __launch_bounds__(BX) k_pcg_p(size_t n, const float *__restrict__ zv,
                                              float *__restrict__ p, const CgScalars *__restrict__ s)
{
    pcg_p_range((int)n, zv, p, s, (int)blockIdx.x, (int)gridDim.x);
}

// q = A p with the operator of this step (from eps and the node classes; the multigrid
// hierarchy may be a few steps old, which only changes the preconditioner) and partials of
// p . q. Dirichlet neighbours hold no correction (p = 0 there).
template <int D>
__device__ __forceinline__ float pcg_Ap_value(const MgDims &d, const float *eps,
                                              const uint8_t *info, const float *Dg,
                                              const float *p, int x, int y, int z,
                                              float (&v)[1])
{
    {
        const int i = cell(d, x, y, z);
        const Nb6 nb = nb6(d, i, x, y, z);
        const float Di = Dg[i], ei = eps[i], pi = p[i];
        int pt[2 * D];
        float ej[2 * D], pj[2 * D];
#pragma unroll
        for (int f = 0; f < 2 * D; f++) {
            const int j = nb.n[f];
            pt[f] = info[j] & 3;
            ej[f] = eps[j];
            pj[f] = p[j];
        }
        float qi = 0.0f;
        if (Di > 0.0f) {
#pragma unroll
            for (int f = 0; f < 2 * D; f++) {
                if (pt[f] == PT_FLUID)
                    qi = __fmaf_rn(__fmul_rn(0.5f, __fadd_rn(ei, ej[f])), __fsub_rn(pi, pj[f]), qi);
                else if (pt[f] == PT_DIRICHLET)
                    qi = __fmaf_rn(ei, pi, qi);
            }
            v[0] = __fmul_rn(pi, qi);
        }
        return qi;
    }
}

template <int D>
__device__ __forceinline__ void pcg_Ap_site(const MgDims &d, const float *eps,
                                            const uint8_t *info,
                                            const float *Dg,
                                            const float *p, float *q,
                                            int x, int y, int z, float (&v)[1])
{
    q[cell(d, x, y, z)] = pcg_Ap_value<D>(d, eps, info, Dg, p, x, y, z, v);
}

template <int D>
__global__ void __launch_bounds__(BX) k_pcg_Ap(MgDims d, const float *__restrict__ eps,
                                               const uint8_t *__restrict__ info,
                                               const float *__restrict__ Dg,
                                               const float *__restrict__ p, float *__restrict__ q,
                                               double *__restrict__ partials)
{
    const int i = blockIdx.x * BX + threadIdx.x;
    float v[1] = {0.f};
    if (i < d.nx * d.ny * d.nz) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        pcg_Ap_site<D>(d, eps, info, Dg, p, q, x, y, z, v);
    }
    block_partials<1>(v, partials);
}

// ---------------------------------------------------------------- minimal-residual start
//
// The forward solve may start from x0 = a1 d1 + a2 d2, the increments of the last two steps
// (d1 the last one's, d2 the one before), with (a1, a2) minimising ||b - A (phi + x0)||_2 over
// their span. With r0 = b - A phi and q_k = A d_k (Dirichlet values held, so A acts on the
// increments alone) that is the 2 x 2 normal system G a = c, G_kl = q_k . q_l, c_k = q_k . r0,
// and the least residual is ||r0||^2 - a . c. The sums only choose the start and estimate its
// residual for the convergence test; they are FP32 block sums (the FP64 pipe of this part is
// narrow), summed in a fixed order by one 1024-thread block. ||r0||^2 and ||b||^2 are the FP64
// partials of every other residual. A step whose start meets the tolerance applies x0 and
// stops; one that does not forms x0 and r = r0 - a1 q1 - a2 q2 site by site and iterates.
// A singular or nearly singular system (the first solve: d1 = d2 = 0) falls back to one
// increment or to none.
constexpr int MR_NV = 5;   // q1.r0, q2.r0, q1.q1, q1.q2, q2.q2

// Threads of the one-block scalar reductions (the CG scalars, the start's coefficients).
constexpr int SCALAR_THREADS = 1024;

// out = (a1, a2, a . c) from the totals (c1, c2, G11, G12, G22). Written with the rounding
// intrinsics, so that every kernel that inlines it (the persistent solve, k_mr_alpha,
// k_mr_alpha_batch) gets the same bits.
__device__ __forceinline__ void mr_solve(const float (&m)[MR_NV], double *out)
{
    const double c1 = m[0], c2 = m[1], g11 = m[2], g12 = m[3], g22 = m[4];
    const double gg = __dmul_rn(g11, g22);
    const double det = __dsub_rn(gg, __dmul_rn(g12, g12));
    double a1 = 0.0, a2 = 0.0;
    if (g11 > 0.0 && g22 > 0.0 && det > __dmul_rn(1e-6, gg)) {
        a1 = __ddiv_rn(__dsub_rn(__dmul_rn(c1, g22), __dmul_rn(c2, g12)), det);
        a2 = __ddiv_rn(__dsub_rn(__dmul_rn(c2, g11), __dmul_rn(c1, g12)), det);
    } else if (g22 > 0.0) {
        a2 = __ddiv_rn(c2, g22);
    } else if (g11 > 0.0) {
        a1 = __ddiv_rn(c1, g11);
    }
    out[0] = a1;
    out[1] = a2;
    out[2] = __dadd_rn(__dmul_rn(a1, c1), __dmul_rn(a2, c2));
}

// The coefficients from the first pass's block sums mr_part[k * nblk + b], by one block of
// SCALAR_THREADS threads in a fixed order: thread t adds blocks t, t + SCALAR_THREADS, ... in
// order (the MR_NV loads of a block issued together), then the warps' butterflies and the
// warps in order. Every thread of the block gets out (shared or global memory, written by
// thread 0, visible after the block barrier this ends with).
__device__ __forceinline__ void mr_alpha_block(const float *part, int nblk, double *out)
{
    constexpr int NW = SCALAR_THREADS / 32;
    __shared__ float sm[MR_NV][NW];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float acc[MR_NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = threadIdx.x; j < nblk; j += SCALAR_THREADS) {
        float v[MR_NV];
#pragma unroll
        for (int k = 0; k < MR_NV; k++)
            v[k] = __ldcg(part + (size_t)k * nblk + j);
#pragma unroll
        for (int k = 0; k < MR_NV; k++)
            acc[k] = __fadd_rn(acc[k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < MR_NV; k++) {
        const float sv = warp_sum(acc[k]);
        if (lane == 0)
            sm[k][wid] = sv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot[MR_NV];
#pragma unroll
        for (int k = 0; k < MR_NV; k++) {
            tot[k] = 0.0f;
            for (int w = 0; w < NW; w++)
                tot[k] = __fadd_rn(tot[k], sm[k][w]);
        }
        mr_solve(tot, out);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(SCALAR_THREADS) k_mr_alpha(const float *__restrict__ part,
                                                             int nblk, double *__restrict__ out)
{
    mr_alpha_block(part, nblk, out);
}

// First pass, one block `blk` of nblk BX-site blocks: r0 = b - A phi (k_pcg_init's start
// residual with a zero increment, and its FP64 block partials of ||r0||^2 and ||b||^2) into r,
// q1 = A d1 and q2 = A d2, and FP32 block sums of the five products into
// mr_part[k * nblk + blk]. The shared scratch is free again on return.
template <int D>
__device__ __forceinline__ void mr_init_block(const MgDims &d, const float *pot,
                                              const float *pot_lo, const float *d1,
                                              const float *d2, const float *eps,
                                              const float *rho, const uint8_t *info,
                                              const float *Dg, float *r, float *q1, float *q2,
                                              double *partials, float *mr_part, int blk, int nblk)
{
    const int i = blk * BX + threadIdx.x;
    float v[2] = {0.f, 0.f}, m[MR_NV] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < d.nx * d.ny * d.nz) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        const float r0 = pcg_init_value<D>(d, pot, pot_lo, nullptr, eps, rho, info, Dg, x, y, z,
                                           v, true);
        float w[1] = {0.f};
        const float a = pcg_Ap_value<D>(d, eps, info, Dg, d1, x, y, z, w);
        const float b = pcg_Ap_value<D>(d, eps, info, Dg, d2, x, y, z, w);
        r[i] = r0;
        q1[i] = a;
        q2[i] = b;
        m[0] = __fmul_rn(a, r0);
        m[1] = __fmul_rn(b, r0);
        m[2] = __fmul_rn(a, a);
        m[3] = __fmul_rn(a, b);
        m[4] = __fmul_rn(b, b);
    }
    block_partials<2>(v, partials, (size_t)blk, (size_t)nblk);
    __shared__ float sm[MR_NV][BX / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MR_NV; k++) {
        const float s = warp_sum(m[k]);
        if (lane == 0)
            sm[k][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < MR_NV) {
        float acc = 0.0f;
#pragma unroll
        for (int w = 0; w < BX / 32; w++)
            acc = __fadd_rn(acc, sm[threadIdx.x][w]);
        mr_part[threadIdx.x * nblk + blk] = acc;
    }
    __syncthreads();
}

template <int D>
__global__ void __launch_bounds__(BX) k_pcg_init_mr(MgDims d, const float *__restrict__ pot,
                                                    const float *__restrict__ pot_lo,
                                                    const float *__restrict__ d1,
                                                    const float *__restrict__ d2,
                                                    const float *__restrict__ eps,
                                                    const float *__restrict__ rho,
                                                    const uint8_t *__restrict__ info,
                                                    const float *__restrict__ Dg,
                                                    float *__restrict__ r, float *__restrict__ q1,
                                                    float *__restrict__ q2,
                                                    double *__restrict__ partials,
                                                    float *__restrict__ mr_part,
                                                    unsigned *zero = nullptr)
{
    if (zero && blockIdx.x == 0 && threadIdx.x == 0)   // the persistent solve's barrier counter
        *zero = 0u;
    mr_init_block<D>(d, pot, pot_lo, d1, d2, eps, rho, info, Dg, r, q1, q2, partials, mr_part,
                     (int)blockIdx.x, (int)gridDim.x);
}

// At one site: x0 = a1 d1 + a2 d2 written over d2 (x holds d2 on entry); returns x0.
__device__ __forceinline__ float mr_x0_site(int i, float a1, float a2, const float *d1,
                                            float *x)
{
    const float x0 = __fmaf_rn(a2, x[i], __fmul_rn(a1, d1[i]));
    x[i] = x0;
    return x0;
}

// At one site: x0 as mr_x0_site and r = r0 - a1 q1 - a2 q2 over r0.
__device__ __forceinline__ void mr_start_site(int i, float a1, float a2, const float *d1,
                                              float *x, float *r, const float *q1,
                                              const float *q2)
{
    mr_x0_site(i, a1, a2, d1, x);
    r[i] = __fmaf_rn(-a2, q2[i], __fmaf_rn(-a1, q1[i], r[i]));
}

// x0 and r for every site (grid-stride).
__global__ void __launch_bounds__(BX) k_pcg_start_mr(int n, const double *__restrict__ alpha,
                                                     const float *__restrict__ d1,
                                                     float *__restrict__ x, float *__restrict__ r,
                                                     const float *__restrict__ q1,
                                                     const float *__restrict__ q2)
{
    const float a1 = (float)alpha[0], a2 = (float)alpha[1];
    for (int i = blockIdx.x * BX + threadIdx.x; i < n; i += gridDim.x * BX)
        mr_start_site(i, a1, a2, d1, x, r, q1, q2);
}

// delta += alpha p, r -= alpha q, partials of ||r||^2.
__device__ __forceinline__ void pcg_update_range_t(int n, const float *p,
                                                   const float *q,
                                                   float *delta, float *r,
                                                   const CgScalars *s, int b, int nb, int t,
                                                   float (&v)[1])
{
    const float a = (float)s->alpha;
    for (int i = b * BX + t; i < n; i += nb * BX) {
        delta[i] = __fmaf_rn(a, p[i], delta[i]);
        const float ri = __fmaf_rn(-a, q[i], r[i]);
        r[i] = ri;
        v[0] = __fmaf_rn(ri, ri, v[0]);
    }
}

__device__ __forceinline__ void pcg_update_range(int n, const float *p,
                                                 const float *q,
                                                 float *delta, float *r,
                                                 const CgScalars *s, int b, int nb,
                                                 float (&v)[1])
{
    pcg_update_range_t(n, p, q, delta, r, s, b, nb, (int)threadIdx.x, v);
}

__global__ void __launch_bounds__(BX) k_pcg_update(size_t n, const float *__restrict__ p,
                                                   const float *__restrict__ q,
                                                   float *__restrict__ delta, float *__restrict__ r,
                                                   const CgScalars *__restrict__ s,
                                                   double *__restrict__ partials)
{
    float v[1] = {0.f};
    pcg_update_range((int)n, p, q, delta, r, s, (int)blockIdx.x, (int)gridDim.x, v);
    block_partials<1>(v, partials);
}

// partials of r . z
__device__ __forceinline__ void pcg_dot_range_t(int n, const float *a,
                                                const float *b, int blk, int nb, int t,
                                                float (&v)[1])
{
    for (int i = blk * BX + t; i < n; i += nb * BX)
        v[0] = __fmaf_rn(a[i], b[i], v[0]);
}

__device__ __forceinline__ void pcg_dot_range(int n, const float *a,
                                              const float *b, int blk, int nb,
                                              float (&v)[1])
{
    pcg_dot_range_t(n, a, b, blk, nb, (int)threadIdx.x, v);
}

__global__ void __launch_bounds__(BX) k_pcg_dot(size_t n, const float *__restrict__ a,
                                                const float *__restrict__ b,
                                                double *__restrict__ partials)
{
    float v[1] = {0.0f};
    pcg_dot_range((int)n, a, b, (int)blockIdx.x, (int)gridDim.x, v);
    block_partials<1>(v, partials);
}

// Fixed-order FP64 sum of nv partial arrays and the CG scalar update that follows.
//   op 0: start     rr, bb            -> done if rr <= tol2 bb (resets the step counter)
//   op 4: restart   as op 0 for a refinement pass (keeps the step counter)
//   op 1: r.z       rz                -> beta = rz / rz_old, rz_old = rz
//   op 2: p.Ap      pq                -> alpha = rz / pq
//   op 3: ||r||^2   rr                -> iters++, done / converged, refine = 1 from the
//                                        second iteration on
//   op 5: ||r||^2   as op 3, for a refinement pass (leaves refine alone)
// (op 0 clears refine.) pcg_scalar_block returns true in thread 0 after updating *s.
// k_pcg_scalar: with use_cond, ops 0, 4, 3 and 5 also set the graph's while-loop condition
// to !done; with use_ref, op 0 clears and op 3 sets the condition of the refinement block.

// The fixed summation order, in two pieces that may run on different SMs: the sum of
// virtual warp w (lanes = threads 32 w .. 32 w + 31 of the 1024-thread order: each lane's
// strided pair of accumulators, then a butterfly), and the butterfly over the 32 warp sums.
__device__ __forceinline__ double pcg_vwarp_sum(const double *p, long long nblocks, int vt)
{
    double a0 = 0.0, a1 = 0.0;
    long long b = vt;
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
    return a;
}

// CG scalar update (thread 0) from the totals of the op's partial arrays.
// rr_sub (op 0 only): subtracted from the reduced ||r||^2 (the minimal-residual start's a . c,
// so that rr is its least residual's norm).
__device__ __forceinline__ void pcg_scalar_update(const double (&tot)[2], int op, CgScalars *s,
                                                  double rr_sub = 0.0)
{
    if (op == 0 || op == 4) {
        s->rr = op == 0 && rr_sub != 0.0 ? fmax(tot[0] - rr_sub, 0.0) : tot[0];
        s->bb = tot[1];
        s->iters = 0;
        if (op == 0) {
            s->step_iters = 0;
            s->refine = 0;
        }
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
        // A refinement pass re-forms the true residual and corrects the drift of the CG's
        // recursive one. One iteration from the warm start leaves r0 within a few times the
        // tolerance, and the FP32 rounding of that single update is ~1e-7 of r0, far below the
        // tolerance: only a pass of two or more iterations (large increments, the first
        // solve, an electrode switch) needs the check.
        if (op == 3 && s->iters >= 2)
            s->refine = 1;
        s->converged = s->rr <= s->tol2 * s->bb || s->rr < 1e-60;
        s->done = s->converged || s->iters >= s->max_iter;
        if (s->done && !s->converged)
            s->nonconv = 1;
    }
}

__device__ __forceinline__ bool pcg_scalar_block(const double *partials,
                                                 long long nblocks, int nv, int op,
                                                 CgScalars *s, double rr_sub = 0.0)
{
    __shared__ double sm[2][SCALAR_THREADS / 32];
    double tot[2] = {0.0, 0.0};
    for (int k = 0; k < nv; k++) {
        const double a = pcg_vwarp_sum(partials + k * nblocks, nblocks, (int)threadIdx.x);
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
        return false;
    pcg_scalar_update(tot, op, s, rr_sub);
    return true;
}

__global__ void __launch_bounds__(SCALAR_THREADS) k_pcg_scalar(const double *__restrict__ partials,
                                                               long long nblocks, int nv, int op,
                                                               CgScalars *__restrict__ s,
                                                               cudaGraphConditionalHandle cond,
                                                               int use_cond,
                                                               cudaGraphConditionalHandle cond_ref,
                                                               int use_ref,
                                                               const double *__restrict__ mr = nullptr)
{
    // mr: the minimal-residual start's (a1, a2, a . c); op 0 then tests its least residual
    if (!pcg_scalar_block(partials, nblocks, nv, op, s, mr ? mr[2] : 0.0))
        return;
    if (use_cond && op != 1 && op != 2)
        cudaGraphSetConditional(cond, s->done ? 0u : 1u);
    // refinement check runs only when the main pass took two or more iterations
    if (use_ref && op == 0)
        cudaGraphSetConditional(cond_ref, 0u);
    if (use_ref && op == 3)
        cudaGraphSetConditional(cond_ref, s->refine ? 1u : 0u);
}

// phi += delta on active cells, phi kept as the compensated pair hi + lo (two-sum in FP32:
// the rounding error of hi + delta is carried into lo); acc += delta when acc is given
// (accumulates a refinement correction into the step's increment).
// (hi, lo) + d as a renormalised pair (two-sum of hi + d, error carried into lo).
__device__ __forceinline__ void pcg_apply_pair(float hi, float lo0, float d, float &hi_out,
                                               float &lo_out)
{
    const float t = __fadd_rn(hi, d);             // two-sum: t + err = hi + d exactly
    const float bv = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(d, bv));
    const float lo = __fadd_rn(lo0, err);
    const float s = __fadd_rn(t, lo);             // renormalise the pair
    hi_out = s;
    lo_out = __fsub_rn(lo, __fsub_rn(s, t));
}

__device__ __forceinline__ void pcg_apply_site(int i, const float *Dg, const float *delta,
                                               float *acc, float *pot, float *pot_lo)
{
    if (Dg[i] <= 0.0f)
        return;
    const float d = delta[i];
    if (acc)
        acc[i] = __fadd_rn(acc[i], d);
    pcg_apply_pair(pot[i], pot_lo[i], d, pot[i], pot_lo[i]);
}

__device__ __forceinline__ void pcg_apply_range(int n, const float *Dg,
                                                const float *delta,
                                                float *acc, float *pot,
                                                float *pot_lo, int b, int nb)
{
    for (int i = b * BX + threadIdx.x; i < n; i += nb * BX)
        pcg_apply_site(i, Dg, delta, acc, pot, pot_lo);
}

__global__ void __launch_bounds__(BX) k_pcg_apply(size_t n, const float *__restrict__ Dg,
                                                  const float *__restrict__ delta,
                                                  float *__restrict__ acc,
                                                  float *__restrict__ pot,
                                                  float *__restrict__ pot_lo)
{
    pcg_apply_range((int)n, Dg, delta, acc, pot, pot_lo, (int)blockIdx.x, (int)gridDim.x);
}

}  // namespace lbehd

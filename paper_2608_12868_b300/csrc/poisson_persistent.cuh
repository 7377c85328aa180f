// poisson_persistent.cuh -- the Gauss-law solve of one step (Eq. 13) as one persistent
// kernel after the launch that forms the start residual: the start's reduction, every
// preconditioned-CG iteration (the V-cycle included), the update of the potential and the
// refinement pass, with grid-wide barriers in place of kernel boundaries.
//
// One CTA of PS_THREADS = 1024 threads per SM, launched cooperatively (all CTAs resident).
// The CG loop of the multi-launch form is latency-bound: a V-cycle of ~36 small dependent
// launches plus 7 CG launches per iteration. Here each of those becomes a phase of this
// kernel ended by a barrier instead of a launch.
//
// Same bits as the multi-launch form, by construction:
//  * each phase calls the same per-cell bodies (poisson.cuh), which are written with explicit
//    rounding intrinsics; smoothing, restriction and prolongation results do not depend on
//    which thread handles which cell (a red-black half sweep reads only the other colour);
//  * dot products keep their partition into BX-site virtual blocks: the 128-thread group g of
//    a CTA plays virtual block blockIdx.x * PS_GROUPS + g, ... and reduces like
//    block_partials (warp sums in FP32, then FP64 over the four warps in order);
//  * the partial arrays are summed in the fixed order of k_pcg_scalar (1024 threads: per
//    thread two strided accumulators, butterflies within and across warps); every CTA keeps
//    an identical copy of the CG scalars, so all CTAs take the same branches. Small sums are
//    done by every CTA; large ones are split: 32 CTAs (per array) each form one warp's sum,
//    then, after a barrier, every CTA finishes the butterfly (FP64 adds are slow on this
//    part, and the split spreads them over SMs);
//  * the shared-memory tail runs in CTA 0 with the 1024-thread k_mg_tail body;
//  * fused phases reproduce a sequence of launches exactly: "zero, then the first red half
//    sweep" (every neighbour is 0, so x = (b + 0) / D on red cells and 0 elsewhere),
//    "residual, then the sum over each coarse cell's children, then the coarse level's zero
//    start and first red half sweep" (each child's residual on its own lane, summed in the
//    restriction's order; the red update needs only the cell's own new b), and
//    "prolongation, then the first black half sweep" (neighbours read as prolongation
//    leaves them).
//
// Barrier: a monotonic arrival counter (zeroed by the start launch before each solve) that
// barrier k waits to reach k * gridDim.x; thread 0 of each CTA spins with a backoff and an
// iteration limit. On time-out it raises the error word, and every CTA leaves at its next
// barrier; the host reads the word and reports the step as failed.
#pragma once

#include "poisson.cuh"

namespace lbehd {

constexpr int PS_THREADS = 1024;
constexpr int PS_GROUPS = PS_THREADS / BX;        // virtual blocks per CTA
constexpr int PS_MAX_LEVELS = 12;
constexpr unsigned PS_SPIN_LIMIT = 1u << 24;      // x >= 32 ns backoff: ~0.5 s at least

static_assert(PS_THREADS == SCALAR_THREADS && PS_THREADS == TAIL_THREADS,
              "the persistent solve runs the 1024-thread scalar and tail bodies as they are");

struct PsBarrier {
    unsigned int count;    // arrivals (zeroed before each launch)
    unsigned int error;    // sticky: a barrier timed out
    unsigned int where;    // barrier index of the first time-out
    unsigned int pad;
};

struct PsLevel {
    MgDims d;
    int cz2, n;
    const float *D, *kx, *ky, *kz;
    float *b, *x;
    int nbj;       // blocks of the block-local smoother
    float *xo;     // its output on the way up (the level's restriction scratch)
};

struct PsArgs {
    int mode;                  // PS_FORWARD or PS_ADJOINT
    int nl;                    // levels smoothed by grid phases: 0 .. nl - 1
    int nu;                    // red-black sweeps before and after the coarse correction
    int bj;                    // 1: block-local smoother (mg_bj_block), 0: whole-level sweeps
    int nu_bj;                 // its sweep pairs per block
    int N, nbs, nb1;           // sites, BX-site blocks, 1D blocks (the partial partitions)
    PsLevel L[PS_MAX_LEVELS];  // 0 .. nl (level nl is the tail's finest)
    TailLevels tail;           // b0 = L[nl].b, x0 = L[nl].x
    // forward: compensated potential, this step's charge, the warm-started increment
    float *pot, *pot_lo;
    const float *eps, *rho;
    const uint8_t *info;
    float *x, *delta2;
    // forward with the minimal-residual start (mr = 1): k_pcg_init_mr's block sums, the last
    // step's increment d1 and the products q1 = A d1, q2 = A d2 (x holds d2 and r holds
    // b - A phi on entry, part[1] the partials of their norms)
    int mr;
    const float *mr_part;
    const float *mr_d1, *mr_q1, *mr_q2;
    // adjoint: right-hand side (the solution is in x)
    const float *rhs;
    float *r, *p, *p2, *q;     // r is L[0].b; z is L[0].x; p and p2 alternate
    double *part[2];           // partial arrays, alternating so a scalar read never races
    double *wsum;              // [2][32] virtual-warp sums of a split scalar reduction
    CgScalars *s;
    PsBarrier *bar;
    unsigned spin_limit;       // polls before a barrier wait gives up (PS_SPIN_LIMIT)
    int extra;                 // arrivals expected beyond the CTAs (0; 1 only to test the
                               // time-out: every barrier then runs out)
};

constexpr int PS_FORWARD = 0, PS_ADJOINT = 1;

// Reductions of at least PS_SPLIT_MIN partials have their 32 virtual-warp sums computed on
// separate CTAs (FP64 adds are slow on this part; one CTA summing 8192 partials takes ~10 us).
constexpr long long PS_SPLIT_MIN = 2048;

__device__ __forceinline__ void ps_named_sync(int id)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(BX) : "memory");
}

__device__ __forceinline__ unsigned ps_load_volatile(const unsigned *p)
{
    return *(const volatile unsigned *)p;
}

// The barrier's arrival is a GPU-scope acquire-release add and its polling an acquire load:
// the release publishes the CTA's writes of the phase (ordered before it by __syncthreads),
// the acquire makes every other CTA's visible to this one. Measured against explicit
// fence.acq_rel fences around a relaxed add and volatile polling: 0.35 us less per barrier
// (0.256 -> 0.245 ms per step with ~0.85 CG iterations per step on 96x64x64).
__device__ __forceinline__ unsigned ps_arrive(unsigned *p)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}

__device__ __forceinline__ unsigned ps_load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `epoch` (1, 2, ...). Returns false once any CTA has timed out.
__device__ __forceinline__ bool ps_sync(PsBarrier *bar, unsigned &epoch, int *ok_sh,
                                        unsigned spin_limit, int extra)
{
    epoch++;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = epoch * (gridDim.x + (unsigned)extra);
        const unsigned last = ps_arrive(&bar->count) + 1u;   // == target: everyone is in
        unsigned spins = 0;
        while (last < target && ps_load_acquire(&bar->count) < target) {
            if (ps_load_volatile(&bar->error)) {
                ok = 0;
                break;
            }
            if (++spins > spin_limit) {
                if (atomicExch(&bar->error, 1u) == 0u)
                    bar->where = epoch;
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// block_partials for the virtual block played by this thread's 128-thread group.
template <int NV>
__device__ __forceinline__ void ps_group_partials(float (&v)[NV], double *partials, int blk,
                                                  int nblk, double (*sm)[2][BX / 32])
{
    const int g = threadIdx.x / BX, t = threadIdx.x % BX;
    const int lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        const float s = warp_sum(v[k]);
        if (lane == 0)
            sm[g][k][wid] = (double)s;
    }
    ps_named_sync(1 + g);
    if (t < NV) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < BX / 32; w++)
            acc += sm[g][t][w];
        partials[(size_t)t * nblk + blk] = acc;
    }
    ps_named_sync(1 + g);   // the group's slice is rewritten by its next virtual block
}

// Flat grid-stride loop over n items.
template <class F>
__device__ __forceinline__ void ps_for(int n, F &&f)
{
    for (int i = blockIdx.x * PS_THREADS + threadIdx.x; i < n; i += gridDim.x * PS_THREADS)
        f(i);
}

// Loop over virtual blocks 0 .. nvb - 1 (group-uniform): f(vb, t).
template <class F>
__device__ __forceinline__ void ps_for_vblocks(int nvb, F &&f)
{
    const int g = threadIdx.x / BX, t = threadIdx.x % BX;
    for (int vb = blockIdx.x * PS_GROUPS + g; vb < nvb; vb += gridDim.x * PS_GROUPS)
        f(vb, t);
}

// Pointwise and 1D phases handle up to PS_B sites per thread per pass with every load issued
// before any store (the bodies carry no restrict qualifiers, so otherwise each site's loads
// would wait for the previous site's stores); per-site arithmetic and accumulation order
// are those of the range bodies in poisson.cuh.
constexpr int PS_B = 4;

// phi += delta (compensated pair), acc += delta, on active cells. With d1 (the
// minimal-residual start, delta holding d2): delta = a1 d1 + a2 d2 first, at every site
// (mr_x0_site's arithmetic), then the update.
__device__ __forceinline__ void ps_apply(int n, const float *Dg, float *delta, float *acc,
                                         float *pot, float *pot_lo, float a1 = 0.0f,
                                         float a2 = 0.0f, const float *d1 = nullptr)
{
    const int S = gridDim.x * PS_THREADS;
    for (int i0 = blockIdx.x * PS_THREADS + threadIdx.x; i0 < n; i0 += PS_B * S) {
        float dg[PS_B], d[PS_B], hi[PS_B], lo[PS_B], ac[PS_B], e[PS_B];
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int i = i0 + j * S;
            dg[j] = d[j] = hi[j] = lo[j] = ac[j] = e[j] = 0.0f;
            if (i < n) {
                dg[j] = Dg[i];
                d[j] = delta[i];
                hi[j] = pot[i];
                lo[j] = pot_lo[i];
                if (acc)
                    ac[j] = acc[i];
                if (d1)
                    e[j] = d1[i];
            }
        }
        if (d1) {
#pragma unroll
            for (int j = 0; j < PS_B; j++) {
                const int i = i0 + j * S;
                if (i < n) {
                    d[j] = __fmaf_rn(a2, d[j], __fmul_rn(a1, e[j]));
                    delta[i] = d[j];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int i = i0 + j * S;
            if (i < n && dg[j] > 0.0f) {
                if (acc)
                    acc[i] = __fadd_rn(ac[j], d[j]);
                float h, l;
                pcg_apply_pair(hi[j], lo[j], d[j], h, l);
                pot[i] = h;
                pot_lo[i] = l;
            }
        }
    }
}

// Level 0's zero start and first red half sweep at one cell, from its own b (= r) and D:
// (b + 0) / D on active red cells, 0 elsewhere (the neighbours are all 0).
__device__ __forceinline__ float ps_first_red(int x, int y, int z, float bi, float di)
{
    return ((x + y + z) & 1) == 0 && di > 0.0f ? __fdiv_rn(__fadd_rn(bi, 0.0f), di) : 0.0f;
}

// delta += alpha p, r -= alpha q, ||r||^2 over the sites of virtual block b, in site order;
// then, with first_red, level 0's first red half sweep of the next V-cycle at the same sites
// (from the new r; the block-local smoother starts from zero by itself).
__device__ __forceinline__ void ps_update_range(int n, const float *p, const float *q,
                                                float *delta, float *r, float a, int b, int nb,
                                                int t, float (&v)[1], const PsLevel &L0,
                                                bool first_red)
{
    const int S = nb * BX;
    for (int i0 = b * BX + t; i0 < n; i0 += PS_B * S) {
        float pp[PS_B], qq[PS_B], dd[PS_B], rr[PS_B], dg[PS_B];
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int i = i0 + j * S;
            pp[j] = qq[j] = dd[j] = rr[j] = dg[j] = 0.0f;
            if (i < n) {
                pp[j] = p[i];
                qq[j] = q[i];
                dd[j] = delta[i];
                rr[j] = r[i];
                dg[j] = L0.D[i];
            }
        }
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int i = i0 + j * S;
            if (i < n) {
                delta[i] = __fmaf_rn(a, pp[j], dd[j]);
                const float ri = __fmaf_rn(-a, qq[j], rr[j]);
                r[i] = ri;
                v[0] = __fmaf_rn(ri, ri, v[0]);
                if (first_red) {
                    int x, y, z;
                    cell_xyz(L0.d, i, x, y, z);
                    L0.x[i] = ps_first_red(x, y, z, ri, dg[j]);
                }
            }
        }
    }
}

// Level 0's last red half sweep at the sites of 1D virtual block b (red cells updated from
// their black neighbours, which this phase does not write), and r . z over the same sites in
// site order (z = the level's x after the sweep).
__device__ __forceinline__ void ps_gs0_dot_range(const PsLevel &L0, const float *r, int b,
                                                 int nb, int t, float (&v)[1])
{
    const MgDims &d = L0.d;
    const int S = nb * BX, n = L0.n;
    for (int i = b * BX + t; i < n; i += S) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        if (((x + y + z) & 1) == 0)
            mg_gs_cell(d, L0.D, L0.kx, L0.ky, L0.kz, L0.b, L0.x, x, y, z);
        v[0] = __fmaf_rn(r[i], L0.x[i], v[0]);
    }
}

// q_i = (A p)_i with p = z + beta p_old formed at the site and its neighbours as pcg_p_site
// forms it (p_i returned for storing); the arithmetic of pcg_Ap_value.
template <int D>
__device__ __forceinline__ float ps_Ap_value(const MgDims &d, const float *eps,
                                             const uint8_t *info, const float *Dg,
                                             const float *p_old, const float *zv, float beta,
                                             int x, int y, int z, float &pi_out, float (&v)[1])
{
    const int i = cell(d, x, y, z);
    const Nb6 nb = nb6(d, i, x, y, z);
    const float Di = Dg[i], ei = eps[i];
    const float pi = beta != 0.0f ? __fmaf_rn(beta, p_old[i], zv[i]) : zv[i];
    int pt[2 * D];
    float ej[2 * D], pj[2 * D];
#pragma unroll
    for (int f = 0; f < 2 * D; f++) {
        const int j = nb.n[f];
        pt[f] = info[j] & 3;
        ej[f] = eps[j];
        pj[f] = beta != 0.0f ? __fmaf_rn(beta, p_old[j], zv[j]) : zv[j];
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
    pi_out = pi;
    return qi;
}

// One red-black half sweep (colour c) of level L, cells in flat order (nx even).
__device__ __forceinline__ void ps_gs(const PsLevel &L, int color)
{
    const MgDims &d = L.d;
    const int hx = d.nx >> 1;
    ps_for(L.n >> 1, [&](int k) {
        const int row = fdiv(k, d.mh, d.sh);
        const int j = k - row * hx;
        const int z = fdiv(row, d.my, d.sy);
        const int y = row - z * d.ny;
        const int x = 2 * j + ((y + z + color) & 1);
        mg_gs_cell(d, L.D, L.kx, L.ky, L.kz, L.b, L.x, x, y, z);
    });
}

// x = 0 then the first red half sweep: every neighbour is 0, so the update of a red cell is
// (b + 0) / D (offdiag_sum of zeros is +0), black and inactive cells keep 0.
__device__ __forceinline__ void ps_gs_first(const PsLevel &L)
{
    const MgDims &d = L.d;
    const int S = gridDim.x * PS_THREADS, n = L.n;
    for (int c0 = blockIdx.x * PS_THREADS + threadIdx.x; c0 < n; c0 += PS_B * S) {
        float dg[PS_B], bb[PS_B];
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int c = c0 + j * S;
            dg[j] = bb[j] = 0.0f;
            if (c < n) {
                dg[j] = L.D[c];
                bb[j] = L.b[c];
            }
        }
#pragma unroll
        for (int j = 0; j < PS_B; j++) {
            const int c = c0 + j * S;
            if (c < n) {
                int x, y, z;
                cell_xyz(d, c, x, y, z);
                float v = 0.0f;
                if (((x + y + z) & 1) == 0 && dg[j] > 0.0f)
                    v = __fdiv_rn(__fadd_rn(bb[j], 0.0f), dg[j]);
                L.x[c] = v;
            }
        }
    }
}

// Residual b - A x of one fine cell (0 on inactive cells), as mg_resid_cell computes it.
__device__ __forceinline__ float ps_resid(const PsLevel &F, int x, int y, int z)
{
    const MgDims &f = F.d;
    const int i = cell(f, x, y, z);
    const float di = F.D[i], xi = F.x[i], bi = F.b[i];
    const float Ax = __fmaf_rn(di, xi, -offdiag_sum(f, i, x, y, z, F.kx, F.ky, F.kz, F.x));
    return di > 0.0f ? __fsub_rn(bi, Ax) : 0.0f;
}

// b_c = sum over each coarse cell's children of the fine residual, in the order of
// mg_restrict_sum_cell ((x, y, z) = (2X + a, 2Y + b, z0 + g), a outermost). Eight lanes per
// coarse cell: lane ch = 4a + 2b + g of the group evaluates one child, the group's first
// lane gathers the eight by shuffles and sums them in that order. With `start`, the same
// lane also does the coarse level's zero start and first red half sweep at that cell (the
// value ps_gs_first writes there, from the b just formed), which saves that phase's grid
// barrier.
__device__ __forceinline__ void ps_resid_restrict(const PsLevel &F, const PsLevel &C, bool start)
{
    const MgDims &f = F.d, &c = C.d;
    const int span = (C.n * 8 + 31) & ~31;   // whole warps: every lane reaches the shuffles
    const int lane = threadIdx.x & 31;
    for (int k = blockIdx.x * PS_THREADS + threadIdx.x; k < span; k += gridDim.x * PS_THREADS) {
        const int I = k >> 3, ch = k & 7;
        bool z1 = false;
        float r = 0.0f;
        if (I < C.n) {
            int X, Y, Z;
            cell_xyz(c, I, X, Y, Z);
            const int z0 = F.cz2 ? 2 * Z : Z;
            z1 = F.cz2 && z0 + 1 < f.nz;
            const int a = ch >> 2, b = (ch >> 1) & 1, g = ch & 1;
            if (g == 0 || z1)
                r = ps_resid(F, 2 * X + a, 2 * Y + b, z0 + g);
        }
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; j++)
            v[j] = __shfl_sync(0xffffffffu, r, (lane & ~7) + j);
        if (ch == 0 && I < C.n) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if ((j & 1) == 0 || z1)
                    acc = __fadd_rn(acc, v[j]);
            C.b[I] = acc;
            if (start) {
                int X, Y, Z;
                cell_xyz(c, I, X, Y, Z);
                C.x[I] = ps_first_red(X, Y, Z, acc, C.D[I]);
            }
        }
    }
}

// Prolongation fused into the first black half sweep after it: a black cell's update reads
// its (red) neighbours as the prolongation would have left them, x_j + x_c(parent of j) on
// active cells, computed on the fly in the order offdiag_sum uses. Red cells are not
// written: the red half sweep that follows overwrites every active red cell without reading
// it, and prolongation leaves inactive cells alone. Same bits as prolong, then sweep.
__device__ __forceinline__ void ps_prolong_gs1(const PsLevel &F, const PsLevel &C)
{
    const MgDims &d = F.d, &c = C.d;
    const int hx = d.nx >> 1;
    auto xp = [&](int j, int x, int y, int z) {
        const float xj = F.x[j];
        return F.D[j] > 0.0f
                   ? __fadd_rn(xj, C.x[cell(c, x >> 1, y >> 1, F.cz2 ? (z >> 1) : z)])
                   : xj;
    };
    ps_for(F.n >> 1, [&](int k) {
        const int row = fdiv(k, d.mh, d.sh);
        const int jx = k - row * hx;
        const int z = fdiv(row, d.my, d.sy);
        const int y = row - z * d.ny;
        const int x = 2 * jx + ((y + z + 1) & 1);
        const int i = cell(d, x, y, z);
        const Nb6 nb = nb6(d, i, x, y, z);
        const int xm = x == 0 ? d.nx - 1 : x - 1, xq = x + 1 == d.nx ? 0 : x + 1;
        const int ym = y == 0 ? d.ny - 1 : y - 1, yq = y + 1 == d.ny ? 0 : y + 1;
        const float di = F.D[i], bi = F.b[i];
        float s = __fmul_rn(F.kx[i], xp(nb.n[0], xq, y, z));
        s = __fmaf_rn(F.kx[nb.n[1]], xp(nb.n[1], xm, y, z), s);
        s = __fmaf_rn(F.ky[i], xp(nb.n[2], x, yq, z), s);
        s = __fmaf_rn(F.ky[nb.n[3]], xp(nb.n[3], x, ym, z), s);
        if (d.nz > 1) {
            const int zm = z == 0 ? d.nz - 1 : z - 1, zq = z + 1 == d.nz ? 0 : z + 1;
            s = __fmaf_rn(F.kz[i], xp(nb.n[4], x, y, zq), s);
            s = __fmaf_rn(F.kz[nb.n[5]], xp(nb.n[5], x, y, zm), s);
        }
        if (di > 0.0f)
            F.x[i] = __fdiv_rn(__fadd_rn(bi, s), di);
    });
}

template <int D>
__global__ void __launch_bounds__(PS_THREADS, 1) k_poisson_solve(const __grid_constant__ PsArgs A)
{
    extern __shared__ float tail_sm[];
    __shared__ CgScalars s;
    __shared__ double gsm[PS_GROUPS][2][BX / 32];
    __shared__ int ok_sh;
    unsigned epoch = 0;
    if (threadIdx.x == 0)
        s = *A.s;
    __syncthreads();
    bool ok = true;
    auto sync = [&]() {
        if (ok)
            ok = ps_sync(A.bar, epoch, &ok_sh, A.spin_limit, A.extra);
    };
    // barrier, then the CG scalar update from the partial arrays, in the fixed order of
    // pcg_scalar_block: small reductions are summed by every CTA; large ones have their 32
    // virtual-warp sums spread over CTAs 0 .. 32 nv - 1, a second barrier, then every CTA
    // finishes the butterfly over the 32 sums and updates its copy of the scalars
    auto sync_scalar = [&](const double *part, int nv, int op, int nblk, bool first = true,
                           double rr_sub = 0.0) {
        if (first)   // not for partials written by the kernel before this one
            sync();
        if (!ok)
            return;
        if ((long long)nv * nblk < PS_SPLIT_MIN || (int)gridDim.x < 32 * nv) {
            pcg_scalar_block(part, nblk, nv, op, &s, rr_sub);
            __syncthreads();
            return;
        }
        if (threadIdx.x < 32 && (int)blockIdx.x < 32 * nv) {
            const int k = blockIdx.x >> 5, w = blockIdx.x & 31;
            const double a = pcg_vwarp_sum(part + (size_t)k * nblk, nblk, 32 * w + threadIdx.x);
            if (threadIdx.x == 0)
                A.wsum[k * 32 + w] = a;
        }
        sync();
        if (!ok)
            return;
        if (threadIdx.x < 32) {
            double tot[2] = {0.0, 0.0};
            for (int k = 0; k < nv; k++) {
                double a = __ldcg(A.wsum + k * 32 + threadIdx.x);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                tot[k] = a;
            }
            if (threadIdx.x == 0)
                pcg_scalar_update(tot, op, &s, rr_sub);
        }
        __syncthreads();
    };
    const PsLevel &L0 = A.L[0];
    float *z = A.bj ? L0.xo : L0.x;

    // the p buffers alternate: Ap reads the previous direction and writes the new one
    float *p_old = A.p, *p_new = A.p2;

    // one symmetric V-cycle, z ~= A^-1 r. After an iteration's update, level 0's zero start
    // and first red half sweep were done by that update (z_ready); the last red half sweep of
    // level 0 also forms the r . z partials (then the caller's op-1 reduction ends the phase).
    bool z_ready = false, tail_ops = false;
    auto vcycle = [&]() {
        for (int l = 0; l < A.nl && ok; l++) {
            const PsLevel &L = A.L[l];
            if (l == 0 && !z_ready) {   // coarser levels were started by the restriction
                ps_gs_first(L);
                sync();
            }
            ps_gs(L, 1);
            sync();
            for (int k = 1; k < A.nu && ok; k++) {
                ps_gs(L, 0);
                sync();
                ps_gs(L, 1);
                sync();
            }
            ps_resid_restrict(L, A.L[l + 1], l + 1 < A.nl);
            sync();
        }
        if (!ok)
            return;
        if (blockIdx.x == 0) {   // the tail's operators stay in shared memory after the first
            mg_tail_block(A.tail, tail_sm, tail_ops);
            tail_ops = true;
        }
        sync();
        for (int l = A.nl - 1; l >= 0 && ok; l--) {
            const PsLevel &L = A.L[l];
            for (int k = 0; k < A.nu && ok; k++) {
                if (k == 0)
                    ps_prolong_gs1(L, A.L[l + 1]);
                else
                    ps_gs(L, 1);
                sync();
                if (l == 0 && k == A.nu - 1) {
                    ps_for_vblocks(A.nb1, [&](int vb, int t) {
                        float v[1] = {0.0f};
                        ps_gs0_dot_range(L0, A.r, vb, A.nb1, t, v);
                        ps_group_partials<1>(v, A.part[0], vb, A.nb1, gsm);
                    });
                } else {
                    ps_gs(L, 0);
                    sync();
                }
            }
        }
    };

    // the same V-cycle with the block-local smoother: per level on the way down one
    // smoothing phase from zero and the residual + restriction phase, on the way up one
    // phase of prolongation + smoothing (into the level's xo); level 0's last phase also
    // forms the r . z partials, one per block
    auto vcycle_bj = [&]() {
        for (int l = 0; l < A.nl && ok; l++) {
            const PsLevel &L = A.L[l];
            for (int blk = blockIdx.x; blk < L.nbj; blk += gridDim.x)
                mg_bj_block<D>(L.d, L.D, L.kx, L.ky, L.kz, L.b, nullptr, L.x, blk, A.nu_bj, false,
                               L.d, 0, nullptr, nullptr, nullptr);
            sync();
            ps_resid_restrict(L, A.L[l + 1], false);
            sync();
        }
        if (!ok)
            return;
        if (blockIdx.x == 0) {
            mg_tail_block(A.tail, tail_sm, tail_ops);
            tail_ops = true;
        }
        sync();
        for (int l = A.nl - 1; l >= 0 && ok; l--) {
            const PsLevel &L = A.L[l], &C = A.L[l + 1];
            const float *xc = l + 1 == A.nl ? C.x : C.xo;
            for (int blk = blockIdx.x; blk < L.nbj; blk += gridDim.x)
                mg_bj_block<D>(L.d, L.D, L.kx, L.ky, L.kz, L.b, L.x, L.xo, blk, A.nu_bj, true,
                               C.d, L.cz2, xc, l == 0 ? A.r : nullptr, A.part[0]);
            if (l > 0)
                sync();
        }
    };

    // one preconditioned CG iteration on the increment (or adjoint potential) xv
    auto iteration = [&](float *xv) {
        if (A.bj)
            vcycle_bj();
        else
            vcycle();
        sync_scalar(A.part[0], 1, 1, A.bj ? L0.nbj : A.nb1);   // r . z
        if (!ok)
            return;
        const float beta = pcg_beta(&s);
        ps_for_vblocks(A.nbs, [&](int vb, int t) {
            // p = z + beta p and q = A p, p formed on the fly at the site and its neighbours
            const int i = vb * BX + t;
            float v[1] = {0.0f};
            if (i < A.N) {
                int x, y, zz;
                cell_xyz(L0.d, i, x, y, zz);
                float pi;
                A.q[i] = ps_Ap_value<D>(L0.d, A.eps, A.info, L0.D, p_old, z, beta, x, y, zz, pi,
                                        v);
                p_new[i] = pi;
            }
            ps_group_partials<1>(v, A.part[1], vb, A.nbs, gsm);
        });
        sync_scalar(A.part[1], 1, 2, A.nbs);   // p . Ap
        if (!ok)
            return;
        const float alpha = (float)s.alpha;
        ps_for_vblocks(A.nb1, [&](int vb, int t) {
            float v[1] = {0.0f};
            ps_update_range(A.N, p_new, A.q, xv, A.r, alpha, vb, A.nb1, t, v, L0, !A.bj);
            ps_group_partials<1>(v, A.part[0], vb, A.nb1, gsm);
        });
        float *tp = p_old;
        p_old = p_new;
        p_new = tp;
        z_ready = true;
        sync_scalar(A.part[0], 1, 3, A.nb1);   // ||r||^2
    };

    // the refinement pass's start: r = b - A phi of the updated potential, with its increment
    // delta2 read as zero and zeroed in the same pass, then op 4 (this phase does nothing for
    // the V-cycle: most refinement passes stop here)
    auto refine_start = [&]() {
        ps_for_vblocks(A.nbs, [&](int vb, int t) {
            const int i = vb * BX + t;
            float v[2] = {0.0f, 0.0f};
            if (i < A.N) {
                int x, y, zz;
                cell_xyz(L0.d, i, x, y, zz);
                A.r[i] = pcg_init_value<D>(L0.d, A.pot, A.pot_lo, A.delta2, A.eps, A.rho,
                                           A.info, L0.D, x, y, zz, v, true);
                A.delta2[i] = 0.0f;
            }
            ps_group_partials<2>(v, A.part[1], vb, A.nbs, gsm);
        });
        z_ready = false;
        sync_scalar(A.part[1], 2, 4, A.nbs);
    };

    // the start residual r and its partials part[1] come from the k_pcg_init (forward) or
    // k_adj_pcg_init (adjoint) launch just before this kernel: only their reduction is left.
    // The minimal-residual start (k_pcg_init_mr before this kernel) first sums its coefficients
    // in every CTA, in k_mr_alpha's order, and tests its least residual; if that meets the
    // tolerance, the potential update forms x0 as it goes, else a phase forms x0 and r.
    z_ready = false;
    const bool mr = A.mode == PS_FORWARD && A.mr;
    __shared__ double mra[3];
    if (mr)
        mr_alpha_block(A.mr_part, A.nbs, mra);
    sync_scalar(A.part[1], 2, 0, A.nbs, false, mr ? mra[2] : 0.0);
    bool x0_formed = !mr;
    if (ok && mr && !s.done) {
        const float a1 = (float)mra[0], a2 = (float)mra[1];
        ps_for(A.N, [&](int i) { mr_start_site(i, a1, a2, A.mr_d1, A.x, A.r, A.mr_q1, A.mr_q2); });
        x0_formed = true;
        sync();
    }
    while (ok && !s.done)
        iteration(A.x);
    if (ok && A.mode == PS_FORWARD) {
        if (x0_formed)
            ps_apply(A.N, L0.D, A.x, nullptr, A.pot, A.pot_lo);
        else
            ps_apply(A.N, L0.D, A.x, nullptr, A.pot, A.pot_lo, (float)mra[0], (float)mra[1],
                     A.mr_d1);
        // refinement: the true residual of the updated potential, once, if the pass iterated
        // (s.refine is the same in every CTA; without it the kernel's end is the barrier)
        if (ok && s.refine)
            sync();
        if (ok && s.refine) {
            refine_start();
            while (ok && !s.done)
                iteration(A.delta2);
            if (ok)
                ps_apply(A.N, L0.D, A.delta2, A.x, A.pot, A.pot_lo);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!ok) {
            s.done = 1;
            s.nonconv = 1;
        }
        *A.s = s;
    }
}

}  // namespace lbehd

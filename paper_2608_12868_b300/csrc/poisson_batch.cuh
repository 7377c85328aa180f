// poisson_batch.cuh -- the Gauss-law solve (Eq. 13) of many instances in lockstep: every
// multigrid and CG stage is one launch over all instances, and one device-side loop
// iterates while any instance's CG pass is unconverged.
//
// Each launch is a fixed grid of CTAs walking work items (instance k, block b of that
// instance's partition of this stage). At start a CTA builds, in shared memory, the table of
// the instances taking part in the launch: all of them, or those the activity mode selects
// (a list the CG scalar kernel rewrites after every update, so a converged instance
// costs nothing), with their block offsets. The launch's per-instance parameters travel in
// kernel parameter space. The per-site arithmetic is the single-instance kernels' own (the
// *_cell / *_site / *_range bodies of poisson.cuh), and every reduction keeps that
// instance's single-instance partition (blocks of BX consecutive sites for the stencil
// reductions, a grid stride over nb1d blocks for the vector reductions), so the partial
// sums, and hence every CG scalar, are bitwise those of the single-instance solve.
#pragma once

#include "batch.cuh"
#include "poisson.cuh"

namespace lbehd {

// Activity modes: 0 every instance; 1 instances whose current CG pass is not done; 2
// instances refining this step (their first pass iterated); 3 refining and not done.
__device__ __forceinline__ bool batch_active(int mode, const CgScalars *s)
{
    if (mode == 0)
        return true;
    const int done = s->done, ref = s->refine;
    if (mode == 1)
        return !done;
    if (mode == 2)
        return ref != 0;
    return ref != 0 && !done;
}

// Instances active in modes 1-3 (index 0 unused), rewritten by k_pcg_scalar_batch_split.
struct ActiveLists {
    int count[4];
    int ids[4][BATCH_MAX];
};

struct GridSet {
    int n, mode;
    int blocks[BATCH_MAX];              // work items of instance k in this launch (0: none)
    CgScalars *s[BATCH_MAX];
    const ActiveLists *act;
};

// The CTA's table of the launch's instances: ids[j] owns work items [start[j], start[j+1]).
struct WorkTable {
    int n;
    int ids[BATCH_MAX];
    int start[BATCH_MAX + 1];
};

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int &total)
{
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += t;
    }
    total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

__device__ __forceinline__ void load_work(const GridSet &g, WorkTable &W)
{
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int cnt = g.mode == 0 ? g.n : g.act->count[g.mode];
        int base = 0;
#pragma unroll
        for (int h = 0; h < BATCH_MAX / 32; h++) {
            const int j = h * 32 + lane;
            const int id = j < cnt ? (g.mode == 0 ? j : g.act->ids[g.mode][j]) : 0;
            const int nb = j < cnt ? g.blocks[id] : 0;
            int tot;
            const int ex = warp_excl_scan(nb, lane, tot);
            W.ids[j] = id;
            W.start[j] = base + ex;
            base += tot;
        }
        if (lane == 0) {
            W.n = cnt;
            W.start[cnt] = base;
        }
    }
    __syncthreads();
}

// Largest j with W.start[j] <= w (w < W.start[W.n]).
__device__ __forceinline__ int work_slot(const WorkTable &W, int w)
{
    int lo = 0, hi = W.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (W.start[mid] <= w)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// for (each work item of this CTA) body(k, b); uniform across the CTA.
template <class F>
__device__ __forceinline__ void for_work(const GridSet &g, F &&body)
{
    __shared__ WorkTable W;
    load_work(g, W);
    const int total = W.start[W.n];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int j = work_slot(W, w);
        body(W.ids[j], w - W.start[j]);
    }
}

// block_partials for use inside a work loop: the shared scratch is free again on return.
template <int NV>
__device__ __forceinline__ void block_partials_loop(float (&v)[NV], double *partials, int blk,
                                                    int nblk)
{
    block_partials<NV>(v, partials, (size_t)blk, (size_t)nblk);
    __syncthreads();
}

// ---------------------------------------------------------------- multigrid

struct MgInst {
    MgDims f, c;                              // this level and the next coarser one
    int cz2, reps;                            // coarsening halves z; sweeps of this instance
    float scale;
    const float *eps;                         // level-0 set-up
    const uint8_t *info;
    float *D, *kx, *ky, *kz, *b, *x, *r;      // this level (r: residual scratch)
    float *Dc, *kxc, *kyc, *kzc, *bc, *xc;    // the coarser level
    // block-local smoother (k_mg_bj_batch): the coarse correction's source on the way up
    // (the coarser level's way-up output, or the tail's x), and on level 0 the CG residual
    // and the r . z partials the way-up pass writes (null on other levels)
    const float *xcu, *rdot;
    double *pdot;
};

struct MgBatch {
    GridSet g;
    int color, sweep;                         // Gauss-Seidel colour and sweep index
    MgInst m[BATCH_MAX];
};

__device__ __forceinline__ int cells(const MgDims &d) { return d.nx * d.ny * d.nz; }

// x = 0 on this level (one cell per thread).
__global__ void __launch_bounds__(BX) k_mg_zero_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const int i = b * BX + threadIdx.x;
        if (i < cells(A.m[k].f))
            A.m[k].x[i] = 0.0f;
    });
}

template <int D>
__global__ void __launch_bounds__(BX) k_mg_setup0_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const int i = b * BX + threadIdx.x;
        if (i >= cells(m.f))
            return;
        int x, y, z;
        cell_xyz(m.f, i, x, y, z);
        mg_setup0_cell<D>(m.f, m.eps, m.info, m.D, m.kx, m.ky, m.kz, x, y, z);
    });
}

__global__ void __launch_bounds__(BX) k_mg_coarsen_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const int i = b * BX + threadIdx.x;
        if (i >= cells(m.c))
            return;
        int X, Y, Z;
        cell_xyz(m.c, i, X, Y, Z);
        mg_coarsen_cell(m.f, m.c, m.cz2, m.scale, m.D, m.kx, m.ky, m.kz, m.Dc, m.kxc, m.kyc,
                        m.kzc, X, Y, Z);
    });
}

// One red-black half sweep: thread -> cell (2 x2 + colour offset, y, z) of this level (nx is
// even on every level). Instances whose sweep count is below A.sweep + 1 take no part.
__global__ void __launch_bounds__(BX) k_mg_gs_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const int half = m.f.nx >> 1;
        const int i = b * BX + threadIdx.x;
        if (i >= half * m.f.ny * m.f.nz)
            return;
        const int r = fdiv(i, m.f.mh, m.f.sh), z = fdiv(r, m.f.my, m.f.sy), y = r - z * m.f.ny;
        const int x = 2 * (i - r * half) + ((y + z + A.color) & 1);
        mg_gs_cell(m.f, m.D, m.kx, m.ky, m.kz, m.b, m.x, x, y, z);
    });
}

// x = 0 on this level, then the first red half sweep. Every neighbour is 0, so a red cell
// with D > 0 gets (b + 0) / D (offdiag_sum of zeros is +0) and every other cell 0: the same
// bits as k_mg_zero_batch followed by k_mg_gs_batch with colour 0, in one pass.
__global__ void __launch_bounds__(BX) k_mg_gs_first_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const int i = b * BX + threadIdx.x;
        if (i >= cells(m.f))
            return;
        int x, y, z;
        cell_xyz(m.f, i, x, y, z);
        const float di = m.D[i];
        float v = 0.0f;
        if (((x + y + z) & 1) == 0 && di > 0.0f)
            v = __fdiv_rn(__fadd_rn(m.b[i], 0.0f), di);
        m.x[i] = v;
    });
}

// The fine level's residual and its restriction in one pass: 8 lanes per coarse cell form
// the residuals of its children, and the first lane sums them in the child order of
// mg_restrict_sum_cell (the same bits as mg_resid_cell on every fine cell, then
// mg_restrict_sum_cell).
// A work item is BX / 8 coarse cells. Needs even fine x and y extents (every coarsened
// level has them).
__global__ void __launch_bounds__(BX) k_mg_resid_restrict_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const MgDims &f = m.f;
        const int lane = threadIdx.x & 31, ch = threadIdx.x & 7;
        const int I = b * (BX / 8) + (threadIdx.x >> 3);
        const bool own = I < cells(m.c);
        bool z1 = false;
        float r = 0.0f;
        if (own) {
            int X, Y, Z;
            cell_xyz(m.c, I, X, Y, Z);
            const int z0 = m.cz2 ? 2 * Z : Z;
            z1 = m.cz2 && z0 + 1 < f.nz;
            const int g = ch & 1;
            if (g == 0 || z1) {
                const int x = 2 * X + (ch >> 2), y = 2 * Y + ((ch >> 1) & 1), z = z0 + g;
                const int i = cell(f, x, y, z);
                const float di = m.D[i], xi = m.x[i], bi = m.b[i];
                const float Ax =
                    __fmaf_rn(di, xi, -offdiag_sum(f, i, x, y, z, m.kx, m.ky, m.kz, m.x));
                r = di > 0.0f ? __fsub_rn(bi, Ax) : 0.0f;
            }
        }
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; j++)
            v[j] = __shfl_sync(0xffffffffu, r, (lane & ~7) + j);
        if (ch == 0 && own) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if ((j & 1) == 0 || z1)
                    acc = __fadd_rn(acc, v[j]);
            m.bc[I] = acc;
        }
    });
}

// The block-local smoother's pass (mg_bj_block) on every listed instance, one work item per
// block, reps sweep pairs per block; A.color = 1 on the way up (prolongation, output in r),
// 0 on the way down (zero start, output in x).
template <int D>
__global__ void __launch_bounds__(BJ_THREADS, 1) k_mg_bj_batch(const __grid_constant__ MgBatch A)
{
    const bool up = A.color != 0;
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        mg_bj_block<D>(m.f, m.D, m.kx, m.ky, m.kz, m.b, up ? m.x : nullptr, up ? m.r : m.x, b,
                       m.reps, up, m.c, m.cz2, m.xcu, up ? m.rdot : nullptr, m.pdot);
    });
}

__global__ void __launch_bounds__(BX) k_mg_prolong_batch(const __grid_constant__ MgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const MgInst &m = A.m[k];
        const int i = b * BX + threadIdx.x;
        if (i >= cells(m.f))
            return;
        int x, y, z;
        cell_xyz(m.f, i, x, y, z);
        mg_prolong_cell(m.f, m.c, m.cz2, m.D, m.xc, m.x, x, y, z);
    });
}

struct TailBatch {
    GridSet g;                                // one work item per instance with a tail
    const TailLevels *T[BATCH_MAX];           // device copies (b0, x0 set)
};

// The shared-memory tail of every active instance that has one, one CTA each.
__global__ void __launch_bounds__(TAIL_THREADS) k_mg_tail_batch(const __grid_constant__ TailBatch A)
{
    __shared__ TailLevels T;
    extern __shared__ float sm[];
    for_work(A.g, [&](int k, int) {
        constexpr int W = (int)(sizeof(TailLevels) / sizeof(int));
        static_assert(sizeof(TailLevels) % sizeof(int) == 0, "TailLevels copied as ints");
        const int *src = reinterpret_cast<const int *>(A.T[k]);
        int *dst = reinterpret_cast<int *>(&T);
        for (int w = threadIdx.x; w < W; w += blockDim.x)
            dst[w] = src[w];
        __syncthreads();
        mg_tail_block(T, sm);
        __syncthreads();
    });
}

// ---------------------------------------------------------------- CG on level 0

struct CgInst {
    MgDims d;
    int nbs, nb1d;             // site partition: nbs blocks of BX consecutive sites; grid
                               // stride: nb1d blocks
    float *pot, *pot_lo;
    const float *eps, *rho;
    const uint8_t *info;
    const float *Dg;           // level-0 diagonal
    float *r, *p, *q, *z;      // z: the level-0 V-cycle output
    float *x, *acc;            // the increment solved for; where apply accumulates it (or null)
    double *partials;
    // the least-residual start (LBEHD_OPT_WARM_START 1): the last step's increment (x holds
    // the one before), the start pass's block sums and the coefficients (a1, a2, a . c)
    const float *d1;
    float *mr_part;
    double *mr_alpha;
};

struct CgBatch {
    GridSet g;
    CgInst c[BATCH_MAX];
};

template <int D>
__global__ void __launch_bounds__(BX) k_pcg_init_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        const int i = b * BX + threadIdx.x;
        float v[2] = {0.f, 0.f};
        if (i < cells(c.d)) {
            int x, y, z;
            cell_xyz(c.d, i, x, y, z);
            pcg_init_site<D>(c.d, c.pot, c.pot_lo, c.x, c.eps, c.rho, c.info, c.Dg, c.r, x, y, z,
                             v);
        }
        block_partials_loop<2>(v, c.partials, b, c.nbs);
    });
}

// The least-residual start of every instance in the set: the first pass (mr_init_block over
// the instance's BX-site blocks, r0 into r, A d1 into q, A d2 into p), the coefficients (one
// SCALAR_THREADS block per instance, k_mr_alpha's order), then x0 and r (k_pcg_start_mr's
// per-site arithmetic).
template <int D>
__global__ void __launch_bounds__(BX) k_pcg_init_mr_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        mr_init_block<D>(c.d, c.pot, c.pot_lo, c.d1, c.x, c.eps, c.rho, c.info, c.Dg, c.r, c.q,
                         c.p, c.partials, c.mr_part, b, c.nbs);
    });
}

__global__ void __launch_bounds__(SCALAR_THREADS) k_mr_alpha_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int) {
        const CgInst &c = A.c[k];
        mr_alpha_block(c.mr_part, c.nbs, c.mr_alpha);
    });
}

__global__ void __launch_bounds__(BX) k_pcg_start_mr_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        const float a1 = (float)c.mr_alpha[0], a2 = (float)c.mr_alpha[1];
        const int n = cells(c.d);
        for (int i = b * BX + threadIdx.x; i < n; i += c.nb1d * BX)
            mr_start_site(i, a1, a2, c.d1, c.x, c.r, c.q, c.p);
    });
}

template <int D>
__global__ void __launch_bounds__(BX) k_pcg_Ap_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        const int i = b * BX + threadIdx.x;
        float v[1] = {0.f};
        if (i < cells(c.d)) {
            int x, y, z;
            cell_xyz(c.d, i, x, y, z);
            pcg_Ap_site<D>(c.d, c.eps, c.info, c.Dg, c.p, c.q, x, y, z, v);
        }
        block_partials_loop<1>(v, c.partials, b, c.nbs);
    });
}

__global__ void __launch_bounds__(BX) k_pcg_dot_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        float v[1] = {0.f};
        pcg_dot_range(cells(c.d), c.r, c.z, b, c.nb1d, v);
        block_partials_loop<1>(v, c.partials, b, c.nb1d);
    });
}

__global__ void __launch_bounds__(BX) k_pcg_p_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        pcg_p_range(cells(c.d), c.z, c.p, A.g.s[k], b, c.nb1d);
    });
}

__global__ void __launch_bounds__(BX) k_pcg_update_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        float v[1] = {0.f};
        pcg_update_range(cells(c.d), c.p, c.q, c.x, c.r, A.g.s[k], b, c.nb1d, v);
        block_partials_loop<1>(v, c.partials, b, c.nb1d);
    });
}

__global__ void __launch_bounds__(BX) k_pcg_apply_batch(const __grid_constant__ CgBatch A)
{
    for_work(A.g, [&](int k, int b) {
        const CgInst &c = A.c[k];
        pcg_apply_range(cells(c.d), c.Dg, c.x, c.acc, c.pot, c.pot_lo, b, c.nb1d);
    });
}

struct ScalarBatch {
    GridSet g;                                // one block per instance (blocks[] unused)
    const double *partials[BATCH_MAX];
    long long nblocks[BATCH_MAX];
    int nv, op;
    int loop_mode;                            // >= 0: set `cond` to "some instance active in
                                              // this mode" after the update
    int set_ref;                              // set `cond_ref` to "some instance refining"
    int eager;                                // no graph: write the two conditions to
                                              // counters[6], [7] for the host instead
    cudaGraphConditionalHandle cond, cond_ref;
    int *counters;                            // [2] arrivals (zero between launches); [3..5]
                                              // pass counts (ops 3, 5, 4); [6..7] eager
    ActiveLists *act;                         // rewritten after ops 0, 3, 4, 5
    unsigned *icnt;                           // [BATCH_MAX] arrivals per instance (split form)
    double *wsum;                             // [BATCH_MAX][2][32] virtual-warp sums
    const double *mr[BATCH_MAX];              // op 0: the instance's least-residual start
                                              // coefficients (a1, a2, a . c), or null
};

// The last block's work after every instance's update: rewrite the active lists, set the
// batch's loop conditions (or, eager, hand them to the host) and zero the arrival count.
// Run by one warp.
__device__ __forceinline__ void batch_scalar_finish(const ScalarBatch &A, int lane)
{
    const int n = A.g.n;
    int cnt[4] = {0, 0, 0, 0};
#pragma unroll
    for (int h = 0; h < BATCH_MAX / 32; h++) {
        const int j = h * 32 + lane;
        int done = 1, ref = 0;
        if (j < n) {
            const volatile CgScalars *sj = A.g.s[j];
            done = sj->done;
            ref = sj->refine;
        }
        const bool in[4] = {false, j < n && !done, j < n && ref != 0, j < n && ref != 0 && !done};
#pragma unroll
        for (int m = 1; m < 4; m++) {
            const unsigned bal = __ballot_sync(0xffffffffu, in[m]);
            if (in[m])
                A.act->ids[m][cnt[m] + __popc(bal & ((1u << lane) - 1u))] = j;
            cnt[m] += __popc(bal);
        }
    }
    if (lane != 0)
        return;
    for (int m = 1; m < 4; m++)
        A.act->count[m] = cnt[m];
    A.counters[2] = 0;
    const int any_act = A.loop_mode >= 0 ? cnt[A.loop_mode] : 0, any_ref = cnt[2];
    if (A.eager) {
        A.counters[6] = any_act;
        A.counters[7] = any_ref;
        return;
    }
    // passes of the main loop, of the refinement loop, refinement blocks entered
    if (A.op == 3 || A.op == 5 || A.op == 4)
        A.counters[A.op == 3 ? 3 : (A.op == 5 ? 4 : 5)] += 1;
    if (A.loop_mode >= 0)
        cudaGraphSetConditional(A.cond, any_act > 0 ? 1u : 0u);
    if (A.set_ref)
        cudaGraphSetConditional(A.cond_ref, any_ref > 0 ? 1u : 0u);
}

// The CG scalar update of every active instance, each instance's sums split over 32
// one-warp CTAs (FP64 adds are slow on this part, so one 1024-thread CTA per instance is
// latency-bound): CTA (k, w) forms virtual warp w's sums of pcg_scalar_block's order, the
// last CTA of instance k adds them (the butterfly over 32) and updates its scalars (same bits
// as pcg_scalar_block), and the last instance to finish does the lists and conditions
// (batch_scalar_finish). icnt must be zero before the first launch; it is reset as it is used.
__global__ void __launch_bounds__(32) k_pcg_scalar_batch_split(const __grid_constant__ ScalarBatch A)
{
    const int k = blockIdx.x >> 5, w = blockIdx.x & 31, lane = threadIdx.x;
    const int ninst = (int)gridDim.x >> 5;
    CgScalars *s = A.g.s[k];
    const bool act = batch_active(A.g.mode, s);   // read before the instance's update
    if (act)
        for (int v = 0; v < A.nv; v++) {
            const double a = pcg_vwarp_sum(A.partials[k] + v * A.nblocks[k], A.nblocks[k], 32 * w + lane);
            if (lane == 0)
                A.wsum[(k * 2 + v) * 32 + w] = a;
        }
    int last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&A.icnt[k], 1u) == 31u;
    }
    if (!__shfl_sync(0xffffffffu, last, 0))
        return;
    __threadfence();
    if (act) {
        double tot[2] = {0.0, 0.0};
        for (int v = 0; v < A.nv; v++) {
            double a = __ldcg(A.wsum + (k * 2 + v) * 32 + lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                a += __shfl_xor_sync(0xffffffffu, a, o);
            tot[v] = a;
        }
        if (lane == 0)
            pcg_scalar_update(tot, A.op, s, A.op == 0 && A.mr[k] ? A.mr[k][2] : 0.0);
    }
    if (lane == 0)
        A.icnt[k] = 0u;
    if (A.loop_mode < 0 && !A.set_ref)
        return;
    last = 0;
    if (lane == 0) {
        __threadfence();
        last = atomicAdd(&A.counters[2], 1) == ninst - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0))
        return;
    __threadfence();
    batch_scalar_finish(A, lane);
}

static_assert(sizeof(MgBatch) <= 32000 && sizeof(CgBatch) <= 32000 &&
                  sizeof(ScalarBatch) <= 32000 && sizeof(TailBatch) <= 32000,
              "batch tables must fit the kernel parameter space");

}  // namespace lbehd

// batch.cuh -- batched launches of the moments and collide kernels: one launch covers the
// blocks of up to BATCH_MAX independent instances of different lattice sizes and
// parameters (lubricant viscosity, wettability, electrode potentials).
//
// The instance table travels in the kernel's parameter space (__grid_constant__, a few KB
// below the 32 KB limit), so every block reads its instance's parameters through the
// constant cache; instance k owns the launch's blocks [start[k], start[k + 1]). The
// per-site arithmetic is the single-instance kernels' own (fields_site, collide_*), so a
// batched step is bitwise the single-instance step of each instance.
#pragma once

#include "kernels.cuh"

namespace lbehd {

constexpr int BATCH_MAX = 64;   // instances per batched launch

// Largest k with start[k] <= b (start ascending, start[0] = 0).
__device__ __forceinline__ int batch_instance(const int *start, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

struct FieldsBatch {
    int n;
    int start[BATCH_MAX + 1];
    Params P[BATCH_MAX];
    FieldPtrs F[BATCH_MAX];
};

// Moments + ghosts over the flattened sites of every instance (BX sites per block, no
// idle threads on rows shorter than a block).
template <int D>
__global__ void __launch_bounds__(BX) k_fields_batch(const __grid_constant__ FieldsBatch A)
{
    const int k = batch_instance(A.start, A.n, blockIdx.x);
    const Params P = A.P[k];      // by value: registers, no local copy of the table entry
    const FieldPtrs F = A.F[k];
    // site offsets fit 32 bits (19 N < 2^31 is checked at init)
    const int i = (blockIdx.x - A.start[k]) * BX + threadIdx.x;
    if (i >= (int)P.N)
        return;
    const int r = i / P.nx;
    fields_site<D>(P, F, i - r * P.nx, r % P.ny, r / P.ny);
}

struct CollideBatch {
    int n, first;
    int start[BATCH_MAX + 1];
    int tiles_x[BATCH_MAX], tiles_y[BATCH_MAX];   // staged: tile counts along x and y
    Params P[BATCH_MAX];
    State S[BATCH_MAX];
    const PopMaps *maps;                          // staged: [n] tensor maps in global memory
};

// The block's instance parameters and state pointers, copied from the parameter table into
// shared memory by the first threads (the caller synchronises before use). The collide body
// reads them many times; from the table, every read is an indexed constant load (measured:
// 89.6 -> 82.4 us per 128x64x64 instance for the staged 64x2 kernel with four instances).
__device__ __forceinline__ void batch_entry_to_smem(const CollideBatch &A, int k, Params &sP,
                                                    State &sS)
{
    static_assert(sizeof(Params) % 4 == 0 && sizeof(State) % 4 == 0, "word copies");
    const int t = threadIdx.x;
    if (t < (int)(sizeof(Params) / 4))
        reinterpret_cast<int *>(&sP)[t] = reinterpret_cast<const int *>(&A.P[k])[t];
    if (t < (int)(sizeof(State) / 4))
        reinterpret_cast<int *>(&sS)[t] = reinterpret_cast<const int *>(&A.S[k])[t];
}

// Global-load collide over the flattened sites of every instance.
template <int D>
__global__ void __launch_bounds__(BX, 4) k_collide_batch(const __grid_constant__ CollideBatch A)
{
    const int k = batch_instance(A.start, A.n, blockIdx.x);
    __shared__ __align__(16) Params sP;
    __shared__ __align__(16) State sS;
    batch_entry_to_smem(A, k, sP, sS);
    __syncthreads();
    const Params &P = sP;
    const int b = blockIdx.x - A.start[k];
    const int i = b * BX + threadIdx.x;
    float ob[NOBS];
#pragma unroll
    for (int m = 0; m < NOBS; m++)
        ob[m] = 0.0f;
    if (i < (int)P.N) {
        const int r = i / P.nx;
        collide_global_site<D>(P, sS, A.first, i - r * P.nx, r % P.ny, r / P.ny, ob);
    }
    block_obs_partials(ob, sS.obs_partials, b, A.start[k + 1] - A.start[k]);
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m)
{
    // the maps were written to global memory by a host copy: order that write before the
    // tensor copies that read them
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(m))
                 : "memory");
}

// Staged collide on TX x TY tiles of every instance.
template <int D, int TY>
__global__ void __launch_bounds__(BX, 4) k_collide_staged_batch(const __grid_constant__ CollideBatch A)
{
    const int k = batch_instance(A.start, A.n, blockIdx.x);
    const int b = blockIdx.x - A.start[k];
    const int tx = A.tiles_x[k], ty = A.tiles_y[k];
    const int bx = b % tx, r = b / tx;
    const PopMaps *m = A.maps + k;
    if (threadIdx.x == 0)   // the only map the staged tile reads
        tensormap_acquire(&m->fphi);
    __shared__ __align__(16) Params sP;
    __shared__ __align__(16) State sS;
    batch_entry_to_smem(A, k, sP, sS);   // collide_staged_tile synchronises before reading them
    collide_staged_tile<D, TY>(sP, sS, A.first, m, bx * Halo<D, TY>::TX, (r % ty) * TY, r / ty,
                               b, A.start[k + 1] - A.start[k]);
}

struct ObsBatch {
    int n;
    const double *partials[BATCH_MAX];
    long long nblocks[BATCH_MAX];
    double *obs[BATCH_MAX];
};

// grid (NOBS, n): block (k, j) sums observable k of instance j.
__global__ void __launch_bounds__(OBS_THREADS) k_obs_final_batch(const __grid_constant__ ObsBatch A)
{
    const int j = blockIdx.y;
    obs_final_block(A.partials[j], A.nblocks[j], A.obs[j], blockIdx.x);
}

static_assert(sizeof(FieldsBatch) <= 32000 && sizeof(CollideBatch) <= 32000 &&
                  sizeof(ObsBatch) <= 32000,
              "batch tables must fit the kernel parameter space");

}  // namespace lbehd

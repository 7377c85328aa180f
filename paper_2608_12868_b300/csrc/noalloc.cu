// noalloc.cu -- droplet phase moments of caller-owned device fields, computed without any
// device allocation.
//
// Some callers cannot let a library allocate device memory: a host program that hands
// out all device memory from its own pre-sized pool (a cudaMalloc behind its back can fail
// or fragment the pool), or a framework that calls foreign kernels from a context where it
// forbids allocation. For them this file offers one reduction whose scratch space (the
// per-block partial sums) is a fixed file-scope __device__ array instead of memory from
// cudaMalloc or a caching allocator. The array is part of the loaded library: every GPU
// that loads it holds these bytes until the process exits.
//
// It is the same reduction that lbehd_observe reports for the droplet (volume, centroid,
// velocity, per-component mass), taken from stored fields (Phi_1..3, u) instead of inside
// the fused collide kernel.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lbehd.h"

namespace lbehd {
void set_global_error(const std::string &msg);   // lbehd.cu: message for lbehd_last_error(NULL)
}

namespace {

constexpr int NM_VALS = 9;         // M1, sum Phi1 x (3), sum Phi1 u (3), sum Phi2, sum Phi3
constexpr int NM_THREADS = 256;
constexpr int NM_MAX_BLOCKS = 2048;
constexpr long long NM_SITES_PER_BLOCK = 8192;   // each block reduces <= 8192 sites

// Scratch: one FP64 partial per value and block (2048 * 9 * 8 B = 144 KB per device).
static __device__ __align__(256) double g_partials[NM_MAX_BLOCKS * NM_VALS];

// Device address of g_partials, looked up once per device and context: a device reset (or a
// new primary context) reloads the module, and the array may then sit at another address,
// so the cached address is kept together with the id of the context it belongs to.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    double *ptr = nullptr;
};
ScratchAddr g_scratch[MAX_DEVICES];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if it cannot be read).
unsigned long long current_context_id()
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

__global__ void __launch_bounds__(NM_THREADS) k_moments_partials(int nx, int ny, long long N,
                                                                 const float *__restrict__ phi,
                                                                 const float *__restrict__ u,
                                                                 const uint8_t *__restrict__ solid,
                                                                 double *__restrict__ partials)
{
    double acc[NM_VALS];
#pragma unroll
    for (int k = 0; k < NM_VALS; k++)
        acc[k] = 0.0;
    const long long begin = (long long)blockIdx.x * NM_SITES_PER_BLOCK;
    const long long end = begin + NM_SITES_PER_BLOCK < N ? begin + NM_SITES_PER_BLOCK : N;
    for (long long i = begin + threadIdx.x; i < end; i += NM_THREADS) {
        if (solid[i])
            continue;
        const float p1 = phi[i];
        const long long x = i % nx, y = (i / nx) % ny, z = i / ((long long)nx * ny);
        acc[0] += p1;
        acc[1] += (double)p1 * (double)x;
        acc[2] += (double)p1 * (double)y;
        acc[3] += (double)p1 * (double)z;
        acc[4] += (double)p1 * u[i];
        acc[5] += (double)p1 * u[N + i];
        acc[6] += (double)p1 * u[2 * N + i];
        acc[7] += phi[N + i];
        acc[8] += phi[2 * N + i];
    }
    __shared__ double sm[NM_VALS][NM_THREADS / 32];
#pragma unroll
    for (int k = 0; k < NM_VALS; k++) {
        double a = acc[k];
        for (int o = 16; o > 0; o >>= 1)
            a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0)
            sm[k][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x < NM_VALS) {
        double a = 0.0;
        for (int w = 0; w < NM_THREADS / 32; w++)
            a += sm[threadIdx.x][w];
        partials[threadIdx.x * NM_MAX_BLOCKS + blockIdx.x] = a;
    }
}

// out: M1, centroid[3], velocity[3], mass[3]
__global__ void __launch_bounds__(32 * NM_VALS) k_moments_final(const double *__restrict__ partials,
                                                                int nblocks, double *__restrict__ out)
{
    __shared__ double tot[NM_VALS];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a = 0.0;
    for (int b = lane; b < nblocks; b += 32)
        a += partials[k * NM_MAX_BLOCKS + b];
    for (int o = 16; o > 0; o >>= 1)
        a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0)
        tot[k] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double M1 = tot[0];
        const double inv = M1 != 0.0 ? 1.0 / M1 : 0.0;
        out[0] = M1;
        for (int d = 0; d < 3; d++) {
            out[1 + d] = tot[1 + d] * inv;
            out[4 + d] = tot[4 + d] * inv;
        }
        out[7] = M1;
        out[8] = tot[7];
        out[9] = tot[8];
    }
}

int fail(int code, const std::string &msg)
{
    lbehd::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int lbehd_phase_moments_noalloc(int dim, int nx, int ny, int nz, const float *phi,
                                           const float *u, const uint8_t *solid, double *out,
                                           void *stream)
{
    if ((dim != 2 && dim != 3) || nx < 1 || ny < 1 || nz < 1 || (dim == 2 && nz != 1))
        return fail(LBEHD_ERR_INVALID_ARG, "lbehd_phase_moments_noalloc: bad lattice extents");
    if (!phi || !u || !solid || !out)
        return fail(LBEHD_ERR_INVALID_ARG, "lbehd_phase_moments_noalloc: null pointer");
    const long long N = (long long)nx * ny * nz;
    const long long nblocks = (N + NM_SITES_PER_BLOCK - 1) / NM_SITES_PER_BLOCK;
    if (nblocks > NM_MAX_BLOCKS)
        return fail(LBEHD_ERR_INVALID_ARG,
                    "lbehd_phase_moments_noalloc: lattice larger than the static scratch allows "
                    "(at most 2048 * 8192 = 16777216 sites)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return fail(LBEHD_ERR_CUDA, "lbehd_phase_moments_noalloc: no usable current device");
    // An error left by the caller's own earlier work is reported as such and left in place
    // (cudaGetLastError below would otherwise clear it and blame this call's launches).
    e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return fail(LBEHD_ERR_CUDA, std::string("lbehd_phase_moments_noalloc: an earlier CUDA "
                                                "error is pending: ") +
                                        cudaGetErrorString(e));
    double *scratch = nullptr;
    {
        // once per device and context, with that device current: the device address of the
        // file-scope scratch array (its name in host code is only a host-side handle)
        const unsigned long long ctx = current_context_id();
        std::lock_guard<std::mutex> lock(g_mu);
        ScratchAddr &a = g_scratch[dev];
        if (!a.ptr || ctx == 0 || a.ctx_id != ctx) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_partials);
            if (e != cudaSuccess || !p)
                return fail(LBEHD_ERR_CUDA, std::string("lbehd_phase_moments_noalloc: "
                                                        "cudaGetSymbolAddress failed: ") +
                                                cudaGetErrorString(e));
            a.ptr = (double *)p;
            a.ctx_id = ctx;
        }
        scratch = a.ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    k_moments_partials<<<(unsigned)nblocks, NM_THREADS, 0, s>>>(nx, ny, N, phi, u, solid, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_moments_final<<<1, 32 * NM_VALS, 0, s>>>(scratch, (int)nblocks, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(LBEHD_ERR_CUDA, std::string("lbehd_phase_moments_noalloc: launch failed: ") +
                                        cudaGetErrorString(e));
    return LBEHD_OK;
}

// lbehd.cu -- host side of the C ABI in include/lbehd.h: configuration checks, geometry
// tables, device state, the per-step launch sequence and the Poisson convergence loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbehd.h"
#include "batch.cuh"
#include "kernels.cuh"
#include "poisson.cuh"
#include "poisson_batch.cuh"
#include "adjoint.cuh"
#include "poisson_persistent.cuh"

namespace lbehd {

static thread_local std::string g_init_error;

void set_global_error(const std::string &msg) { g_init_error = msg; }

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace lbehd

using namespace lbehd;

struct lbehd_handle {
    lbehd_config cfg;              // copy; host array pointers cleared after init
    int dim = 0, nx = 0, ny = 0, nz = 0;
    size_t N = 0;
    int Q = 0, QS = 0;
    Params P{};
    ParamsVD PV{};                 // the variable-density kernels' extra parameters (rho_ph)
    bool var_density = false;      // config density_model 1
    cudaStream_t stream = nullptr;
    cudaStream_t ls = nullptr;     // stream the launch helpers enqueue on (stream, or aux
    cudaStream_t aux = nullptr;    //   while a conditional-node body is being captured)
    cudaStream_t aux2 = nullptr;   // body capture of a conditional node nested in another
    cudaStream_t own_stream = nullptr;  // created when cfg->stream is the legacy stream
    std::vector<DevBuf> bufs;
    // device state
    float *g[2] = {}, *fphi[2] = {}, *frho[2] = {};
    float *phi[2] = {}, *rho[2] = {};
    float *u = nullptr, *q = nullptr, *pot = nullptr, *pot_lo = nullptr, *eps = nullptr;
    double *V = nullptr;           // electrode potentials (device, FP64)
    uint8_t *info = nullptr, *normal = nullptr;
    int16_t *elec = nullptr;
    // obs_partials: [2][NOBS][obs_stride] block partials, one set per step parity; obs:
    // [2 NOBS] the last two steps' sums, then [2 NOBS] a copy kept across an adjoint backward
    double *obs_partials = nullptr, *obs = nullptr;
    size_t obs_stride = 0;
    long long obs_nblk[2] = {0, 0};   // blocks of the partial set of each parity
    int obs_pending = 0;              // steps (at most 2 counted) whose sums are not in obs
    double *obs_wsum = nullptr;    // [NOBS][OBS_THREADS / 32] warp sums of k_obs_final_split
    unsigned *obs_cnt = nullptr;   // [NOBS] arrival counters of k_obs_final_split
    int *flag = nullptr;
    // Poisson: multigrid hierarchy (level 0 = the lattice) and CG vectors on level 0
    struct Level {
        MgDims d;
        size_t n = 0;
        int cz2 = 0;               // coarsening to the next level halves z too
        float *D = nullptr, *kx = nullptr, *ky = nullptr, *kz = nullptr, *x = nullptr, *b = nullptr;
        float *r = nullptr;            // residual scratch of the restriction; the
                                       // block-local smoother's output on the way up
        dim3 grid, grid_half;
        int nbj = 0;                   // blocks of the block-local smoother
    };
    std::vector<Level> mg;
    // inc[s & 1] holds the potential increment of step s; the warm start of step s is formed
    // from the increments of steps s-1 and s-2 (LBEHD_OPT_WARM_START), in place in inc[s & 1]
    // (the charge collision with tau_rho ~ 1/2 makes consecutive increments alternate).
    // delta2: correction of a refinement pass.
    float *inc[2] = {}, *delta2 = nullptr;
    float *eps_mg = nullptr;       // eps the multigrid hierarchy was last built from
    float *cg_r = nullptr, *cg_p = nullptr, *cg_q = nullptr;
    double *cg_partials = nullptr;
    CgScalars *cg_s = nullptr;
    // LBEHD_OPT_WARM_START: 1 starts each forward solve from the combination of the last two
    // increments with the least residual (k_pcg_init_mr), 0 from the increment of step s - 2
    int warm_mode = 1;
    double *mr_alpha = nullptr;    // multi-launch form: (a1, a2, a . c) of the current start
    float *mr_part = nullptr;      // MR_NV x nblocks_site FP32 block sums of k_pcg_init_mr
    CgScalars *h_cg = nullptr;     // pinned copy for the host convergence check
    dim3 grid1d;
    size_t nblocks1d = 0;
    size_t nblocks_site = 0;       // blocks of BX consecutive sites (stencil reductions)
    // CUDA graphs of one step per step parity (LBEHD_POISSON_GRAPH)
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [parity][refresh]
    cudaGraphConditionalHandle cond = 0, cond_ref = 0;
    int use_cond = 0, use_ref = 0;
    int mg_refresh = 16;           // multigrid hierarchy rebuilt every mg_refresh steps
    bool mg_valid = false;
    long long graph_launches = 0, graph_static_kernels[2][2] = {{0, 0}, {0, 0}}, iter_kernels = 0;
    long long graph_iters0 = 0;    // device iteration counter when graphs took over
    bool graph_launches_started = false;
    int collide_variant = 0;       // LBEHD_OPT_COLLIDE: 0 auto, 1 global loads, 2-4 staged
    bool batch_owned = false;      // instance of an lbehd_batch (stepped and freed by it)
    bool maps_ok = false;          // tensor maps of both population buffers encoded
    PopMaps maps[3][2];            // [tile shape][buffer]; shapes TY = 4, 2, 8
    dim3 grid_tile[3];             // TX x TY tiles of the staged collide kernel
    size_t nblocks_tile[3] = {0, 0, 0};
    int mg_nu = 2, mg_coarse = 8;
    int mg_smoother = 1;           // LBEHD_OPT_MG_SMOOTHER: 1 block-local, 0 whole-level sweeps
    int bj_nu = 3;                 // sweep pairs per block of the block-local smoother
    bool bj_ok = false;            // this lattice allows it (a tail level; see mg build)
    int tail_level = -1;           // first level handled by k_mg_tail (-1: none)
    TailLevels tail{};
    size_t tail_smem = 0;
    // persistent Gauss-law solve (k_poisson_solve): one cooperative launch per solve
    bool ps_ok = false;            // this lattice allows it (see ps_setup)
    bool ps_on = true;             // LBEHD_OPT_POISSON_KERNEL
    int ps_grid = 0;               // CTAs: one per SM
    PsArgs ps{};                   // arguments but the per-launch ones
    PsBarrier *ps_bar = nullptr;
    double *ps_part = nullptr;
    unsigned *h_ps_err = nullptr;  // pinned copy of ps_bar->error
    unsigned ps_spin_limit = PS_SPIN_LIMIT;
    int ps_extra = 0;              // LBEHD_OPT_BARRIER_TEST
    float mg_scale = 0.6f;
    int cur = 0;                   // population buffer holding the state at time n
    int pcur = 0;                  // phi / rho buffer holding the last step's fields
    bool first = true;
    long long step = 0;
    long long launches = 0;
    int last_iters = 0;
    double last_resid = 0.0;
    int status = LBEHD_OK;
    std::string err;
    dim3 grid, block;
    size_t nblocks = 0;
    // profiling: event pairs recorded around launches, per kernel class
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[LBEHD_NKC];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    // discrete adjoint (lbehd_adjoint_forward / lbehd_adjoint_backward)
    struct HostState {
        long long step;
        int cur, pcur;
        bool first, mg_valid;
    };
    struct Adj {
        int S = 0, E = 0, seg = 0, T = 0, K = 0;   // segments, electrodes, steps per segment,
                                                   // steps, checkpoint spacing
        std::vector<double> V;                      // [S][E] schedule of the recorded run
        std::vector<float *> ckpt, slot;            // states at 0, K, 2K, ...; one interval
        std::vector<HostState> ckpt_host;
        float *fin = nullptr;                       // state after the last step
        HostState fin_host{};
        bool have = false;                          // a forward run is recorded
        double xc = 0.0, M1 = 0.0;                  // loss (x centroid) and droplet volume
        float *lg[2] = {}, *lf[2] = {}, *lr[2] = {}, *lp[2] = {};
        float *rec = nullptr, *loc = nullptr, *phibar = nullptr, *potbar = nullptr, *jb = nullptr;
        float *mu = nullptr, *rhs = nullptr, *seed = nullptr;
        float *ptraj = nullptr;                     // [T][2][N] potential (hi, lo) of each step
        size_t ptraj_cap = 0;                       //   (null: replays re-solve Gauss's law)
        bool use_traj = true;
        int mg_age = 0;                             // reversed steps since the multigrid rebuild
        float *mu3[3] = {};                         // adjoint potentials, rotating by step
        cudaGraphExec_t solve[3] = {};              // adjoint Gauss-law solve into mu3[k]
        double *grad = nullptr;
        size_t grad_cap = 0;
        long long steps_replayed = 0, adj_steps = 0, adj_iters = 0;   // last backward pass
        size_t bytes = 0;                                              // device memory held
        long long fwd_iters = 0;                    // CG iterations of the recorded run
        int dev_seg = -1;                           // segment whose potentials are on the device
    } adj;
};

namespace {

int fail(lbehd_handle *h, int code, const std::string &msg)
{
    if (h)
        h->err = msg;
    else
        g_init_error = msg;
    return code;
}

int cuda_fail(lbehd_handle *h, cudaError_t e, const char *what)
{
    return fail(h, LBEHD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess)                        \
            return cuda_fail((h), e_, #call);         \
    } while (0)

void *dev_alloc(lbehd_handle *h, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0)
        bytes = 16;
    if (h->cfg.alloc) {
        p = h->cfg.alloc(bytes, h->cfg.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p)
        h->bufs.push_back({p, bytes});
    return p;
}

void dev_free(lbehd_handle *h, void *p)
{
    for (size_t k = 0; k < h->bufs.size(); k++)
        if (h->bufs[k].ptr == p) {
            if (h->cfg.free)
                h->cfg.free(p, h->cfg.alloc_ctx);
            else
                cudaFree(p);
            h->bufs.erase(h->bufs.begin() + (long)k);
            return;
        }
}

// Lattice normal of a boundary solid node: the fluid neighbour direction maximising
// e_k . v / |e_k| with v = sum_n w_n e_n [fluid neighbour n]; integer weights (x36),
// ties to the lowest index. 0 when the node has no fluid neighbour.
template <int D>
void build_normals(const lbehd_handle *h, const uint8_t *solid, std::vector<uint8_t> &normal)
{
    using L = Lat<D>;
    const int nx = h->nx, ny = h->ny, nz = h->nz;
    normal.assign(h->N, 0);
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                const size_t i = x + (size_t)nx * (y + (size_t)ny * z);
                if (!solid[i])
                    continue;
                long v[3] = {0, 0, 0};
                bool fl[L::Q] = {};
                bool any = false;
                for (int n = 1; n < L::Q; n++) {
                    const int X = (x + L::ex(n) + nx) % nx, Y = (y + L::ey(n) + ny) % ny,
                              Z = (z + L::ez(n) + nz) % nz;
                    fl[n] = solid[X + (size_t)nx * (Y + (size_t)ny * Z)] == 0;
                    if (fl[n]) {
                        const long iw = std::lround(36.0 * L::w(n));
                        v[0] += iw * L::ex(n);
                        v[1] += iw * L::ey(n);
                        v[2] += iw * L::ez(n);
                        any = true;
                    }
                }
                if (!any)
                    continue;
                int best = 0;
                long bdot = 0, blen2 = 1;
                for (int n = 1; n < L::Q; n++) {
                    if (!fl[n])
                        continue;
                    const long dot = L::ex(n) * v[0] + L::ey(n) * v[1] + L::ez(n) * v[2];
                    const long len2 = L::ex(n) * L::ex(n) + L::ey(n) * L::ey(n) + L::ez(n) * L::ez(n);
                    // dot/sqrt(len2) > bdot/sqrt(blen2), compared through signed squares
                    const long a = dot * std::labs(dot) * blen2, b = bdot * std::labs(bdot) * len2;
                    if (best == 0 || a > b) {
                        best = n;
                        bdot = dot;
                        blen2 = len2;
                    }
                }
                normal[i] = (uint8_t)best;
            }
}

// Launch through here: counts launches and, while profiling, brackets them with events.
template <class F>
void launch(lbehd_handle *h, int kc, int nlaunch, F &&fn)
{
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (h->prof) {
        if (!h->ev_pool.empty()) {
            ev = h->ev_pool.back();
            h->ev_pool.pop_back();
        } else if (cudaEventCreate(&ev.first) != cudaSuccess ||
                   cudaEventCreate(&ev.second) != cudaSuccess) {
            ev = {nullptr, nullptr};
        }
        if (ev.first)
            cudaEventRecord(ev.first, h->ls);
    }
    fn();
    h->launches += nlaunch;
    if (ev.first) {
        cudaEventRecord(ev.second, h->ls);
        h->ev_pending[kc].push_back(ev);
    }
}

FieldPtrs field_ptrs(const lbehd_handle *h, int cur, int pcur)
{
    return FieldPtrs{h->fphi[cur], h->frho[cur], h->phi[pcur], h->rho[pcur], h->eps, h->pot,
                     h->pot_lo, h->info, h->normal, h->elec, h->V};
}

template <int D>
int launch_fields(lbehd_handle *h)
{
    const FieldPtrs F = field_ptrs(h, h->cur, h->pcur);
    launch(h, LBEHD_KC_FIELDS, 1, [&] { k_fields<D><<<h->grid, h->block, 0, h->ls>>>(h->P, F); });
    return LBEHD_OK;
}

// The persistent solve needs the shared-memory tail below at least one level smoothed by grid
// phases, an even nx on those levels, cooperative launches and one resident 1024-thread CTA
// (with the tail's shared memory) per SM; otherwise the multi-launch form runs.
template <int D>
int ps_setup(lbehd_handle *h)
{
    int coop = 0, dev = 0, nsm = 0;
    CK(h, cudaGetDevice(&dev));
    CK(h, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CK(h, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    bool ok = coop != 0 && h->tail_level >= 1 && h->tail_level < PS_MAX_LEVELS &&
              h->N < (size_t)1 << 30;
    for (int l = 0; ok && l < h->tail_level; l++)
        ok = h->mg[l].d.nx % 2 == 0;
    if (!ok)
        return LBEHD_OK;
    CK(h, cudaFuncSetAttribute(k_poisson_solve<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)TAIL_SMEM_MAX));
    int per_sm = 0;
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_poisson_solve<D>, PS_THREADS,
                                                        h->tail_smem));
    if (per_sm < 1)
        return LBEHD_OK;
    const size_t pn = 2 * std::max(h->nblocks_site, h->nblocks1d);
    h->ps_part = (double *)dev_alloc(h, 2 * pn * sizeof(double));
    h->ps_bar = (PsBarrier *)dev_alloc(h, sizeof(PsBarrier));
    h->ps.wsum = (double *)dev_alloc(h, 2 * 32 * sizeof(double));
    h->ps.p2 = (float *)dev_alloc(h, h->N * sizeof(float));
    if (!h->ps_part || !h->ps_bar || !h->ps.wsum || !h->ps.p2)
        return fail(h, LBEHD_ERR_OOM, "device allocation failed (persistent Poisson)");
    CK(h, cudaMemsetAsync(h->ps_bar, 0, sizeof(PsBarrier), h->stream));
    CK(h, cudaMallocHost(&h->h_ps_err, sizeof(unsigned)));
    *h->h_ps_err = 0;
    PsArgs &A = h->ps;
    A.nl = h->tail_level;
    A.nu = h->mg_nu;
    A.N = (int)h->N;
    A.nbs = (int)h->nblocks_site;
    A.nb1 = (int)h->nblocks1d;
    for (int l = 0; l <= h->tail_level; l++) {
        const auto &L = h->mg[l];
        A.L[l] = PsLevel{L.d, L.cz2, (int)L.n, L.D, L.kx, L.ky, L.kz, L.b, L.x, L.nbj, L.r};
    }
    A.tail = h->tail;
    A.tail.b0 = h->mg[h->tail_level].b;
    A.tail.x0 = h->mg[h->tail_level].x;
    A.pot = h->pot;
    A.pot_lo = h->pot_lo;
    A.eps = h->eps;
    A.info = h->info;
    A.delta2 = h->delta2;
    A.r = h->cg_r;
    A.p = h->cg_p;
    A.q = h->cg_q;
    A.part[0] = h->ps_part;
    A.part[1] = h->ps_part + pn;
    A.s = h->cg_s;
    A.bar = h->ps_bar;
    h->ps_grid = nsm;
    h->ps_ok = true;
    return LBEHD_OK;
}

bool ps_use(const lbehd_handle *h) { return h->ps_ok && h->ps_on; }

bool mr_use(const lbehd_handle *h) { return h->warm_mode == 1; }

// The other increment buffer: d1 (the last step's increment) when x holds d2.
const float *mr_other(const lbehd_handle *h, const float *x)
{
    return x == h->inc[0] ? h->inc[1] : h->inc[0];
}

bool bj_use(const lbehd_handle *h) { return h->bj_ok && h->mg_smoother == 1; }

// One persistent solve on h->ls: the forward step's (increment x, this step's charge rho) or
// the adjoint's (solution x, right-hand side rhs), after the launch that forms its start.
template <int D>
int ps_launch(lbehd_handle *h, int mode, float *x, const float *rho, const float *rhs)
{
    PsArgs A = h->ps;
    A.spin_limit = h->ps_spin_limit;
    A.extra = h->ps_extra;
    A.bj = bj_use(h) ? 1 : 0;
    A.nu_bj = h->bj_nu;
    A.mode = mode;
    A.x = x;
    A.rho = rho;
    A.rhs = rhs;
    // The start r = b - A (phi + x) (forward) or rhs - A x (adjoint) as an ordinary launch:
    // at full occupancy it runs near bandwidth, where the persistent kernel's 1024-thread
    // CTAs take it in four latency-bound rounds. Same per-site body and block partition as
    // the kernel's own start phase. It also resets the barrier counter.
    const auto &L0 = h->mg[0];
    A.mr = mode == PS_FORWARD && mr_use(h) ? 1 : 0;
    if (A.mr) {
        // minimal-residual start: r0, q1 = A d1 (into q), q2 = A d2 (into p: the first
        // iteration does not read the old direction) and the block sums; the kernel sums the
        // coefficients and forms x0 (and r, if it iterates)
        A.mr_part = h->mr_part;
        A.mr_d1 = mr_other(h, x);
        A.mr_q1 = h->cg_q;
        A.mr_q2 = h->cg_p;
        k_pcg_init_mr<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(
            L0.d, A.pot, A.pot_lo, A.mr_d1, x, A.eps, rho, A.info, L0.D, A.r, h->cg_q, h->cg_p,
            A.part[1], h->mr_part, &h->ps_bar->count);
    } else if (mode == PS_FORWARD)
        k_pcg_init<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(
            L0.d, A.pot, A.pot_lo, x, A.eps, rho, A.info, L0.D, A.r, A.part[1], &h->ps_bar->count);
    else
        k_adj_pcg_init<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(
            L0.d, A.eps, A.info, L0.D, x, rhs, A.r, A.part[1], &h->ps_bar->count);
    h->launches += 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)h->ps_grid);
    cfg.blockDim = dim3(PS_THREADS);
    cfg.dynamicSmemBytes = h->tail_smem;
    cfg.stream = h->ls;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(h, cudaLaunchKernelEx(&cfg, k_poisson_solve<D>, A));
    h->launches += 1;
    return LBEHD_OK;
}

void mg_gs(lbehd_handle *h, const lbehd_handle::Level &L, int color)
{
    k_mg_gs<<<L.grid_half, h->block, 0, h->ls>>>(L.d, L.D, L.kx, L.ky, L.kz, L.b, L.x, color);
}

// One symmetric V-cycle: x_l ~= A_l^-1 b_l, starting from x_l = 0. Levels from
// h->tail_level down run in one shared-memory kernel.
void vcycle(lbehd_handle *h, size_t l)
{
    const auto &L = h->mg[l];
    if ((int)l == h->tail_level) {
        TailLevels T = h->tail;
        T.b0 = L.b;
        T.x0 = L.x;
        k_mg_tail<<<1, TAIL_THREADS, h->tail_smem, h->ls>>>(T);
        return;
    }
    cudaMemsetAsync(L.x, 0, L.n * sizeof(float), h->ls);
    if (l + 1 == h->mg.size()) {
        for (int s = 0; s < h->mg_coarse; s++) {
            mg_gs(h, L, 0);
            mg_gs(h, L, 1);
            mg_gs(h, L, 1);
            mg_gs(h, L, 0);
        }
        return;
    }
    for (int s = 0; s < h->mg_nu; s++) {
        mg_gs(h, L, 0);
        mg_gs(h, L, 1);
    }
    const auto &C = h->mg[l + 1];
    k_mg_resid<<<L.grid, h->block, 0, h->ls>>>(L.d, L.D, L.kx, L.ky, L.kz, L.b, L.x, L.r);
    k_mg_restrict_sum<<<C.grid, h->block, 0, h->ls>>>(L.d, C.d, L.cz2, L.r, C.b);
    vcycle(h, l + 1);
    k_mg_prolong<<<L.grid, h->block, 0, h->ls>>>(L.d, C.d, L.cz2, L.D, C.x, L.x);
    for (int s = 0; s < h->mg_nu; s++) {
        mg_gs(h, L, 1);
        mg_gs(h, L, 0);
    }
}

// The same V-cycle with the block-local smoother (mg_bj_block): on the way down one smoothing
// launch from zero per level, then the residual and the restriction; on the way up one
// launch of prolongation + smoothing per level into the level's r array; level 0's also
// writes the r . z partials (one per block) into the CG partials. z ends in mg[0].r.
template <int D>
void vcycle_bj(lbehd_handle *h, size_t l)
{
    const auto &L = h->mg[l];
    if ((int)l == h->tail_level) {
        TailLevels T = h->tail;
        T.b0 = L.b;
        T.x0 = L.x;
        k_mg_tail<<<1, TAIL_THREADS, h->tail_smem, h->ls>>>(T);
        return;
    }
    const auto &C = h->mg[l + 1];
    k_mg_bj<D><<<L.nbj, BJ_THREADS, 0, h->ls>>>(L.d, L.D, L.kx, L.ky, L.kz, L.b, nullptr, L.x,
                                                h->bj_nu, 0, L.d, 0, nullptr, nullptr, nullptr);
    k_mg_resid<<<L.grid, h->block, 0, h->ls>>>(L.d, L.D, L.kx, L.ky, L.kz, L.b, L.x, L.r);
    k_mg_restrict_sum<<<C.grid, h->block, 0, h->ls>>>(L.d, C.d, L.cz2, L.r, C.b);
    vcycle_bj<D>(h, l + 1);
    const float *xc = (int)l + 1 == h->tail_level ? C.x : C.r;
    k_mg_bj<D><<<L.nbj, BJ_THREADS, 0, h->ls>>>(L.d, L.D, L.kx, L.ky, L.kz, L.b, L.x, L.r,
                                                h->bj_nu, 1, C.d, L.cz2, xc,
                                                l == 0 ? h->cg_r : nullptr,
                                                l == 0 ? h->cg_partials : nullptr);
}

int vcycle_launches(const lbehd_handle *h)
{
    if (bj_use(h))
        return 4 * h->tail_level + 1;
    const int levels = (int)h->mg.size();
    if (h->tail_level >= 0)
        return h->tail_level * (4 * h->mg_nu + 3) + 1;   // memsets not counted
    return (levels - 1) * (4 * h->mg_nu + 3) + 4 * h->mg_coarse;
}

void cg_scalar(lbehd_handle *h, int nv, int op, size_t nblk, const double *mr = nullptr)
{
    k_pcg_scalar<<<1, SCALAR_THREADS, 0, h->ls>>>(h->cg_partials, (long long)nblk, nv, op, h->cg_s,
                                                   h->cond, h->use_cond, h->cond_ref, h->use_ref,
                                                   mr);
}

// One preconditioned CG iteration on level 0 (z = V-cycle(r) lives in mg[0].x), updating
// the increment x.
template <int D>
void pcg_iteration(lbehd_handle *h, float *x)
{
    auto &L0 = h->mg[0];
    const bool bj = bj_use(h);
    launch(h, LBEHD_KC_MG, vcycle_launches(h), [&] {
        if (bj)
            vcycle_bj<D>(h, 0);
        else
            vcycle(h, 0);
    });
    launch(h, LBEHD_KC_CG, bj ? 7 : 8, [&] {
        if (!bj)
            k_pcg_dot<<<h->grid1d, h->block, 0, h->ls>>>(h->N, h->cg_r, L0.x, h->cg_partials);
        cg_scalar(h, 1, 1, bj ? (size_t)L0.nbj : h->nblocks1d);
        k_pcg_p<<<h->grid1d, h->block, 0, h->ls>>>(h->N, bj ? L0.r : L0.x, h->cg_p, h->cg_s);
        k_pcg_Ap<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(L0.d, h->eps, h->info, L0.D,
                                                                       h->cg_p, h->cg_q,
                                                                       h->cg_partials);
        cg_scalar(h, 1, 2, h->nblocks_site);
        k_pcg_update<<<h->grid1d, h->block, 0, h->ls>>>(h->N, h->cg_p, h->cg_q, x, h->cg_r,
                                                             h->cg_s, h->cg_partials);
        cg_scalar(h, 1, 3, h->nblocks1d);
    });
}

int read_cg(lbehd_handle *h)
{
    CK(h, cudaMemcpyAsync(h->h_cg, h->cg_s, sizeof(CgScalars), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

// r = b - A (phi + x) in FP64 and the CG start (op 0: first pass of a step, 4: refinement).
// The first pass of a step with the minimal-residual start (x holds d2, the other increment
// buffer d1) replaces x by x0 = a1 d1 + a2 d2 and forms r = b - A (phi + x0) from r0, q1, q2.
template <int D>
void pcg_start(lbehd_handle *h, float *x, int op = 0)
{
    auto &L0 = h->mg[0];
    if (op == 0 && mr_use(h)) {
        // the persistent kernel's order: coefficients, x0 and r (here always formed: the same
        // x0 as the persistent solve forms in its update when the start meets the tolerance),
        // then the test of the least residual
        launch(h, LBEHD_KC_CG, 4, [&] {
            const float *d1 = mr_other(h, x);
            k_pcg_init_mr<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(
                L0.d, h->pot, h->pot_lo, d1, x, h->eps, h->rho[h->pcur], h->info, L0.D,
                h->cg_r, h->cg_q, h->cg_p, h->cg_partials, h->mr_part);
            k_mr_alpha<<<1, SCALAR_THREADS, 0, h->ls>>>(h->mr_part, (int)h->nblocks_site,
                                                         h->mr_alpha);
            k_pcg_start_mr<<<h->grid1d, h->block, 0, h->ls>>>((int)h->N, h->mr_alpha, d1, x,
                                                              h->cg_r, h->cg_q, h->cg_p);
            cg_scalar(h, 2, op, h->nblocks_site, h->mr_alpha);
        });
        return;
    }
    launch(h, LBEHD_KC_CG, 2, [&] {
        k_pcg_init<D><<<(unsigned)h->nblocks_site, h->block, 0, h->ls>>>(
            L0.d, h->pot, h->pot_lo, x, h->eps, h->rho[h->pcur], h->info, L0.D, h->cg_r,
            h->cg_partials);
        cg_scalar(h, 2, op, h->nblocks_site);
    });
}

// phi += x (compensated); acc += x when acc is given.
void pcg_apply(lbehd_handle *h, const float *x, float *acc)
{
    launch(h, LBEHD_KC_CG, 1, [&] {
        k_pcg_apply<<<h->grid1d, h->block, 0, h->ls>>>(h->N, h->mg[0].D, x, acc, h->pot,
                                                            h->pot_lo);
    });
}

// Run CG iterations on x until the device flag says done (host reads it back).
template <int D>
int pcg_host_loop(lbehd_handle *h, float *x)
{
    int rc = read_cg(h);
    if (rc)
        return rc;
    const int every = std::max(h->cfg.poisson_check_every, 1);
    while (!h->h_cg->done) {
        for (int k = 0; k < every; k++)
            pcg_iteration<D>(h, x);
        rc = read_cg(h);
        if (rc)
            return rc;
    }
    return LBEHD_OK;
}

// Gauss law (Eq. 13) for this step: operator set-up; FP64 defect of the warm start;
// preconditioned CG on the increment; phi += increment. In LBEHD_POISSON_HOST mode the
// true FP64 residual is then re-checked and, if the FP32 iteration stopped short of the
// tolerance (a large increment, e.g. the first solve from phi = 0), up to three
// refinement passes solve for a further correction.
template <int D>
void mg_setup(lbehd_handle *h)
{
    auto &L0 = h->mg[0];
    launch(h, LBEHD_KC_MG, (int)h->mg.size(), [&] {
        k_mg_setup0<D><<<h->grid, h->block, 0, h->ls>>>(L0.d, h->eps, h->info, L0.D, L0.kx,
                                                             L0.ky, L0.kz);
        for (size_t l = 0; l + 1 < h->mg.size(); l++) {
            const auto &F = h->mg[l];
            const auto &C = h->mg[l + 1];
            k_mg_coarsen<<<C.grid, h->block, 0, h->ls>>>(F.d, C.d, F.cz2, h->mg_scale, F.D,
                                                             F.kx, F.ky, F.kz, C.D, C.kx, C.ky,
                                                             C.kz);
        }
    });
    // the eps of this build (saved with a state, so that a restore rebuilds this hierarchy)
    cudaMemcpyAsync(h->eps_mg, h->eps, h->N * sizeof(float), cudaMemcpyDeviceToDevice, h->ls);
    h->mg_valid = true;
}

// The multigrid hierarchy only preconditions (the CG operator is formed from eps each step),
// so it is rebuilt every mg_refresh steps; eps moves with the slowly moving interfaces.
bool mg_due(const lbehd_handle *h) { return !h->mg_valid || h->step % h->mg_refresh == 0; }

template <int D>
int poisson(lbehd_handle *h)
{
    const lbehd_config &c = h->cfg;
    if (mg_due(h))
        mg_setup<D>(h);
    if (c.poisson_mode == LBEHD_POISSON_GRAPH && !h->first && ps_use(h)) {
        // eager form of a graph step (profiling): the same persistent solve
        int rc = LBEHD_OK;
        launch(h, LBEHD_KC_CG, 0, [&] {
            rc = ps_launch<D>(h, PS_FORWARD, h->inc[h->step & 1], h->rho[h->pcur], nullptr);
        });
        return rc;
    }
    float *x = h->inc[h->step & 1];   // holds the increment of step - 2: the warm start
    pcg_start<D>(h, x);
    bool converged = true;
    if (c.poisson_mode == LBEHD_POISSON_FIXED) {
        for (int k = 0; k < c.poisson_fixed_iters; k++)
            pcg_iteration<D>(h, x);
        pcg_apply(h, x, nullptr);
        h->last_iters = c.poisson_fixed_iters;
        h->last_resid = -1.0;
        return LBEHD_OK;
    }
    int rc = pcg_host_loop<D>(h, x);
    if (rc)
        return rc;
    int iters = h->h_cg->iters;
    pcg_apply(h, x, nullptr);
    // refinement: only after a pass of two or more iterations (with none, the start residual
    // was the true residual and already within the tolerance; after one, the recursive
    // residual still is, to FP32 rounding of one update far below it)
    for (int pass = 0; pass < 3 && (pass > 0 || h->h_cg->refine) && h->h_cg->iters > 0;
         pass++) {
        CK(h, cudaMemsetAsync(h->delta2, 0, h->N * sizeof(float), h->ls));
        pcg_start<D>(h, h->delta2, 4);   // true residual of the updated potential
        rc = pcg_host_loop<D>(h, h->delta2);
        if (rc)
            return rc;
        if (h->h_cg->iters == 0)
            break;
        iters += h->h_cg->iters;
        pcg_apply(h, h->delta2, x);
    }
    converged = h->h_cg->converged != 0;
    h->last_iters = iters;
    h->last_resid = h->h_cg->bb > 0.0 ? std::sqrt(h->h_cg->rr / h->h_cg->bb) : 0.0;
    if (!converged) {
        h->status = h->status ? h->status : LBEHD_ERR_POISSON_NOCONV;
        return LBEHD_ERR_POISSON_NOCONV;
    }
    return LBEHD_OK;
}

// Block partials of the observables written by the collide kernel of a step of parity `cur`.
double *obs_buf(const lbehd_handle *h, int cur)
{
    return h->obs_partials + (size_t)cur * NOBS * h->obs_stride;
}

State collide_state(const lbehd_handle *h, int cur, int pcur)
{
    State S;
    S.g = h->g[cur];
    S.fphi = h->fphi[cur];
    S.frho = h->frho[cur];
    S.g_out = h->g[cur ^ 1];
    S.fphi_out = h->fphi[cur ^ 1];
    S.frho_out = h->frho[cur ^ 1];
    S.phi = h->phi[pcur];
    S.phi_prev = h->phi[pcur ^ 1];
    S.rho = h->rho[pcur];
    S.rho_prev = h->rho[pcur ^ 1];
    S.u = h->u;
    S.q = h->q;
    S.pot = h->pot;
    S.pot_lo = h->pot_lo;
    S.info = h->info;
    S.obs_partials = obs_buf(h, cur);
    S.flag = h->flag;
    return S;
}

// Collide variant actually run: 0 (automatic) resolves to the 32x4 staged kernel when the
// tensor maps exist, else to the global-load kernel.
int resolved_variant(const lbehd_handle *h)
{
    const int v = h->collide_variant;
    if (v == 1 || !h->maps_ok)
        return 1;
    if (h->var_density)   // the variable-density scheme has the 32x4 staged kernel only
        return 2;
    return v == 0 ? 2 : v;
}

// tile shape index of a staged variant: 2 -> TY 4, 3 -> TY 2, 4 -> TY 8
int tile_shape(int v) { return v == 3 ? 1 : (v == 4 ? 2 : 0); }

// Blocks of the collide launch in effect (one observable partial per block).
long long collide_launch_blocks(const lbehd_handle *h)
{
    const int v = resolved_variant(h);
    return v == 1 ? (long long)h->nblocks : (long long)h->nblocks_tile[tile_shape(v)];
}

// The fused collide + stream kernel of one step. Its block partials of the observables stay
// in the partial set of the step's parity; obs_finalize sums them when they are read.
template <int D>
void collide(lbehd_handle *h)
{
    const State S = collide_state(h, h->cur, h->pcur);
    // variants: 1 global loads, 2/3/4 staged tiles with TY = 4 / 2 / 8
    const int v = resolved_variant(h);
    const int shape = tile_shape(v);
    const bool staged = v != 1;
    const int first = h->first ? 1 : 0;
    launch(h, LBEHD_KC_COLLIDE, 1, [&] {
        if (h->var_density) {
            ParamsVD PV = h->PV;
            static_cast<Params &>(PV) = h->P;
            if (!staged)
                k_collide<D, true><<<h->grid, h->block, 0, h->ls>>>(PV, S, first);
            else
                k_collide_staged<D, 4, true>
                    <<<h->grid_tile[0], h->block, staged_smem_bytes<D, 4>(), h->ls>>>(
                        PV, S, first, h->maps[0][h->cur]);
        } else if (!staged)
            k_collide<D><<<h->grid, h->block, 0, h->ls>>>(h->P, S, first);
        else if (shape == 0)
            k_collide_staged<D, 4><<<h->grid_tile[0], h->block, staged_smem_bytes<D, 4>(), h->ls>>>(
                h->P, S, first, h->maps[0][h->cur]);
        else if (shape == 1)
            k_collide_staged<D, 2><<<h->grid_tile[1], h->block, staged_smem_bytes<D, 2>(), h->ls>>>(
                h->P, S, first, h->maps[1][h->cur]);
        else
            k_collide_staged<D, 8><<<h->grid_tile[2], h->block, staged_smem_bytes<D, 8>(), h->ls>>>(
                h->P, S, first, h->maps[2][h->cur]);
    });
}

// A step of parity h->cur has left its observable partials (called before cur flips).
void obs_note_step(lbehd_handle *h)
{
    h->obs_nblk[h->cur] = collide_launch_blocks(h);
    h->obs_pending = std::min(h->obs_pending + 1, 2);
}

// Sum the partials of the steps not yet reduced into obs: [0, NOBS) the last step's sums,
// [NOBS, 2 NOBS) the step's before. Each reduction is the fixed-order k_obs_final_split,
// which moves the previous sums up before writing the new ones, so the sums are the same
// bits as a reduction after every step.
int obs_finalize(lbehd_handle *h)
{
    if (!h->obs_pending)
        return LBEHD_OK;
    const int last = h->cur ^ 1;
    h->ls = h->stream;
    for (int k = h->obs_pending; k >= 1; k--) {
        const int par = k == 2 ? last ^ 1 : last;
        launch(h, LBEHD_KC_OBS, 1, [&] {
            k_obs_final_split<<<NOBS * (OBS_THREADS / 32), 32, 0, h->ls>>>(
                obs_buf(h, par), h->obs_nblk[par], h->obs_wsum, h->obs_cnt, h->obs);
        });
    }
    h->obs_pending = 0;
    CK(h, cudaGetLastError());
    return LBEHD_OK;
}

// Append a conditional node (while or if, on handle `cond`) to the ongoing capture of
// stream `cap`; its body is captured from `body` on stream `bs`.
template <class F>
int add_cond(lbehd_handle *h, cudaStream_t cap, cudaStream_t bs, cudaGraphConditionalHandle cond,
             cudaGraphConditionalNodeType type, F &&body)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(h, cudaStreamGetCaptureInfo(cap, &st, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(h, cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
    cudaGraph_t bodyg = np.conditional.phGraph_out[0];
    CK(h, cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed));
    const cudaStream_t prev = h->ls;
    h->ls = bs;
    const int rc = body();
    h->ls = prev;
    cudaGraph_t out = nullptr;
    CK(h, cudaStreamEndCapture(bs, &out));
    if (rc)
        return rc;
    CK(h, cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1,
                                              cudaStreamSetCaptureDependencies));
    return LBEHD_OK;
}

// Enqueue one coupled step on h->stream, which must be capturing into `g` (the
// conditional handles are created in `g`): moments, Poisson (multigrid rebuild when
// `refresh`, device-side CG loop, then, if that loop iterated, one refinement check with
// its own loop), collide + stream. Buffers are those of a step with the given parity.
// With full == false only the Poisson part is recorded (the batched step launches the
// moments and collide kernels of all instances itself).
template <int D>
int record_step(lbehd_handle *h, cudaGraph_t g, int parity, int refresh, bool full = true)
{
    const int cur = h->cur, pcur = h->pcur;
    const long long step = h->step, launches = h->launches;
    const bool prof = h->prof;
    h->cur = h->pcur = parity;
    h->step = parity;
    h->prof = false;
    cudaGraphConditionalHandle c1 = 0, c2 = 0, cr = 0;
    auto body = [&]() -> int {
        h->ls = h->stream;
        if (ps_use(h)) {   // one persistent solve: no conditional nodes
            if (full)
                launch_fields<D>(h);
            if (refresh)
                mg_setup<D>(h);
            const int r = ps_launch<D>(h, PS_FORWARD, h->inc[parity], h->rho[h->pcur], nullptr);
            if (r)
                return r;
            h->iter_kernels = 0;
            if (full)
                collide<D>(h);
            return LBEHD_OK;
        }
        CK(h, cudaGraphConditionalHandleCreate(&c1, g, 0, 0));
        CK(h, cudaGraphConditionalHandleCreate(&c2, g, 0, 0));
        CK(h, cudaGraphConditionalHandleCreate(&cr, g, 0, 0));
        h->use_cond = 1;
        if (full)
            launch_fields<D>(h);
        if (refresh)
            mg_setup<D>(h);
        float *x = h->inc[parity];
        h->cond = c1;
        h->cond_ref = cr;
        h->use_ref = 1;
        pcg_start<D>(h, x, 0);
        int r = add_cond(h, h->stream, h->aux, c1, cudaGraphCondTypeWhile, [&]() -> int {
            const long long k0 = h->launches;
            pcg_iteration<D>(h, x);
            h->iter_kernels = h->launches - k0;
            h->launches = k0;
            return LBEHD_OK;
        });
        h->use_ref = 0;
        if (r)
            return r;
        pcg_apply(h, x, nullptr);
        r = add_cond(h, h->stream, h->aux, cr, cudaGraphCondTypeIf, [&]() -> int {
            const long long k0 = h->launches;
            cudaMemsetAsync(h->delta2, 0, h->N * sizeof(float), h->ls);
            h->cond = c2;
            pcg_start<D>(h, h->delta2, 4);
            const int r2 = add_cond(h, h->aux, h->aux2, c2, cudaGraphCondTypeWhile, [&]() -> int {
                const long long k1 = h->launches;
                pcg_iteration<D>(h, h->delta2);
                h->launches = k1;
                return LBEHD_OK;
            });
            pcg_apply(h, h->delta2, x);
            h->launches = k0;   // the refinement block rarely runs: not counted as static
            return r2;
        });
        if (r)
            return r;
        if (full)
            collide<D>(h);
        return LBEHD_OK;
    };
    const int rc = body();
    h->graph_static_kernels[parity][refresh] = h->launches - launches;
    h->use_cond = 0;
    h->use_ref = 0;
    h->cond = h->cond_ref = 0;
    h->ls = h->stream;
    h->cur = cur;
    h->pcur = pcur;
    h->step = step;
    h->launches = launches;
    h->prof = prof;
    return rc;
}

void abort_capture(cudaStream_t sx)
{
    cudaStreamCaptureStatus st;
    if (sx && cudaStreamIsCapturing(sx, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(sx, &junk);
        if (junk)
            cudaGraphDestroy(junk);
    }
}

// One whole coupled step as a CUDA graph for the given step parity (see record_step).
template <int D>
int capture_step(lbehd_handle *h, int parity, int refresh)
{
    cudaGraph_t g = nullptr;
    int rc = LBEHD_OK;
    if (cudaGraphCreate(&g, 0) != cudaSuccess)
        return fail(h, LBEHD_ERR_CUDA, "cudaGraphCreate failed");
    if (cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
        rc = fail(h, LBEHD_ERR_CUDA, "cudaStreamBeginCaptureToGraph failed");
    if (!rc)
        rc = record_step<D>(h, g, parity, refresh);
    if (!rc) {
        cudaGraph_t out = nullptr;
        if (cudaStreamEndCapture(h->stream, &out) != cudaSuccess ||
            cudaGraphInstantiate(&h->gexec[parity][refresh], g, 0) != cudaSuccess)
            rc = fail(h, LBEHD_ERR_CUDA, "step graph capture failed");
    }
    if (rc) {
        for (cudaStream_t sx : {h->aux2, h->aux, h->stream})
            abort_capture(sx);
        cudaGetLastError();
    }
    cudaGraphDestroy(g);
    return rc;
}

template <int D>
int do_step(lbehd_handle *h)
{
    // graph replay (profiling brackets eager launches with events, so it runs eagerly)
    if (h->cfg.poisson_mode == LBEHD_POISSON_GRAPH && !h->first && !h->prof) {
        const int parity = (int)(h->step & 1), refresh = mg_due(h) ? 1 : 0;
        if (!h->gexec[parity][refresh]) {
            const int rc = capture_step<D>(h, parity, refresh);
            if (rc)
                return rc;
        }
        if (!h->graph_launches && !h->graph_launches_started) {
            h->graph_launches_started = true;
            CgScalars s0;
            CK(h, cudaMemcpyAsync(&s0, h->cg_s, sizeof(s0), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            h->graph_iters0 = s0.total_iters;
        }
        CK(h, cudaGraphLaunch(h->gexec[parity][refresh], h->stream));
        h->graph_launches++;
        h->launches += h->graph_static_kernels[parity][refresh];
        obs_note_step(h);
        h->cur ^= 1;
        h->pcur ^= 1;
        h->step++;
        return LBEHD_OK;
    }
    int rc = launch_fields<D>(h);
    if (rc)
        return rc;
    const int prc = poisson<D>(h);
    if (prc && prc != LBEHD_ERR_POISSON_NOCONV)
        return prc;
    collide<D>(h);
    CK(h, cudaGetLastError());
    obs_note_step(h);
    h->cur ^= 1;
    h->pcur ^= 1;
    h->first = false;
    h->step++;
    return prc;
}

int set_params(lbehd_handle *h)
{
    const lbehd_config &c = h->cfg;
    Params &P = h->P;
    P.nx = h->nx;
    P.ny = h->ny;
    P.nz = h->nz;
    P.N = (long long)h->N;
    for (int k = 0; k < 3; k++) {
        P.nu[k] = (float)c.nu[k];
        P.eps[k] = (float)c.eps[k];
        P.sig[k] = (float)c.sigma[k];
        P.body[k] = (float)c.body_force[k];
        P.body1[k] = (float)c.body_force_droplet[k];
    }
    // Eq. 11
    const double Y1 = c.gamma12 + c.gamma13 - c.gamma23;
    const double Y2 = c.gamma12 + c.gamma23 - c.gamma13;
    const double Y3 = c.gamma13 + c.gamma23 - c.gamma12;
    if (Y1 == 0.0 || Y2 == 0.0 || Y3 == 0.0)
        return fail(h, LBEHD_ERR_INVALID_ARG, "surface tensions give a zero Upsilon (Eq. 11)");
    P.Y[0] = (float)Y1;
    P.Y[1] = (float)Y2;
    P.Y[2] = (float)Y3;
    P.YT = (float)(3.0 / (1.0 / Y1 + 1.0 / Y2 + 1.0 / Y3));
    const double d2r = 3.14159265358979323846 / 180.0;
    P.cos12 = (float)std::cos(c.theta12 * d2r);
    P.cos13 = (float)std::cos(c.theta13 * d2r);
    P.cos23 = (float)std::cos(c.theta23 * d2r);
    P.W = (float)c.W;
    const double cs2 = 1.0 / 3.0, cs2s = h->dim == 3 ? 0.25 : 1.0 / 3.0;
    P.inv_tau_phi = (float)(1.0 / (0.5 + c.mobility / cs2));
    P.inv_tau_rho = (float)(1.0 / (0.5 + c.alpha / cs2s));
    P.s_bulk = (float)c.s_bulk;
    if (c.density_model != 0 && c.density_model != 1)
        return fail(h, LBEHD_ERR_INVALID_ARG, "density_model takes 0 or 1");
    h->var_density = c.density_model == 1;
    for (int k = 0; k < 3; k++) {
        if (c.density_model == 1 && !(c.rho_phase[k] > 0.0))
            return fail(h, LBEHD_ERR_INVALID_ARG, "rho_phase must be > 0 with density_model 1");
        h->PV.rho_ph[k] = (float)c.rho_phase[k];
    }
    h->mg_nu = c.mg_nu > 0 ? c.mg_nu : 2;
    h->bj_nu = c.mg_nu > 0 ? c.mg_nu : 3;
    h->mg_coarse = c.mg_coarse_sweeps > 0 ? c.mg_coarse_sweeps : 8;
    h->mg_scale = c.mg_scale > 0.0 ? (float)c.mg_scale : 0.6f;
    return LBEHD_OK;
}

// Tensor maps (x, y, z, array) of the population sets of both buffers, box TX x TY x 1 x
// (all arrays), for the staged collide kernel. cuTensorMapEncodeTiled comes from the driver
// through the runtime's entry-point query (no link-time dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int encode_pop_maps(lbehd_handle *h)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return fail(h, LBEHD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    EncodeTiledFn encode = (EncodeTiledFn)fn;
    const cuuint64_t N = h->N;
    auto one = [&](CUtensorMap *m, float *base, int narr, int ty) -> bool {
        const cuuint64_t dims[4] = {(cuuint64_t)h->nx, (cuuint64_t)h->ny, (cuuint64_t)h->nz,
                                    (cuuint64_t)narr};
        const cuuint64_t strides[3] = {(cuuint64_t)h->nx * 4, (cuuint64_t)h->nx * h->ny * 4, N * 4};
        const cuuint32_t box[4] = {(cuuint32_t)(BX / ty), (cuuint32_t)ty, 1u, (cuuint32_t)narr};
        const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    const int tys[3] = {4, 2, 8};
    for (int k = 0; k < 3; k++)
        for (int b = 0; b < 2; b++)
            if (!one(&h->maps[k][b].g, h->g[b], h->Q, tys[k]) ||
                !one(&h->maps[k][b].fphi, h->fphi[b], 3 * h->Q, tys[k]) ||
                !one(&h->maps[k][b].frho, h->frho[b], h->QS, tys[k]))
                return fail(h, LBEHD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    h->maps_ok = true;
    return LBEHD_OK;
}

template <int D>
int init_impl(lbehd_handle *h)
{
    const lbehd_config &c = h->cfg;
    const size_t N = h->N;
    h->Q = Lat<D>::Q;
    h->QS = Lat<D>::QS;
    // geometry tables
    std::vector<uint8_t> info(N), normal;
    std::vector<int16_t> elec(N, -1);
    for (size_t i = 0; i < N; i++) {
        const uint8_t s = c.solid[i];
        if (s > 2)
            return fail(h, LBEHD_ERR_INVALID_ARG, "solid class must be 0, 1 or 2");
        const int id = c.electrode_id ? c.electrode_id[i] : -1;
        if (id < -2 || id >= c.n_electrodes)
            return fail(h, LBEHD_ERR_INVALID_ARG, "electrode id out of range");
        uint8_t pt = PT_FLUID;
        if (s)
            pt = (id >= 0 || id == -2) ? PT_DIRICHLET : PT_NEUMANN;
        info[i] = (uint8_t)(pt | (s << 2));
        elec[i] = (int16_t)(s ? id : -1);
    }
    build_normals<D>(h, c.solid, normal);
    if (D == 3 && h->nz % 2) {
        const size_t plane = (size_t)h->nx * h->ny;
        for (size_t k = 0; k < plane; k++)
            if (!c.solid[k] && !c.solid[(h->nz - 1) * plane + k])
                return fail(h, LBEHD_ERR_INVALID_ARG,
                            "odd nz needs a solid bottom or top layer (red-black colouring)");
    }
    // device buffers
    const size_t fb = sizeof(float);
    for (int b = 0; b < 2; b++) {
        h->g[b] = (float *)dev_alloc(h, h->Q * N * fb);
        h->fphi[b] = (float *)dev_alloc(h, 3 * h->Q * N * fb);
        h->frho[b] = (float *)dev_alloc(h, h->QS * N * fb);
        h->phi[b] = (float *)dev_alloc(h, 3 * N * fb);
        h->rho[b] = (float *)dev_alloc(h, N * fb);
        if (!h->g[b] || !h->fphi[b] || !h->frho[b] || !h->phi[b] || !h->rho[b])
            return fail(h, LBEHD_ERR_OOM, "device allocation failed (populations)");
    }
    h->u = (float *)dev_alloc(h, 3 * N * fb);
    h->q = (float *)dev_alloc(h, N * fb);
    h->pot = (float *)dev_alloc(h, N * fb);
    h->pot_lo = (float *)dev_alloc(h, N * fb);
    h->eps = (float *)dev_alloc(h, N * fb);
    h->V = (double *)dev_alloc(h, LBEHD_MAX_ELECTRODES * sizeof(double));
    h->info = (uint8_t *)dev_alloc(h, N);
    h->normal = (uint8_t *)dev_alloc(h, N);
    h->elec = (int16_t *)dev_alloc(h, N * sizeof(int16_t));
    h->block = dim3(BX, 1, 1);
    h->grid = dim3((h->nx + BX - 1) / BX, h->ny, h->nz);
    h->nblocks = (size_t)h->grid.x * h->grid.y * h->grid.z;
    size_t nblk_max = h->nblocks;
    {
        const int tys[3] = {4, 2, 8};
        for (int k = 0; k < 3; k++) {
            const int tx = BX / tys[k];
            h->grid_tile[k] = dim3((h->nx + tx - 1) / tx, (h->ny + tys[k] - 1) / tys[k], h->nz);
            h->nblocks_tile[k] = (size_t)h->grid_tile[k].x * h->grid_tile[k].y * h->grid_tile[k].z;
            nblk_max = std::max(nblk_max, h->nblocks_tile[k]);
        }
    }
    h->obs_stride = nblk_max;
    h->obs_partials = (double *)dev_alloc(h, 2 * NOBS * nblk_max * sizeof(double));
    h->obs = (double *)dev_alloc(h, 4 * NOBS * sizeof(double));
    h->obs_wsum = (double *)dev_alloc(h, NOBS * (OBS_THREADS / 32) * sizeof(double));
    h->obs_cnt = (unsigned *)dev_alloc(h, NOBS * sizeof(unsigned));
    h->flag = (int *)dev_alloc(h, sizeof(int));
    if (!h->u || !h->q || !h->pot || !h->pot_lo || !h->eps || !h->V || !h->info || !h->normal || !h->elec ||
        !h->obs_partials || !h->obs || !h->flag || !h->obs_wsum || !h->obs_cnt)
        return fail(h, LBEHD_ERR_OOM, "device allocation failed (fields)");
    CK(h, cudaMemsetAsync(h->obs_cnt, 0, NOBS * sizeof(unsigned), h->stream));
    // Poisson: CG vectors, reductions, multigrid hierarchy
    {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const size_t want = (N + BX - 1) / BX, cap = (size_t)nsm * 8;
        h->grid1d = dim3((unsigned)std::min(want, cap), 1, 1);
    }
    h->nblocks1d = h->grid1d.x;
    h->nblocks_site = (N + BX - 1) / BX;
    h->inc[0] = (float *)dev_alloc(h, N * fb);
    h->inc[1] = (float *)dev_alloc(h, N * fb);
    h->eps_mg = (float *)dev_alloc(h, N * fb);
    if (!h->eps_mg)
        return fail(h, LBEHD_ERR_OOM, "device allocation failed (multigrid eps)");
    h->delta2 = (float *)dev_alloc(h, N * fb);
    h->cg_r = (float *)dev_alloc(h, N * fb);
    h->cg_p = (float *)dev_alloc(h, N * fb);
    h->cg_q = (float *)dev_alloc(h, N * fb);
    h->cg_partials = (double *)dev_alloc(h, 2 * std::max(h->nblocks, h->nblocks1d) * sizeof(double));
    h->cg_s = (CgScalars *)dev_alloc(h, sizeof(CgScalars));
    h->mr_alpha = (double *)dev_alloc(h, 3 * sizeof(double));
    h->mr_part = (float *)dev_alloc(h, MR_NV * h->nblocks_site * sizeof(float));
    if (!h->inc[0] || !h->inc[1] || !h->delta2 || !h->cg_r || !h->cg_p || !h->cg_q ||
        !h->cg_partials || !h->cg_s || !h->mr_alpha || !h->mr_part)
        return fail(h, LBEHD_ERR_OOM, "device allocation failed (Poisson)");
    {
        MgDims d = mg_dims(h->nx, h->ny, h->nz);
        const int maxl = c.mg_max_levels > 0 ? c.mg_max_levels : 16;
        while ((int)h->mg.size() < maxl) {
            lbehd_handle::Level L;
            L.d = d;
            L.n = (size_t)d.nx * d.ny * d.nz;
            L.grid = dim3((d.nx + BX - 1) / BX, d.ny, d.nz);
            L.grid_half = dim3((d.nx / 2 + 1 + BX - 1) / BX, d.ny, d.nz);
            L.D = (float *)dev_alloc(h, L.n * fb);
            L.kx = (float *)dev_alloc(h, L.n * fb);
            L.ky = (float *)dev_alloc(h, L.n * fb);
            L.kz = (float *)dev_alloc(h, L.n * fb);
            L.x = (float *)dev_alloc(h, L.n * fb);
            L.b = h->mg.empty() ? h->cg_r : (float *)dev_alloc(h, L.n * fb);
            L.r = (float *)dev_alloc(h, L.n * fb);
            if (!L.D || !L.kx || !L.ky || !L.kz || !L.x || !L.b || !L.r)
                return fail(h, LBEHD_ERR_OOM, "device allocation failed (multigrid)");
            // keep x and y even on every level (red-black colouring across the periodic wrap)
            const bool more = d.nx % 4 == 0 && d.ny % 4 == 0 && (h->dim == 2 || d.nz >= 4);
            L.cz2 = (more && h->dim == 3) ? 1 : 0;
            h->mg.push_back(L);
            if (!more)
                break;
            d = mg_dims(d.nx / 2, d.ny / 2, h->dim == 3 ? (d.nz + 1) / 2 : 1);
        }
        h->mg.back().cz2 = 0;
        // shared-memory tail: from the first level with <= 1024 cells; when no level is that
        // small, the coarsest level alone if it has <= TAIL_MAX_TOTAL cells (one CTA then
        // replaces its many sweep launches)
        int tail_from = -1;
        for (size_t l = 0; l < h->mg.size() && tail_from < 0; l++)
            if (h->mg[l].n <= 1024 && h->mg.size() - l <= (size_t)TAIL_MAX_LEVELS)
                tail_from = (int)l;
        if (tail_from < 0 && h->mg.back().n <= (size_t)TAIL_MAX_TOTAL)
            tail_from = (int)h->mg.size() - 1;
        for (size_t l = 0; l < h->mg.size(); l++) {
            const size_t nl = h->mg.size() - l;
            if ((int)l == tail_from) {
                TailLevels &T = h->tail;
                T.nl = (int)nl;
                T.nu = h->mg_nu;
                T.coarse = h->mg_coarse;
                int off = 0;
                for (size_t k = 0; k < nl; k++) {
                    const auto &L = h->mg[l + k];
                    T.d[k] = L.d;
                    T.cz2[k] = L.cz2;
                    T.off[k] = off;
                    T.D[k] = L.D;
                    T.kx[k] = L.kx;
                    T.ky[k] = L.ky;
                    T.kz[k] = L.kz;
                    off += (int)L.n;
                }
                T.total = off;
                h->tail_smem = 6 * (size_t)off * sizeof(float);
                h->tail_level = (int)l;
                // the attribute belongs to the kernel, not the handle: set it to the largest
                // tail any handle can have
                CK(h, cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)TAIL_SMEM_MAX));
                break;
            }
        }
        // the block-local smoother runs on the levels above a tail, and level 0's r . z
        // partials (one per block) must fit the CG partial array
        for (auto &L : h->mg)
            L.nbj = bj_blocks<D>(L.d);
        h->bj_ok = h->tail_level > 0 &&
                   (size_t)h->mg[0].nbj <= std::max(h->nblocks, h->nblocks1d);
    }
    CK(h, cudaMallocHost(&h->h_cg, sizeof(CgScalars)));
    {
        int rc = ps_setup<D>(h);
        if (rc)
            return rc;
    }
    CK(h, cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    CK(h, cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking));
    if (h->nx % 4 == 0) {
        int rc = encode_pop_maps(h);
        if (rc)
            return rc;
        CK(h, cudaFuncSetAttribute(k_collide_staged<D, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)staged_smem_bytes<D, 4>()));
        CK(h, cudaFuncSetAttribute(k_collide_staged<D, 4, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)staged_smem_bytes<D, 4>()));
        CK(h, cudaFuncSetAttribute(k_collide_staged<D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)staged_smem_bytes<D, 2>()));
        CK(h, cudaFuncSetAttribute(k_collide_staged<D, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)staged_smem_bytes<D, 8>()));
    }
    {
        CgScalars s0{};
        s0.tol2 = c.poisson_tol * c.poisson_tol;
        s0.max_iter = c.poisson_max_iter;
        CK(h, cudaMemcpyAsync(h->cg_s, &s0, sizeof(s0), cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        CK(h, cudaMemsetAsync(h->inc[0], 0, N * fb, h->stream));
        CK(h, cudaMemsetAsync(h->inc[1], 0, N * fb, h->stream));
        CK(h, cudaMemsetAsync(h->cg_p, 0, N * fb, h->stream));
    }
    std::vector<float> phi0(3 * N);
    std::vector<double> V(LBEHD_MAX_ELECTRODES, 0.0);
    for (size_t k = 0; k < 3 * N; k++)
        phi0[k] = (float)c.phi_init[k];
    for (int k = 0; k < c.n_electrodes; k++)
        V[k] = c.electrode_V[k];
    cudaStream_t s = h->stream;
    CK(h, cudaMemcpyAsync(h->info, info.data(), N, cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->normal, normal.data(), N, cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->elec, elec.data(), N * sizeof(int16_t), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->phi[1], phi0.data(), 3 * N * fb, cudaMemcpyHostToDevice, s));
    for (int b = 0; b < 2; b++) {
        CK(h, cudaMemsetAsync(h->g[b], 0, h->Q * N * fb, s));
        CK(h, cudaMemsetAsync(h->fphi[b], 0, 3 * h->Q * N * fb, s));
        CK(h, cudaMemsetAsync(h->frho[b], 0, h->QS * N * fb, s));
        CK(h, cudaMemsetAsync(h->rho[b], 0, N * fb, s));
    }
    CK(h, cudaMemsetAsync(h->phi[0], 0, 3 * N * fb, s));
    CK(h, cudaMemsetAsync(h->u, 0, 3 * N * fb, s));
    CK(h, cudaMemsetAsync(h->q, 0, N * fb, s));
    CK(h, cudaMemsetAsync(h->pot, 0, N * fb, s));
    CK(h, cudaMemsetAsync(h->pot_lo, 0, N * fb, s));
    CK(h, cudaMemsetAsync(h->eps, 0, N * fb, s));
    CK(h, cudaMemsetAsync(h->obs, 0, 4 * NOBS * sizeof(double), s));
    CK(h, cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    k_init<D><<<h->grid, h->block, 0, s>>>(h->P, h->phi[1], h->g[0], h->fphi[0], h->frho[0], h->info);
    h->launches++;
    CK(h, cudaGetLastError());
    // host staging vectors die here: wait for the copies
    CK(h, cudaStreamSynchronize(s));
    h->cur = 0;
    h->pcur = 0;
    return LBEHD_OK;
}

void drop_events(lbehd_handle *h)
{
    for (auto &v : h->ev_pending) {
        for (auto &e : v)
            h->ev_pool.push_back(e);
        v.clear();
    }
}

void release(lbehd_handle *h)
{
    if (!h)
        return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    drop_events(h);
    for (auto &e : h->ev_pool) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    h->ev_pool.clear();
    for (auto &b : h->bufs) {
        if (h->cfg.free)
            h->cfg.free(b.ptr, h->cfg.alloc_ctx);
        else
            cudaFree(b.ptr);
    }
    h->bufs.clear();
    if (h->h_cg)
        cudaFreeHost(h->h_cg);
    if (h->h_ps_err)
        cudaFreeHost(h->h_ps_err);
    h->h_ps_err = nullptr;
    h->h_cg = nullptr;
    for (auto &row : h->gexec)
        for (auto &e : row)
            if (e)
                cudaGraphExecDestroy(e);
    for (auto &e : h->adj.solve)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    if (h->aux)
        cudaStreamDestroy(h->aux);
    h->aux = nullptr;
    if (h->aux2)
        cudaStreamDestroy(h->aux2);
    h->aux2 = nullptr;
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    h->own_stream = nullptr;
}


// ------------------------------------------------------------ collide autotuner

// Time every collide kernel the instance can run on its current state (see lbehd_autotune)
// and keep the fastest. The timed launches write the other population buffer and the
// observable partials (both overwritten first by the next step) and u, q and the error
// flag, which are saved in the CG work vectors (dead between steps) and restored.
template <int D>
int autotune_impl(lbehd_handle *h, int reps, double *ms_out)
{
    reps = std::max(1, std::min(reps, 1000));
    const size_t N = h->N, fb = sizeof(float);
    if (int rc0 = obs_finalize(h))   // the timed launches overwrite the partial sets
        return rc0;
    CK(h, cudaStreamSynchronize(h->stream));
    float *save[4] = {h->cg_r, h->cg_p, h->cg_q, h->delta2};
    for (int c = 0; c < 3; c++)
        CK(h, cudaMemcpyAsync(save[c], h->u + c * N, N * fb, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(save[3], h->q, N * fb, cudaMemcpyDeviceToDevice, h->stream));
    int flag0 = 0;
    CK(h, cudaMemcpyAsync(&flag0, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    const int v0 = h->collide_variant;
    const bool prof = h->prof, first = h->first;
    h->prof = false;
    h->first = false;
    h->ls = h->stream;
    int best = 1;
    float best_ms = 0.0f;
    int rc = LBEHD_OK;
    for (int v = 1; v <= 4 && !rc; v++) {
        double ms = -1.0;
        if (v == 1 || h->maps_ok) {
            h->collide_variant = v;
            collide<D>(h);
            collide<D>(h);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps; r++)
                collide<D>(h);
            cudaEventRecord(e1, h->stream);
            float t = 0.0f;
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&t, e0, e1);
            if (e != cudaSuccess) {
                rc = cuda_fail(h, e, "autotune timing");
                break;
            }
            t /= (float)reps;
            ms = t;
            if (v == 1 || t < best_ms) {
                best = v;
                best_ms = t;
            }
        }
        if (ms_out)
            ms_out[v - 1] = ms;
    }
    h->prof = prof;
    h->first = first;
    h->collide_variant = rc ? v0 : best;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int c = 0; c < 3; c++)
        CK(h, cudaMemcpyAsync(h->u + c * N, save[c], N * fb, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->q, save[3], N * fb, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->flag, &flag0, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    for (auto &row : h->gexec)   // captured graphs hold the previous choice
        for (auto &e : row)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    return rc ? rc : best;
}

int set_option_impl(lbehd_handle *h, int option, long long value)
{
    if (option == LBEHD_OPT_COLLIDE) {
        if (value < 0 || value > 4)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_COLLIDE takes 0 to 4");
        if (value >= 2 && !h->maps_ok)
            return fail(h, LBEHD_ERR_INVALID_ARG, "the staged collide kernel needs nx % 4 == 0");
        CK(h, cudaStreamSynchronize(h->stream));
        h->collide_variant = (int)value;
    } else if (option == LBEHD_OPT_MG_REFRESH) {
        if (value < 1 || value > (1 << 20))
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_MG_REFRESH must be >= 1");
        CK(h, cudaStreamSynchronize(h->stream));
        h->mg_refresh = (int)value;
        h->mg_valid = false;
    } else if (option == LBEHD_OPT_POISSON_KERNEL) {
        if (value < 0 || value > 1)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_POISSON_KERNEL takes 0 or 1");
        CK(h, cudaStreamSynchronize(h->stream));
        h->ps_on = value != 0;
        for (auto &e : h->adj.solve)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    } else if (option == LBEHD_OPT_WARM_START) {
        if (value < 0 || value > 1)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_WARM_START takes 0 or 1");
        CK(h, cudaStreamSynchronize(h->stream));
        h->warm_mode = (int)value;
    } else if (option == LBEHD_OPT_MG_SMOOTHER) {
        if (value < 0 || value > 1)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_MG_SMOOTHER takes 0 or 1");
        CK(h, cudaStreamSynchronize(h->stream));
        h->mg_smoother = (int)value;
        for (auto &e : h->adj.solve)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    } else if (option == LBEHD_OPT_BARRIER_TEST) {
        if (value < 0 || value > (long long)PS_SPIN_LIMIT)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_BARRIER_TEST takes 0 to 2^24");
        CK(h, cudaStreamSynchronize(h->stream));
        h->ps_extra = value > 0 ? 1 : 0;
        h->ps_spin_limit = value > 0 ? (unsigned)value : PS_SPIN_LIMIT;
        for (auto &e : h->adj.solve)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    } else if (option == LBEHD_OPT_ADJ_TRAJECTORY) {
        if (value < 0 || value > 1)
            return fail(h, LBEHD_ERR_INVALID_ARG, "LBEHD_OPT_ADJ_TRAJECTORY takes 0 or 1");
        CK(h, cudaStreamSynchronize(h->stream));
        h->adj.use_traj = value != 0;
        if (!h->adj.use_traj && h->adj.ptraj) {   // a recorded run needs its trajectory
            dev_free(h, h->adj.ptraj);
            h->adj.bytes -= h->adj.ptraj_cap * sizeof(float);
            h->adj.ptraj = nullptr;
            h->adj.ptraj_cap = 0;
            h->adj.have = false;
        }
        return LBEHD_OK;
    } else {
        return fail(h, LBEHD_ERR_INVALID_ARG, "unknown option");
    }
    for (auto &row : h->gexec)   // captured graphs hold the previous choice
        for (auto &e : row)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    return LBEHD_OK;
}

// Observables: enqueue the copies (o[2 NOBS], flag, CG scalars into h->h_cg), then, after
// the stream is synchronised, fill *out.
int observe_enqueue(lbehd_handle *h, double *o, int *flag)
{
    if (int rc = obs_finalize(h))
        return rc;
    CK(h, cudaMemcpyAsync(o, h->obs, 2 * NOBS * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(h->h_cg, h->cg_s, sizeof(CgScalars), cudaMemcpyDeviceToHost, h->stream));
    if (h->ps_bar)
        CK(h, cudaMemcpyAsync(h->h_ps_err, &h->ps_bar->error, sizeof(unsigned),
                              cudaMemcpyDeviceToHost, h->stream));
    return LBEHD_OK;
}

int observe_fill(lbehd_handle *h, const double *o, int flag, lbehd_obs *out)
{
    std::memset(out, 0, sizeof(*out));
    out->step = h->step - 1;
    const double M1 = o[0], M1p = o[NOBS];
    out->M1 = M1;
    for (int a = 0; a < 3; a++) {
        out->centroid[a] = M1 != 0.0 ? o[1 + a] / M1 : 0.0;
        out->velocity[a] = M1 != 0.0 ? o[4 + a] / M1 : 0.0;
        out->f_ele[a] = o[7 + a];
        out->f_ele_total[a] = o[10 + a];
        const double Vp = M1p != 0.0 ? o[NOBS + 4 + a] / M1p : 0.0;
        const double drive = h->cfg.body_force[a] + h->cfg.body_force_droplet[a];
        out->f_drag[a] =
            h->step >= 2 ? o[7 + a] + M1 * drive - M1 * (out->velocity[a] - Vp) : 0.0;
    }
    out->mass[0] = M1;
    out->mass[1] = o[13];
    out->mass[2] = o[14];
    out->charge = o[15];
    out->poisson_iters = h->h_cg->step_iters;
    out->poisson_resid = h->h_cg->bb > 0.0 ? std::sqrt(h->h_cg->rr / h->h_cg->bb) : 0.0;
    out->status = flag ? LBEHD_ERR_NONFINITE
                       : (h->status ? h->status : (h->h_cg->nonconv ? LBEHD_ERR_POISSON_NOCONV : 0));
    if (h->h_ps_err && *h->h_ps_err) {   // the root cause when both are set
        out->status = LBEHD_ERR_CUDA;
        return fail(h, LBEHD_ERR_CUDA, "persistent Poisson solve: a grid barrier timed out");
    }
    if (flag)
        return fail(h, LBEHD_ERR_NONFINITE, "non-finite value in the state");
    return LBEHD_OK;
}

// ------------------------------------------------------------ discrete adjoint

// Floats per site of a saved state: populations, Phi^{n-1}, rho^{n-1}, u^{n-1}, Q^{n-1},
// then the potential (hi, lo), both warm-start increments and the multigrid's eps.
size_t adj_state_floats(const lbehd_handle *h) { return (size_t)(4 * h->Q + h->QS + 13); }

struct StateView {
    float *g, *fphi, *frho, *phi_prev, *rho_prev, *u, *q, *pot, *pot_lo, *inc0, *inc1, *eps_mg;
};

StateView state_view(const lbehd_handle *h, float *base)
{
    const size_t N = h->N;
    StateView v;
    v.g = base;
    v.fphi = v.g + h->Q * N;
    v.frho = v.fphi + 3 * h->Q * N;
    v.phi_prev = v.frho + h->QS * N;
    v.rho_prev = v.phi_prev + 3 * N;
    v.u = v.rho_prev + N;
    v.q = v.u + 3 * N;
    v.pot = v.q + N;
    v.pot_lo = v.pot + N;
    v.inc0 = v.pot_lo + N;
    v.inc1 = v.inc0 + N;
    v.eps_mg = v.inc1 + N;
    return v;
}

// Copy the handle's state into / out of a saved state (device to device, on the stream).
// The device-side count of CG iterations so far (synchronises).
int cg_total_iters(lbehd_handle *h, long long *v)
{
    CgScalars s0;
    CK(h, cudaMemcpyAsync(&s0, h->cg_s, sizeof(s0), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *v = s0.total_iters;
    return LBEHD_OK;
}

// Device allocation held by the adjoint (counted in adj.bytes).
float *adj_alloc_floats(lbehd_handle *h, size_t n)
{
    float *p = (float *)dev_alloc(h, n * sizeof(float));
    if (p)
        h->adj.bytes += n * sizeof(float);
    return p;
}

int adj_save(lbehd_handle *h, float *dst, bool with_potential = true)
{
    const size_t N = h->N, fb = sizeof(float);
    const StateView v = state_view(h, dst);
    auto cp = [&](float *d, const float *s, size_t n) {
        return cudaMemcpyAsync(d, s, n * fb, cudaMemcpyDeviceToDevice, h->stream);
    };
    CK(h, cp(v.g, h->g[h->cur], h->Q * N));
    CK(h, cp(v.fphi, h->fphi[h->cur], 3 * h->Q * N));
    CK(h, cp(v.frho, h->frho[h->cur], h->QS * N));
    CK(h, cp(v.phi_prev, h->phi[h->pcur ^ 1], 3 * N));
    CK(h, cp(v.rho_prev, h->rho[h->pcur ^ 1], N));
    CK(h, cp(v.u, h->u, 3 * N));
    CK(h, cp(v.q, h->q, N));
    if (!with_potential)
        return LBEHD_OK;
    CK(h, cp(v.pot, h->pot, N));
    CK(h, cp(v.pot_lo, h->pot_lo, N));
    CK(h, cp(v.inc0, h->inc[0], N));
    CK(h, cp(v.inc1, h->inc[1], N));
    CK(h, cp(v.eps_mg, h->eps_mg, N));
    return LBEHD_OK;
}

lbehd_handle::HostState host_state(const lbehd_handle *h)
{
    return lbehd_handle::HostState{h->step, h->cur, h->pcur, h->first, h->mg_valid};
}

// Restore a saved state (with its potential). The multigrid hierarchy is rebuilt from the
// saved eps of its last build, so the next steps repeat the saved run's iterates exactly.
template <int D>
int adj_restore(lbehd_handle *h, const float *src, const lbehd_handle::HostState &hs)
{
    h->step = hs.step;
    h->cur = hs.cur;
    h->pcur = hs.pcur;
    h->first = hs.first;
    h->mg_valid = false;
    const size_t N = h->N, fb = sizeof(float);
    const StateView v = state_view(h, const_cast<float *>(src));
    auto cp = [&](float *d, const float *s, size_t n) {
        return cudaMemcpyAsync(d, s, n * fb, cudaMemcpyDeviceToDevice, h->stream);
    };
    CK(h, cp(h->g[h->cur], v.g, h->Q * N));
    CK(h, cp(h->fphi[h->cur], v.fphi, 3 * h->Q * N));
    CK(h, cp(h->frho[h->cur], v.frho, h->QS * N));
    CK(h, cp(h->phi[h->pcur ^ 1], v.phi_prev, 3 * N));
    CK(h, cp(h->rho[h->pcur ^ 1], v.rho_prev, N));
    CK(h, cp(h->u, v.u, 3 * N));
    CK(h, cp(h->q, v.q, N));
    CK(h, cp(h->pot, v.pot, N));
    CK(h, cp(h->pot_lo, v.pot_lo, N));
    CK(h, cp(h->inc[0], v.inc0, N));
    CK(h, cp(h->inc[1], v.inc1, N));
    if (hs.mg_valid) {   // eps is formed again by the next step's moments kernel
        CK(h, cp(h->eps, v.eps_mg, N));
        h->ls = h->stream;
        mg_setup<D>(h);
        CK(h, cudaGetLastError());
    }
    return LBEHD_OK;
}

// Electrode potentials of step t on the device (copied only when the segment changes).
int adj_set_V(lbehd_handle *h, int t)
{
    auto &a = h->adj;
    if (a.E == 0 || t / a.seg == a.dev_seg)
        return LBEHD_OK;
    a.dev_seg = t / a.seg;
    const double *v = a.V.data() + (size_t)(t / a.seg) * a.E;
    CK(h, cudaMemcpyAsync(h->V, v, a.E * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    return LBEHD_OK;
}

template <int D>
int adjoint_forward(lbehd_handle *h, const double *V, int S, int seg, double *loss)
{
    auto &a = h->adj;
    const size_t N = h->N, fb = sizeof(float), SS = adj_state_floats(h);
    a.S = S;
    a.seg = seg;
    a.E = h->cfg.n_electrodes;
    a.T = S * seg;
    // checkpoints every K steps: K ~ sqrt(T), a multiple of the 16-step multigrid refresh
    a.K = std::max(16, (int)std::ceil(std::sqrt((double)a.T) / 16.0) * 16);
    const int nck = (a.T + a.K - 1) / a.K;
    a.V.assign(V, V + (size_t)S * a.E);
    while ((int)a.ckpt.size() < nck) {
        float *p = adj_alloc_floats(h, SS * N);
        if (!p)
            return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint checkpoints)");
        a.ckpt.push_back(p);
    }
    a.ckpt_host.assign(nck, lbehd_handle::HostState{});
    a.dev_seg = -1;
    if (!a.fin && !(a.fin = adj_alloc_floats(h, SS * N)))
        return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint final state)");
    // the potential of every step (8 N bytes a step), so that replays need no Gauss-law solve;
    // without room for it the replays solve again (same iterates, same bits)
    const size_t ptraj_need = (size_t)a.T * 2 * N;
    if (a.use_traj && a.ptraj_cap < ptraj_need) {
        if (a.ptraj) {
            dev_free(h, a.ptraj);
            a.bytes -= a.ptraj_cap * fb;
        }
        a.ptraj = adj_alloc_floats(h, ptraj_need);
        a.ptraj_cap = a.ptraj ? ptraj_need : 0;
    }
    int worst = LBEHD_OK;
    long long it0 = 0;
    int rc0 = cg_total_iters(h, &it0);
    if (rc0)
        return rc0;
    for (int t = 0; t < a.T; t++) {
        if (t % a.K == 0) {
            int rc = adj_save(h, a.ckpt[t / a.K]);
            if (rc)
                return rc;
            a.ckpt_host[t / a.K] = host_state(h);
        }
        int rc = adj_set_V(h, t);
        if (rc)
            return rc;
        rc = do_step<D>(h);
        if (rc == LBEHD_ERR_POISSON_NOCONV)
            worst = rc;
        else if (rc)
            return rc;
        if (a.ptraj) {
            float *pt = a.ptraj + (size_t)t * 2 * N;
            CK(h, cudaMemcpyAsync(pt, h->pot, N * fb, cudaMemcpyDeviceToDevice, h->stream));
            CK(h, cudaMemcpyAsync(pt + N, h->pot_lo, N * fb, cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    if ((rc0 = obs_finalize(h)))
        return rc0;
    // the backward's replays overwrite the sums: keep this run's last two
    CK(h, cudaMemcpyAsync(h->obs + 2 * NOBS, h->obs, 2 * NOBS * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
    double o[2 * NOBS];
    CK(h, cudaMemcpyAsync(o, h->obs, sizeof(o), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    a.M1 = o[0];
    a.xc = o[0] != 0.0 ? o[1] / o[0] : 0.0;
    long long it1 = 0;
    if ((rc0 = cg_total_iters(h, &it1)))
        return rc0;
    a.fwd_iters = it1 - it0;
    int rc = adj_save(h, a.fin);
    if (rc)
        return rc;
    a.fin_host = host_state(h);
    a.have = true;
    *loss = a.xc;
    return worst;
}

int adj_alloc(lbehd_handle *h)
{
    auto &a = h->adj;
    const size_t N = h->N, SS = adj_state_floats(h);
    while ((int)a.slot.size() < a.K) {
        float *p = adj_alloc_floats(h, SS * N);
        if (!p)
            return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint replay)");
        a.slot.push_back(p);
    }
    if (!a.rec) {
        for (int b = 0; b < 2; b++) {
            a.lg[b] = adj_alloc_floats(h, h->Q * N);
            a.lf[b] = adj_alloc_floats(h, 3 * h->Q * N);
            a.lr[b] = adj_alloc_floats(h, h->QS * N);
            a.lp[b] = adj_alloc_floats(h, 8 * N);
            if (!a.lg[b] || !a.lf[b] || !a.lr[b] || !a.lp[b])
                return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint state)");
        }
        a.rec = adj_alloc_floats(h, ADJ_REC * N);
        a.jb = adj_alloc_floats(h, 12 * N);
        a.loc = adj_alloc_floats(h, 5 * N);
        a.phibar = adj_alloc_floats(h, 3 * N);
        a.potbar = adj_alloc_floats(h, N);
        for (int k = 0; k < 3; k++)
            a.mu3[k] = adj_alloc_floats(h, N);
        a.mu = a.mu3[0];
        a.rhs = adj_alloc_floats(h, N);
        a.seed = adj_alloc_floats(h, 3 * N);
        if (!a.rec || !a.jb || !a.loc || !a.phibar || !a.potbar || !a.mu3[0] || !a.mu3[1] ||
            !a.mu3[2] || !a.rhs || !a.seed)
            return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint work arrays)");
    }
    const size_t ng = (size_t)std::max(1, a.S * a.E);
    if (a.grad_cap < ng) {
        a.grad = (double *)dev_alloc(h, ng * sizeof(double));
        if (!a.grad)
            return fail(h, LBEHD_ERR_OOM, "device allocation failed (adjoint gradient)");
        a.bytes += ng * sizeof(double);
        a.grad_cap = ng;
    }
    return LBEHD_OK;
}

// The adjoint Gauss-law solve as a graph: r = rhs - A mu, then CG iterations on mu while the
// residual is above ADJ_POISSON_TOL (conditional while node).
template <int D>
int capture_adj_solve(lbehd_handle *h, int km)
{
    auto &a = h->adj;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess)
        return fail(h, LBEHD_ERR_CUDA, "cudaGraphCreate failed");
    const long long launches = h->launches;
    int rc = LBEHD_OK;
    auto body = [&]() -> int {
        CK(h, cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeRelaxed));
        h->ls = h->stream;
        if (ps_use(h)) {   // one persistent solve
            const int r = ps_launch<D>(h, PS_ADJOINT, a.mu3[km], nullptr, a.rhs);
            if (r)
                return r;
            cudaGraph_t out = nullptr;
            CK(h, cudaStreamEndCapture(h->stream, &out));
            CK(h, cudaGraphInstantiate(&a.solve[km], g, 0));
            return LBEHD_OK;
        }
        cudaGraphConditionalHandle c = 0;
        CK(h, cudaGraphConditionalHandleCreate(&c, g, 0, 0));
        h->use_cond = 1;
        h->use_ref = 0;
        h->cond = c;
        k_adj_pcg_init<D><<<(unsigned)h->nblocks_site, h->block, 0, h->stream>>>(
            h->mg[0].d, h->eps, h->info, h->mg[0].D, a.mu3[km], a.rhs, h->cg_r, h->cg_partials);
        cg_scalar(h, 2, 0, h->nblocks_site);
        const int r = add_cond(h, h->stream, h->aux, c, cudaGraphCondTypeWhile, [&]() -> int {
            pcg_iteration<D>(h, a.mu3[km]);
            return LBEHD_OK;
        });
        if (r)
            return r;
        cudaGraph_t out = nullptr;
        CK(h, cudaStreamEndCapture(h->stream, &out));
        CK(h, cudaGraphInstantiate(&a.solve[km], g, 0));
        return LBEHD_OK;
    };
    rc = body();
    if (rc) {
        for (cudaStream_t sx : {h->aux, h->stream})
            abort_capture(sx);
        cudaGetLastError();
    }
    h->use_cond = 0;
    h->cond = 0;
    h->launches = launches;
    cudaGraphDestroy(g);
    return rc;
}

// One reversed step t: lambda[ia] holds lambda^{t+1}; lambda[ia ^ 1] receives lambda^t.
template <int D>
int adjoint_step(lbehd_handle *h, int t, int ia, float *slot)
{
    auto &a = h->adj;
    const size_t N = h->N;
    const int ib = ia ^ 1;
    const StateView v = state_view(h, slot);
    int rc = adj_set_V(h, t);
    if (rc)
        return rc;
    h->ls = h->stream;
    // the step's potential (recorded trajectory, else the replay's copy in the slot)
    float *pot = a.ptraj ? a.ptraj + (size_t)t * 2 * N : v.pot;
    float *pot_lo = a.ptraj ? pot + N : v.pot_lo;
    // the step's fields Phi^n, rho^n, eps^n from its populations
    const FieldPtrs F{v.fphi, v.frho, h->phi[0], h->rho[0], h->eps, pot, pot_lo,
                      h->info, h->normal, h->elec, h->V};
    k_fields<D><<<h->grid, h->block, 0, h->stream>>>(h->P, F);
    AdjFwd fw{v.g, v.fphi, v.frho, v.phi_prev, v.rho_prev, v.u, v.q, h->phi[0], h->rho[0],
              h->eps, pot, pot_lo, h->info, h->normal};
    const bool last = t == a.T - 1;
    if (last)
        k_adj_seed<<<h->nblocks1d, BX, 0, h->stream>>>(h->P, h->info, a.xc, a.M1, a.seed);
    AdjBuf ab;
    ab.lg_in = a.lg[ia];
    ab.lf_in = a.lf[ia];
    ab.lr_in = a.lr[ia];
    ab.lPp_in = a.lp[ia];
    ab.lrp_in = a.lp[ia] + 3 * N;
    ab.lup_in = a.lp[ia] + 4 * N;
    ab.lqp_in = a.lp[ia] + 7 * N;
    ab.lg_out = a.lg[ib];
    ab.lf_out = a.lf[ib];
    ab.lr_out = a.lr[ib];
    ab.lPp_out = a.lp[ib];
    ab.lrp_out = a.lp[ib] + 3 * N;
    ab.lup_out = a.lp[ib] + 4 * N;
    ab.lqp_out = a.lp[ib] + 7 * N;
    ab.rec = a.rec;
    ab.jb = a.jb;
    ab.loc = a.loc;
    ab.phibar = a.phibar;
    ab.potbar = a.potbar;
    // the adjoint potential of step t, warm-started from the linear extrapolation of those of
    // steps t + 1 and t + 2 (buffers rotate with t)
    const int km = t % 3;
    a.mu = a.mu3[km];
    ab.mu = a.mu;
    ab.seed = last ? a.seed : nullptr;
    const int first = (t == 0 && a.ckpt_host[0].first) ? 1 : 0;
    k_adj_collide<D><<<h->grid, h->block, 0, h->stream>>>(h->P, fw, ab, first);
    k_adj_gather<D><<<h->grid, h->block, 0, h->stream>>>(h->P, fw, ab);
    k_adj_rhs<<<h->grid1d, h->block, 0, h->stream>>>((long long)N, h->info, a.potbar, a.rhs);
    // adjoint Gauss-law solve A mu = phi_bar (A symmetric, built from eps^n): one graph launch
    // (start, device-side CG loop). The multigrid preconditioner is rebuilt from eps^n every
    // 16 reversed steps, as in the forward run.
    if (a.mg_age++ % 16 == 0)
        mg_setup<D>(h);
    if (!a.solve[km] && (rc = capture_adj_solve<D>(h, km)))
        return rc;
    k_adj_extrapolate<<<h->grid1d, h->block, 0, h->stream>>>((long long)N, a.mu3[(t + 1) % 3],
                                                              a.mu3[(t + 2) % 3], a.mu);
    CK(h, cudaGraphLaunch(a.solve[km], h->stream));
    AdjFieldsArgs fa{h->P.cos12, h->P.cos13, h->P.cos23, 4.0f / h->P.W, a.rhs};
    k_adj_fields<D><<<h->grid, h->block, 0, h->stream>>>(h->P, fw, ab, fa);
    k_adj_vgrad<D><<<std::min<size_t>(h->nblocks1d, 148 * 4), VGRAD_THREADS, 0, h->stream>>>(
        h->P, fw, ab, h->elec, a.E, a.grad + (size_t)(t / a.seg) * a.E);
    CK(h, cudaGetLastError());
    h->launches += 9 + (last ? 1 : 0);
    a.adj_steps++;
    return LBEHD_OK;
}

// A replayed forward step t with the recorded potential of that step in place of the
// Gauss-law solve: the same moments and collide kernels as the recorded step, so the same
// bits.
template <int D>
int replay_step(lbehd_handle *h, int t)
{
    auto &a = h->adj;
    const size_t N = h->N, fb = sizeof(float);
    h->ls = h->stream;
    int rc = launch_fields<D>(h);
    if (rc)
        return rc;
    const float *pt = a.ptraj + (size_t)t * 2 * N;
    CK(h, cudaMemcpyAsync(h->pot, pt, N * fb, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->pot_lo, pt + N, N * fb, cudaMemcpyDeviceToDevice, h->stream));
    collide<D>(h);
    CK(h, cudaGetLastError());
    h->cur ^= 1;
    h->pcur ^= 1;
    h->first = false;
    h->step++;
    return LBEHD_OK;
}

template <int D>
int adjoint_backward(lbehd_handle *h, double *grad)
{
    auto &a = h->adj;
    if (!a.have)
        return fail(h, LBEHD_ERR_INVALID_ARG, "no recorded forward run (lbehd_adjoint_forward)");
    int rc = adj_alloc(h);
    if (rc)
        return rc;
    const size_t N = h->N, fb = sizeof(float), SS = adj_state_floats(h);
    CK(h, cudaMemsetAsync(a.grad, 0, (size_t)std::max(1, a.S * a.E) * sizeof(double), h->stream));
    a.dev_seg = -1;
    a.mg_age = 0;
    a.steps_replayed = a.adj_steps = 0;
    long long it0 = 0, it1 = 0;
    if ((rc = cg_total_iters(h, &it0)))
        return rc;
    int ia = 0;
    CK(h, cudaMemsetAsync(a.lg[ia], 0, h->Q * N * fb, h->stream));
    CK(h, cudaMemsetAsync(a.lf[ia], 0, 3 * h->Q * N * fb, h->stream));
    CK(h, cudaMemsetAsync(a.lr[ia], 0, h->QS * N * fb, h->stream));
    CK(h, cudaMemsetAsync(a.lp[ia], 0, 8 * N * fb, h->stream));
    for (int k = 0; k < 3; k++)
        CK(h, cudaMemsetAsync(a.mu3[k], 0, N * fb, h->stream));
    // the adjoint solves stop at a relative residual of ADJ_POISSON_TOL
    const double tol2 = ADJ_POISSON_TOL * ADJ_POISSON_TOL;
    const double tol2_fwd = h->cfg.poisson_tol * h->cfg.poisson_tol;
    const int nck = (a.T + a.K - 1) / a.K;
    for (int ck = nck - 1; ck >= 0; ck--) {
        const int t0 = ck * a.K, t1 = std::min(a.T, t0 + a.K);
        if ((rc = adj_restore<D>(h, a.ckpt[ck], a.ckpt_host[ck])))
            return rc;
        // replay the interval, keeping every step's input state (and, without a recorded
        // trajectory, its potential)
        for (int t = t0; t < t1; t++) {
            float *sl = a.slot[t - t0];
            if ((rc = adj_save(h, sl, a.ptraj == nullptr)))
                return rc;
            if ((rc = adj_set_V(h, t)))
                return rc;
            if (a.ptraj) {
                if ((rc = replay_step<D>(h, t)))
                    return rc;
            } else {
                rc = do_step<D>(h);
                if (rc && rc != LBEHD_ERR_POISSON_NOCONV)
                    return rc;
                const StateView v = state_view(h, sl);
                CK(h, cudaMemcpyAsync(v.pot, h->pot, N * fb, cudaMemcpyDeviceToDevice, h->stream));
                CK(h, cudaMemcpyAsync(v.pot_lo, h->pot_lo, N * fb, cudaMemcpyDeviceToDevice,
                                      h->stream));
            }
            a.steps_replayed++;
        }
        CK(h, cudaMemcpyAsync(&h->cg_s->tol2, &tol2, sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
        a.mg_age = 0;   // preconditioner rebuilt at the interval's last step, then every 16
        for (int t = t1 - 1; t >= t0; t--) {
            if ((rc = adjoint_step<D>(h, t, ia, a.slot[t - t0])))
                return rc;
            ia ^= 1;
        }
        CK(h, cudaMemcpyAsync(&h->cg_s->tol2, &tol2_fwd, sizeof(double), cudaMemcpyHostToDevice,
                              h->stream));
    }
    std::vector<double> g((size_t)std::max(1, a.S * a.E));
    CK(h, cudaMemcpyAsync(g.data(), a.grad, g.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    if ((rc = cg_total_iters(h, &it1)))
        return rc;
    // replays without a trajectory repeat the recorded run's solves, iteration for iteration
    a.adj_iters = it1 - it0 - (a.ptraj ? 0 : a.fwd_iters);
    std::copy(g.begin(), g.begin() + (size_t)a.S * a.E, grad);
    (void)SS;
    // leave the handle as the forward run left it, observables included
    if ((rc = adj_restore<D>(h, a.fin, a.fin_host)))
        return rc;
    CK(h, cudaMemcpyAsync(h->obs, h->obs + 2 * NOBS, 2 * NOBS * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
    h->obs_pending = 0;
    if ((rc = adj_set_V(h, a.T - 1)))
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

// A saved state for lbehd_save_state / lbehd_load_state: this header (padded to
// STATE_HEADER bytes), then the arrays of adj_save.
constexpr size_t STATE_HEADER = 1024;
constexpr uint32_t STATE_MAGIC = 0x4C424548u;   // "LBEH"
struct StateHeader {
    uint32_t magic, version, dim, nx, ny, nz, Q, QS, n_electrodes;
    int32_t cur, pcur, first, mg_valid, pad;
    int64_t step;
};
static_assert(sizeof(StateHeader) + (LBEHD_MAX_ELECTRODES + 2 * NOBS) * sizeof(double) <=
                  STATE_HEADER, "state header too large");

size_t state_bytes(const lbehd_handle *h)
{
    return STATE_HEADER + adj_state_floats(h) * h->N * sizeof(float);
}

int save_state(lbehd_handle *h, void *dst)
{
    char *d = (char *)dst;
    StateHeader H{STATE_MAGIC, 1u, (uint32_t)h->dim, (uint32_t)h->nx, (uint32_t)h->ny,
                  (uint32_t)h->nz, (uint32_t)h->Q, (uint32_t)h->QS,
                  (uint32_t)h->cfg.n_electrodes, h->cur, h->pcur, h->first ? 1 : 0,
                  h->mg_valid ? 1 : 0, 0, h->step};
    if (int rc0 = obs_finalize(h))
        return rc0;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(d, &H, sizeof(H), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpyAsync(d + sizeof(H), h->V, LBEHD_MAX_ELECTRODES * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(d + sizeof(H) + LBEHD_MAX_ELECTRODES * sizeof(double), h->obs,
                          2 * NOBS * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    int rc = adj_save(h, (float *)(d + STATE_HEADER), true);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

template <int D>
int load_state(lbehd_handle *h, const void *src)
{
    const char *s = (const char *)src;
    StateHeader H;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(&H, s, sizeof(H), cudaMemcpyDeviceToHost));
    if (H.magic != STATE_MAGIC || H.version != 1u)
        return fail(h, LBEHD_ERR_INVALID_ARG, "not a saved lbehd state");
    if (H.dim != (uint32_t)h->dim || H.nx != (uint32_t)h->nx || H.ny != (uint32_t)h->ny ||
        H.nz != (uint32_t)h->nz || H.Q != (uint32_t)h->Q || H.QS != (uint32_t)h->QS ||
        H.n_electrodes != (uint32_t)h->cfg.n_electrodes)
        return fail(h, LBEHD_ERR_INVALID_ARG, "saved state is of another lattice");
    if ((H.cur & ~1) || (H.pcur & ~1) || H.step < 0)
        return fail(h, LBEHD_ERR_INVALID_ARG, "saved state header is corrupt");
    CK(h, cudaMemcpyAsync(h->V, s + sizeof(H), LBEHD_MAX_ELECTRODES * sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->obs, s + sizeof(H) + LBEHD_MAX_ELECTRODES * sizeof(double),
                          2 * NOBS * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    h->obs_pending = 0;
    const lbehd_handle::HostState hs{H.step, H.cur, H.pcur, H.first != 0, H.mg_valid != 0};
    int rc = adj_restore<D>(h, (const float *)(s + STATE_HEADER), hs);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

}  // namespace

// ------------------------------------------------------------ batched form

struct lbehd_batch {
    std::vector<lbehd_handle *> inst;
    int dim = 0;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free)(void *, void *) = nullptr;
    void *alloc_ctx = nullptr;
    PopMaps *maps = nullptr;           // device: [2][n] tensor maps, per step parity
    TailLevels *tails = nullptr;       // device: [n] shared-memory tails (b0, x0 set)
    ActiveLists *act = nullptr;        // device: instances active in each mode
    unsigned *icnt = nullptr;          // device: per-instance arrivals of the split scalar kernel
    double *wsum = nullptr;            // device: its virtual-warp sums
    int cta_cap = 2368;                // CTAs of a batched Poisson launch (16 per SM)
    int *counters = nullptr;           // device: loop-condition counts [3], then loop passes
                                       //   [3] main CG, [4] refinement CG, [5] refinement blocks
    double *h_obs = nullptr;           // pinned: [n][2 NOBS] observables, then [n] flags
    cudaStream_t aux = nullptr, aux2 = nullptr;   // capture of conditional-node bodies
    cudaStream_t ls = nullptr;         // stream the batched launches are enqueued on
    size_t tail_smem = 0;              // largest tail's shared memory
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [parity][refresh]
    long long static_kernels[2][2] = {{0, 0}, {0, 0}};
    long long loop_kernels[3] = {0, 0, 0};   // kernels per main / refinement CG pass, per
                                             //   refinement block (outside its loop)
    long long *count = nullptr;        // where the launch being recorded is counted
    long long counters0[3] = {0, 0, 0};   // loop passes when graph replays began
    long long launches = 0, graph_launches = 0, launches_rec = 0;
    bool graphs_started = false;
    int *h_flags = nullptr;            // pinned: loop conditions of an eager step
    bool prof = false;                 // eager steps with CUDA events around every launch
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending[LBEHD_NKC];
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::string err;
};

namespace {

int bfail(lbehd_batch *b, int code, const std::string &msg)
{
    b->err = msg;
    return code;
}

#define BCK(b, call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return bfail((b), LBEHD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void drop_batch_graphs(lbehd_batch *b)
{
    for (auto &row : b->gexec)
        for (auto &e : row)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
}

// Current capture dependencies of a stream (copied: the returned array is only valid until
// the next call on the stream).
int capture_deps(lbehd_batch *b, std::vector<cudaGraphNode_t> &out)
{
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    BCK(b, cudaStreamGetCaptureInfo(b->stream, &st, nullptr, nullptr, &deps, nullptr, &nd));
    out.assign(deps, deps + nd);
    return LBEHD_OK;
}

int set_deps(lbehd_batch *b, const std::vector<cudaGraphNode_t> &deps)
{
    BCK(b, cudaStreamUpdateCaptureDependencies(b->stream, const_cast<cudaGraphNode_t *>(deps.data()),
                                               nullptr, deps.size(),
                                               cudaStreamSetCaptureDependencies));
    return LBEHD_OK;
}

template <int D>
void launch_collide_chunk(lbehd_batch *b, int v, const CollideBatch &A, int blocks)
{
    if (v == 1)
        k_collide_batch<D><<<blocks, BX, 0, b->ls>>>(A);
    else if (v == 2)
        k_collide_staged_batch<D, 4><<<blocks, BX, staged_smem_bytes<D, 4>(), b->ls>>>(A);
    else if (v == 3)
        k_collide_staged_batch<D, 2><<<blocks, BX, staged_smem_bytes<D, 2>(), b->ls>>>(A);
    else
        k_collide_staged_batch<D, 8><<<blocks, BX, staged_smem_bytes<D, 8>(), b->ls>>>(A);
}

// ------------------------------------------------------------ batched Gauss-law solve

// Table header of a batched Poisson launch over instances `ids` with `blocks(k)` blocks for
// instance k; returns the launch's block count.
// Table header of a batched Poisson launch: instances `ids` take part with blocks(k) work
// items each (the others with none); returns the grid: one CTA per work item of all of
// them, capped at b->cta_cap (the CTAs then walk the work items of the active instances).
template <class NB>
int fill_grid_set(lbehd_batch *b, GridSet &g, const std::vector<int> &ids, int mode, NB blocks)
{
    const int n = (int)b->inst.size();
    g.n = n;
    g.mode = mode;
    g.act = b->act;
    for (int k = 0; k < n; k++) {
        g.blocks[k] = 0;
        g.s[k] = b->inst[k]->cg_s;
    }
    long long tot = 0;
    for (int k : ids) {
        g.blocks[k] = (int)blocks(k);
        tot += g.blocks[k];
    }
    return (int)std::min<long long>(tot, b->cta_cap);
}

inline int ceil_div(long long a, int b) { return (int)((a + b - 1) / b); }
inline long long dims_cells(const MgDims &d) { return (long long)d.nx * d.ny * d.nz; }

// MgBatch for level level(k) of each instance k in ids (the coarser level's arrays too).
template <class LV>
void fill_mg(lbehd_batch *b, MgBatch &A, const std::vector<int> &ids, LV level)
{
    for (int k : ids) {
        const lbehd_handle *h = b->inst[k];
        const int l = level(k);
        const auto &L = h->mg[l];
        MgInst &m = A.m[k];
        std::memset(&m, 0, sizeof(m));
        m.f = L.d;
        m.cz2 = L.cz2;
        m.scale = h->mg_scale;
        m.eps = h->eps;
        m.info = h->info;
        m.D = L.D;
        m.kx = L.kx;
        m.ky = L.ky;
        m.kz = L.kz;
        m.b = L.b;
        m.x = L.x;
        m.r = L.r;
        if (l + 1 < (int)h->mg.size()) {
            const auto &C = h->mg[l + 1];
            m.c = C.d;
            m.Dc = C.D;
            m.kxc = C.kx;
            m.kyc = C.ky;
            m.kzc = C.kz;
            m.bc = C.b;
            m.xc = C.x;
        }
    }
}

// Launch through here: counts the launch and, while profiling, brackets it with events.
template <class F>
void blaunch_fn(lbehd_batch *b, int kc, F &&fn)
{
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (b->prof) {
        if (!b->ev_pool.empty()) {
            ev = b->ev_pool.back();
            b->ev_pool.pop_back();
        } else if (cudaEventCreate(&ev.first) != cudaSuccess ||
                   cudaEventCreate(&ev.second) != cudaSuccess) {
            ev = {nullptr, nullptr};
        }
        if (ev.first)
            cudaEventRecord(ev.first, b->ls);
    }
    fn();
    if (b->count)
        ++*b->count;
    if (ev.first) {
        cudaEventRecord(ev.second, b->ls);
        b->ev_pending[kc].push_back(ev);
    }
}

template <class K, class T>
void blaunch(lbehd_batch *b, K kernel, const T &tab, int blocks, int threads, size_t smem = 0,
             int kc = LBEHD_KC_MG)
{
    if (blocks <= 0)
        return;
    blaunch_fn(b, kc, [&] { kernel<<<blocks, threads, smem, b->ls>>>(tab); });
}

// Multigrid levels of instance k handled by separate launches: those above its shared-memory
// tail, or all but the coarsest when it has none.
int mg_depth(const lbehd_handle *h)
{
    return h->tail_level >= 0 ? h->tail_level : (int)h->mg.size() - 1;
}

// One symmetric V-cycle of every active instance, level-synchronous: the same sequence of
// operations as vcycle() per instance.
template <int D>
void batch_vcycle(lbehd_batch *b, MgBatch &A, int mode)
{
    const int n = (int)b->inst.size();
    int maxd = 0, max_nu = 0, max_coarse = 0;
    for (int k = 0; k < n; k++) {
        maxd = std::max(maxd, mg_depth(b->inst[k]));
        max_nu = std::max(max_nu, b->inst[k]->mg_nu);
        max_coarse = std::max(max_coarse, b->inst[k]->mg_coarse);
    }
    // instances with level l above their tail, split by smoother: block-local (bj) or
    // whole-level red-black sweeps
    auto above = [&](int l, int bj) {
        std::vector<int> ids;
        for (int k = 0; k < n; k++)
            if (l < mg_depth(b->inst[k]) && (bj < 0 || (int)bj_use(b->inst[k]) == bj))
                ids.push_back(k);
        return ids;
    };
    auto at = [](int l) { return [l](int) { return l; }; };
    // the instances of ids still sweeping at sweep index sw (reps(k) sweeps each)
    auto sweeping = [](const std::vector<int> &ids, int sw, auto reps) {
        std::vector<int> out;
        for (int k : ids)
            if (sw < reps(k))
                out.push_back(k);
        return out;
    };
    auto nu_of = [&b](int k) { return b->inst[k]->mg_nu; };
    auto cells_f = [&](int l) {
        return [&b, l](int k) { return ceil_div(dims_cells(b->inst[k]->mg[l].d), BX); };
    };
    // block-local passes of level l on the instances of ids
    auto bj_pass = [&](int l, const std::vector<int> &ids, bool up) {
        if (ids.empty())
            return;
        fill_mg(b, A, ids, at(l));
        for (int k : ids) {
            const lbehd_handle *h = b->inst[k];
            MgInst &m = A.m[k];
            m.reps = h->bj_nu;
            m.xcu = l + 1 == h->tail_level ? h->mg[l + 1].x : h->mg[l + 1].r;
            m.rdot = l == 0 ? h->cg_r : nullptr;
            m.pdot = l == 0 ? h->cg_partials : nullptr;
        }
        A.color = up ? 1 : 0;
        blaunch(b, k_mg_bj_batch<D>, A,
                fill_grid_set(b, A.g, ids, mode, [&b, l](int k) { return b->inst[k]->mg[l].nbj; }),
                BJ_THREADS);
    };
    for (int l = 0; l < maxd; l++) {
        bj_pass(l, above(l, 1), false);
        const std::vector<int> ids = above(l, 0);
        if (!ids.empty()) {
            fill_mg(b, A, ids, at(l));
            // zero + the first red half sweep in one pass when every instance sweeps at least once
            const bool fused = sweeping(ids, 0, nu_of).size() == ids.size();
            blaunch(b, fused ? k_mg_gs_first_batch : k_mg_zero_batch, A,
                    fill_grid_set(b, A.g, ids, mode, cells_f(l)), BX);
            auto half = [&b, l](int k) {
                const MgDims &d = b->inst[k]->mg[l].d;
                return ceil_div((long long)(d.nx / 2) * d.ny * d.nz, BX);
            };
            for (int sw = 0; sw < max_nu; sw++) {
                const int hb = fill_grid_set(b, A.g, sweeping(ids, sw, nu_of), mode, half);
                for (int color = (fused && sw == 0) ? 1 : 0; color < 2; color++) {
                    A.color = color;
                    A.sweep = sw;
                    blaunch(b, k_mg_gs_batch, A, hb, BX);
                }
            }
        }
        // residual + restriction in one pass, 8 lanes per coarse cell
        const std::vector<int> all = above(l, -1);
        fill_mg(b, A, all, at(l));
        auto coarse_lanes = [&b, l](int k) {
            return ceil_div(dims_cells(b->inst[k]->mg[l + 1].d) * 8, BX);
        };
        blaunch(b, k_mg_resid_restrict_batch, A, fill_grid_set(b, A.g, all, mode, coarse_lanes),
                BX);
    }
    // bottom: shared-memory tails, and the coarsest-level sweeps of instances without one
    {
        std::vector<int> tail_ids, coarse_ids;
        for (int k = 0; k < n; k++)
            (b->inst[k]->tail_level >= 0 ? tail_ids : coarse_ids).push_back(k);
        if (!tail_ids.empty()) {
            std::unique_ptr<TailBatch> T(new TailBatch);
            std::memset(T.get(), 0, sizeof(TailBatch));
            const int blocks = fill_grid_set(b, T->g, tail_ids, mode, [](int) { return 1; });
            for (int k : tail_ids)
                T->T[k] = b->tails + k;
            blaunch(b, k_mg_tail_batch, *T, blocks, TAIL_THREADS, b->tail_smem);
        }
        if (!coarse_ids.empty()) {
            auto lev = [&b](int k) { return (int)b->inst[k]->mg.size() - 1; };
            fill_mg(b, A, coarse_ids, lev);
            blaunch(b, k_mg_zero_batch, A, fill_grid_set(b, A.g, coarse_ids, mode, [&b, &lev](int k) {
                        return ceil_div(dims_cells(b->inst[k]->mg[lev(k)].d), BX);
                    }), BX);
            auto coarse_of = [&b](int k) { return b->inst[k]->mg_coarse; };
            for (int sw = 0; sw < max_coarse; sw++) {
                const int hb = fill_grid_set(b, A.g, sweeping(coarse_ids, sw, coarse_of), mode,
                                             [&b, &lev](int k) {
                                                 const MgDims &d = b->inst[k]->mg[lev(k)].d;
                                                 return ceil_div((long long)(d.nx / 2) * d.ny * d.nz, BX);
                                             });
                for (int color : {0, 1, 1, 0}) {
                    A.color = color;
                    A.sweep = sw;
                    blaunch(b, k_mg_gs_batch, A, hb, BX);
                }
            }
        }
    }
    for (int l = maxd - 1; l >= 0; l--) {
        bj_pass(l, above(l, 1), true);
        const std::vector<int> ids = above(l, 0);
        if (ids.empty())
            continue;
        fill_mg(b, A, ids, at(l));
        blaunch(b, k_mg_prolong_batch, A, fill_grid_set(b, A.g, ids, mode, cells_f(l)), BX);
        auto half = [&b, l](int k) {
            const MgDims &d = b->inst[k]->mg[l].d;
            return ceil_div((long long)(d.nx / 2) * d.ny * d.nz, BX);
        };
        for (int sw = 0; sw < max_nu; sw++) {
            const int hb = fill_grid_set(b, A.g, sweeping(ids, sw, nu_of), mode, half);
            for (int color = 1; color >= 0; color--) {
                A.color = color;
                A.sweep = sw;
                blaunch(b, k_mg_gs_batch, A, hb, BX);
            }
        }
    }
}

// CG table of every instance; x(h) is the increment solved for, acc(h) where apply adds it.
template <class XF, class AF>
void fill_cg(lbehd_batch *b, CgBatch &C, int parity, XF xsel, AF accsel)
{
    for (size_t k = 0; k < b->inst.size(); k++) {
        lbehd_handle *h = b->inst[k];
        CgInst &c = C.c[k];
        std::memset(&c, 0, sizeof(c));
        c.d = h->mg[0].d;
        c.nbs = (int)h->nblocks_site;
        c.nb1d = (int)h->nblocks1d;
        c.pot = h->pot;
        c.pot_lo = h->pot_lo;
        c.eps = h->eps;
        c.rho = h->rho[parity];
        c.info = h->info;
        c.Dg = h->mg[0].D;
        c.r = h->cg_r;
        c.p = h->cg_p;
        c.q = h->cg_q;
        c.z = bj_use(h) ? h->mg[0].r : h->mg[0].x;   // the level-0 V-cycle output
        c.x = xsel(h);
        c.acc = accsel(h);
        c.partials = h->cg_partials;
        c.d1 = c.x == h->inc[parity] ? h->inc[parity ^ 1] : nullptr;
        c.mr_part = h->mr_part;
        c.mr_alpha = h->mr_alpha;
    }
}

std::vector<int> all_ids(const lbehd_batch *b)
{
    std::vector<int> ids(b->inst.size());
    for (size_t k = 0; k < ids.size(); k++)
        ids[k] = (int)k;
    return ids;
}

int part3d(const lbehd_handle *h) { return (int)h->nblocks_site; }
int part1d(const lbehd_handle *h) { return (int)h->nblocks1d; }

// part: the partition of the partials being summed, 0 the 1D grid stride, 1 the BX-site
// blocks, 2 that of r . z (the block-local smoother's blocks of level 0 for the instances on
// it, else the 1D grid stride).
void batch_scalar(lbehd_batch *b, ScalarBatch &S, int mode, int nv, int op, int part,
                  int loop_mode, cudaGraphConditionalHandle cond, bool set_ref,
                  cudaGraphConditionalHandle cond_ref, bool mr = false)
{
    std::memset(&S, 0, sizeof(S));
    const std::vector<int> ids = all_ids(b);
    fill_grid_set(b, S.g, ids, mode, [](int) { return 1; });
    for (size_t k = 0; k < ids.size(); k++) {
        const lbehd_handle *h = b->inst[k];
        S.partials[k] = h->cg_partials;
        S.nblocks[k] = part == 1 ? part3d(h)
                       : part == 2 && bj_use(h) ? h->mg[0].nbj
                                                : part1d(h);
        S.mr[k] = mr && mr_use(h) ? h->mr_alpha : nullptr;
    }
    S.nv = nv;
    S.op = op;
    S.loop_mode = loop_mode;
    S.set_ref = set_ref ? 1 : 0;
    S.cond = cond;
    S.cond_ref = cond_ref;
    S.counters = b->counters;
    S.act = b->act;
    S.icnt = b->icnt;
    S.wsum = b->wsum;
    S.eager = b->prof ? 1 : 0;
    blaunch(b, k_pcg_scalar_batch_split, S, 32 * (int)ids.size(), 32, 0, LBEHD_KC_CG);
}

// r = b - A (phi + x) and the CG start of every instance active in `mode`.
template <int D>
void batch_pcg_start(lbehd_batch *b, CgBatch &C, ScalarBatch &S, int mode, int op, int loop_mode,
                     cudaGraphConditionalHandle cond, bool set_ref,
                     cudaGraphConditionalHandle cond_ref)
{
    const std::vector<int> ids = all_ids(b);
    // a step's first pass: the least-residual start on the instances that use it (the
    // multi-launch form's order: start pass, coefficients, x0 and r, then the test)
    std::vector<int> plain_ids, mr_ids;
    for (int k : ids)
        (op == 0 && mr_use(b->inst[k]) ? mr_ids : plain_ids).push_back(k);
    const int blocks = fill_grid_set(b, C.g, plain_ids, mode,
                                     [&b](int k) { return part3d(b->inst[k]); });
    if (blocks > 0)
        blaunch(b, k_pcg_init_batch<D>, C, blocks, BX, 0, LBEHD_KC_CG);
    if (!mr_ids.empty()) {
        const int b3 = fill_grid_set(b, C.g, mr_ids, mode,
                                     [&b](int k) { return part3d(b->inst[k]); });
        blaunch(b, k_pcg_init_mr_batch<D>, C, b3, BX, 0, LBEHD_KC_CG);
        const int ba = fill_grid_set(b, C.g, mr_ids, mode, [](int) { return 1; });
        blaunch(b, k_mr_alpha_batch, C, ba, SCALAR_THREADS, 0, LBEHD_KC_CG);
        const int b1 = fill_grid_set(b, C.g, mr_ids, mode,
                                     [&b](int k) { return part1d(b->inst[k]); });
        blaunch(b, k_pcg_start_mr_batch, C, b1, BX, 0, LBEHD_KC_CG);
    }
    batch_scalar(b, S, mode, 2, op, 1, loop_mode, cond, set_ref, cond_ref, op == 0);
}

// One preconditioned CG iteration of every instance active in `mode`.
template <int D>
void batch_pcg_iteration(lbehd_batch *b, MgBatch &A, CgBatch &C, ScalarBatch &S, int mode,
                         int op, cudaGraphConditionalHandle cond, bool set_ref,
                         cudaGraphConditionalHandle cond_ref)
{
    const std::vector<int> ids = all_ids(b);
    batch_vcycle<D>(b, A, mode);
    // r . z: k_pcg_dot_batch for the instances on whole-level sweeps; the block-local
    // smoother's last pass wrote the others' partials
    std::vector<int> gs_ids;
    for (int k : ids)
        if (!bj_use(b->inst[k]))
            gs_ids.push_back(k);
    const int bd = fill_grid_set(b, C.g, gs_ids, mode, [&b](int k) { return part1d(b->inst[k]); });
    blaunch(b, k_pcg_dot_batch, C, bd, BX, 0, LBEHD_KC_CG);
    batch_scalar(b, S, mode, 1, 1, 2, -1, cond, false, cond_ref);
    const int b1 = fill_grid_set(b, C.g, ids, mode, [&b](int k) { return part1d(b->inst[k]); });
    blaunch(b, k_pcg_p_batch, C, b1, BX, 0, LBEHD_KC_CG);
    const int b3 = fill_grid_set(b, C.g, ids, mode, [&b](int k) { return part3d(b->inst[k]); });
    blaunch(b, k_pcg_Ap_batch<D>, C, b3, BX, 0, LBEHD_KC_CG);
    batch_scalar(b, S, mode, 1, 2, 1, -1, cond, false, cond_ref);
    fill_grid_set(b, C.g, ids, mode, [&b](int k) { return part1d(b->inst[k]); });
    blaunch(b, k_pcg_update_batch, C, b1, BX, 0, LBEHD_KC_CG);
    batch_scalar(b, S, mode, 1, op, 0, mode, cond, set_ref, cond_ref);
}

void batch_pcg_apply(lbehd_batch *b, CgBatch &C, int mode)
{
    const int b1 = fill_grid_set(b, C.g, all_ids(b), mode, [&b](int k) { return part1d(b->inst[k]); });
    blaunch(b, k_pcg_apply_batch, C, b1, BX, 0, LBEHD_KC_CG);
}

// Conditional node on the ongoing capture of `cap`, body captured from `body` on `bs`.
template <class F>
int batch_add_cond(lbehd_batch *b, cudaStream_t cap, cudaStream_t bs,
                   cudaGraphConditionalHandle cond, cudaGraphConditionalNodeType type, F &&body)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    BCK(b, cudaStreamGetCaptureInfo(cap, &st, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BCK(b, cudaGraphAddNode(&node, cg, deps, nullptr, nd, &np));
    BCK(b, cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
    const cudaStream_t prev = b->ls;
    b->ls = bs;
    const int rc = body();
    b->ls = prev;
    cudaGraph_t out = nullptr;
    BCK(b, cudaStreamEndCapture(bs, &out));
    if (rc)
        return rc;
    BCK(b, cudaStreamUpdateCaptureDependencies(cap, &node, nullptr, 1,
                                               cudaStreamSetCaptureDependencies));
    return LBEHD_OK;
}

// Multigrid hierarchy of every instance from this step's permittivity.
template <int D>
void batch_mg_setup(lbehd_batch *b, MgBatch &A)
{
    const std::vector<int> ids = all_ids(b);
    const int n = (int)ids.size();
    fill_mg(b, A, ids, [](int) { return 0; });
    blaunch(b, k_mg_setup0_batch<D>, A, fill_grid_set(b, A.g, ids, 0, [&b](int k) {
                return ceil_div((long long)b->inst[k]->N, BX);
            }), BX);
    int levels = 0;
    for (int k = 0; k < n; k++)
        levels = std::max(levels, (int)b->inst[k]->mg.size());
    for (int l = 0; l + 1 < levels; l++) {
        std::vector<int> lid;
        for (int k = 0; k < n; k++)
            if (l + 1 < (int)b->inst[k]->mg.size())
                lid.push_back(k);
        fill_mg(b, A, lid, [l](int) { return l; });
        blaunch(b, k_mg_coarsen_batch, A, fill_grid_set(b, A.g, lid, 0, [&b, l](int k) {
                    return ceil_div(dims_cells(b->inst[k]->mg[l + 1].d), BX);
                }), BX);
    }
}

// delta2 = 0 on the instances active in `mode`.
void batch_zero_delta2(lbehd_batch *b, MgBatch &A, int mode)
{
    const std::vector<int> ids = all_ids(b);
    fill_mg(b, A, ids, [](int) { return 0; });
    for (size_t k = 0; k < ids.size(); k++)
        A.m[k].x = b->inst[k]->delta2;
    blaunch(b, k_mg_zero_batch, A, fill_grid_set(b, A.g, ids, mode, [&b](int k) {
                return ceil_div((long long)b->inst[k]->N, BX);
            }), BX, 0, LBEHD_KC_CG);
}

int read_flags(lbehd_batch *b, int &act, int &ref)
{
    BCK(b, cudaMemcpyAsync(b->h_flags, b->counters + 6, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    act = b->h_flags[0];
    ref = b->h_flags[1];
    return LBEHD_OK;
}

// The same solve as record_batch_poisson with the loop conditions read back by the host
// (eager launches, for profiling).
template <int D>
int eager_batch_poisson(lbehd_batch *b, int parity, int refresh)
{
    std::unique_ptr<MgBatch> A(new MgBatch);
    std::unique_ptr<CgBatch> C(new CgBatch);
    std::unique_ptr<ScalarBatch> S(new ScalarBatch);
    std::memset(A.get(), 0, sizeof(MgBatch));
    std::memset(C.get(), 0, sizeof(CgBatch));
    if (refresh)
        batch_mg_setup<D>(b, *A);
    auto inc = [parity](lbehd_handle *h) { return h->inc[parity]; };
    auto none = [](lbehd_handle *) -> float * { return nullptr; };
    auto del = [](lbehd_handle *h) { return h->delta2; };
    int act = 0, ref = 0, junk = 0, rc;
    fill_cg(b, *C, parity, inc, none);
    batch_pcg_start<D>(b, *C, *S, 0, 0, 1, 0, true, 0);
    if ((rc = read_flags(b, act, ref)))
        return rc;
    while (act) {
        batch_pcg_iteration<D>(b, *A, *C, *S, 1, 3, 0, true, 0);
        if ((rc = read_flags(b, act, ref)))
            return rc;
    }
    batch_pcg_apply(b, *C, 0);
    if (!ref)
        return LBEHD_OK;
    batch_zero_delta2(b, *A, 2);
    fill_cg(b, *C, parity, del, none);
    batch_pcg_start<D>(b, *C, *S, 2, 4, 3, 0, false, 0);
    if ((rc = read_flags(b, act, junk)))
        return rc;
    while (act) {
        batch_pcg_iteration<D>(b, *A, *C, *S, 3, 5, 0, false, 0);
        if ((rc = read_flags(b, act, junk)))
            return rc;
    }
    fill_cg(b, *C, parity, del, inc);
    batch_pcg_apply(b, *C, 2);
    return LBEHD_OK;
}

// The Gauss-law solves of all instances for one step (the batched counterpart of the
// Poisson part of record_step): multigrid rebuild when `refresh`; start; CG loop while any
// instance is unconverged; apply; then, if any instance iterated, the refinement block for
// those instances with its own loop.
template <int D>
int record_batch_poisson(lbehd_batch *b, cudaGraph_t g, int parity, int refresh)
{
    std::unique_ptr<MgBatch> A(new MgBatch);
    std::unique_ptr<CgBatch> C(new CgBatch);
    std::unique_ptr<ScalarBatch> S(new ScalarBatch);
    std::memset(A.get(), 0, sizeof(MgBatch));
    std::memset(C.get(), 0, sizeof(CgBatch));
    const std::vector<int> ids = all_ids(b);
    if (refresh)
        batch_mg_setup<D>(b, *A);
    cudaGraphConditionalHandle c1 = 0, c2 = 0, cr = 0;
    BCK(b, cudaGraphConditionalHandleCreate(&c1, g, 0, 0));
    BCK(b, cudaGraphConditionalHandleCreate(&c2, g, 0, 0));
    BCK(b, cudaGraphConditionalHandleCreate(&cr, g, 0, 0));
    auto inc = [parity](lbehd_handle *h) { return h->inc[parity]; };
    auto none = [](lbehd_handle *) -> float * { return nullptr; };
    auto del = [](lbehd_handle *h) { return h->delta2; };
    fill_cg(b, *C, parity, inc, none);
    batch_pcg_start<D>(b, *C, *S, 0, 0, 1, c1, true, cr);
    int rc = batch_add_cond(b, b->stream, b->aux, c1, cudaGraphCondTypeWhile, [&]() -> int {
        long long *prev = b->count;
        b->loop_kernels[0] = 0;
        b->count = &b->loop_kernels[0];
        batch_pcg_iteration<D>(b, *A, *C, *S, 1, 3, c1, true, cr);
        b->count = prev;
        return LBEHD_OK;
    });
    if (rc)
        return rc;
    batch_pcg_apply(b, *C, 0);
    rc = batch_add_cond(b, b->stream, b->aux, cr, cudaGraphCondTypeIf, [&]() -> int {
        long long *prev = b->count;
        b->loop_kernels[2] = 0;
        b->count = &b->loop_kernels[2];
        batch_zero_delta2(b, *A, 2);
        fill_cg(b, *C, parity, del, none);
        batch_pcg_start<D>(b, *C, *S, 2, 4, 3, c2, false, cr);
        const int r2 = batch_add_cond(b, b->aux, b->aux2, c2, cudaGraphCondTypeWhile, [&]() -> int {
            long long *prev2 = b->count;
            b->loop_kernels[1] = 0;
            b->count = &b->loop_kernels[1];
            batch_pcg_iteration<D>(b, *A, *C, *S, 3, 5, c2, false, cr);
            b->count = prev2;
            return LBEHD_OK;
        });
        fill_cg(b, *C, parity, del, inc);
        batch_pcg_apply(b, *C, 2);
        b->count = prev;
        return r2;
    });
    return rc;
}

// Blocks of one instance in the batched collide launch of variant v.
long long collide_blocks(const lbehd_handle *h, int v)
{
    return v == 1 ? (long long)((h->N + BX - 1) / BX) : (long long)h->nblocks_tile[tile_shape(v)];
}

// Instances grouped by collide kernel (order[]), and their tensor maps for `parity` in that
// order in the device table.
int batch_prepare_collide(lbehd_batch *b, int parity, std::vector<int> &order)
{
    const int n = (int)b->inst.size();
    order.clear();
    for (int v = 1; v <= 4; v++)
        for (int i = 0; i < n; i++)
            if (resolved_variant(b->inst[i]) == v)
                order.push_back(i);
    std::vector<PopMaps> hm(n);
    for (int k = 0; k < n; k++) {
        const lbehd_handle *h = b->inst[order[k]];
        const int v = resolved_variant(h);
        if (v != 1)
            hm[k] = h->maps[tile_shape(v)][parity];
        else
            std::memset(&hm[k], 0, sizeof(PopMaps));
    }
    BCK(b, cudaMemcpyAsync(b->maps + (size_t)parity * n, hm.data(), n * sizeof(PopMaps),
                           cudaMemcpyHostToDevice, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    return LBEHD_OK;
}

// Moments + ghosts of every instance, one launch.
template <int D>
void batch_fields(lbehd_batch *b, int parity)
{
    std::unique_ptr<FieldsBatch> FA(new FieldsBatch);
    std::memset(FA.get(), 0, sizeof(FieldsBatch));
    const int n = (int)b->inst.size();
    FA->n = n;
    long long blocks = 0;
    for (int k = 0; k < n; k++) {
        const lbehd_handle *h = b->inst[k];
        FA->start[k] = (int)blocks;
        FA->P[k] = h->P;
        FA->F[k] = field_ptrs(h, parity, parity);
        blocks += (long long)((h->N + BX - 1) / BX);
    }
    FA->start[n] = (int)blocks;
    blaunch_fn(b, LBEHD_KC_FIELDS,
               [&] { k_fields_batch<D><<<(unsigned)blocks, BX, 0, b->ls>>>(*FA); });
}

// Collide + stream: one launch per group of instances running the same collide kernel (in
// a capture, the groups are parallel branches), then the observable sums of every instance.
template <int D>
int batch_collide(lbehd_batch *b, int parity, const std::vector<int> &order, bool capture)
{
    const int n = (int)b->inst.size();
    std::unique_ptr<CollideBatch> CA(new CollideBatch);
    std::unique_ptr<ObsBatch> OA(new ObsBatch);
    std::vector<cudaGraphNode_t> ends, cends, tmp;
    int r;
    if (capture && (r = capture_deps(b, ends)))
        return r;
    const PopMaps *dmaps = b->maps + (size_t)parity * n;
    for (int k0 = 0; k0 < n;) {
        const int v = resolved_variant(b->inst[order[k0]]);
        int m = 0;
        while (k0 + m < n && resolved_variant(b->inst[order[k0 + m]]) == v)
            m++;
        std::memset(CA.get(), 0, sizeof(CollideBatch));
        CA->n = m;
        CA->first = 0;
        CA->maps = dmaps + k0;
        long long blocks = 0;
        for (int k = 0; k < m; k++) {
            const lbehd_handle *h = b->inst[order[k0 + k]];
            CA->start[k] = (int)blocks;
            if (v != 1) {
                CA->tiles_x[k] = (int)h->grid_tile[tile_shape(v)].x;
                CA->tiles_y[k] = (int)h->grid_tile[tile_shape(v)].y;
            }
            CA->P[k] = h->P;
            CA->S[k] = collide_state(h, parity, parity);
            blocks += collide_blocks(h, v);
        }
        CA->start[m] = (int)blocks;
        if (capture && (r = set_deps(b, ends)))
            return r;
        blaunch_fn(b, LBEHD_KC_COLLIDE, [&] { launch_collide_chunk<D>(b, v, *CA, (int)blocks); });
        if (capture) {
            if ((r = capture_deps(b, tmp)))
                return r;
            cends.insert(cends.end(), tmp.begin(), tmp.end());
        }
        k0 += m;
    }
    if (capture && (r = set_deps(b, cends)))
        return r;
    std::memset(OA.get(), 0, sizeof(ObsBatch));
    OA->n = n;
    for (int k = 0; k < n; k++) {
        const lbehd_handle *h = b->inst[k];
        OA->partials[k] = obs_buf(h, parity);
        OA->nblocks[k] = collide_blocks(h, resolved_variant(h));
        OA->obs[k] = h->obs;
    }
    blaunch_fn(b, LBEHD_KC_OBS,
               [&] { k_obs_final_batch<<<dim3(NOBS, n), OBS_THREADS, 0, b->ls>>>(*OA); });
    return LBEHD_OK;
}

// The whole batch's step for one parity as one graph: the moments of every instance (one
// launch), the Gauss-law solves of all instances in lockstep, the collide kernels (one
// launch per group of instances running the same kernel, the groups as parallel branches),
// then the observable sums of every instance.
template <int D>
int capture_batch(lbehd_batch *b, int parity, int refresh)
{
    std::vector<int> order;
    int rc = batch_prepare_collide(b, parity, order);
    if (rc)
        return rc;
    cudaGraph_t g = nullptr;
    BCK(b, cudaGraphCreate(&g, 0));
    b->launches_rec = 0;
    b->count = &b->launches_rec;
    const bool prof = b->prof;
    b->prof = false;
    auto body = [&]() -> int {
        BCK(b, cudaStreamBeginCaptureToGraph(b->stream, g, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
        b->ls = b->stream;
        batch_fields<D>(b, parity);
        int r = record_batch_poisson<D>(b, g, parity, refresh);
        if (r)
            return r;
        if ((r = batch_collide<D>(b, parity, order, true)))
            return r;
        BCK(b, cudaGetLastError());
        cudaGraph_t out = nullptr;
        BCK(b, cudaStreamEndCapture(b->stream, &out));
        BCK(b, cudaGraphInstantiate(&b->gexec[parity][refresh], g, 0));
        return LBEHD_OK;
    };
    rc = body();
    if (rc) {
        for (cudaStream_t sx : {b->aux2, b->aux, b->stream})
            abort_capture(sx);
        cudaGetLastError();
    }
    cudaGraphDestroy(g);
    b->static_kernels[parity][refresh] = b->launches_rec;
    b->count = nullptr;
    b->prof = prof;
    return rc;
}

// One batch step of eager launches (profiling): the graph's sequence, loops checked on the
// host.
template <int D>
int eager_batch_step(lbehd_batch *b, int parity, int refresh)
{
    std::vector<int> order;
    int rc = batch_prepare_collide(b, parity, order);
    if (rc)
        return rc;
    b->ls = b->stream;
    b->count = &b->launches;
    batch_fields<D>(b, parity);
    if (!(rc = eager_batch_poisson<D>(b, parity, refresh)))
        rc = batch_collide<D>(b, parity, order, false);
    b->count = nullptr;
    if (!rc) {
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            rc = bfail(b, LBEHD_ERR_CUDA, std::string("eager batch step: ") + cudaGetErrorString(e));
    }
    return rc;
}

template <int D>
int batch_step_one(lbehd_batch *b)
{
    bool any_first = false;
    for (lbehd_handle *h : b->inst)
        any_first = any_first || h->first;
    if (any_first) {
        // the first step (initial fields, host-checked Poisson solve) runs per instance
        int worst = LBEHD_OK;
        for (lbehd_handle *h : b->inst) {
            const int rc = do_step<D>(h);
            if (rc == LBEHD_ERR_POISSON_NOCONV)
                worst = rc;
            else if (rc)
                return bfail(b, rc, "first step: " + h->err);
            // the batched steps reduce every instance's observables after each step
            if (const int r2 = obs_finalize(h))
                return bfail(b, r2, "first step: " + h->err);
        }
        return worst;
    }
    const lbehd_handle *h0 = b->inst[0];
    const int parity = (int)(h0->step & 1);
    int refresh = 0;
    for (lbehd_handle *h : b->inst) {
        if (h->step != h0->step || h->cur != parity || h->pcur != parity)
            return bfail(b, LBEHD_ERR_INVALID_ARG, "batch instances are out of step");
        refresh |= mg_due(h) ? 1 : 0;
    }
    if (b->prof) {
        const int rc = eager_batch_step<D>(b, parity, refresh);
        if (rc)
            return rc;
        for (lbehd_handle *h : b->inst) {
            h->cur ^= 1;
            h->pcur ^= 1;
            h->step++;
            if (refresh)
                h->mg_valid = true;
        }
        return LBEHD_OK;
    }
    if (!b->gexec[parity][refresh]) {
        const int rc = capture_batch<D>(b, parity, refresh);
        if (rc)
            return rc;
    }
    if (!b->graphs_started) {
        // kernels inside the batch's loops are counted from the device loop-pass counters:
        // remember where they stood
        int c[6] = {0, 0, 0, 0, 0, 0};
        BCK(b, cudaMemcpyAsync(c, b->counters, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        for (int k = 0; k < 3; k++)
            b->counters0[k] = c[3 + k];
        b->graphs_started = true;
    }
    BCK(b, cudaGraphLaunch(b->gexec[parity][refresh], b->stream));
    b->graph_launches++;
    b->launches += b->static_kernels[parity][refresh];
    for (lbehd_handle *h : b->inst) {
        h->cur ^= 1;
        h->pcur ^= 1;
        h->step++;
        h->graph_launches++;
        if (refresh)
            h->mg_valid = true;   // the graph rebuilt the hierarchy
    }
    return LBEHD_OK;
}

void batch_release(lbehd_batch *b)
{
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    drop_batch_graphs(b);
    for (lbehd_handle *h : b->inst) {
        release(h);
        delete h;
    }
    b->inst.clear();
    for (void *p : {(void *)b->maps, (void *)b->tails, (void *)b->counters, (void *)b->act,
                    (void *)b->icnt, (void *)b->wsum}) {
        if (!p)
            continue;
        if (b->free)
            b->free(p, b->alloc_ctx);
        else
            cudaFree(p);
    }
    b->maps = nullptr;
    b->tails = nullptr;
    b->counters = nullptr;
    b->act = nullptr;
    b->icnt = nullptr;
    b->wsum = nullptr;
    for (cudaStream_t *sx : {&b->aux, &b->aux2})
        if (*sx) {
            cudaStreamDestroy(*sx);
            *sx = nullptr;
        }
    if (b->h_obs)
        cudaFreeHost(b->h_obs);
    b->h_obs = nullptr;
    if (b->h_flags)
        cudaFreeHost(b->h_flags);
    b->h_flags = nullptr;
    for (auto &v : b->ev_pending) {
        for (auto &e : v)
            b->ev_pool.push_back(e);
        v.clear();
    }
    for (auto &e : b->ev_pool) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    b->ev_pool.clear();
    if (b->own_stream)
        cudaStreamDestroy(b->own_stream);
    b->own_stream = nullptr;
}

template <int D>
int batch_kernel_attributes()
{
    if (cudaFuncSetAttribute(k_collide_staged_batch<D, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)staged_smem_bytes<D, 4>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_collide_staged_batch<D, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)staged_smem_bytes<D, 2>()) != cudaSuccess ||
        cudaFuncSetAttribute(k_collide_staged_batch<D, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)staged_smem_bytes<D, 8>()) != cudaSuccess)
        return LBEHD_ERR_CUDA;
    return LBEHD_OK;
}

}  // namespace

extern "C" {

int lbehd_abi_version(void) { return LBEHD_ABI_VERSION; }

size_t lbehd_config_size(void) { return sizeof(lbehd_config); }

int lbehd_init(const lbehd_config *cfg, lbehd_handle **out)
{
    if (!cfg || !out)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null config or output pointer");
    *out = nullptr;
    if (cfg->dim != 2 && cfg->dim != 3)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (cfg->nx < 2 || cfg->ny < 2 || cfg->nz < 1 || (cfg->dim == 2 && cfg->nz != 1) ||
        (cfg->dim == 3 && cfg->nz < 2))
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "bad lattice extents");
    if (cfg->nx % 2 || (cfg->dim == 3 && cfg->ny % 2))
        return fail(nullptr, LBEHD_ERR_INVALID_ARG,
                    "periodic extents must be even (red-black ordering of the Poisson smoother)");
    if (cfg->ny > 65535 || cfg->nz > 65535)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "ny and nz must be <= 65535");
    if ((long long)cfg->nx * cfg->ny * cfg->nz * 19 >= (1LL << 31))
        return fail(nullptr, LBEHD_ERR_INVALID_ARG,
                    "lattice too large: 32-bit site offsets need 19 * N < 2^31");
    if (!cfg->solid || !cfg->phi_init)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "solid and phi_init are required");
    if (cfg->n_electrodes < 0 || cfg->n_electrodes > LBEHD_MAX_ELECTRODES ||
        (cfg->n_electrodes > 0 && !cfg->electrode_V))
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "bad electrode table");
    if (!(cfg->W > 0.0) || !(cfg->mobility > 0.0) || !(cfg->alpha >= 0.0) ||
        !(cfg->poisson_tol > 0.0) || cfg->poisson_max_iter < 1)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "W, mobility, poisson_tol must be > 0");
    for (int k = 0; k < 3; k++)
        if (!(cfg->nu[k] > 0.0) || !(cfg->eps[k] > 0.0) || !(cfg->sigma[k] >= 0.0))
            return fail(nullptr, LBEHD_ERR_INVALID_ARG, "nu, eps > 0 and sigma >= 0 required");
    lbehd_handle *h = new (std::nothrow) lbehd_handle();
    if (!h)
        return fail(nullptr, LBEHD_ERR_OOM, "host allocation failed");
    h->cfg = *cfg;
    h->dim = cfg->dim;
    h->nx = cfg->nx;
    h->ny = cfg->ny;
    h->nz = cfg->nz;
    h->N = (size_t)cfg->nx * cfg->ny * cfg->nz;
    h->stream = (cudaStream_t)cfg->stream;
    if (!h->stream) {
        // the legacy default stream cannot be captured into a graph: use an own blocking
        // stream, which stays ordered with the legacy stream
        if (cudaStreamCreate(&h->own_stream) != cudaSuccess) {
            delete h;
            return fail(nullptr, LBEHD_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->stream = h->own_stream;
    }
    h->ls = h->stream;
    int rc = set_params(h);
    if (!rc)
        rc = h->dim == 2 ? init_impl<2>(h) : init_impl<3>(h);
    h->cfg.solid = nullptr;
    h->cfg.electrode_id = nullptr;
    h->cfg.phi_init = nullptr;
    h->cfg.electrode_V = nullptr;
    if (rc) {
        g_init_error = h->err;
        release(h);
        delete h;
        return rc;
    }
    *out = h;
    return LBEHD_OK;
}

int lbehd_step(lbehd_handle *h, int n)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: use lbehd_batch_step");
    if (n < 0)
        return fail(h, LBEHD_ERR_INVALID_ARG, "n must be >= 0");
    int worst = LBEHD_OK;
    for (int s = 0; s < n; s++) {
        const int rc = h->dim == 2 ? do_step<2>(h) : do_step<3>(h);
        if (rc == LBEHD_ERR_POISSON_NOCONV)
            worst = rc;
        else if (rc)
            return rc;
    }
    if (worst)
        h->err = "Poisson solve reached poisson_max_iter";
    return worst;
}

int lbehd_set_electrodes(lbehd_handle *h, const double *V, int n)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (n != h->cfg.n_electrodes || (n > 0 && !V))
        return fail(h, LBEHD_ERR_INVALID_ARG, "electrode count differs from the configuration");
    // pageable source: the copy is staged before this call returns
    CK(h, cudaMemcpyAsync(h->V, V, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

int lbehd_set_body_force(lbehd_handle *h, const double *body, const double *body_droplet)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: body forces are set at init");
    for (int k = 0; k < 3; k++)
        if ((body && !std::isfinite(body[k])) || (body_droplet && !std::isfinite(body_droplet[k])))
            return fail(h, LBEHD_ERR_INVALID_ARG, "body force must be finite");
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 3; k++) {
        if (body)
            h->cfg.body_force[k] = body[k];
        if (body_droplet)
            h->cfg.body_force_droplet[k] = body_droplet[k];
        h->P.body[k] = (float)h->cfg.body_force[k];
        h->P.body1[k] = (float)h->cfg.body_force_droplet[k];
    }
    for (auto &row : h->gexec)   // captured graphs hold the previous parameters
        for (auto &e : row)
            if (e) {
                cudaGraphExecDestroy(e);
                e = nullptr;
            }
    h->adj.have = false;
    return LBEHD_OK;
}

int lbehd_observe(lbehd_handle *h, lbehd_obs *out)
{
    if (!h || !out)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or output");
    double o[2 * NOBS];
    int flag = 0;
    const int rc = observe_enqueue(h, o, &flag);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    return observe_fill(h, o, flag, out);
}

static int array_info(lbehd_handle *h, int which, void **ptr, size_t *bytes)
{
    const size_t N = h->N, fb = sizeof(float);
    switch (which) {
    case LBEHD_G: *ptr = h->g[h->cur]; *bytes = h->Q * N * fb; break;
    case LBEHD_FPHI: *ptr = h->fphi[h->cur]; *bytes = 3 * h->Q * N * fb; break;
    case LBEHD_FRHO: *ptr = h->frho[h->cur]; *bytes = h->QS * N * fb; break;
    case LBEHD_PHI: *ptr = h->phi[h->pcur ^ 1]; *bytes = 3 * N * fb; break;
    case LBEHD_RHO: *ptr = h->rho[h->pcur ^ 1]; *bytes = N * fb; break;
    case LBEHD_POT: *ptr = h->pot; *bytes = N * fb; break;
    case LBEHD_U: *ptr = h->u; *bytes = 3 * N * fb; break;
    case LBEHD_QSRC: *ptr = h->q; *bytes = N * fb; break;
    case LBEHD_EPS: *ptr = h->eps; *bytes = N * fb; break;
    case LBEHD_POT_LO: *ptr = h->pot_lo; *bytes = N * fb; break;
    default: return fail(h, LBEHD_ERR_INVALID_ARG, "unknown array id");
    }
    return LBEHD_OK;
}

int lbehd_copy_out(lbehd_handle *h, int which, void *dst, size_t bytes)
{
    if (!h || !dst)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or destination");
    void *p = nullptr;
    size_t nb = 0;
    int rc = array_info(h, which, &p, &nb);
    if (rc)
        return rc;
    if (bytes < nb)
        return fail(h, LBEHD_ERR_INVALID_ARG, "destination too small");
    CK(h, cudaMemcpyAsync(dst, p, nb, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return LBEHD_OK;
}

int lbehd_device_ptr(lbehd_handle *h, int which, void **ptr, size_t *bytes)
{
    if (!h || !ptr || !bytes)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null argument");
    return array_info(h, which, ptr, bytes);
}

long long lbehd_launch_count(lbehd_handle *h)
{
    if (!h)
        return 0;
    long long n = h->launches;
    if (h->graph_launches_started) {
        // kernels inside the graphs' while loops: iterations since graphs took over
        CgScalars s0;
        if (cudaMemcpyAsync(&s0, h->cg_s, sizeof(s0), cudaMemcpyDeviceToHost, h->stream) ==
                cudaSuccess &&
            cudaStreamSynchronize(h->stream) == cudaSuccess)
            n += (s0.total_iters - h->graph_iters0) * h->iter_kernels;
    }
    return n;
}

int lbehd_set_option(lbehd_handle *h, int option, long long value)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: use lbehd_batch_set_option");
    return set_option_impl(h, option, value);
}

size_t lbehd_state_bytes(lbehd_handle *h)
{
    return h ? state_bytes(h) : 0;
}

int lbehd_save_state(lbehd_handle *h, void *dst)
{
    if (!h || !dst)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or destination");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: states are saved per handle");
    if ((uintptr_t)dst % 16)
        return fail(h, LBEHD_ERR_INVALID_ARG, "state buffer must be 16-byte aligned");
    return save_state(h, dst);
}

int lbehd_load_state(lbehd_handle *h, const void *src)
{
    if (!h || !src)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or source");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: states are loaded per handle");
    if ((uintptr_t)src % 16)
        return fail(h, LBEHD_ERR_INVALID_ARG, "state buffer must be 16-byte aligned");
    return h->dim == 2 ? load_state<2>(h, src) : load_state<3>(h, src);
}

int lbehd_get_option(lbehd_handle *h, int option, long long *value)
{
    if (!h || !value)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or output");
    if (option == LBEHD_OPT_COLLIDE)
        *value = resolved_variant(h);
    else if (option == LBEHD_OPT_MG_REFRESH)
        *value = h->mg_refresh;
    else if (option == LBEHD_OPT_ADJ_TRAJECTORY)
        *value = h->adj.use_traj ? 1 : 0;
    else if (option == LBEHD_OPT_POISSON_KERNEL)
        *value = ps_use(h) ? 1 : 0;
    else if (option == LBEHD_OPT_MG_SMOOTHER)
        *value = bj_use(h) ? 1 : 0;
    else if (option == LBEHD_OPT_WARM_START)
        *value = h->warm_mode;
    else
        return fail(h, LBEHD_ERR_INVALID_ARG, "unknown option");
    return LBEHD_OK;
}

int lbehd_adjoint_forward(lbehd_handle *h, const double *V, int n_segments, int seg_steps,
                          double *loss)
{
    if (!h || !loss || (h->cfg.n_electrodes > 0 && !V))
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle, schedule or loss");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: the adjoint is per handle");
    if (h->var_density)
        return fail(h, LBEHD_ERR_INVALID_ARG,
                    "the adjoint runs equal densities (density_model 0)");
    if (n_segments < 1 || seg_steps < 1 || (long long)n_segments * seg_steps > (1 << 24))
        return fail(h, LBEHD_ERR_INVALID_ARG, "need n_segments >= 1, seg_steps >= 1");
    if (h->prof)
        return fail(h, LBEHD_ERR_INVALID_ARG, "disable profiling before an adjoint run");
    return h->dim == 2 ? adjoint_forward<2>(h, V, n_segments, seg_steps, loss)
                       : adjoint_forward<3>(h, V, n_segments, seg_steps, loss);
}

int lbehd_adjoint_get_info(lbehd_handle *h, lbehd_adjoint_info *out)
{
    if (!h || !out)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or output");
    const auto &a = h->adj;
    std::memset(out, 0, sizeof(*out));
    if (a.T == 0)
        return LBEHD_OK;
    out->steps = a.T;
    out->checkpoint_every = a.K;
    out->checkpoints = (a.T + a.K - 1) / a.K;
    out->trajectory = a.ptraj ? 1 : 0;
    out->steps_replayed = a.steps_replayed;
    out->steps_reversed = a.adj_steps;
    out->adjoint_cg_iters = a.adj_iters;
    out->device_bytes = (long long)a.bytes;
    return LBEHD_OK;
}

int lbehd_adjoint_backward(lbehd_handle *h, double *grad)
{
    if (!h || !grad)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null handle or gradient");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: the adjoint is per handle");
    return h->dim == 2 ? adjoint_backward<2>(h, grad) : adjoint_backward<3>(h, grad);
}

int lbehd_autotune(lbehd_handle *h, int reps, double *ms)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: use lbehd_batch_autotune");
    return h->dim == 2 ? autotune_impl<2>(h, reps, ms) : autotune_impl<3>(h, reps, ms);
}

int lbehd_get_stats(lbehd_handle *h, lbehd_stats *out)
{
    if (!h || !out)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null argument");
    CgScalars s0;
    CK(h, cudaMemcpyAsync(&s0, h->cg_s, sizeof(s0), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    out->steps = h->step;
    out->poisson_iters = s0.total_iters;
    out->graph_launches = h->graph_launches;
    out->kernels = h->launches +
                   (h->graph_launches_started ? (s0.total_iters - h->graph_iters0) * h->iter_kernels : 0);
    return LBEHD_OK;
}

int lbehd_profile_enable(lbehd_handle *h, int enable)
{
    if (!h)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null handle");
    if (h->batch_owned)
        return fail(h, LBEHD_ERR_INVALID_ARG, "instance of a batch: profiling is per handle");
    CK(h, cudaStreamSynchronize(h->stream));
    drop_events(h);
    h->prof = enable != 0;
    return LBEHD_OK;
}

int lbehd_profile_read(lbehd_handle *h, double *ms, long long *count)
{
    if (!h || !ms || !count)
        return fail(h, LBEHD_ERR_INVALID_ARG, "null argument");
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < LBEHD_NKC; k++) {
        double acc = 0.0;
        for (auto &e : h->ev_pending[k]) {
            float t = 0.0f;
            CK(h, cudaEventElapsedTime(&t, e.first, e.second));
            acc += t;
        }
        ms[k] = acc;
        count[k] = (long long)h->ev_pending[k].size();
    }
    return LBEHD_OK;
}

const char *lbehd_last_error(lbehd_handle *h)
{
    return h ? h->err.c_str() : g_init_error.c_str();
}

void lbehd_destroy(lbehd_handle *h)
{
    if (h && h->batch_owned)
        return;
    release(h);
    delete h;
}

// ---------------------------------------------------------------- batched form

int lbehd_batch_init(const lbehd_config *cfgs, int n, lbehd_batch **out)
{
    if (!cfgs || !out || n < 1)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null configs or output, or n < 1");
    if (n > BATCH_MAX)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "at most 64 instances per batch");
    *out = nullptr;
    for (int i = 1; i < n; i++)
        if (cfgs[i].dim != cfgs[0].dim)
            return fail(nullptr, LBEHD_ERR_INVALID_ARG, "batch instances must share dim");
    if (cfgs[0].dim != 2 && cfgs[0].dim != 3)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "dim must be 2 or 3");
    lbehd_batch *b = new (std::nothrow) lbehd_batch();
    if (!b)
        return fail(nullptr, LBEHD_ERR_OOM, "host allocation failed");
    b->dim = cfgs[0].dim;
    b->alloc = cfgs[0].alloc;
    b->free = cfgs[0].free;
    b->alloc_ctx = cfgs[0].alloc_ctx;
    b->stream = (cudaStream_t)cfgs[0].stream;
    auto bail = [&](int code, const std::string &msg) {
        batch_release(b);
        delete b;
        return fail(nullptr, code, msg);
    };
    if (!b->stream) {
        if (cudaStreamCreate(&b->own_stream) != cudaSuccess)
            return bail(LBEHD_ERR_CUDA, "cudaStreamCreate failed");
        b->stream = b->own_stream;
    }
    {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        b->cta_cap = 16 * nsm;
    }
    if ((b->dim == 2 ? batch_kernel_attributes<2>() : batch_kernel_attributes<3>()) != LBEHD_OK)
        return bail(LBEHD_ERR_CUDA, "cudaFuncSetAttribute failed for the batched kernels");
    for (int i = 0; i < n; i++) {
        if (cfgs[i].density_model != 0)
            return bail(LBEHD_ERR_INVALID_ARG,
                        "instance " + std::to_string(i) +
                            ": the batched form runs equal densities (density_model 0)");
        lbehd_config c = cfgs[i];
        c.stream = b->stream;
        c.poisson_mode = LBEHD_POISSON_GRAPH;
        lbehd_handle *h = nullptr;
        const int rc = lbehd_init(&c, &h);
        if (rc)
            return bail(rc, "instance " + std::to_string(i) + ": " + g_init_error);
        h->batch_owned = true;
        // whole-level sweeps by default: on the 64-instance sweep they cost fewer CG
        // iterations than the block-local smoother (0.86 against 1.04 per instance-step) and
        // run faster as full-occupancy launches over all instances (2786 against 2465 MLUPS)
        h->mg_smoother = 0;
        // and the start from the increment of step s - 2: on the 64-instance sweep the
        // least-residual start lowers the CG iterations per instance-step from 0.31 to 0.25,
        // but every pass of the batched loop still runs while any instance iterates, and the
        // start's two extra passes over all instances cost more (3186 against 3594 MLUPS)
        h->warm_mode = 0;
        b->inst.push_back(h);
    }
    auto balloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (b->alloc)
            p = b->alloc(bytes, b->alloc_ctx);
        else if (cudaMalloc(&p, bytes) != cudaSuccess)
            p = nullptr;
        return p;
    };
    b->maps = (PopMaps *)balloc(2 * (size_t)n * sizeof(PopMaps));
    b->tails = (TailLevels *)balloc((size_t)n * sizeof(TailLevels));
    b->counters = (int *)balloc(8 * sizeof(int));
    b->act = (ActiveLists *)balloc(sizeof(ActiveLists));
    b->icnt = (unsigned *)balloc(BATCH_MAX * sizeof(unsigned));
    b->wsum = (double *)balloc(BATCH_MAX * 2 * 32 * sizeof(double));
    if (!b->maps || !b->tails || !b->counters || !b->act || !b->icnt || !b->wsum)
        return bail(LBEHD_ERR_OOM, "device allocation of the batch tables failed");
    {
        // shared-memory tails of the instances, with their level's arrays filled in
        std::vector<TailLevels> T(n);
        for (int i = 0; i < n; i++) {
            const lbehd_handle *h = b->inst[i];
            std::memset(&T[i], 0, sizeof(TailLevels));
            if (h->tail_level >= 0) {
                T[i] = h->tail;
                T[i].b0 = h->mg[h->tail_level].b;
                T[i].x0 = h->mg[h->tail_level].x;
                b->tail_smem = std::max(b->tail_smem, h->tail_smem);
            }
        }
        if (cudaMemcpyAsync(b->tails, T.data(), n * sizeof(TailLevels), cudaMemcpyHostToDevice,
                            b->stream) != cudaSuccess ||
            cudaMemsetAsync(b->counters, 0, 8 * sizeof(int), b->stream) != cudaSuccess ||
            cudaMemsetAsync(b->icnt, 0, BATCH_MAX * sizeof(unsigned), b->stream) != cudaSuccess ||
            cudaMemsetAsync(b->act, 0, sizeof(ActiveLists), b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return bail(LBEHD_ERR_CUDA, "upload of the batch tables failed");
        if (cudaFuncSetAttribute(k_mg_tail_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TAIL_SMEM_MAX) != cudaSuccess)
            return bail(LBEHD_ERR_CUDA, "cudaFuncSetAttribute failed for the batched tail");
    }
    if (cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->aux2, cudaStreamNonBlocking) != cudaSuccess)
        return bail(LBEHD_ERR_CUDA, "cudaStreamCreate failed");
    if (cudaMallocHost((void **)&b->h_obs, (size_t)n * (2 * NOBS + 1) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_flags, 8 * sizeof(int)) != cudaSuccess)
        return bail(LBEHD_ERR_OOM, "pinned host allocation failed");
    *out = b;
    return LBEHD_OK;
}

int lbehd_batch_step(lbehd_batch *b, int n)
{
    if (!b)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch");
    if (n < 0)
        return bfail(b, LBEHD_ERR_INVALID_ARG, "n must be >= 0");
    int worst = LBEHD_OK;
    for (int s = 0; s < n; s++) {
        const int rc = b->dim == 2 ? batch_step_one<2>(b) : batch_step_one<3>(b);
        if (rc == LBEHD_ERR_POISSON_NOCONV)
            worst = rc;
        else if (rc)
            return rc;
    }
    if (worst)
        b->err = "Poisson solve reached poisson_max_iter";
    return worst;
}

int lbehd_batch_size(lbehd_batch *b) { return b ? (int)b->inst.size() : 0; }

lbehd_handle *lbehd_batch_instance(lbehd_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->inst.size())
        return nullptr;
    return b->inst[i];
}

int lbehd_batch_observe(lbehd_batch *b, lbehd_obs *out)
{
    if (!b || !out)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch or output");
    const int n = (int)b->inst.size();
    int *flags = reinterpret_cast<int *>(b->h_obs + (size_t)n * 2 * NOBS);
    for (int i = 0; i < n; i++) {
        lbehd_handle *h = b->inst[i];
        if (observe_enqueue(h, b->h_obs + (size_t)i * 2 * NOBS, flags + i))
            return bfail(b, LBEHD_ERR_CUDA, "instance " + std::to_string(i) + ": " + h->err);
    }
    BCK(b, cudaStreamSynchronize(b->stream));
    int worst = LBEHD_OK;
    for (int i = 0; i < n; i++) {
        lbehd_handle *h = b->inst[i];
        const int rc = observe_fill(h, b->h_obs + (size_t)i * 2 * NOBS, flags[i], out + i);
        if (rc) {
            worst = rc;
            b->err = "instance " + std::to_string(i) + ": " + h->err;
        }
    }
    return worst;
}

int lbehd_batch_set_option(lbehd_batch *b, int option, long long value)
{
    if (!b)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch");
    for (size_t i = 0; i < b->inst.size(); i++) {
        const int rc = set_option_impl(b->inst[i], option, value);
        if (rc)
            return bfail(b, rc, "instance " + std::to_string(i) + ": " + b->inst[i]->err);
    }
    drop_batch_graphs(b);
    return LBEHD_OK;
}

int lbehd_batch_autotune(lbehd_batch *b, int reps, int *variants, double *ms)
{
    if (!b)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch");
    for (size_t i = 0; i < b->inst.size(); i++) {
        lbehd_handle *h = b->inst[i];
        const int rc = b->dim == 2 ? autotune_impl<2>(h, reps, ms ? ms + 4 * i : nullptr)
                                   : autotune_impl<3>(h, reps, ms ? ms + 4 * i : nullptr);
        if (rc < 0)
            return bfail(b, rc, "instance " + std::to_string(i) + ": " + h->err);
        if (variants)
            variants[i] = rc;
    }
    drop_batch_graphs(b);
    return LBEHD_OK;
}

int lbehd_batch_get_stats(lbehd_batch *b, lbehd_stats *out)
{
    if (!b || !out)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch or output");
    for (lbehd_handle *h : b->inst)
        BCK(b, cudaMemcpyAsync(h->h_cg, h->cg_s, sizeof(CgScalars), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    std::memset(out, 0, sizeof(*out));
    out->steps = b->inst.empty() ? 0 : b->inst[0]->step;
    out->graph_launches = b->graph_launches;
    out->kernels = b->launches;
    for (lbehd_handle *h : b->inst) {
        out->poisson_iters += h->h_cg->total_iters;
        out->kernels += h->launches;   // eager launches: first step, autotuning
    }
    if (b->graphs_started) {
        // kernels inside the batch graphs' loops and refinement blocks
        int c[6] = {0, 0, 0, 0, 0, 0};
        BCK(b, cudaMemcpyAsync(c, b->counters, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
        BCK(b, cudaStreamSynchronize(b->stream));
        for (int k = 0; k < 3; k++)
            out->kernels += (c[3 + k] - b->counters0[k]) * b->loop_kernels[k];
    }
    return LBEHD_OK;
}

int lbehd_batch_profile_enable(lbehd_batch *b, int enable)
{
    if (!b)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null batch");
    BCK(b, cudaStreamSynchronize(b->stream));
    for (auto &v : b->ev_pending) {
        for (auto &e : v)
            b->ev_pool.push_back(e);
        v.clear();
    }
    b->prof = enable != 0;
    return LBEHD_OK;
}

int lbehd_batch_profile_read(lbehd_batch *b, double *ms, long long *count)
{
    if (!b || !ms || !count)
        return fail(nullptr, LBEHD_ERR_INVALID_ARG, "null argument");
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int k = 0; k < LBEHD_NKC; k++) {
        double acc = 0.0;
        for (auto &e : b->ev_pending[k]) {
            float t = 0.0f;
            BCK(b, cudaEventElapsedTime(&t, e.first, e.second));
            acc += t;
        }
        ms[k] = acc;
        count[k] = (long long)b->ev_pending[k].size();
    }
    return LBEHD_OK;
}

const char *lbehd_batch_last_error(lbehd_batch *b) { return b ? b->err.c_str() : g_init_error.c_str(); }

void lbehd_batch_destroy(lbehd_batch *b)
{
    if (!b)
        return;
    batch_release(b);
    delete b;
}

}  // extern "C"

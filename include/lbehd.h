/*
 * lbehd.h -- C ABI of the B300 (sm_103a) coupled lattice Boltzmann electrohydrodynamics
 * step: ternary conservative phase field (droplet, lubricant, ambient), incompressible
 * momentum, leaky-dielectric charge transport and Gauss law, on micropillar geometry.
 *
 * Method: "Controlling the dynamics of an electric-field-driven droplet on a
 * lubricant-infused micropillar surface", Methods:
 *   conservative Allen-Cahn (Eq. 8), Navier-Stokes with capillary and electric forces
 *   (Eq. 9), ternary chemical potential (Eqs. 10-11), electric force (Eq. 12),
 *   Gauss law (Eq. 13), charge transport (Eq. 14), raw-moment MRT collision of the phase
 *   field (Eqs. 15-19), wetting condition (Eq. 20a), momentum and charge collisions
 *   (Eq. 20b), and the inner Poisson iterations that precede each hydrodynamic step.
 *
 * Conventions for every entry point:
 *  - Return value 0 (LBEHD_OK) on success, a negative LBEHD_ERR_* code otherwise.
 *    No C++ exception crosses this boundary. lbehd_last_error() gives a message.
 *  - Host pointers passed in are borrowed for the duration of the call only.
 *  - Device memory is owned by the handle until lbehd_destroy(); it is obtained from
 *    cfg->alloc/cfg->free when given (e.g. PyTorch's caching allocator), else cudaMalloc.
 *  - All GPU work is enqueued on cfg->stream (a cudaStream_t). For NULL the library creates
 *    its own blocking stream (ordered with the legacy default stream), because graph
 *    capture is not possible on the legacy stream.
 *    lbehd_step() returns after enqueueing, except for the host round trips of the
 *    Poisson convergence test in LBEHD_POISSON_HOST mode. lbehd_observe(),
 *    lbehd_copy_out() and lbehd_destroy() synchronise the stream.
 *  - Lattice: site index i = x + nx * (y + ny * z), x fastest. 2D runs use nz = 1 and the
 *    vertical axis is y; 3D runs use z. All axes are periodic; walls are solid nodes.
 *  - Velocity order (shared with the parity tests): rest first, then each moving
 *    velocity followed by its opposite.
 *      D2Q9 : (0,0) (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1)
 *      D3Q19: (0,0,0) +-x +-y +-z (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *             (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *      D2Q5 / D3Q7 (charge): rest, +-x, +-y (, +-z)
 */
#ifndef LBEHD_H
#define LBEHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBEHD_ABI_VERSION 4

#define LBEHD_OK 0
#define LBEHD_ERR_INVALID_ARG (-1)
#define LBEHD_ERR_OOM (-2)
#define LBEHD_ERR_POISSON_NOCONV (-3) /* step completed, Poisson hit its iteration cap */
#define LBEHD_ERR_NONFINITE (-4)      /* a NaN/Inf appeared in the state, or a bounded device
                                       * wait (shared-memory staging) gave up */
#define LBEHD_ERR_CUDA (-5)
#define LBEHD_ERR_STATE (-6)          /* call not valid in the handle's current state */

#define LBEHD_MAX_ELECTRODES 64

/* Poisson (Eq. 13) solve per step: preconditioned CG on the potential increment, one
 * multigrid V-cycle as preconditioner. Convergence control: */
#define LBEHD_POISSON_HOST 0   /* host reads the FP64 residual every poisson_check_every iterations */
#define LBEHD_POISSON_FIXED 1  /* exactly poisson_fixed_iters iterations, no host round trip */
#define LBEHD_POISSON_GRAPH 2  /* each step after the first replays a CUDA graph whose CG loop
                                * (and one refinement check) runs as device-side conditional
                                * while nodes: no host round trip, convergence to poisson_tol */

/* Solid classes (cfg->solid): 0 fluid, 1 substrate (wetting angles theta_ij apply),
 * 2 neutral wall (all angles 90 degrees). Electrode ids (cfg->electrode_id), meaningful
 * on solid nodes only: -1 zero-flux wall, -2 grounded (phi = 0), k >= 0 electrode k held
 * at electrode_V[k]. */
typedef struct lbehd_config {
    int dim;                 /* 2 (D2Q9 + D2Q5) or 3 (D3Q19 + D3Q7) */
    int nx, ny, nz;          /* lattice extents; nz = 1 in 2D; nx (and ny in 3D) even */
    const uint8_t *solid;    /* host, N solid classes */
    const int16_t *electrode_id; /* host, N ids */
    const double *phi_init;  /* host, 3*N initial Phi_1..3 (droplet, lubricant, ambient) */
    double nu[3];            /* kinematic viscosity per phase; nu = sum Phi_i nu_i */
    double eps[3];           /* permittivity per phase; eps = sum Phi_i eps_i */
    double sigma[3];         /* conductivity per phase; sigma = sum Phi_i sigma_i */
    double gamma12, gamma13, gamma23; /* pairwise surface tensions (Eq. 11) */
    double theta12, theta13, theta23; /* contact angles on class-1 solid, degrees (Eq. 20a) */
    double mobility;         /* M of Eq. 8 (0.0025); tau_Phi = 1/2 + M / c_s^2 */
    double W;                /* interface width (5) */
    double alpha;            /* charge diffusivity of Eq. 14 */
    double body_force[3];    /* uniform body force density added to F */
    double body_force_droplet[3]; /* force density on the droplet phase alone: F gains
                                   * Phi_1 * body_force_droplet (gravity on a droplet much
                                   * denser than its surroundings, the sliding droplet of the
                                   * Methods' validation; zero for the electrically driven
                                   * runs) */
    double s_bulk;           /* relaxation rate of the trace of the momentum flux (1) */
    int density_model;       /* 0: equal densities (the incompressible momentum scheme with the
                              * raw-moment MRT collision); 1: phase densities rho_phase (Table
                              * 1's water / oil / air, Eq. 9 with a variable rho): the momentum
                              * populations carry the gauge pressure p and rho u,
                              * g_eq,n = w_n p/c_s^2 + rho s_n(u) (n > 0),
                              * g_eq,0 = (w_0 - 1) p/c_s^2 + rho s_0(u),
                              * s_n(u) = w_n [e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)],
                              * the force term (e_n - u).[(w_n + s_n) F + s_n c_s^2 grad rho]
                              * / c_s^2, rho = sum Phi_i rho_i, rho u = sum e g + F/2,
                              * p = c_s^2/(1 - w_0) [sum_{n>0} g_n + u.grad(rho)/2 +
                              * rho s_0(u)], one relaxation time tau = 1/2 + nu/c_s^2 (nu is
                              * kinematic). The momentum populations are then stored as g
                              * itself and start at 0 (p = 0, u = 0). Not with the batched
                              * form or the adjoint (LBEHD_ERR_INVALID_ARG). */
    double rho_phase[3];     /* phase densities rho_i (density_model 1; all > 0) */
    double poisson_tol;      /* relative residual ||b - A phi||_2 / ||b||_2 to stop at */
    int poisson_max_iter;    /* cap on preconditioned-CG iterations per step */
    int poisson_mode;        /* LBEHD_POISSON_HOST or LBEHD_POISSON_FIXED */
    int poisson_check_every; /* iterations between host convergence checks (HOST mode) */
    int poisson_fixed_iters; /* iterations per step in LBEHD_POISSON_FIXED */
    int mg_nu;               /* red-black pre/post smoothing sweep pairs per level
                              * (0 -> 2; with the block-local smoother of
                              * LBEHD_OPT_MG_SMOOTHER, pairs per block, 0 -> 3) */
    int mg_coarse_sweeps;    /* symmetric sweep pairs on the coarsest level (0 -> 8) */
    int mg_max_levels;       /* multigrid levels (0 -> as many as the extents allow) */
    double mg_scale;         /* scale of the Galerkin coarse operators (0 -> 0.6) */
    int n_electrodes;
    const double *electrode_V; /* host, n_electrodes initial potentials */
    void *(*alloc)(size_t bytes, void *ctx); /* optional device allocator */
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
    void *stream;            /* cudaStream_t */
} lbehd_config;

/* Droplet observables of the last completed step (FP64 sums over fluid nodes of the
 * fields computed in that step). */
typedef struct lbehd_obs {
    long long step;          /* index of the step the fields belong to */
    double M1;               /* sum Phi_1 (droplet volume) */
    double centroid[3];      /* sum Phi_1 x / M1 */
    double velocity[3];      /* sum Phi_1 u / M1 */
    double f_ele[3];         /* electric force on the droplet, sum Phi_1 F_e */
    double f_ele_total[3];   /* sum F_e over the fluid */
    double f_drag[3];        /* drag from the force balance (Results, Eqs. 1 and 5): the
                              * driving force on the droplet minus its inertia,
                              * f_ele + M1 (body_force + body_force_droplet) - M1 (V^n - V^{n-1})
                              * (unit density, m = M1), with the body forces in effect when
                              * lbehd_observe is called; -M1 dV/dt for an undriven droplet */
    double mass[3];          /* sum Phi_i, per component */
    double charge;           /* sum rho_e */
    int poisson_iters;       /* CG iterations of the last step's Poisson solve */
    double poisson_resid;    /* its final relative residual */
    int status;              /* LBEHD_OK or the first error code recorded */
} lbehd_obs;

typedef struct lbehd_handle lbehd_handle;

/* Arrays that lbehd_copy_out / lbehd_device_ptr can reach. Populations are the
 * pre-collision state at the current time; fields are those computed in the last step.
 * FP32 throughout. Layouts (N = nx*ny*nz, Q = 9/19, QS = 5/7):
 *   LBEHD_G     Q*N     momentum populations stored SHIFTED: g_n - w_n
 *   LBEHD_FPHI  3*Q*N   phase-field populations [component][velocity][site]
 *   LBEHD_FRHO  QS*N    charge populations
 *   LBEHD_PHI   3*N     Phi_1..3 (boundary solid nodes hold the wetting ghosts)
 *   LBEHD_RHO   N       rho_e
 *   LBEHD_POT   N       electric potential, high part (Dirichlet nodes hold their value)
 *   LBEHD_U     3*N     velocity u = j + F/2
 *   LBEHD_QSRC  N       conduction source div(sigma grad phi)
 *   LBEHD_EPS   N       permittivity
 *   LBEHD_POT_LO N      low part of the potential: phi = POT + POT_LO (compensated pair) */
enum lbehd_array {
    LBEHD_G = 0, LBEHD_FPHI, LBEHD_FRHO, LBEHD_PHI, LBEHD_RHO, LBEHD_POT, LBEHD_U,
    LBEHD_QSRC, LBEHD_EPS, LBEHD_POT_LO, LBEHD_NARRAYS
};

/* ABI version and sizeof(lbehd_config), for binding checks. */
int lbehd_abi_version(void);
size_t lbehd_config_size(void);

/* Validate cfg, build the geometry tables (node classes, wetting normals), allocate the
 * state and set the populations to equilibrium with u = 0, p = 1, rho_e = 0 and
 * Phi = cfg->phi_init. Writes the new handle to *out. */
int lbehd_init(const lbehd_config *cfg, lbehd_handle **out);

/* Advance n >= 0 coupled steps: phase moments and wetting ghosts, Poisson solve, forces,
 * fused collide + push-stream of the momentum, three phase-field and charge populations,
 * block partial sums of the observables. Returns LBEHD_ERR_POISSON_NOCONV if any solve hit
 * the cap (the steps are still completed). */
int lbehd_step(lbehd_handle *h, int n);

/* Set the electrode potentials used from the next step on (Dirichlet values of the
 * Gauss law; the programmable switching of the Results). n must equal cfg->n_electrodes. */
int lbehd_set_electrodes(lbehd_handle *h, const double *V, int n);

/* Set the uniform and the droplet-phase body force densities (3 components each, as
 * cfg->body_force and cfg->body_force_droplet) used from the next step on: the sliding and
 * deceleration runs switch the drive on and off. Either pointer may be NULL to keep that
 * force. Synchronises the stream and discards captured step graphs (the next step captures
 * them again). A recorded adjoint run is dropped (its replays would no longer match).
 * Errors: LBEHD_ERR_INVALID_ARG (null handle, non-finite value, instance of a batch). */
int lbehd_set_body_force(lbehd_handle *h, const double *body, const double *body_droplet);

/* Sum the last two steps' observable partials on the device (fixed order, FP64; the drag
 * force uses both), synchronise the stream and fill *out with the last step's observables.
 * Returns LBEHD_ERR_NONFINITE if a non-finite value was detected. */
int lbehd_observe(lbehd_handle *h, lbehd_obs *out);

/* Copy one array (enum lbehd_array) to host memory dst of at least *bytes; synchronises. */
int lbehd_copy_out(lbehd_handle *h, int which, void *dst, size_t bytes);

/* Device pointer and size in bytes of one array (valid until the next lbehd_step). */
int lbehd_device_ptr(lbehd_handle *h, int which, void **ptr, size_t *bytes);

/* Implementation options (synchronises; discards captured step graphs).
 *   LBEHD_OPT_COLLIDE: which fused collide kernel runs: 0 automatic (2 when nx % 4 == 0,
 *   else 1), 1 populations and stencil fields loaded straight from global memory (128-site
 *   row blocks), 2 / 3 / 4 tile staged into shared memory (populations by TMA tensor copies,
 *   stencil halo by cooperative loads) on 32x4 / 64x2 / 16x8 tiles (needs nx % 4 == 0).
 *   All give the same arithmetic. */
#define LBEHD_OPT_COLLIDE 1
/*   LBEHD_OPT_MG_REFRESH: rebuild the multigrid hierarchy (the Poisson preconditioner)
 *   every `value` steps (default 16). The CG operator itself is formed from this step's
 *   permittivity every step, so the refresh period only affects convergence speed. */
#define LBEHD_OPT_MG_REFRESH 2
/*   LBEHD_OPT_ADJ_TRAJECTORY: 1 (default) lbehd_adjoint_forward records every step's
 *   potential (8 bytes per site per step) when the allocation succeeds, so that the
 *   backward replays need no Gauss-law solve; 0 never records it (replays solve again and
 *   reproduce the same potential bit for bit). */
#define LBEHD_OPT_ADJ_TRAJECTORY 3
/*   LBEHD_OPT_POISSON_KERNEL: 1 (default) in LBEHD_POISSON_GRAPH mode each Gauss-law solve
 *   is one launch that forms the start residual, then one persistent cooperative kernel with
 *   grid-wide barriers (CG iterations with their V-cycles, potential update, refinement
 *   pass), where the lattice allows it (a shared-memory tail level, even nx on the levels
 *   above it); 0 the multi-launch graph with conditional nodes. Both give the same bits. */
#define LBEHD_OPT_POISSON_KERNEL 4
/*   LBEHD_OPT_BARRIER_TEST: test hook for the persistent solve's time-out path. value > 0:
 *   its grid barriers wait for one CTA more than is launched and give up after `value`
 *   polls, so every solve times out; each CTA leaves at its next barrier, the kernel ends and
 *   the next lbehd_observe returns LBEHD_ERR_CUDA ("grid barrier timed out"). The error is
 *   sticky for the handle. 0 (default): normal barriers. */
#define LBEHD_OPT_BARRIER_TEST 5
/*   LBEHD_OPT_MG_SMOOTHER: the smoother of the multigrid preconditioner on the levels above
 *   the shared-memory tail. 1 (default where the lattice has such levels): block-local,
 *   block-Jacobi between blocks of 16x8x8 (2D: 32x32) cells, red-black Gauss-Seidel sweeps
 *   within a block against its halo as it was when the pass began (mg_nu pairs per pass,
 *   default 3); one grid-wide dependency per level and direction of a V-cycle. 0:
 *   red-black Gauss-Seidel half sweeps over whole levels (mg_nu pairs, default 2). Both are
 *   symmetric, so CG converges to the same tolerance with either; the solutions differ
 *   within it. The persistent, the multi-launch and the batched solves give the same bits
 *   for either value: a batch instance with the same setting as a single handle steps bit
 *   for bit like it. A batch starts with 0 (lbehd_batch_set_option changes it for every
 *   instance). */
#define LBEHD_OPT_MG_SMOOTHER 6
/*   LBEHD_OPT_WARM_START: the start of each step's Gauss-law solve (Eq. 13). 1 (a handle's
 *   default): x0 = a1 d1 + a2 d2 from the increments of the last two steps, with (a1, a2)
 *   minimising the residual ||b - A (phi + x0)||_2 over their span (a 2 x 2 least-squares
 *   system from one extra pass over the lattice: A d1, A d2 and five dot products). 0: x0 =
 *   d2, the increment of two steps back (the increments of consecutive steps alternate in
 *   sign). Both stop at the same tolerance; the solutions differ within it. On the 128x64x64
 *   droplet in steady state, 86 % of the steps then converge on their start alone against
 *   74 %. The persistent, the multi-launch and the batched solves give the same bits for
 *   either value. A batch starts with 0 (on the 64-instance sweep 1 lowers the CG
 *   iterations per instance-step from 0.31 to 0.25 but runs at 3186 against 3594 MLUPS: the
 *   batched CG loop runs while any instance iterates, and the start's extra passes cover
 *   all of them); lbehd_batch_set_option changes it for every instance. */
#define LBEHD_OPT_WARM_START 7
int lbehd_set_option(lbehd_handle *h, int option, long long value);
/* The value in effect: for LBEHD_OPT_COLLIDE the kernel the automatic choice resolved to,
 * for LBEHD_OPT_POISSON_KERNEL and LBEHD_OPT_MG_SMOOTHER 1 only if the option is on and this
 * lattice allows it. Errors: LBEHD_ERR_INVALID_ARG (unknown option, null output). */
int lbehd_get_option(lbehd_handle *h, int option, long long *value);

/* Counters since init (synchronises: reads the device-side iteration counter). */
typedef struct lbehd_stats {
    long long steps;          /* coupled steps taken */
    long long poisson_iters;  /* preconditioned-CG iterations, all steps and passes */
    long long graph_launches; /* step graphs replayed (LBEHD_POISSON_GRAPH) */
    long long kernels;        /* kernels launched, as lbehd_launch_count() */
} lbehd_stats;
int lbehd_get_stats(lbehd_handle *h, lbehd_stats *out);

/* Number of kernels launched by this handle since init (for launch accounting; kernels run
 * inside graph replays are counted from the device-side iteration counter; synchronises). */
long long lbehd_launch_count(lbehd_handle *h);

/* Per-kernel device time, for roofline accounting: while profiling is enabled every
 * launch of the handle is bracketed by CUDA events recorded on cfg->stream. Kernel
 * classes: */
#define LBEHD_KC_FIELDS 0   /* moments + wetting ghosts */
#define LBEHD_KC_MG 1       /* multigrid setup, smoothing and transfers */
#define LBEHD_KC_CG 2       /* CG vector kernels, reductions and the increment update */
#define LBEHD_KC_COLLIDE 3  /* fused forces + collide + stream of all populations */
#define LBEHD_KC_OBS 4      /* observable reduction */
#define LBEHD_NKC 5

/* Start (enable != 0) or stop recording. Enabling clears earlier records. While profiling,
 * steps run as eager launches even in LBEHD_POISSON_GRAPH mode. */
int lbehd_profile_enable(lbehd_handle *h, int enable);

/* Synchronise and return, per kernel class, the summed device time in ms (ms[LBEHD_NKC])
 * and the number of launches (count[LBEHD_NKC]) recorded since profiling was enabled. */
int lbehd_profile_read(lbehd_handle *h, double *ms, long long *count);

/* Droplet phase moments of caller-owned device fields, computed without allocating any
 * device memory. The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate, such as a host program that hands out all device memory
 * from its own pre-sized pool (an allocation behind its back could fail or fragment the
 * pool) or a framework that calls foreign kernels where it forbids allocation.
 * Inputs (device, FP32, site index i = x + nx (y + ny z)): phi = 3*N values Phi_1..3,
 * u = 3*N velocity components, solid = N solid classes (0 = fluid; only fluid sites count).
 * Output (device, written asynchronously on `stream`): out[10] = M1 = sum Phi_1,
 * centroid[3] = sum Phi_1 x / M1, velocity[3] = sum Phi_1 u / M1, mass[3] = sum Phi_i,
 * the quantities lbehd_observe reports for the droplet.
 * Scratch: the per-block partial sums live in one file-scope __device__ array of
 * 2048 x 9 doubles (144 KB), which every GPU that loads the library holds until the
 * process exits. This caps the lattice at 2048 x 8192 = 16 777 216 sites; larger lattices
 * are rejected with LBEHD_ERR_INVALID_ARG. The first call on a device (and the first after a
 * device reset, which gives the device a new context) looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call before any stream
 * capture. Every call overwrites the partials it reads, so nothing needs clearing, but all
 * calls share the array: calls whose kernels overlap on the GPU (other streams, other
 * threads) race and must be serialised by the caller.
 * Errors: LBEHD_ERR_INVALID_ARG (bad extents, null pointer, too large), LBEHD_ERR_CUDA (also
 * when a CUDA error from the caller's earlier work is still pending; it is left in place);
 * the message is in lbehd_last_error(NULL). */
int lbehd_phase_moments_noalloc(int dim, int nx, int ny, int nz, const float *phi,
                                const float *u, const uint8_t *solid, double *out, void *stream);

/* Collide-kernel autotuner. Times each collide kernel the instance can run (1 global
 * loads; 2, 3, 4 staged 32x4, 64x2, 16x8 tiles when nx % 4 == 0) on the current state,
 * `reps` launches each after two untimed ones, keeps the fastest as LBEHD_OPT_COLLIDE and
 * writes the mean time per launch in ms to ms[v - 1] (ms[4], -1 for a kernel that cannot
 * run; may be NULL). The state is left as it was: the timed launches write only the
 * buffers the next step overwrites first, and u, the conduction source and the error flag
 * are saved and restored around them. Synchronises; discards captured step graphs. Returns
 * the chosen variant (>= 1) or a negative error code. Must not be called on an instance
 * owned by a batch (use lbehd_batch_autotune). */
int lbehd_autotune(lbehd_handle *h, int reps, double *ms);

/* ---------------------------------------------------------------- discrete adjoint
 * Gradients of the droplet's x centroid after a run with respect to the electrode
 * potentials, which are piecewise constant in time (the programmable switching of the
 * Results): V[k * n_electrodes + e] is electrode e's potential during segment k, which
 * lasts seg_steps steps.
 *
 * lbehd_adjoint_forward runs the n_segments * seg_steps steps from the handle's current state
 * (as lbehd_step would, the potentials set segment by segment). On the way it keeps the state
 * every K ~ sqrt(steps) steps (K a multiple of 16) in device memory, and (see
 * LBEHD_OPT_ADJ_TRAJECTORY) the potential of every step. It returns the loss
 * L = sum Phi_1 x / sum Phi_1 over the fluid nodes after the last step (the x centroid
 * lbehd_observe reports). The handle is left after the last step.
 *
 * lbehd_adjoint_backward returns grad[k * n_electrodes + e] = dL/dV[k][e], the discrete
 * adjoint of the recorded run. It replays one checkpoint interval at a time (moments and
 * collide with the recorded potential, or whole steps without a recorded trajectory),
 * keeping every step's input state, and runs the reversed steps: the reverse of the fused
 * collide kernel, the gather of the stencils' adjoints, one adjoint Gauss-law solve with the
 * same symmetric operator (preconditioned CG), the reverse of the moments and wetting ghosts,
 * and the per-electrode sums. The first step of a fresh handle has no backward differences
 * and contributes none. Afterwards the handle is again in the state after the last step.
 * Memory: (ceil(steps / K) + K + 1) saved states of (4 Q + Q_s + 13) floats per site, plus
 * 2 floats per site per step for the recorded potential.
 * Synchronise. Errors: LBEHD_ERR_INVALID_ARG (no recorded run, bad sizes, batch instance),
 * LBEHD_ERR_OOM, LBEHD_ERR_CUDA; LBEHD_ERR_POISSON_NOCONV from the forward is reported but
 * the run completes. */
int lbehd_adjoint_forward(lbehd_handle *h, const double *V, int n_segments, int seg_steps,
                          double *loss);
int lbehd_adjoint_backward(lbehd_handle *h, double *grad);

/* The recorded adjoint run: its steps, checkpoint spacing K and count, whether every step's
 * potential was recorded, the steps replayed and reversed by the last backward pass, the
 * adjoint CG iterations it took, and the device bytes the adjoint holds (checkpoints,
 * replay slots, trajectory, work arrays). All zero before the first forward run. */
typedef struct lbehd_adjoint_info {
    long long steps, checkpoint_every, checkpoints, trajectory;
    long long steps_replayed, steps_reversed, adjoint_cg_iters, device_bytes;
} lbehd_adjoint_info;
int lbehd_adjoint_get_info(lbehd_handle *h, lbehd_adjoint_info *out);

/* ---------------------------------------------------------------- checkpoint / restore
 * A handle's whole state in one caller-owned device buffer of lbehd_state_bytes(h) bytes
 * (16-byte aligned): a 1 KiB header (lattice extents, step counter and parities, electrode
 * potentials, the last two steps' observable sums), then per site the populations,
 * Phi^{n-1}, rho^{n-1}, u^{n-1}, Q^{n-1}, the potential pair, both warm-start increments
 * and the permittivity the multigrid preconditioner was last built from (4 Q + Q_s + 13
 * floats per site). lbehd_load_state into a handle of the same lattice and configuration
 * continues the saved run bit for bit (the preconditioner is rebuilt from the saved
 * permittivity). Both synchronise the handle's stream. Errors: LBEHD_ERR_INVALID_ARG (null
 * or unaligned buffer, batch instance, a buffer that is not a state of this lattice),
 * LBEHD_ERR_CUDA. The paper's runs are long; this is the restart point of one. */
size_t lbehd_state_bytes(lbehd_handle *h);
int lbehd_save_state(lbehd_handle *h, void *dst_device);
int lbehd_load_state(lbehd_handle *h, const void *src_device);

/* Message of the last error on this handle (or of the last failed init when h is NULL). */
const char *lbehd_last_error(lbehd_handle *h);

/* Free every device buffer (through cfg->free when given) and the handle. A handle owned
 * by a batch is left alone (lbehd_batch_destroy frees it). */
void lbehd_destroy(lbehd_handle *h);

/* ---------------------------------------------------------------- batched form
 * Many independent instances of the coupled step (a sweep over lubricant viscosity,
 * wettability and field strength on lattices of different sizes) advanced together, one
 * CUDA graph launch per step for the whole batch. In each step graph the moments kernel and
 * the collide kernels are each one launch over all instances (an instance table in the
 * kernel parameters; instances grouped by their collide kernel, up to 64 per launch), while
 * every instance's Poisson solve runs as its own branch with its own device-side CG loop,
 * so instances that converge in fewer iterations never wait for the others. Each instance
 * computes exactly what lbehd_step computes for it alone in LBEHD_POISSON_GRAPH mode with
 * the same LBEHD_OPT_COLLIDE and LBEHD_OPT_MG_REFRESH (bitwise on the state).
 * All instances must have the same dim; they share one stream (cfgs[0].stream, or a
 * stream the batch creates when that is NULL) and run in LBEHD_POISSON_GRAPH mode whatever
 * cfgs[i].poisson_mode says. */
typedef struct lbehd_batch lbehd_batch;

/* Initialise 1 <= n <= 64 instances from cfgs[0..n) (each as lbehd_init would; host arrays
 * are borrowed for the call). On failure nothing is left allocated and the message is in
 * lbehd_last_error(NULL). */
int lbehd_batch_init(const lbehd_config *cfgs, int n, lbehd_batch **out);

/* Advance every instance by n steps (the first step of a fresh batch runs instance by
 * instance; from then on one graph launch per step). Asynchronous; returns
 * LBEHD_ERR_POISSON_NOCONV if a host-checked solve hit its cap. */
int lbehd_batch_step(lbehd_batch *b, int n);

/* Number of instances, and instance i (0 <= i < n; NULL otherwise). The instance handle is
 * borrowed: lbehd_observe, lbehd_copy_out, lbehd_device_ptr, lbehd_set_electrodes,
 * lbehd_get_stats and lbehd_last_error work on it; lbehd_step, lbehd_set_option,
 * lbehd_autotune and lbehd_profile_enable are refused with LBEHD_ERR_INVALID_ARG. */
int lbehd_batch_size(lbehd_batch *b);
lbehd_handle *lbehd_batch_instance(lbehd_batch *b, int i);

/* Observables of every instance (out[n]) with one synchronisation. Returns
 * LBEHD_ERR_NONFINITE if any instance saw a non-finite value (its out[i].status says so). */
int lbehd_batch_observe(lbehd_batch *b, lbehd_obs *out);

/* Options for every instance (LBEHD_OPT_COLLIDE, LBEHD_OPT_MG_REFRESH as for one handle). */
int lbehd_batch_set_option(lbehd_batch *b, int option, long long value);

/* Run lbehd_autotune on every instance: each gets the collide kernel that is fastest for
 * its own lattice (ragged tiles, solid fraction), and the batched collide launches are
 * regrouped accordingly. variants[n] (may be NULL) receives the choices and ms[4 n] (may be
 * NULL) the timings. Synchronises. */
int lbehd_batch_autotune(lbehd_batch *b, int reps, int *variants, double *ms);

/* Counters of the whole batch: steps (per instance), Poisson iterations and kernels summed
 * over instances, graph_launches = batch step graphs launched. Synchronises. */
int lbehd_batch_get_stats(lbehd_batch *b, lbehd_stats *out);

/* Per-kernel device time of the batch, as lbehd_profile_enable / lbehd_profile_read for one
 * handle: while enabled, batch steps run as eager launches (the same kernels as the step
 * graph, the loop conditions read back by the host) bracketed by CUDA events. */
int lbehd_batch_profile_enable(lbehd_batch *b, int enable);
int lbehd_batch_profile_read(lbehd_batch *b, double *ms, long long *count);

/* Message of the batch's last error. */
const char *lbehd_batch_last_error(lbehd_batch *b);

/* Free every instance and the batch. */
void lbehd_batch_destroy(lbehd_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LBEHD_H */

"""Python binding of the C ABI in include/lbehd.h (argument marshalling only).

Every step of the method runs in the CUDA library ``liblbehd.so`` built next to this file
for sm_103a. There is no CPU fallback: if the library is missing, loading it raises.
PyTorch supplies device memory (its caching allocator, through the ABI's allocator hooks)
and the CUDA stream the library enqueues on.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbehd.so")

# enum lbehd_array
G, FPHI, FRHO, PHI, RHO, POT, U, QSRC, EPS, POT_LO = range(10)
ARRAY_NAMES = {"g": G, "fphi": FPHI, "frho": FRHO, "phi": PHI, "rho": RHO, "pot": POT,
               "u": U, "qsrc": QSRC, "eps": EPS, "pot_lo": POT_LO}
POISSON_HOST, POISSON_FIXED, POISSON_GRAPH = 0, 1, 2
OPT_COLLIDE, OPT_MG_REFRESH, OPT_ADJ_TRAJECTORY, OPT_POISSON_KERNEL, OPT_BARRIER_TEST = 1, 2, 3, 4, 5
OPT_MG_SMOOTHER = 6
OPT_WARM_START = 7
COLLIDE_AUTO, COLLIDE_GLOBAL, COLLIDE_STAGED = 0, 1, 2
COLLIDE_STAGED_64x2, COLLIDE_STAGED_16x8 = 3, 4

# Storage convention of LBEHD_G: the library keeps g_n - w_n (lattice weights in the
# documented velocity order).
STORAGE_SHIFT = {
    2: np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4),
    3: np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12),
}

ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "POISSON_NOCONV", -4: "NONFINITE", -5: "CUDA",
          -6: "STATE"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_D3 = ctypes.c_double * 3


class Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int),
                ("solid", ctypes.POINTER(ctypes.c_uint8)),
                ("electrode_id", ctypes.POINTER(ctypes.c_int16)),
                ("phi_init", ctypes.POINTER(ctypes.c_double)),
                ("nu", _D3), ("eps", _D3), ("sigma", _D3),
                ("gamma12", ctypes.c_double), ("gamma13", ctypes.c_double),
                ("gamma23", ctypes.c_double),
                ("theta12", ctypes.c_double), ("theta13", ctypes.c_double),
                ("theta23", ctypes.c_double),
                ("mobility", ctypes.c_double), ("W", ctypes.c_double), ("alpha", ctypes.c_double),
                ("body_force", _D3), ("body_force_droplet", _D3), ("s_bulk", ctypes.c_double),
                ("density_model", ctypes.c_int), ("rho_phase", _D3),
                ("poisson_tol", ctypes.c_double), ("poisson_max_iter", ctypes.c_int),
                ("poisson_mode", ctypes.c_int), ("poisson_check_every", ctypes.c_int),
                ("poisson_fixed_iters", ctypes.c_int), ("mg_nu", ctypes.c_int),
                ("mg_coarse_sweeps", ctypes.c_int), ("mg_max_levels", ctypes.c_int),
                ("mg_scale", ctypes.c_double),
                ("n_electrodes", ctypes.c_int),
                ("electrode_V", ctypes.POINTER(ctypes.c_double)),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("stream", ctypes.c_void_p)]


class Obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("M1", ctypes.c_double), ("centroid", _D3),
                ("velocity", _D3), ("f_ele", _D3), ("f_ele_total", _D3), ("f_drag", _D3),
                ("mass", _D3), ("charge", ctypes.c_double), ("poisson_iters", ctypes.c_int),
                ("poisson_resid", ctypes.c_double), ("status", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("poisson_iters", ctypes.c_longlong),
                ("graph_launches", ctypes.c_longlong), ("kernels", ctypes.c_longlong)]


class AdjointInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_longlong) for k in (
        "steps", "checkpoint_every", "checkpoints", "trajectory", "steps_replayed",
        "steps_reversed", "adjoint_cg_iters", "device_bytes")]


class LBEHDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbehd error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


_lib = None

EXPORTS = ("lbehd_abi_version", "lbehd_config_size", "lbehd_init", "lbehd_step",
           "lbehd_set_electrodes", "lbehd_set_body_force", "lbehd_observe", "lbehd_copy_out",
           "lbehd_device_ptr",
           "lbehd_launch_count", "lbehd_set_option", "lbehd_get_option", "lbehd_get_stats", "lbehd_profile_enable",
           "lbehd_profile_read", "lbehd_autotune", "lbehd_adjoint_forward",
           "lbehd_adjoint_backward", "lbehd_adjoint_get_info", "lbehd_state_bytes",
           "lbehd_save_state", "lbehd_load_state", "lbehd_last_error",
           "lbehd_destroy",
           "lbehd_batch_init", "lbehd_batch_step", "lbehd_batch_size", "lbehd_batch_instance",
           "lbehd_batch_observe", "lbehd_batch_set_option", "lbehd_batch_autotune",
           "lbehd_batch_get_stats", "lbehd_batch_profile_enable", "lbehd_batch_profile_read",
           "lbehd_batch_last_error", "lbehd_batch_destroy")
KERNEL_CLASSES = ("fields", "mg", "cg", "collide", "obs")


def load():
    """Load liblbehd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; build it with "
                           "`python -m paper_2608_12868_b300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    lib.lbehd_abi_version.restype = ctypes.c_int
    lib.lbehd_config_size.restype = ctypes.c_size_t
    lib.lbehd_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(P)]
    lib.lbehd_step.argtypes = [P, ctypes.c_int]
    lib.lbehd_set_electrodes.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.lbehd_set_body_force.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.lbehd_observe.argtypes = [P, ctypes.POINTER(Obs)]
    lib.lbehd_copy_out.argtypes = [P, ctypes.c_int, P, ctypes.c_size_t]
    lib.lbehd_device_ptr.argtypes = [P, ctypes.c_int, ctypes.POINTER(P),
                                     ctypes.POINTER(ctypes.c_size_t)]
    lib.lbehd_launch_count.argtypes = [P]
    lib.lbehd_launch_count.restype = ctypes.c_longlong
    lib.lbehd_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.lbehd_set_option.argtypes = [P, ctypes.c_int, ctypes.c_longlong]
    lib.lbehd_get_option.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    lib.lbehd_profile_enable.argtypes = [P, ctypes.c_int]
    lib.lbehd_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
    lib.lbehd_last_error.argtypes = [P]
    lib.lbehd_last_error.restype = ctypes.c_char_p
    lib.lbehd_destroy.argtypes = [P]
    lib.lbehd_destroy.restype = None
    lib.lbehd_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.lbehd_adjoint_forward.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.lbehd_adjoint_backward.argtypes = [P, ctypes.POINTER(ctypes.c_double)]
    lib.lbehd_adjoint_get_info.argtypes = [P, ctypes.POINTER(AdjointInfo)]
    lib.lbehd_state_bytes.argtypes = [P]
    lib.lbehd_state_bytes.restype = ctypes.c_size_t
    lib.lbehd_save_state.argtypes = [P, P]
    lib.lbehd_load_state.argtypes = [P, P]
    lib.lbehd_batch_init.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(P)]
    lib.lbehd_batch_step.argtypes = [P, ctypes.c_int]
    lib.lbehd_batch_size.argtypes = [P]
    lib.lbehd_batch_instance.argtypes = [P, ctypes.c_int]
    lib.lbehd_batch_instance.restype = P
    lib.lbehd_batch_observe.argtypes = [P, ctypes.POINTER(Obs)]
    lib.lbehd_batch_set_option.argtypes = [P, ctypes.c_int, ctypes.c_longlong]
    lib.lbehd_batch_autotune.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.lbehd_batch_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
    lib.lbehd_batch_profile_enable.argtypes = [P, ctypes.c_int]
    lib.lbehd_batch_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_longlong)]
    lib.lbehd_batch_last_error.argtypes = [P]
    lib.lbehd_batch_last_error.restype = ctypes.c_char_p
    lib.lbehd_batch_destroy.argtypes = [P]
    lib.lbehd_batch_destroy.restype = None
    if lib.lbehd_config_size() != ctypes.sizeof(Config):
        raise RuntimeError("lbehd_config layout mismatch between the binding and the library")
    _lib = lib
    return lib


def _dptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _obs_dict(o):
    return {
        "step": o.step, "M1": o.M1, "centroid": np.array(o.centroid[:]),
        "velocity": np.array(o.velocity[:]), "f_ele": np.array(o.f_ele[:]),
        "f_ele_total": np.array(o.f_ele_total[:]), "f_drag": np.array(o.f_drag[:]),
        "mass": np.array(o.mass[:]), "charge": o.charge, "poisson_iters": o.poisson_iters,
        "poisson_resid": o.poisson_resid, "status": o.status,
    }


def make_config(w, c, *, poisson_mode=POISSON_HOST, poisson_check_every=1, poisson_fixed_iters=2,
                mg_nu=0, mg_coarse_sweeps=0, mg_max_levels=0, mg_scale=0.0):
    """Fill Config ``c`` from a ``workloads.Workload``; returns the host arrays it points
    to (keep them alive until the init call returns)."""
    nz, ny, nx = w.shape
    p = w.params
    solid = np.ascontiguousarray(w.solid, dtype=np.uint8).reshape(-1)
    elec = np.ascontiguousarray(w.elec, dtype=np.int16).reshape(-1)
    phi = np.ascontiguousarray(w.phi_init, dtype=np.float64).reshape(-1)
    V = np.ascontiguousarray(p.get("V", []), dtype=np.float64)
    c.dim, c.nx, c.ny, c.nz = w.dim, nx, ny, nz
    c.solid, c.electrode_id, c.phi_init = (_dptr(solid, ctypes.c_uint8),
                                           _dptr(elec, ctypes.c_int16),
                                           _dptr(phi, ctypes.c_double))
    for k in range(3):
        c.nu[k], c.eps[k], c.sigma[k] = p["nu"][k], p["eps"][k], p["sig"][k]
        c.body_force[k] = p.get("body", (0.0, 0.0, 0.0))[k]
        c.body_force_droplet[k] = p.get("body_droplet", (0.0, 0.0, 0.0))[k]
    c.gamma12, c.gamma13, c.gamma23 = p["gamma12"], p["gamma13"], p["gamma23"]
    c.theta12, c.theta13, c.theta23 = p["theta12"], p["theta13"], p["theta23"]
    c.mobility, c.W, c.alpha = p["mobility"], p["W"], p["alpha"]
    c.s_bulk = p.get("s_bulk", 1.0)
    c.density_model = int(p.get("density_model", 0))
    for k in range(3):
        c.rho_phase[k] = p.get("rho_phase", (1.0, 1.0, 1.0))[k]
    c.poisson_tol = p.get("poisson_tol", 1e-7)
    c.poisson_max_iter = int(p.get("poisson_max_iter", 100))
    c.poisson_check_every = int(poisson_check_every)
    c.poisson_mode = int(poisson_mode)
    c.poisson_fixed_iters = int(poisson_fixed_iters)
    c.mg_nu, c.mg_coarse_sweeps = int(mg_nu), int(mg_coarse_sweeps)
    c.mg_max_levels, c.mg_scale = int(mg_max_levels), float(mg_scale)
    c.n_electrodes = len(V)
    c.electrode_V = _dptr(V, ctypes.c_double) if len(V) else None
    return (solid, elec, phi, V)


def _torch_allocator(torch, device, stream):
    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=device, stream=stream)
        except torch.cuda.OutOfMemoryError:
            return 0   # the library reports LBEHD_ERR_OOM (or takes its low-memory path)

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(_alloc), FREE_FN(_free)


class _HandleOps:
    """Calls on one lbehd_handle (a Simulation, or one instance of a Batch)."""

    def _setup_shape(self, w):
        self.workload = w
        self.dim, self.shape = w.dim, tuple(w.shape)
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.Q, self.QS = (9, 5) if w.dim == 2 else (19, 7)
        self.n_electrodes = len(w.params.get("V", []))

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise LBEHDError(rc, self._lib.lbehd_last_error(self._h).decode())
        return rc

    def set_electrodes(self, V):
        V = np.ascontiguousarray(V, dtype=np.float64)
        self._check(self._lib.lbehd_set_electrodes(self._h, _dptr(V, ctypes.c_double), len(V)))

    def observe(self):
        o = Obs()
        self._check(self._lib.lbehd_observe(self._h, ctypes.byref(o)))
        return _obs_dict(o)

    def _shape_of(self, which):
        nz, ny, nx = self.shape
        return {G: (self.Q,), FPHI: (3, self.Q), FRHO: (self.QS,), PHI: (3,), RHO: (), POT: (),
                U: (3,), QSRC: (), EPS: (), POT_LO: ()}[which] + (nz, ny, nx)

    def array(self, which):
        """Host copy (float32 numpy) of one array; ``which`` is a name or an enum value."""
        which = ARRAY_NAMES.get(which, which)
        out = np.empty(self._shape_of(which), dtype=np.float32)
        self._check(self._lib.lbehd_copy_out(self._h, which, out.ctypes.data_as(ctypes.c_void_p),
                                             out.nbytes))
        return out

    def potential(self):
        """Electric potential in float64 from its compensated pair (hi + lo)."""
        return self.array(POT).astype(np.float64) + self.array(POT_LO).astype(np.float64)

    def populations_g(self):
        """Momentum populations g_n in float64 (the library stores g_n - w_n; with the
        variable-density scheme, density_model 1, g_n itself)."""
        g = self.array(G).astype(np.float64)
        if self.workload.params.get("density_model", 0) == 1:
            return g
        return g + STORAGE_SHIFT[self.dim].reshape((-1, 1, 1, 1))

    def tensor(self, which):
        """Zero-copy torch view of one device array (valid until the next step)."""
        which = ARRAY_NAMES.get(which, which)
        ptr, nb = ctypes.c_void_p(), ctypes.c_size_t()
        self._check(self._lib.lbehd_device_ptr(self._h, which, ctypes.byref(ptr), ctypes.byref(nb)))
        shape = self._shape_of(which)

        class _View:
            __cuda_array_interface__ = {"shape": shape, "typestr": "<f4",
                                        "data": (ptr.value, False), "version": 3,
                                        "stream": None}
        return self._torch.as_tensor(_View(), device=self.device)

    def stats(self):
        """Counters since init: steps, Poisson CG iterations, graph replays, kernels."""
        st = Stats()
        self._check(self._lib.lbehd_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def launch_count(self):
        return int(self._lib.lbehd_launch_count(self._h))


class Simulation(_HandleOps):
    """One coupled LB-EHD run on the GPU.

    ``workload``: a ``workloads.Workload`` (geometry, initial Phi, parameters).
    ``stream``: a ``torch.cuda.Stream`` (default: torch's current stream).
    ``torch_alloc``: take device memory from PyTorch's caching allocator.
    """

    def __init__(self, workload, *, stream=None, torch_alloc=True, device=0, **config_kw):
        import torch
        self._torch = torch
        lib = load()
        self._setup_shape(workload)
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        c = Config()
        keep = make_config(workload, c, **config_kw)
        if torch_alloc:
            self._alloc_cb, self._free_cb = _torch_allocator(torch, self.device, self.stream)
            c.alloc, c.free = self._alloc_cb, self._free_cb
        c.stream = ctypes.c_void_p(self.stream.cuda_stream)
        self._cfg = c
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.lbehd_init(ctypes.byref(c), ctypes.byref(h))
        del keep
        if rc != 0:
            raise LBEHDError(rc, lib.lbehd_last_error(None).decode())
        self._h = h
        self._lib = lib

    # ----------------------------------------------------------------- calls

    def step(self, n=1):
        """Advance n steps; returns 0 or -3 (a Poisson solve hit its cap)."""
        return self._check(self._lib.lbehd_step(self._h, int(n)), allow=(-3,))

    def set_body_force(self, body=None, body_droplet=None):
        """Uniform and droplet-phase body force densities from the next step on (None keeps
        the current one)."""
        arrs = [None if b is None else np.ascontiguousarray(b, dtype=np.float64)
                for b in (body, body_droplet)]
        for a in arrs:
            if a is not None and a.shape != (3,):
                raise ValueError("body forces have 3 components")
        ptrs = [None if a is None else _dptr(a, ctypes.c_double) for a in arrs]
        self._check(self._lib.lbehd_set_body_force(self._h, *ptrs))

    def profile(self, enable=True):
        """Record per-kernel device time with CUDA events on the library's stream."""
        self._check(self._lib.lbehd_profile_enable(self._h, int(bool(enable))))

    def profile_read(self):
        """{kernel class: (total ms, launches)} since profiling was enabled."""
        n = len(KERNEL_CLASSES)
        ms, cnt = (ctypes.c_double * n)(), (ctypes.c_longlong * n)()
        self._check(self._lib.lbehd_profile_read(self._h, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def set_option(self, option, value):
        self._check(self._lib.lbehd_set_option(self._h, int(option), int(value)))

    def get_option(self, option):
        """The value in effect (see lbehd_get_option)."""
        v = ctypes.c_longlong()
        self._check(self._lib.lbehd_get_option(self._h, int(option), ctypes.byref(v)))
        return v.value

    def autotune(self, reps=20):
        """Time every collide kernel this lattice can run (state untouched), keep the
        fastest; returns (chosen variant, {variant: ms per launch})."""
        ms = (ctypes.c_double * 4)()
        rc = self._lib.lbehd_autotune(self._h, int(reps), ms)
        if rc < 0:
            self._check(rc)
        return rc, {v + 1: ms[v] for v in range(4) if ms[v] >= 0}

    def adjoint_forward(self, V, seg_steps):
        """Run the potential schedule V ((segments, electrodes), seg_steps steps each) from
        the current state, recording it for adjoint_backward; returns the loss (the droplet's
        x centroid after the last step)."""
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.ndim != 2 or V.shape[1] != self.n_electrodes:
            raise ValueError("V must have shape (segments, n_electrodes)")
        loss = ctypes.c_double()
        self._check(self._lib.lbehd_adjoint_forward(self._h, _dptr(V, ctypes.c_double),
                                                    V.shape[0], int(seg_steps),
                                                    ctypes.byref(loss)), allow=(-3,))
        self._adj_shape = V.shape
        return loss.value

    def adjoint_backward(self):
        """dL/dV of the recorded run, shape (segments, electrodes)."""
        g = np.zeros(self._adj_shape, dtype=np.float64)
        self._check(self._lib.lbehd_adjoint_backward(self._h, _dptr(g, ctypes.c_double)))
        return g

    def save_state(self, out=None):
        """The handle's whole state (lbehd_save_state) in a uint8 CUDA tensor (allocated here
        unless `out` is given)."""
        import torch
        n = int(self._lib.lbehd_state_bytes(self._h))
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, device=self.device)
        if out.numel() * out.element_size() < n or not out.is_cuda:
            raise ValueError(f"need a CUDA tensor of at least {n} bytes")
        self._check(self._lib.lbehd_save_state(self._h, ctypes.c_void_p(out.data_ptr())))
        return out

    def load_state(self, state):
        """Continue from a state saved by save_state on a handle of the same lattice."""
        if not state.is_cuda:
            raise ValueError("the state must be a CUDA tensor")
        self._check(self._lib.lbehd_load_state(self._h, ctypes.c_void_p(state.data_ptr())))

    def adjoint_info(self):
        """The recorded adjoint run: steps, checkpoint spacing and count, whether the
        potential trajectory was recorded, the last backward pass's replayed and reversed
        steps and adjoint CG iterations, and the adjoint's device bytes."""
        out = AdjointInfo()
        self._check(self._lib.lbehd_adjoint_get_info(self._h, ctypes.byref(out)))
        return {k: getattr(out, k) for k, _ in AdjointInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbehd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchInstance(_HandleOps):
    """Instance i of a Batch: observables, arrays and electrode switching of that
    instance. Stepping and options go through the Batch."""

    def __init__(self, batch, i, h, workload):
        self._batch = batch   # keeps the batch (which owns the handle) alive
        self._torch = batch._torch
        self._lib = batch._lib
        self._h = ctypes.c_void_p(h)
        self.index = i
        self.device = batch.device
        self._setup_shape(workload)


class Batch:
    """Many independent instances (``workloads``, same dim, any sizes and parameters)
    advanced together: one CUDA graph launch per step for the whole batch."""

    def __init__(self, workloads, *, stream=None, torch_alloc=True, device=0, **config_kw):
        import torch
        self._torch = torch
        lib = load()
        self._lib = lib
        self.workloads = list(workloads)
        n = len(self.workloads)
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        cfgs = (Config * n)()
        keep = [make_config(w, cfgs[i], **config_kw) for i, w in enumerate(self.workloads)]
        if torch_alloc:
            self._alloc_cb, self._free_cb = _torch_allocator(torch, self.device, self.stream)
        for c in cfgs:
            if torch_alloc:
                c.alloc, c.free = self._alloc_cb, self._free_cb
            c.stream = ctypes.c_void_p(self.stream.cuda_stream)
        b = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = lib.lbehd_batch_init(cfgs, n, ctypes.byref(b))
        del keep
        if rc != 0:
            raise LBEHDError(rc, lib.lbehd_last_error(None).decode())
        self._b = b
        self.instances = [BatchInstance(self, i, lib.lbehd_batch_instance(b, i), w)
                          for i, w in enumerate(self.workloads)]

    def __len__(self):
        return len(self.instances)

    def __getitem__(self, i):
        return self.instances[i]

    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            raise LBEHDError(rc, self._lib.lbehd_batch_last_error(self._b).decode())
        return rc

    def step(self, n=1):
        """Advance every instance n steps; returns 0 or -3 (a Poisson solve hit its cap)."""
        return self._check(self._lib.lbehd_batch_step(self._b, int(n)), allow=(-3,))

    def observe(self):
        """Observables of every instance (one synchronisation)."""
        n = len(self.instances)
        out = (Obs * n)()
        self._check(self._lib.lbehd_batch_observe(self._b, out))
        return [_obs_dict(o) for o in out]

    def set_option(self, option, value):
        self._check(self._lib.lbehd_batch_set_option(self._b, int(option), int(value)))

    def autotune(self, reps=20):
        """Per-instance collide kernel choice; returns (variants, [{variant: ms}])."""
        n = len(self.instances)
        var, ms = (ctypes.c_int * n)(), (ctypes.c_double * (4 * n))()
        self._check(self._lib.lbehd_batch_autotune(self._b, int(reps), var, ms))
        return list(var), [{v + 1: ms[4 * i + v] for v in range(4) if ms[4 * i + v] >= 0}
                           for i in range(n)]

    def profile(self, enable=True):
        """Eager batch steps with CUDA events around every launch."""
        self._check(self._lib.lbehd_batch_profile_enable(self._b, int(bool(enable))))

    def profile_read(self):
        """{kernel class: (total ms, launches)} since profiling was enabled."""
        n = len(KERNEL_CLASSES)
        ms, cnt = (ctypes.c_double * n)(), (ctypes.c_longlong * n)()
        self._check(self._lib.lbehd_batch_profile_read(self._b, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def stats(self):
        st = Stats()
        self._check(self._lib.lbehd_batch_get_stats(self._b, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def close(self):
        if getattr(self, "_b", None):
            for inst in self.instances:
                inst._h = None
            self._lib.lbehd_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _ScheduleLoss:
    """Built lazily so that importing this module does not import torch."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            import torch

            class ScheduleLoss(torch.autograd.Function):
                @staticmethod
                def forward(ctx, V, sim, seg_steps):
                    loss = sim.adjoint_forward(V.detach().cpu().double().numpy(), seg_steps)
                    ctx.sim = sim
                    ctx.meta = (V.dtype, V.device)
                    return torch.tensor(loss, dtype=V.dtype, device=V.device)

                @staticmethod
                def backward(ctx, gL):
                    dtype, device = ctx.meta
                    g = torch.as_tensor(ctx.sim.adjoint_backward(), dtype=dtype, device=device)
                    return g * gL, None, None

            cls.fn = ScheduleLoss
        return cls.fn


def schedule_loss(sim, V, seg_steps):
    """L(V) = droplet x centroid after running the electrode-potential schedule V
    (tensor (segments, electrodes), seg_steps steps per segment) on ``sim`` from its current
    state; differentiable: backward runs the library's discrete adjoint."""
    return _ScheduleLoss.get().apply(V, sim, seg_steps)

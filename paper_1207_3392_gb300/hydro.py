"""Thin Python binding of the C ABI in include/genasis_hydro.h.

Argument marshalling only: every step of the update runs in the CUDA library
``_lib/libgenasis_hydro.so``.  There is no fallback: if the library is missing
or fails to load, every call raises.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); they must be C-contiguous and of the documented
dtype.  PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libgenasis_hydro.so")

OK, EINVAL, ENOMEM, ECUDA, ENONPHYS, ETIMEOUT = 0, -1, -2, -3, -4, -5
HLL, HLLC, HLLC_SWITCH = 0, 1, 2  # HLLC_SWITCH: HLLC with HLL transverse to shocks
BC_PERIODIC, BC_REFLECT, BC_OUTFLOW = 0, 1, 2
FP64, FP32_MIXED, FP64_DW = 0, 1, 2  # FP64_DW: double-word FP32 pairs on the device, FP64 on the host
OPT_STEP_TOTALS = 1
OPT_ONE_LAUNCH = 2
OPT_MLP_TCGEN05 = 3


class HydroError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"genasis_hydro error {code}: {msg}")
        self.code = code


class NonPhysicalState(HydroError):
    pass


class Desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("widths", ctypes.c_void_p * 3),
                ("origin", ctypes.c_double * 3), ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("gamma", ctypes.c_double),
                ("solver", ctypes.c_int), ("theta", ctypes.c_double), ("precision", ctypes.c_int),
                ("stream", ctypes.c_void_p)]


_lib = None

# (name, argtypes); every function returns int except last_error.
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "genasis_hydro_create": [ctypes.POINTER(Desc), ctypes.POINTER(_P)],
    "genasis_hydro_destroy": [_P],
    "genasis_hydro_set_primitive": [_P, _P, _P, _P],
    "genasis_hydro_set_conserved": [_P, _P, _I],
    "genasis_hydro_get_conserved": [_P, _P, _I],
    "genasis_hydro_compute_dt": [_P, _D, _P],
    "genasis_hydro_step": [_P, _D],
    "genasis_hydro_advance": [_P, _I, _D, _D, _P],
    "genasis_hydro_get_time": [_P, _P],
    "genasis_hydro_set_time": [_P, _D],
    "genasis_hydro_get_totals": [_P, _P],
    "genasis_hydro_status": [_P],
    "genasis_hydro_clear_status": [_P],
    "genasis_hydro_set_conserved_async": [_P, _P, _I],
    "genasis_hydro_get_conserved_async": [_P, _P, _I],
    "genasis_hydro_sync": [_P],
    "genasis_hydro_set_potential_gradient": [_P, _P],
    "genasis_fmr_create": [_P, _P],
    "genasis_fmr_destroy": [_P],
    "genasis_fmr_set_level": [_P, _I, _P],
    "genasis_fmr_get_level": [_P, _I, _P],
    "genasis_fmr_step": [_P, _I, ctypes.c_double, _P],
    "genasis_fmr_autotune": [_P, _I],
    "genasis_hydro_set_tile": [_P, _I, _I],
    "genasis_hydro_get_tile": [_P, _P],
    "genasis_hydro_autotune": [_P, _I, ctypes.c_char_p],
    "genasis_hydro_launches_per_step": [_P],
    "genasis_hydro_profile_step": [_P, _D, _P],
    "genasis_hydro_set_option": [_P, _I, _I],
    "genasis_hydro_get_step_totals": [_P, _P],
    "genasis_hydro_step_noalloc": [ctypes.POINTER(Desc), _P, _P, _D],
    "genasis_hydro_accumulate_face_flux": [_P, _I, _D, _P],
    "genasis_hydro_restrict": [_P, _I, _P],
    "genasis_learned_create": [ctypes.POINTER(Desc), ctypes.POINTER(_P)],
    "genasis_learned_destroy": [_P],
    "genasis_learned_set_params": [_P, _P],
    "genasis_learned_set_limit": [_P, ctypes.c_float],
    "genasis_learned_set_fct": [_P, _I],
    "genasis_learned_step": [_P, ctypes.c_double],
    "genasis_learned_set_primitive": [_P, _P, _P, _P],
    "genasis_learned_set_conserved": [_P, _P],
    "genasis_learned_get_conserved": [_P, _P],
    "genasis_learned_advance": [_P, _I, _D, _D, _P],
    "genasis_learned_fallbacks": [_P, _P],
    "genasis_measure_link_rate": [ctypes.c_int, _P],
    "genasis_check_bounded_waits": [_P, _P],
    "genasis_learned_set_option": [_P, ctypes.c_int, ctypes.c_int],
    "genasis_learned_launches_per_step": [_P],
    "genasis_learned_features": [_P, _P, _P],
    "genasis_learned_targets": [_P, _P, _P, _P, _P],
    "genasis_mlp_param_count": [],
    "genasis_mlp_forward": [_P, _P, ctypes.c_longlong, _P, _P],
    "genasis_mlp_gradient": [_P, _P, _P, ctypes.c_longlong, _P, _P, _P],
    "genasis_mlp_opt_create": [_P, _P, ctypes.POINTER(_P)],
    "genasis_mlp_opt_destroy": [_P],
    "genasis_mlp_opt_step": [_P, _P, _P, ctypes.c_longlong, ctypes.c_float, _P],
    "genasis_mlp_opt_get_params": [_P, _P],
    "genasis_batch_create": [_I, _P, _I, _D, _I, _P, ctypes.POINTER(_P)],
    "genasis_batch_destroy": [_P],
    "genasis_batch_set_primitive": [_P, _I, _P, _P, _P],
    "genasis_batch_get_conserved": [_P, _I, _P, _I],
    "genasis_batch_run": [_P, _I, _D, _D],
    "genasis_batch_get_times": [_P, _P],
    "genasis_batch_status": [_P, _P],
    "genasis_batch_set_tile": [_P, _I, _I],
    "genasis_batch_get_tile": [_P, _P],
    "genasis_batch_autotune": [_P, _I, ctypes.c_char_p],
    "genasis_batch_profile_step": [_P, _D, _P],
    "genasis_hydro_get_centers": [_P, _I, _P],
    "genasis_hydro_batch_create": [_I, _P, ctypes.POINTER(_P)],
    "genasis_hydro_batch_set_primitive": [_P, _I, _P, _P, _P],
    "genasis_hydro_batch_run": [_P, _I, _D, _D],
    "genasis_hydro_batch_get_conserved": [_P, _I, _P, _I],
    "genasis_hydro_batch_get_times": [_P, _P],
    "genasis_hydro_set_flux_mlp": [_P, _P, ctypes.c_size_t],
    "genasis_measure_fma_rate": [_I, _P],
}


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise HydroError(ECUDA, f"CUDA library not built: {path} is missing "
                                    "(run `python -m paper_1207_3392_gb300.build`)")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.genasis_hydro_last_error.argtypes = []
        lib.genasis_hydro_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def check(rc):
    if rc == OK or (isinstance(rc, int) and rc > 0):
        return rc
    msg = load().genasis_hydro_last_error().decode()
    if rc == ENONPHYS:
        raise NonPhysicalState(rc, msg)
    raise HydroError(rc, msg)


def _ptr(a, dtype, count=None, name="array"):
    """Raw address of a contiguous numpy array or torch tensor (host or CUDA)."""
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {want} tensor")
        if count is not None and a.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {a.numel()}")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if count is not None and arr.size != count:
        raise ValueError(f"{name}: expected {count} elements, got {arr.size}")
    return arr.ctypes.data, arr


class Hydro:
    """One mesh + state on the GPU (a genasis_hydro_t handle)."""

    def __init__(self, ndim, n, widths, bc_lo, bc_hi, gamma=1.4, solver=HLLC, theta=1.4,
                 precision=FP64, stream=None, origin=(0.0, 0.0, 0.0)):
        lib = load()
        self.ndim = int(ndim)
        self.n = tuple(int(x) for x in (list(n) + [1, 1, 1])[:3])
        self.precision = int(precision)
        # host arrays: FP32 for the FP32 state, FP64 otherwise
        self.host_precision = FP32_MIXED if self.precision == FP32_MIXED else FP64
        self.dtype = np.float64 if self.host_precision == FP64 else np.float32
        self._widths = [np.ascontiguousarray(widths[q], dtype=np.float64) for q in range(self.ndim)]
        d = Desc()
        d.ndim = self.ndim
        for q in range(3):
            d.n[q] = self.n[q] if q < self.ndim else 1
            d.widths[q] = self._widths[q].ctypes.data if q < self.ndim else None
            d.bc_lo[q] = int(bc_lo[q]) if q < self.ndim else 0
            d.bc_hi[q] = int(bc_hi[q]) if q < self.ndim else 0
            d.origin[q] = float(origin[q]) if q < len(origin) else 0.0
        d.gamma, d.solver, d.theta, d.precision = float(gamma), int(solver), float(theta), self.precision
        # stream: a cudaStream_t handle (int) or torch.cuda.Stream; None or 0
        # (the legacy default stream) gives the handle a stream of its own
        if stream is not None:
            d.stream = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
        self._h = ctypes.c_void_p()
        check(lib.genasis_hydro_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.ncell = int(np.prod(self.n[: self.ndim]))
        self.nvar = self.ndim + 2
        self.shape = tuple(reversed(self.n[: self.ndim]))

    @classmethod
    def from_problem(cls, prob, precision=FP64, solver=None, stream=None, set_state=True):
        h = cls(prob.ndim, prob.n, prob.widths, prob.bc_lo, prob.bc_hi, prob.gamma,
                prob.solver if solver is None else solver, prob.theta, precision, stream,
                origin=getattr(prob, "origin", (0.0, 0.0, 0.0)))
        if any(getattr(prob, "grad_phi", (0.0, 0.0, 0.0))):
            h.set_potential_gradient(prob.grad_phi)
        if set_state:
            h.set_primitive(prob.rho, prob.vel, prob.p)
        return h

    # -- state ---------------------------------------------------------------
    def set_primitive(self, rho, vel, p):
        pr, a = _ptr(rho, np.float64, self.ncell, "rho")
        pv, b = _ptr(vel, np.float64, self.ncell * self.ndim, "vel")
        pp, c = _ptr(p, np.float64, self.ncell, "p")
        check(load().genasis_hydro_set_primitive(self._h, pr, pv, pp))

    def set_conserved(self, U, precision=None):
        precision = self.host_precision if precision is None else precision
        dt = np.float64 if precision == FP64 else np.float32
        pu, keep = _ptr(U, dt, self.ncell * self.nvar, "U")
        check(load().genasis_hydro_set_conserved(self._h, pu, precision))

    def get_conserved(self, out=None, precision=None):
        """Return the conserved state, shape (nvar,) + shape; into `out` (numpy
        or torch, host or CUDA) if given."""
        precision = self.host_precision if precision is None else precision
        dt = np.float64 if precision == FP64 else np.float32
        if out is None:
            out = np.empty((self.nvar,) + self.shape, dtype=dt)
        po, _ = _ptr(out, dt, self.ncell * self.nvar, "out")
        check(load().genasis_hydro_get_conserved(self._h, po, precision))
        return out

    def set_conserved_async(self, U, precision=None):
        """Enqueue the copy of U (page-locked host or device) without waiting;
        U must stay unchanged until sync()."""
        precision = self.host_precision if precision is None else precision
        dt = np.float64 if precision == FP64 else np.float32
        pu, keep = _ptr(U, dt, self.ncell * self.nvar, "U")
        if keep is not U:
            raise ValueError("U: an asynchronous copy needs a contiguous array of the exact dtype (no temporary)")
        check(load().genasis_hydro_set_conserved_async(self._h, pu, precision))

    def get_conserved_async(self, out, precision=None):
        """Enqueue the copy of the state into `out` without waiting; read it
        after sync()."""
        precision = self.host_precision if precision is None else precision
        dt = np.float64 if precision == FP64 else np.float32
        po, keep = _ptr(out, dt, self.ncell * self.nvar, "out")
        if keep is not out:
            raise ValueError("out: an asynchronous copy needs a contiguous array of the exact dtype (no temporary)")
        check(load().genasis_hydro_get_conserved_async(self._h, po, precision))
        return out

    def sync(self):
        """Wait for the handle's stream; raises on a non-physical state."""
        check(load().genasis_hydro_sync(self._h))

    def set_potential_gradient(self, grad_phi):
        """External force -grad Phi of a linear potential (Sec. 4.3.2)."""
        g = np.zeros(3)
        g[: len(grad_phi)] = grad_phi
        check(load().genasis_hydro_set_potential_gradient(self._h, g.ctypes.data))

    def centers(self, axis):
        """Geometric cell centres along `axis` measured from the origin."""
        out = np.empty(self.n[axis] if 0 <= axis < self.ndim else 1)
        check(load().genasis_hydro_get_centers(self._h, int(axis), out.ctypes.data))
        return out

    def set_flux_mlp(self, weights_bf16):
        """Attach the flux-correction network from its BF16 parameters (uint16
        bit patterns, numpy or torch, host or CUDA); None detaches it.  With a
        network attached, step/advance run the corrected scheme."""
        if weights_bf16 is None:
            check(load().genasis_hydro_set_flux_mlp(self._h, None, 0))
            return
        if hasattr(weights_bf16, "data_ptr"):
            ptr, nbytes = weights_bf16.data_ptr(), weights_bf16.numel() * weights_bf16.element_size()
            keep = weights_bf16
        else:
            keep = np.ascontiguousarray(weights_bf16, dtype=np.uint16)
            ptr, nbytes = keep.ctypes.data, keep.nbytes
        check(load().genasis_hydro_set_flux_mlp(self._h, ptr, nbytes))

    # -- stepping -------------------------------------------------------------
    def compute_dt(self, cfl):
        out = ctypes.c_double()
        check(load().genasis_hydro_compute_dt(self._h, float(cfl), ctypes.byref(out)))
        return out.value

    def step(self, dt):
        check(load().genasis_hydro_step(self._h, float(dt)))

    def advance(self, nsteps, cfl, t_end=0.0, sync=True):
        t = ctypes.c_double()
        check(load().genasis_hydro_advance(self._h, int(nsteps), float(cfl), float(t_end),
                                           ctypes.byref(t) if sync else None))
        return t.value if sync else None

    def evolve(self, cfl, t_end, chunk=64, max_steps=1 << 30):
        """Advance until t_end in graph launches of `chunk` steps."""
        t = self.time
        steps = 0
        while t < t_end and steps < max_steps:
            t = self.advance(chunk, cfl, t_end)
            steps += chunk
        return t

    @property
    def time(self):
        t = ctypes.c_double()
        check(load().genasis_hydro_get_time(self._h, ctypes.byref(t)))
        return t.value

    @time.setter
    def time(self, value):
        check(load().genasis_hydro_set_time(self._h, float(value)))

    def totals(self):
        out = np.zeros(5)
        check(load().genasis_hydro_get_totals(self._h, out.ctypes.data))
        return out[: self.nvar]

    def step_totals(self):
        """Totals of U^n folded into the last step (GENASIS_OPT_STEP_TOTALS)."""
        out = np.zeros(5)
        check(load().genasis_hydro_get_step_totals(self._h, out.ctypes.data))
        return out[: self.nvar]

    def set_step_totals(self, enabled):
        check(load().genasis_hydro_set_option(self._h, OPT_STEP_TOTALS, int(bool(enabled))))

    def set_one_launch(self, enabled):
        """Small 1D meshes and an attached network: all steps of a call in one
        cooperative launch (default on)."""
        check(load().genasis_hydro_set_option(self._h, OPT_ONE_LAUNCH, int(bool(enabled))))

    def set_mlp_tcgen05(self, enabled):
        """An attached network on tcgen05 (True) or mma.sync (False, default)."""
        check(load().genasis_hydro_set_option(self._h, OPT_MLP_TCGEN05, int(bool(enabled))))

    def status(self):
        return check(load().genasis_hydro_status(self._h))

    def clear_status(self):
        check(load().genasis_hydro_clear_status(self._h))

    # -- launch configuration -------------------------------------------------
    def set_tile(self, tile, kchunk=0):
        check(load().genasis_hydro_set_tile(self._h, int(tile), int(kchunk)))

    def tile_info(self):
        info = (ctypes.c_int * 6)()
        check(load().genasis_hydro_get_tile(self._h, info))
        keys = ("tile", "tx", "ty", "kchunk", "ctas", "tile_count")
        return dict(zip(keys, list(info)))

    def autotune(self, trial_steps=3, cache_path=None):
        check(load().genasis_hydro_autotune(self._h, int(trial_steps),
                                            cache_path.encode() if cache_path else None))
        return self.tile_info()

    def profile_step(self, cfl):
        """One CFL step with per-kernel CUDA-event timing: (stage1, finalize,
        stage2) in milliseconds."""
        ms = (ctypes.c_float * 3)()
        check(load().genasis_hydro_profile_step(self._h, float(cfl), ms))
        return tuple(ms)

    def accumulate_face_flux(self, F, stride=1, weight=1.0):
        """Add the last step's effective RK2 face flux (averaged over `stride`
        fine faces per coarse face) times `weight` into the CUDA float64
        tensor F of shape (2, 4, ny/stride, nx/stride)."""
        pf, _ = _ptr(F, np.float64, None, "F")
        check(load().genasis_hydro_accumulate_face_flux(self._h, int(stride), float(weight), pf))

    def restrict(self, out, factor):
        """Conservative restriction of the state by `factor` into the CUDA
        float32 tensor out of shape (4, ny/factor, nx/factor)."""
        po, _ = _ptr(out, np.float32, None, "out")
        check(load().genasis_hydro_restrict(self._h, int(factor), po))
        return out

    def launches_per_step(self):
        return check(load().genasis_hydro_launches_per_step(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_hydro_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FmrDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int), ("nlevels", ctypes.c_int), ("size", ctypes.c_double),
                ("bc", ctypes.c_int), ("gamma", ctypes.c_double), ("solver", ctypes.c_int),
                ("theta", ctypes.c_double), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


class Fmr:
    """Nested-box multilevel mesh with subcycled evolution (genasis_fmr_t).
    Level l >= 1 is stored with a two-cell exterior ring: (n+4)^d cells."""

    def __init__(self, ndim, n, nlevels, size, bc, gamma=1.4, solver=HLLC, theta=1.4, precision=FP64,
                 stream=None):
        d = FmrDesc(int(ndim), int(n), int(nlevels), float(size), int(bc), float(gamma), int(solver), float(theta),
                    int(precision), None if stream is None else int(getattr(stream, "cuda_stream", stream)))
        self._h = ctypes.c_void_p()
        check(load().genasis_fmr_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.ndim, self.n, self.nlevels = int(ndim), int(n), int(nlevels)

    def stored_shape(self, level):
        m = self.n + (4 if level else 0)
        return (self.ndim + 2,) + (m,) * self.ndim

    def set_level(self, level, U):
        pu, keep = _ptr(U, np.float64, int(np.prod(self.stored_shape(level))), "U")
        check(load().genasis_fmr_set_level(self._h, int(level), pu))

    def get_level(self, level):
        out = np.empty(self.stored_shape(level))
        check(load().genasis_fmr_get_level(self._h, int(level), out.ctypes.data))
        return out

    def autotune(self, trial_steps=2):
        """Autotune every level's launch configuration on its current state."""
        check(load().genasis_fmr_autotune(self._h, int(trial_steps)))

    def step(self, nsteps, cfl):
        t = ctypes.c_double()
        check(load().genasis_fmr_step(self._h, int(nsteps), float(cfl), ctypes.byref(t)))
        return t.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_fmr_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchProblemDesc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 2), ("widths", ctypes.c_void_p * 2),
                ("bc_lo", ctypes.c_int * 2), ("bc_hi", ctypes.c_int * 2), ("gamma", ctypes.c_double)]


class Batch:
    """Many independent 1D/2D problems advanced together (genasis_batch_t)."""

    def __init__(self, problems, solver=HLLC, theta=1.4, precision=FP64, stream=None):
        lib = load()
        self.precision = int(precision)
        self.host_precision = FP32_MIXED if self.precision == FP32_MIXED else FP64
        self.nprob = len(problems)
        self._keep = []
        arr = (BatchProblemDesc * self.nprob)()
        self.meta = []
        for i, pr in enumerate(problems):
            d = arr[i]
            d.ndim = pr.ndim
            ws = []
            for q in range(2):
                active = q < pr.ndim
                d.n[q] = int(pr.n[q]) if active else 1
                if active:
                    w = np.ascontiguousarray(pr.widths[q], dtype=np.float64)
                    ws.append(w)
                    d.widths[q] = w.ctypes.data
                d.bc_lo[q] = int(pr.bc_lo[q]) if active else 2
                d.bc_hi[q] = int(pr.bc_hi[q]) if active else 2
            d.gamma = float(pr.gamma)
            self._keep.append(ws)
            shape = tuple(reversed([int(pr.n[q]) for q in range(pr.ndim)]))
            self.meta.append((pr.ndim, shape, int(np.prod(shape))))
        s = 0
        if stream is not None:
            s = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
        self._h = ctypes.c_void_p()
        check(lib.genasis_batch_create(self.nprob, ctypes.cast(arr, ctypes.c_void_p), int(solver), float(theta),
                                       self.precision, s or None, ctypes.byref(self._h)))
        self._keep = None

    def set_primitive(self, i, rho, vel, p):
        ndim, shape, nc = self.meta[i]
        pr, a = _ptr(rho, np.float64, nc, "rho")
        pv, b = _ptr(vel, np.float64, nc * ndim, "vel")
        pp, c = _ptr(p, np.float64, nc, "p")
        check(load().genasis_batch_set_primitive(self._h, int(i), pr, pv, pp))

    def get_conserved(self, i, precision=FP64):
        ndim, shape, nc = self.meta[i]
        dt = np.float64 if precision == FP64 else np.float32
        out = np.empty((ndim + 2,) + shape, dtype=dt)
        check(load().genasis_batch_get_conserved(self._h, int(i), out.ctypes.data, int(precision)))
        return out

    def run(self, nsteps, cfl, t_end=0.0):
        check(load().genasis_batch_run(self._h, int(nsteps), float(cfl), float(t_end)))

    def times(self):
        t = np.zeros(self.nprob)
        check(load().genasis_batch_get_times(self._h, t.ctypes.data))
        return t

    def status(self):
        bad = ctypes.c_int(-1)
        rc = load().genasis_batch_status(self._h, ctypes.byref(bad))
        if rc != OK:
            check(rc)
        return bad.value

    def set_tile(self, tile, chunk=0):
        check(load().genasis_batch_set_tile(self._h, int(tile), int(chunk)))

    def tile_info(self):
        info = (ctypes.c_int * 7)()
        check(load().genasis_batch_get_tile(self._h, info))
        return dict(zip(("tile", "threads", "chunk", "items", "ctas", "tile_count", "mcells"), list(info)))

    def autotune(self, trial_steps=2, cache_path=None):
        check(load().genasis_batch_autotune(self._h, int(trial_steps), cache_path.encode() if cache_path else None))
        return self.tile_info()

    def profile_step(self, cfl):
        ms = (ctypes.c_float * 3)()
        check(load().genasis_batch_profile_step(self._h, float(cfl), ms))
        return tuple(ms)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_noalloc(prob, U_in, U_out, dt, precision=FP64, solver=None, stream=None):
    """One RK2 step through genasis_hydro_step_noalloc, which allocates no
    device memory (for callers whose device memory is owned by a pooling
    allocator, or that must not allocate after initialisation).  U_in and
    U_out are CUDA tensors of the conserved state in `precision`; prob gives
    the mesh (ndim, n, widths, bc_lo, bc_hi, gamma, theta, solver)."""
    d = Desc()
    d.ndim = int(prob.ndim)
    widths = [np.ascontiguousarray(prob.widths[q], dtype=np.float64) for q in range(prob.ndim)]
    for q in range(3):
        d.n[q] = int(prob.n[q]) if q < prob.ndim else 1
        d.widths[q] = widths[q].ctypes.data if q < prob.ndim else None
        d.bc_lo[q] = int(prob.bc_lo[q]) if q < prob.ndim else 0
        d.bc_hi[q] = int(prob.bc_hi[q]) if q < prob.ndim else 0
    d.gamma = float(prob.gamma)
    d.solver = int(prob.solver if solver is None else solver)
    d.theta = float(prob.theta)
    d.precision = int(precision)
    if stream is not None:
        d.stream = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
    dt_ = np.float64 if precision == FP64 else np.float32
    pin, a = _ptr(U_in, dt_, None, "U_in")
    pout, b = _ptr(U_out, dt_, None, "U_out")
    check(load().genasis_hydro_step_noalloc(ctypes.byref(d), pin, pout, float(dt)))


class HydroBatch:
    """Many independent 1D/2D problems behind one genasis_hydro_t
    (genasis_hydro_batch_create from one genasis_hydro_desc per problem)."""

    def __init__(self, probs, precision=FP64, solver=None, theta=None, stream=None):
        self._keep = []
        arr = (Desc * len(probs))()
        for i, pr in enumerate(probs):
            d, keep = _desc(pr, precision, solver, stream)
            if theta is not None:
                d.theta = float(theta)
            arr[i] = d
            self._keep.append(keep)
        self._h = ctypes.c_void_p()
        check(load().genasis_hydro_batch_create(len(probs), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(self._h)))
        self.probs = [(int(pr.ndim), tuple(int(x) for x in pr.n)) for pr in probs]
        self.precision = int(precision)

    def set_primitive(self, i, rho, vel, p):
        nd, n = self.probs[i]
        nc = int(np.prod(n[:nd]))
        pr, a = _ptr(rho, np.float64, nc, "rho")
        pv, b = _ptr(vel, np.float64, nd * nc, "vel")
        pp, c = _ptr(p, np.float64, nc, "p")
        check(load().genasis_hydro_batch_set_primitive(self._h, int(i), pr, pv, pp))

    def run(self, nsteps, cfl, t_end=0.0):
        check(load().genasis_hydro_batch_run(self._h, int(nsteps), float(cfl), float(t_end)))

    def get_conserved(self, i, precision=None):
        nd, n = self.probs[i]
        precision = FP64 if precision is None else precision
        dt = np.float64 if precision == FP64 else np.float32
        out = np.empty((nd + 2,) + tuple(reversed(n[:nd])), dtype=dt)
        check(load().genasis_hydro_batch_get_conserved(self._h, int(i), out.ctypes.data, int(precision)))
        return out

    def times(self):
        out = np.empty(len(self.probs))
        check(load().genasis_hydro_batch_get_times(self._h, out.ctypes.data))
        return out

    def status(self):
        return check(load().genasis_hydro_status(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_hydro_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_bounded_waits():
    """Run the two waits that cannot complete (grid barrier, mbarrier) and
    return ([status word per wait], [seconds per wait]); a status of 2 means
    the wait gave up within its bound (about a second)."""
    st = (ctypes.c_uint * 2)()
    sec = (ctypes.c_double * 2)()
    check(load().genasis_check_bounded_waits(st, sec))
    return [int(st[0]), int(st[1])], [float(sec[0]), float(sec[1])]


def measure_fma_rate(kind):
    """Measured vector FMA rate of this GPU in TFLOP/s: kind 0 FP64, 1 FP32,
    2 FP32 with the packed two-lane FMA."""
    out = ctypes.c_double()
    check(load().genasis_measure_fma_rate(int(kind), ctypes.byref(out)))
    return out.value


def measure_link_rate(kind):
    """Measured host-link copy rate in GB/s: kind 0 host to device, 1 device
    to host, 2 both directions at once (their sum)."""
    out = ctypes.c_double()
    check(load().genasis_measure_link_rate(int(kind), ctypes.byref(out)))
    return out.value


def _desc(prob, precision, solver=None, stream=None):
    d = Desc()
    d.ndim = int(prob.ndim)
    keep = [np.ascontiguousarray(prob.widths[q], dtype=np.float64) for q in range(prob.ndim)]
    for q in range(3):
        d.n[q] = int(prob.n[q]) if q < prob.ndim else 1
        d.widths[q] = keep[q].ctypes.data if q < prob.ndim else None
        d.bc_lo[q] = int(prob.bc_lo[q]) if q < prob.ndim else 0
        d.bc_hi[q] = int(prob.bc_hi[q]) if q < prob.ndim else 0
        d.origin[q] = float(getattr(prob, "origin", (0.0, 0.0, 0.0))[q]) if q < prob.ndim else 0.0
    d.gamma = float(prob.gamma)
    d.solver = int(prob.solver if solver is None else solver)
    d.theta = float(prob.theta)
    d.precision = int(precision)
    if stream is not None:
        d.stream = stream if isinstance(stream, int) else int(getattr(stream, "cuda_stream", stream))
    return d, keep


def mlp_param_count():
    return load().genasis_mlp_param_count()


def mlp_forward(params, X, Y, stream=None):
    """Y[n, 4] = network(X[n, 32] bf16); CUDA tensors."""
    n = X.shape[0]
    check(load().genasis_mlp_forward(params.data_ptr(), X.data_ptr(), int(n), Y.data_ptr(),
                                     None if stream is None else int(getattr(stream, "cuda_stream", stream))))
    return Y


def mlp_gradient(params, X, T, grad, loss=None, stream=None):
    n = X.shape[0]
    check(load().genasis_mlp_gradient(params.data_ptr(), X.data_ptr(), T.data_ptr(), int(n), grad.data_ptr(),
                                      None if loss is None else loss.data_ptr(),
                                      None if stream is None else int(getattr(stream, "cuda_stream", stream))))
    return grad


class MlpOptimizer:
    """Adam on a device copy of the network parameters (genasis_mlp_opt_t)."""

    def __init__(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32) if not hasattr(params, "data_ptr") else params
        ptr = p.ctypes.data if isinstance(p, np.ndarray) else p.data_ptr()
        self._h = ctypes.c_void_p()
        check(load().genasis_mlp_opt_create(ptr, None if stream is None else int(getattr(stream, "cuda_stream", stream)),
                                            ctypes.byref(self._h)))

    def step(self, X, T, lr, want_loss=True):
        loss = ctypes.c_float()
        check(load().genasis_mlp_opt_step(self._h, X.data_ptr(), T.data_ptr(), int(X.shape[0]), float(lr),
                                          ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def params(self):
        out = np.empty(mlp_param_count(), dtype=np.float32)
        check(load().genasis_mlp_opt_get_params(self._h, out.ctypes.data))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_mlp_opt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Learned:
    """2D FP32 solver with the learned flux correction (genasis_learned_t)."""

    def __init__(self, prob, params=None, solver=None, stream=None):
        lib = load()
        d, keep = _desc(prob, FP32_MIXED, solver, stream)
        self._h = ctypes.c_void_p()
        check(lib.genasis_learned_create(ctypes.byref(d), ctypes.byref(self._h)))
        self.n = (int(prob.n[0]), int(prob.n[1]))
        self.ncell = self.n[0] * self.n[1]
        self.shape = (self.n[1], self.n[0])
        self.set_params(params)

    def set_params(self, params):
        if params is None:
            check(load().genasis_learned_set_params(self._h, None))
            return
        if hasattr(params, "data_ptr"):
            check(load().genasis_learned_set_params(self._h, params.data_ptr()))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            check(load().genasis_learned_set_params(self._h, p.ctypes.data))

    def set_fct(self, enabled):
        """Flux-corrected-transport limiting of the correction (default on)."""
        check(load().genasis_learned_set_fct(self._h, int(bool(enabled))))

    def set_limit(self, ylim):
        """Clamp network outputs to [-ylim, ylim] (math.inf: no bound)."""
        check(load().genasis_learned_set_limit(self._h, float(ylim)))

    def set_primitive(self, rho, vel, p):
        pr, a = _ptr(rho, np.float64, self.ncell, "rho")
        pv, b = _ptr(vel, np.float64, 2 * self.ncell, "vel")
        pp, c = _ptr(p, np.float64, self.ncell, "p")
        check(load().genasis_learned_set_primitive(self._h, pr, pv, pp))

    def set_conserved(self, U):
        pu, keep = _ptr(U, np.float32, 4 * self.ncell, "U")
        check(load().genasis_learned_set_conserved(self._h, pu))

    def get_conserved(self, out=None):
        if out is None:
            out = np.empty((4,) + self.shape, dtype=np.float32)
        po, _ = _ptr(out, np.float32, 4 * self.ncell, "out")
        check(load().genasis_learned_get_conserved(self._h, po))
        return out

    def advance(self, nsteps, cfl, t_end=0.0, sync=True):
        t = ctypes.c_double()
        check(load().genasis_learned_advance(self._h, int(nsteps), float(cfl), float(t_end),
                                             ctypes.byref(t) if sync else None))
        return t.value if sync else None

    def step(self, dt):
        """One corrected RK2 step with a given dt (asynchronous)."""
        check(load().genasis_learned_step(self._h, float(dt)))

    def evolve(self, cfl, t_end, chunk=64, max_chunks=1 << 30):
        """Advance to t_end (the last step clamped); stops early after
        max_chunks calls of `chunk` steps and returns the time reached."""
        t = 0.0
        for _ in range(max_chunks):
            if t >= t_end:
                break
            t = self.advance(chunk, cfl, t_end)
        return t

    def set_one_launch(self, enabled):
        """All steps of a call in one cooperative launch (default on) or the
        per-phase launches; the results are bitwise the same."""
        check(load().genasis_learned_set_option(self._h, OPT_ONE_LAUNCH, int(bool(enabled))))

    def set_mlp_tcgen05(self, enabled):
        """Run the network on tcgen05 (True) or on mma.sync (False, the
        default); the states agree to rounding."""
        check(load().genasis_learned_set_option(self._h, OPT_MLP_TCGEN05, int(bool(enabled))))

    def launches_per_step(self):
        return check(load().genasis_learned_launches_per_step(self._h))

    def fallbacks(self):
        v = ctypes.c_longlong()
        check(load().genasis_learned_fallbacks(self._h, ctypes.byref(v)))
        return v.value

    def features(self, X, scale):
        check(load().genasis_learned_features(self._h, X.data_ptr(), scale.data_ptr()))

    def targets(self, f_target, f_plain, scale, T):
        check(load().genasis_learned_targets(self._h, f_target.data_ptr(), f_plain.data_ptr(), scale.data_ptr(),
                                             T.data_ptr()))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().genasis_learned_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

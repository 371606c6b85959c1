"""CPU oracle of the GenASiS hydrodynamics update (TEST INFRASTRUCTURE ONLY).

The plain FP64 solver is ``hydro_oracle.c`` (built with gcc into
``oracle/_lib``); this module is its ctypes wrapper.  Analytic references that
pin the oracle itself live beside it: ``exact_riemann.py`` (exact solution of
the ideal-gas Riemann problem) and ``sedov.py`` (Sedov-Taylor self-similar
blast).  ``mlp.py`` is the FP64 reference of the learned flux correction.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this package; the CUDA product path never does.  Nothing here shares
code with ``paper_1207_3392_gb300/csrc``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libhydro_oracle.so")
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_COUNT_LIB = os.path.join(_LIBDIR, "libopcount.so")
_COUNT_SRC = os.path.join(_HERE, "opcount.cpp")

ENONPHYS = -4


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so x86 and Arm agree),
    and its operation counter (opcount.cpp) with g++."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or _stale(_LIB, [_SRC]):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    if force or _stale(_COUNT_LIB, [_SRC, _COUNT_SRC]):
        tmp = _COUNT_LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, _COUNT_SRC, "-lm"])
        os.replace(tmp, _COUNT_LIB)
    return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("width", ctypes.c_void_p * 3), ("bc_lo", ctypes.c_int * 3),
                ("bc_hi", ctypes.c_int * 3), ("gamma", ctypes.c_double),
                ("theta", ctypes.c_double), ("solver", ctypes.c_int),
                ("grad_phi", ctypes.c_double * 3)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        D = ctypes.POINTER(_Desc)
        for name, args in [("og_rhs", [D, P, P]), ("og_step", [D, P, ctypes.c_double]),
                           ("og_cfl_dt", [D, P, P]), ("og_totals", [D, P, P]),
                           ("og_evolve", [D, P, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]),
                           ("og_prim_to_cons", [D, P, P, P, P]), ("og_cons_to_prim", [D, P, P, P, P]),
                           ("og_riemann_flux", [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P, P, P]),
                           ("og_physical_flux", [ctypes.c_double, ctypes.c_int, ctypes.c_int, P, P]),
                           ("og_face_fluxes_2d", [D, P, P, P]), ("og_face_fluxes", [D, P, P, P, P])]:
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.og_minmod.argtypes = [ctypes.c_double] * 3
        lib.og_minmod.restype = ctypes.c_double
        _lib = lib
    return _lib


class Grid:
    """Mesh + solver settings for the oracle, taken from a problems.Problem (or
    any object with the same attributes)."""

    def __init__(self, prob, solver=None, theta=None, gamma=None):
        self.ndim = prob.ndim
        self.n = tuple(prob.n)
        self.widths = [np.ascontiguousarray(prob.widths[q], dtype=np.float64) for q in range(prob.ndim)]
        self.bc_lo = tuple(prob.bc_lo)
        self.bc_hi = tuple(prob.bc_hi)
        self.gamma = float(prob.gamma if gamma is None else gamma)
        self.theta = float(prob.theta if theta is None else theta)
        self.solver = int(prob.solver if solver is None else solver)
        self.grad_phi = tuple(float(x) for x in getattr(prob, "grad_phi", (0.0, 0.0, 0.0)))
        d = _Desc()
        d.ndim = self.ndim
        for q in range(3):
            d.n[q] = self.n[q] if q < self.ndim else 1
            d.bc_lo[q] = self.bc_lo[q]
            d.bc_hi[q] = self.bc_hi[q]
            d.width[q] = self.widths[q].ctypes.data if q < self.ndim else None
        d.gamma, d.theta, d.solver = self.gamma, self.theta, self.solver
        for q in range(3):
            d.grad_phi[q] = self.grad_phi[q]
        self._d = d

    @property
    def nvar(self):
        return self.ndim + 2

    @property
    def shape(self):
        return tuple(reversed(self.n[: self.ndim]))

    def _ptr(self):
        return ctypes.byref(self._d)


def _arr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def _check(rc, what):
    if rc == ENONPHYS:
        raise FloatingPointError(f"oracle {what}: non-physical state (rho<=0, p<=0 or NaN)")
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def prim_to_cons(g: Grid, rho, vel, p):
    """U = (D, S_1..S_ndim, G) from (rho, v, p); shape (nvar,) + g.shape."""
    lib = _load()
    rho, pr = _arr(rho)
    vel, pv = _arr(vel)
    p, pp = _arr(p)
    U = np.empty((g.nvar,) + g.shape)
    _check(lib.og_prim_to_cons(g._ptr(), pr, pv, pp, U.ctypes.data), "prim_to_cons")
    return U


def cons_to_prim(g: Grid, U, check=True):
    lib = _load()
    U, pu = _arr(U)
    rho = np.empty(g.shape)
    vel = np.empty((g.ndim,) + g.shape)
    p = np.empty(g.shape)
    rc = lib.og_cons_to_prim(g._ptr(), pu, rho.ctypes.data, vel.ctypes.data, p.ctypes.data)
    if check:
        _check(rc, "cons_to_prim")
    return rho, vel, p


def initial_state(prob, g: Grid | None = None):
    g = g or Grid(prob)
    return prim_to_cons(g, prob.rho, prob.vel, prob.p)


def rhs(g: Grid, U):
    """L[U] (Eq. BalanceEquationAverage without sources)."""
    lib = _load()
    U, pu = _arr(U)
    L = np.empty_like(U)
    _check(lib.og_rhs(g._ptr(), pu, L.ctypes.data), "rhs")
    return L


def step(g: Grid, U, dt):
    """One TVD RK2 step; returns the new state (input untouched)."""
    lib = _load()
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    _check(lib.og_step(g._ptr(), U.ctypes.data, float(dt)), "step")
    return U


def cfl_dt(g: Grid, U):
    """dt_CFL of Eq. courantTimeStep (without the Courant factor)."""
    lib = _load()
    U, pu = _arr(U)
    out = np.zeros(1)
    _check(lib.og_cfl_dt(g._ptr(), pu, out.ctypes.data), "cfl_dt")
    return float(out[0])


def totals(g: Grid, U):
    lib = _load()
    U, pu = _arr(U)
    out = np.zeros(5)
    _check(lib.og_totals(g._ptr(), pu, out.ctypes.data), "totals")
    return out[: g.nvar]


def evolve(g: Grid, U, cfl, t_end=0.0, max_steps=1 << 30):
    """Evolve from t = 0 to t_end (clamping the last step), or exactly max_steps
    steps when t_end <= 0.  Returns (U, t, steps)."""
    lib = _load()
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    t = np.zeros(1)
    n = np.zeros(1, dtype=np.int32)
    _check(lib.og_evolve(g._ptr(), U.ctypes.data, float(cfl), float(t_end), int(max_steps),
                         t.ctypes.data, n.ctypes.data), "evolve")
    return U, float(t[0]), int(n[0])


def riemann_flux(solver, gamma, ndim, axis, primL, primR):
    """Face flux for primitive states (rho, v_1..v_ndim, p); returns (F, diag)
    with diag = (alpha_+, alpha_-, alpha_m, p*_L, p*_R)."""
    lib = _load()
    a, pa = _arr(primL)
    b, pb = _arr(primR)
    F = np.zeros(5)
    diag = np.zeros(5)
    _check(lib.og_riemann_flux(int(solver), float(gamma), int(ndim), int(axis), pa, pb,
                               F.ctypes.data, diag.ctypes.data), "riemann_flux")
    return F[: ndim + 2], diag


def physical_flux(gamma, ndim, axis, prim):
    lib = _load()
    a, pa = _arr(prim)
    F = np.zeros(5)
    _check(lib.og_physical_flux(float(gamma), int(ndim), int(axis), pa, F.ctypes.data), "physical_flux")
    return F[: ndim + 2]


def face_fluxes_2d(g: Grid, U):
    """Plain face fluxes of a 2D state: Fx [4][ny][nx+1], Fy [4][ny+1][nx]."""
    lib = _load()
    U, pu = _arr(U)
    ny, nx = g.shape
    Fx = np.empty((4, ny, nx + 1))
    Fy = np.empty((4, ny + 1, nx))
    _check(lib.og_face_fluxes_2d(g._ptr(), pu, Fx.ctypes.data, Fy.ctypes.data), "face_fluxes_2d")
    return Fx, Fy


def face_fluxes(g: Grid, U):
    """Plain face fluxes along every axis: a list of arrays, axis q of shape
    (nvar,) + (n_2', n_1', n_0') with one more face than cells along q."""
    lib = _load()
    U, pu = _arr(U)
    out = []
    ptrs = []
    for q in range(3):
        if q < g.ndim:
            nf = [g.n[a] if a < g.ndim else 1 for a in range(3)]
            nf[q] += 1
            shape = (g.nvar,) + tuple(reversed(nf[: g.ndim]))
            a = np.empty(shape)
            out.append(a)
            ptrs.append(a.ctypes.data)
        else:
            ptrs.append(None)
    _check(lib.og_face_fluxes(g._ptr(), pu, *ptrs), "face_fluxes")
    return out


def minmod(a, b, c):
    return _load().og_minmod(float(a), float(b), float(c))


def l1_relative(num, ref):
    """Relative L1 norm of Eq. L1ErrorNorm: sum|num - ref| / sum|ref|."""
    num = np.asarray(num, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sum(np.abs(num - ref)) / np.sum(np.abs(ref)))


# ------------------------------------------------------------------ op counts
_count_lib = None
OP_KINDS = ("add", "mul", "div", "sqrt", "minmax", "abs", "total")


def _load_count():
    global _count_lib
    if _count_lib is None:
        build()
        lib = ctypes.CDLL(_COUNT_LIB)
        P = ctypes.c_void_p
        lib.og_count_ops.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, P, ctypes.c_double, P]
        lib.og_count_ops.restype = ctypes.c_int
        _count_lib = lib
    return _count_lib


def count_ops(g: Grid, U, what, param=0.0):
    """Floating-point operations of one oracle call on U, counted by running
    the oracle's code with a counting scalar (opcount.cpp): what = "rhs",
    "step" (dt = param), "cfl_dt" or "totals".  Returns {kind: count}."""
    lib = _load_count()
    code = {"rhs": 0, "step": 1, "cfl_dt": 2, "totals": 3}[what]
    U, pu = _arr(U)
    n = (ctypes.c_int * 3)(*[g.n[q] if q < g.ndim else 1 for q in range(3)])
    w = (ctypes.c_void_p * 3)(*[g.widths[q].ctypes.data if q < g.ndim else None for q in range(3)])
    lo = (ctypes.c_int * 3)(*g.bc_lo[:3])
    hi = (ctypes.c_int * 3)(*g.bc_hi[:3])
    out = (ctypes.c_longlong * 7)()
    rc = lib.og_count_ops(code, g.ndim, n, w, lo, hi, g.gamma, g.theta, g.solver, pu, float(param), out)
    _check(rc, f"count_ops({what})")
    return dict(zip(OP_KINDS, list(out)))


def count_face_flux(solver, gamma, ndim, axis, primL, primR):
    """Operations of the oracle's face flux for primitive states (rho, v, p)."""
    lib = _load_count()
    nv = ndim + 2
    W = np.zeros(2 * nv)
    for s, pr in enumerate((primL, primR)):
        W[s * nv:(s + 1) * nv - 1] = pr[:nv - 1]
        W[s * nv + nv - 1] = pr[nv - 1] / (gamma - 1.0)  # e from p
    n = (ctypes.c_int * 3)(axis, 1, 1)
    out = (ctypes.c_longlong * 7)()
    rc = lib.og_count_ops(4, ndim, n, None, None, None, float(gamma), 1.4, int(solver), W.ctypes.data, 0.0, out)
    _check(rc, "count_face_flux")
    return dict(zip(OP_KINDS, list(out)))

"""Seeded, synthetic initial conditions shaped like the paper's test problems.

This module only builds inputs: mesh widths, boundary codes and primitive
fields (rho, v, p).  It holds none of the solver's arithmetic, so both the CUDA
path and the CPU oracle can take their inputs from here.  Every random number is
drawn from numpy's PCG64 generator with an explicit seed.

Problem setups follow Section 4 of Cardall et al. (arXiv:1207.3392):
advection (Sec. 4.1.1), contact discontinuity and Sod shock tube (Sec. 4.2.1),
double rarefaction (Sec. 4.2.1), implosion (Sec. 4.2.1), interacting blast waves
(Sec. 4.2.2), Sedov-Taylor blast (Sec. 4.2.3), Kelvin-Helmholtz (Sec. 4.3.1),
plus the stretched-mesh pressure pulse and the batched Riemann set that the
benchmark workloads add.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import numpy as np

PERIODIC, REFLECT, OUTFLOW = 0, 1, 2
HLL, HLLC, HLLC_SWITCH = 0, 1, 2  # HLLC_SWITCH: HLLC, with HLL transverse to shocks (Sec. 3.2)


@dataclass
class Problem:
    """A single-level Cartesian problem.

    Arrays are C-ordered with shape ``shape`` = (nz, ny, nx)[-ndim:], x fastest.
    ``vel`` has shape (ndim,) + shape.  ``widths[q]`` has n[q] entries.
    """

    name: str
    ndim: int
    n: tuple
    widths: list
    bc_lo: tuple
    bc_hi: tuple
    gamma: float
    rho: np.ndarray
    vel: np.ndarray
    p: np.ndarray
    solver: int = HLLC
    theta: float = 1.4
    cfl: float = 0.5
    t_end: float = 0.0
    steps: int = 0
    origin: tuple = (0.0, 0.0, 0.0)
    grad_phi: tuple = (0.0, 0.0, 0.0)  # gradient of a linear external potential (force -grad Phi)
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return tuple(reversed(self.n[: self.ndim]))

    @property
    def ncells(self):
        return int(np.prod(self.n[: self.ndim]))

    @property
    def nvar(self):
        return self.ndim + 2

    def centers(self, q):
        """Cell-centre coordinates along axis q (geometric centres)."""
        w = np.asarray(self.widths[q], dtype=np.float64)
        edges = self.origin[q] + np.concatenate([[0.0], np.cumsum(w)])
        return 0.5 * (edges[:-1] + edges[1:])

    def with_(self, **kw):
        d = dict(self.__dict__)
        d.update(kw)
        return Problem(**d)


def _pad3(t, fill):
    t = tuple(t)
    return t + (fill,) * (3 - len(t))


def uniform_widths(n, lo, hi):
    return np.full(n, (hi - lo) / n, dtype=np.float64)


def _make(name, ndim, n, widths, bc, gamma, rho, vel, p, origin, **kw):
    n3 = _pad3(n, 1)
    bc_lo = _pad3(bc[0], PERIODIC)
    bc_hi = _pad3(bc[1], PERIODIC)
    return Problem(name=name, ndim=ndim, n=n3, widths=list(widths), bc_lo=bc_lo, bc_hi=bc_hi,
                   gamma=gamma, rho=np.ascontiguousarray(rho, dtype=np.float64),
                   vel=np.ascontiguousarray(vel, dtype=np.float64),
                   p=np.ascontiguousarray(p, dtype=np.float64), origin=_pad3(origin, 0.0), **kw)


# --------------------------------------------------------------------------- 1D

def riemann_1d(n, left, right, gamma=1.4, x0=0.5, bc=OUTFLOW, name="riemann", axis_len=1.0, **kw):
    """Two constant states (rho, v, p) split at x0 on [0, axis_len]."""
    w = uniform_widths(n, 0.0, axis_len)
    x = (np.arange(n) + 0.5) * (axis_len / n)
    rho = np.where(x < x0, left[0], right[0])
    vel = np.where(x < x0, left[1], right[1])[None, :]
    p = np.where(x < x0, left[2], right[2])
    return _make(name, 1, (n,), [w], ((bc,), (bc,)), gamma, rho, vel, p, (0.0,),
                 meta={"left": tuple(left), "right": tuple(right), "x0": x0}, **kw)


def sod(n=256, t_end=0.2, cfl=0.8, solver=HLLC, paper_states=False):
    """Sod shock tube.  Standard states (1, 0, 1) | (0.125, 0, 0.1); with
    ``paper_states`` the right state is taken as printed in Sec. 4.2.1
    (rho=0.1, p=0.125)."""
    right = (0.1, 0.0, 0.125) if paper_states else (0.125, 0.0, 0.1)
    return riemann_1d(n, (1.0, 0.0, 1.0), right, gamma=1.4, name="sod", t_end=t_end, cfl=cfl,
                      solver=solver)


def contact(n=128, vc=0.0, t_end=2.0, solver=HLLC):
    """Isolated contact discontinuity (Sec. 4.2.1): rho 1.4 | 1.0, p = 1, v = vc."""
    return riemann_1d(n, (1.4, vc, 1.0), (1.0, vc, 1.0), gamma=1.4, name="contact",
                      t_end=t_end, cfl=0.5, solver=solver, bc=PERIODIC)


def double_rarefaction(n=128, t_end=0.15, solver=HLLC):
    """Einfeldt 1-2-0-3 (Sec. 4.2.1): (1, -2, 0.4) | (1, 2, 0.4)."""
    return riemann_1d(n, (1.0, -2.0, 0.4), (1.0, 2.0, 0.4), gamma=1.4, name="double_rarefaction",
                      t_end=t_end, cfl=0.5, solver=solver)


def blast_waves(n=400, t_end=0.038, solver=HLLC):
    """Woodward-Colella interacting blast waves (Sec. 4.2.2), reflecting walls."""
    w = uniform_widths(n, 0.0, 1.0)
    x = (np.arange(n) + 0.5) / n
    rho = np.ones(n)
    p = np.where(x < 0.1, 1000.0, np.where(x > 0.9, 100.0, 0.01))
    return _make("blast_waves", 1, (n,), [w], ((REFLECT,), (REFLECT,)), 1.4, rho,
                 np.zeros((1, n)), p, (0.0,), t_end=t_end, cfl=0.5, solver=solver)


def advection_1d(n, mach=0.6, t_end=1.0, solver=HLLC):
    """Smooth density advection (Sec. 4.1.1): rho = 1 + 0.1 sin(2 pi x), v = 1,
    p = rho0 v^2 / (gamma Ma^2), periodic on [0, 1]."""
    gamma = 1.4
    w = uniform_widths(n, 0.0, 1.0)
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * x)
    p = np.full(n, 1.0 / (gamma * mach * mach))
    return _make("advection_1d", 1, (n,), [w], ((PERIODIC,), (PERIODIC,)), gamma, rho,
                 np.ones((1, n)), p, (0.0,), t_end=t_end, cfl=0.5, solver=solver,
                 meta={"mach": mach})


def sound_wave_1d(n, t_end=1.0, amplitude=1e-6, solver=HLLC):
    """Linear sound wave (Sec. 4.1.2): rho0 = 1, p0 = 3/5, gamma = 5/3 (c0 = 1),
    right-moving eigenvector [c^-2, c^-1 rho^-1, 1] on (rho, v, p)."""
    gamma = 5.0 / 3.0
    w = uniform_widths(n, 0.0, 1.0)
    x = (np.arange(n) + 0.5) / n
    s = amplitude * np.sin(2.0 * np.pi * x)
    return _make("sound_wave_1d", 1, (n,), [w], ((PERIODIC,), (PERIODIC,)), gamma, 1.0 + s,
                 s[None, :], 0.6 + s, (0.0,), t_end=t_end, cfl=0.5, solver=solver)


# --------------------------------------------------------------------------- 2D

def advection_2d(nx, mach=0.6, t_end=1.0, solver=HLLC):
    """Oblique advection (Sec. 4.1.1): Lx = 2 Ly, Ly = sqrt(5)/2, ny = nx / 2,
    domain [0, Lx] x [1, 1 + Ly] as printed (the offset does not matter on a
    periodic domain)."""
    gamma = 1.4
    ly = math.sqrt(5.0) / 2.0
    lx = 2.0 * ly
    ny = nx // 2
    wx = uniform_widths(nx, 0.0, lx)
    wy = uniform_widths(ny, 0.0, ly)
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = 1.0 + (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    rho = 1.0 + 0.1 * np.sin(2.0 * np.pi * (X / lx + Y / ly))
    norm = math.sqrt(lx ** -2 + ly ** -2)
    vx, vy = (1.0 / lx) / norm, (1.0 / ly) / norm
    vel = np.stack([np.full_like(rho, vx), np.full_like(rho, vy)])
    p = np.full_like(rho, 1.0 / (gamma * mach * mach))
    return _make("advection_2d", 2, (nx, ny), [wx, wy], ((PERIODIC,) * 2, (PERIODIC,) * 2), gamma,
                 rho, vel, p, (0.0, 1.0), t_end=t_end, cfl=0.5, solver=solver)


def implosion(n=64, t_end=0.045, solver=HLLC):
    """Liska-Wendroff implosion (Sec. 4.2.1) on [0, 0.3]^2, reflecting walls."""
    w = uniform_widths(n, 0.0, 0.3)
    c = (np.arange(n) + 0.5) * (0.3 / n)
    X, Y = np.meshgrid(c, c)
    inner = (X + Y) <= 0.15
    rho = np.where(inner, 0.125, 1.0)
    p = np.where(inner, 0.14, 1.0)
    return _make("implosion", 2, (n, n), [w, w], ((REFLECT,) * 2, (REFLECT,) * 2), 1.4, rho,
                 np.zeros((2, n, n)), p, (0.0, 0.0), t_end=t_end, cfl=0.5, solver=solver)


def kelvin_helmholtz(n=256, seed=0, solver=HLLC, t_end=1.0, amp_modes=0.01, amp_noise=0.01):
    """Periodic shear layer on [-0.5, 0.5]^2 (the benchmark variant of Sec. 4.3.1):
    rho = 2, vx = +0.5 for |y| < 0.25, else rho = 1, vx = -0.5; p = 2.5;
    vy = [sum_{k=1..4} A sin(2 pi k x + phi_k) + U(-a, a)] psi(y), with
    psi(y) = exp(-0.5 (cos(2 pi y) / (2 pi sigma))^2), sigma = 0.1."""
    rng = np.random.default_rng(seed)
    w = uniform_widths(n, -0.5, 0.5)
    c = -0.5 + (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c)
    inside = np.abs(Y) < 0.25
    rho = np.where(inside, 2.0, 1.0)
    vx = np.where(inside, 0.5, -0.5)
    phases = rng.uniform(0.0, 2.0 * np.pi, size=4)
    modes = sum(amp_modes * np.sin(2.0 * np.pi * k * X + phases[k - 1]) for k in range(1, 5))
    noise = rng.uniform(-amp_noise, amp_noise, size=X.shape)
    sigma = 0.1
    psi = np.exp(-0.5 * (np.cos(2.0 * np.pi * Y) / (2.0 * np.pi * sigma)) ** 2)
    vy = (modes + noise) * psi
    p = np.full_like(rho, 2.5)
    return _make("kelvin_helmholtz", 2, (n, n), [w, w], ((PERIODIC,) * 2, (PERIODIC,) * 2), 1.4,
                 rho, np.stack([vx, vy]), p, (-0.5, -0.5), t_end=t_end, cfl=0.5, solver=solver,
                 meta={"seed": seed, "phases": phases})


def rayleigh_taylor(nx=256, ny=768, solver=HLLC, g=0.1, amp=0.01, t_end=8.5):
    """Rayleigh-Taylor set-up of Sec. 4.3.2: [-0.25, 0.25] x [-0.75, 0.75],
    periodic in x, reflecting in y; rho = 2 above y = 0, 1 below; uniform
    force -g y^ (potential gradient (0, g)); hydrostatic p = 2.5 - rho g y;
    gamma = 1.4; v = A/4 [1 + cos(2 pi x / Lx)] [1 + cos(3 pi y)] y^."""
    lx, ly = 0.5, 1.5
    wx = uniform_widths(nx, -0.25, 0.25)
    wy = uniform_widths(ny, -0.75, 0.75)
    x = -0.25 + (np.arange(nx) + 0.5) * (lx / nx)
    y = -0.75 + (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    rho = np.where(Y > 0.0, 2.0, 1.0)
    p = 2.5 - rho * g * Y
    vy = 0.25 * amp * (1.0 + np.cos(2.0 * np.pi * X / lx)) * (1.0 + np.cos(3.0 * np.pi * Y))
    vel = np.stack([np.zeros_like(vy), vy])
    return _make("rayleigh_taylor", 2, (nx, ny), [wx, wy], ((PERIODIC, REFLECT), (PERIODIC, REFLECT)), 1.4,
                 rho, vel, p, (-0.25, -0.75), t_end=t_end, cfl=0.5, solver=solver, grad_phi=(0.0, g, 0.0))


def free_fall(ndim, n, grad_phi, rho=1.0, p=1.0, gamma=1.4, solver=HLLC):
    """Uniform gas at rest in a periodic box under a uniform force -grad Phi:
    every flux divergence vanishes, so S_q(t) = -rho grad_phi_q t and
    G(t) = G(0) + rho |grad_phi|^2 t^2 / 2 exactly (RK2 integrates both
    exactly)."""
    shape = (n,) * ndim
    w = uniform_widths(n, 0.0, 1.0)
    return _make("free_fall", ndim, shape, [w] * ndim, ((PERIODIC,) * ndim, (PERIODIC,) * ndim), gamma,
                 np.full(shape, rho), np.zeros((ndim,) + shape), np.full(shape, p), (0.0,) * ndim,
                 cfl=0.5, solver=solver, grad_phi=tuple(grad_phi) + (0.0,) * (3 - len(grad_phi)))


def planar_shock(nx=400, ny=20, mach=20.0, solver=HLLC, seed=0, noise=1e-6, gamma=1.4):
    """A strong planar shock moving along +x into gas at rest (rho = 1, p = 1),
    post-shock state from the Rankine-Hugoniot conditions, shock at 10% of the
    channel; outflow in x, periodic in y; density noise of relative size
    `noise` (seeded).  On a Cartesian mesh the HLLC flux lets the noise grow
    into odd-even decoupling behind the shock (Quirk 1994); HLL does not."""
    rho0, p0 = 1.0, 1.0
    c0 = math.sqrt(gamma * p0 / rho0)
    m2 = mach * mach
    rho1 = rho0 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p1 = p0 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    u1 = mach * c0 * (1.0 - rho0 / rho1)
    lx, ly = nx / ny, 1.0
    wx = uniform_widths(nx, 0.0, lx)
    wy = uniform_widths(ny, 0.0, ly)
    X = np.tile((np.arange(nx) + 0.5) * (lx / nx), (ny, 1))
    behind = X < 0.1 * lx
    rng = np.random.default_rng(seed)
    rho = np.where(behind, rho1, rho0) * (1.0 + noise * rng.uniform(-1.0, 1.0, X.shape))
    p = np.where(behind, p1, p0)
    vx = np.where(behind, u1, 0.0)
    return _make("planar_shock", 2, (nx, ny), [wx, wy], ((OUTFLOW, PERIODIC), (OUTFLOW, PERIODIC)), gamma,
                 rho, np.stack([vx, np.zeros_like(vx)]), p, (0.0, 0.0), cfl=0.4, solver=solver,
                 meta={"mach": mach, "post": (rho1, u1, p1)})


def planar_shock_3d(n_long=96, n_cross=12, axis=2, mach=10.0, solver=HLLC, seed=0, noise=1e-6, gamma=1.4):
    """The planar shock of planar_shock in 3D, moving along `axis` (outflow
    along it, periodic across), with seeded density noise."""
    rho0, p0 = 1.0, 1.0
    c0 = math.sqrt(gamma * p0 / rho0)
    m2 = mach * mach
    rho1 = rho0 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p1 = p0 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    u1 = mach * c0 * (1.0 - rho0 / rho1)
    n = [n_cross] * 3
    n[axis] = n_long
    widths = [uniform_widths(n[q], 0.0, n[q] / n_cross) for q in range(3)]
    shape = (n[2], n[1], n[0])
    coord = (np.indices(shape)[2 - axis] + 0.5) / n_cross
    behind = coord < 0.1 * n_long / n_cross
    rng = np.random.default_rng(seed)
    rho = np.where(behind, rho1, rho0) * (1.0 + noise * rng.uniform(-1.0, 1.0, shape))
    p = np.where(behind, p1, p0)
    vel = np.zeros((3,) + shape)
    vel[axis] = np.where(behind, u1, 0.0)
    bc = [PERIODIC] * 3
    bc[axis] = OUTFLOW
    return _make("planar_shock_3d", 3, tuple(n), widths, (tuple(bc), tuple(bc)), gamma, rho, vel, p,
                 (0.0, 0.0, 0.0), cfl=0.3, solver=solver, meta={"mach": mach, "axis": axis})


# --------------------------------------------------------------------------- 3D

def sedov_3d(n=256, solver=HLLC, steps=200, energy=1.0, gamma=1.4, half=1.0):
    """Point blast on [-half, half]^3: rho = 1, p = 1e-5, v = 0, with total
    energy E deposited as internal energy in the central 2^3 cells
    (p = (gamma - 1) E / (8 dV) there), reflecting walls, C_CFL = 0.3."""
    if n % 2:
        raise ValueError("sedov_3d needs an even n so that 2^3 cells sit at the centre")
    w = uniform_widths(n, -half, half)
    dx = w[0]
    rho = np.ones((n, n, n))
    p = np.full((n, n, n), 1e-5)
    c = n // 2
    p[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] = (gamma - 1.0) * energy / (8.0 * dx ** 3)
    return _make("sedov_3d", 3, (n, n, n), [w, w, w], ((REFLECT,) * 3, (REFLECT,) * 3), gamma,
                 rho, np.zeros((3, n, n, n)), p, (-half,) * 3, cfl=0.3, steps=steps, solver=solver,
                 meta={"energy": energy})


def stretched_widths(n_half, d0=1e-3, ratio=1.01):
    """Widths d0 * ratio^k, k = 0..n_half-1, mirrored about the centre."""
    right = d0 * ratio ** np.arange(n_half)
    return np.concatenate([right[::-1], right])


def stretched_pulse_3d(n=320, seed=3, steps=100, solver=HLLC, d0=1e-3, ratio=1.01,
                       amplitude=10.0, sigma=0.05, noise=0.01):
    """Centrally refined rectilinear mesh (widths grow by `ratio` per cell away
    from the centre), Gaussian pressure pulse p = 1 + A exp(-r^2 / (2 sigma^2))
    on rho = 1, seeded velocity noise U(-noise, noise), gamma = 5/3, reflecting
    walls, C_CFL = 0.3."""
    if n % 2:
        raise ValueError("stretched_pulse_3d needs an even n")
    rng = np.random.default_rng(seed)
    w = stretched_widths(n // 2, d0, ratio)
    half = float(np.sum(w[: n // 2]))
    edges = -half + np.concatenate([[0.0], np.cumsum(w)])
    c = 0.5 * (edges[:-1] + edges[1:])
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    p = 1.0 + amplitude * np.exp(-r2 / (2.0 * sigma * sigma))
    rho = np.ones_like(p)
    vel = rng.uniform(-noise, noise, size=(3,) + p.shape)
    return _make("stretched_pulse_3d", 3, (n, n, n), [w, w, w], ((REFLECT,) * 3, (REFLECT,) * 3),
                 5.0 / 3.0, rho, vel, p, (-half,) * 3, cfl=0.3, steps=steps, solver=solver)


def smooth_periodic(ndim, n, seed=0, gamma=1.4, nonuniform=False):
    """Random smooth periodic state (a few Fourier modes) for conservation and
    parity tests; optionally with non-uniform widths."""
    rng = np.random.default_rng(seed)
    ns = (n,) * ndim
    shape = tuple(reversed(ns))
    grids = np.meshgrid(*[(np.arange(m) + 0.5) / m for m in reversed(ns)], indexing="ij")

    def field(amp):
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 3, size=ndim)
            ph = rng.uniform(0, 2 * np.pi)
            arg = sum(2 * np.pi * k[a] * grids[ndim - 1 - a] for a in range(ndim)) + ph
            f += amp * np.sin(arg)
        return f

    rho = 1.0 + field(0.1)
    p = 1.0 + field(0.1)
    vel = np.stack([field(0.3) for _ in range(ndim)])
    widths = []
    for q in range(ndim):
        if nonuniform:
            w = 1.0 + 0.5 * rng.uniform(size=n)
            widths.append(w / w.sum())
        else:
            widths.append(uniform_widths(n, 0.0, 1.0))
    return _make("smooth_periodic", ndim, ns, widths, ((PERIODIC,) * ndim, (PERIODIC,) * ndim),
                 gamma, rho, vel, p, (0.0,) * ndim, cfl=0.5)


def random_blocks(ndim, n, seed=0, bc=REFLECT, gamma=1.4, nonuniform=True):
    """Piecewise-constant random blocks (discontinuities in every direction),
    for parity tests that exercise every HLLC branch and the limiter clipping."""
    rng = np.random.default_rng(seed)
    ns = (n,) * ndim if np.isscalar(n) else tuple(n)
    shape = tuple(reversed(ns))
    blocks = tuple(max(1, m // 5) for m in shape)
    def up(a):
        for ax, m in enumerate(shape):
            reps = -(-m // a.shape[ax])
            a = np.repeat(a, reps, axis=ax)
            a = np.take(a, np.arange(m), axis=ax)
        return a
    rho = up(np.exp(rng.uniform(np.log(0.2), np.log(5.0), size=blocks)))
    p = up(np.exp(rng.uniform(np.log(0.1), np.log(10.0), size=blocks)))
    vel = np.stack([up(rng.uniform(-1.0, 1.0, size=blocks)) for _ in range(ndim)])
    widths = []
    for q in range(ndim):
        m = ns[q]
        if nonuniform:
            w = 1.0 + 0.8 * rng.uniform(size=m)
            widths.append(w / w.sum())
        else:
            widths.append(uniform_widths(m, 0.0, 1.0))
    return _make("random_blocks", ndim, ns, widths, ((bc,) * ndim, (bc,) * ndim), gamma, rho, vel,
                 p, (0.0,) * ndim, cfl=0.4)


# ------------------------------------------------------------------ batched set

@dataclass
class BatchSpec:
    """Compact description of one problem of the batched Riemann set; the
    arrays are only built by ``batch_problem`` so that thousands of problems
    never sit in host memory at once."""

    index: int
    ndim: int
    n: int
    gamma: float
    states: tuple  # 1D: (L, R); 2D: quadrants (lo x lo y, hi x lo y, lo x hi y, hi x hi y); each (rho, vx, vy, p)
    steps: int


def batched_riemann(count=4096, seed=4, n1_range=(128, 4096), n2_range=(64, 512), steps=50):
    """Independent 1D and 2D Riemann problems of uneven size: half 1D (n uniform
    in n1_range on [0, 1], interface at 0.5, outflow), half 2D (n uniform in
    n2_range, square [0, 1]^2, four quadrant states, outflow); rho log-uniform
    in [0.1, 10], p log-uniform in [0.01, 100], v uniform in [-2, 2], gamma in
    {1.4, 5/3}.  States whose velocity jump would open a vacuum
    (dv >= 2 (c_L + c_R) / (gamma - 1)) are redrawn from the same stream."""
    rng = np.random.default_rng(seed)
    out = []

    def state():
        rho = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
        p = math.exp(rng.uniform(math.log(0.01), math.log(100.0)))
        v = rng.uniform(-2.0, 2.0, size=2)
        return (rho, float(v[0]), float(v[1]), p)

    def no_vacuum(a, b, gamma, axis):
        ca = math.sqrt(gamma * a[3] / a[0])
        cb = math.sqrt(gamma * b[3] / b[0])
        return (b[1 + axis] - a[1 + axis]) < 2.0 * (ca + cb) / (gamma - 1.0)

    n1 = count // 2
    for idx in range(count):
        gamma = 1.4 if rng.uniform() < 0.5 else 5.0 / 3.0
        if idx < n1:
            n = int(rng.integers(n1_range[0], n1_range[1] + 1))
            while True:
                L, R = state(), state()
                if no_vacuum(L, R, gamma, 0):
                    break
            out.append(BatchSpec(idx, 1, n, gamma, (L, R), steps))
        else:
            n = int(rng.integers(n2_range[0], n2_range[1] + 1))
            while True:
                q = [state() for _ in range(4)]
                ok = (no_vacuum(q[0], q[1], gamma, 0) and no_vacuum(q[2], q[3], gamma, 0)
                      and no_vacuum(q[0], q[2], gamma, 1) and no_vacuum(q[1], q[3], gamma, 1))
                if ok:
                    break
            out.append(BatchSpec(idx, 2, n, gamma, tuple(q), steps))
    return out


def batch_problem(spec: BatchSpec) -> Problem:
    """Materialise one BatchSpec as a Problem (outflow walls, C_CFL = 0.5, HLLC)."""
    n = spec.n
    if spec.ndim == 1:
        L, R = spec.states
        return riemann_1d(n, (L[0], L[1], L[3]), (R[0], R[1], R[3]), gamma=spec.gamma,
                          name=f"batch1d_{spec.index}", steps=spec.steps, cfl=0.5, solver=HLLC)
    q = spec.states
    w = uniform_widths(n, 0.0, 1.0)
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c)
    sel = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    rho = np.choose(sel, [s[0] for s in q])
    vx = np.choose(sel, [s[1] for s in q])
    vy = np.choose(sel, [s[2] for s in q])
    p = np.choose(sel, [s[3] for s in q])
    return _make(f"batch2d_{spec.index}", 2, (n, n), [w, w], ((OUTFLOW,) * 2, (OUTFLOW,) * 2),
                 spec.gamma, rho, np.stack([vx, vy]), p, (0.0, 0.0), cfl=0.5, steps=spec.steps,
                 solver=HLLC)

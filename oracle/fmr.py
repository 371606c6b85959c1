"""FP64 reference of the multilevel evolution with subcycling (GenASiS I,
Sec. 3.7, Algorithms Evolve, EvolveLevel and StepLevel) on a fixed mesh of
nested levels.  TEST INFRASTRUCTURE ONLY: the CUDA path never imports it.

Readings (the paper's levels are cell-by-cell refinements of an oct-tree; this
reference uses nested boxes):
  * Level 0 is an N^d mesh over the domain with the problem's walls.  Level l
    >= 1 is an N^d mesh over the central half of level l-1 (per axis) at twice
    its resolution, so its cells are the children of the coarse cells
    [N/4, 3N/4) of level l-1.  N is a multiple of 4 and at least 16.
  * A level l >= 1 is stored with a ring of two exterior (ghost) cells.  The
    ring is filled by prolongation from level l-1 before each step of level l
    and held fixed through both RK substeps: each child value is the coarse
    value plus the minmod-limited slopes of the conserved variables times
    the offset of the child centre (+-h_coarse/4 per axis), so the children
    average to the coarse value.
  * Restriction: a covered coarse cell becomes the mean of its 2^d children.
  * Flux replacement: after a step of level l, each uncovered coarse cell
    next to the box of level l+1 has the time integral of the coarse flux
    through the shared face, dt (F1 + F2)/2 (the Heun-effective flux of Eqs.
    RungeKutta1-3), replaced by the one the fine level accumulated over its two
    steps, the mean over the 2^(d-1) fine faces of sum dt_f (F1 + F2)/2.
  * Time step: the deepest level steps with C * min over levels l of
    dt_CFL(l) / 2^(L-1-l) (each level's CFL time divided by its number of
    substeps per coarse step), so every level keeps its own CFL condition;
    coarser levels step by the time their child has advanced.
  * The provisional coarse half-step before a level's second step is one
    forward-Euler substep of the coarse level (Eq. RungeKutta2) by the
    child's first step, without flux replacement; the coarse state is
    restored after the child's second step.  (The paper reuses those coarse
    fluxes in the proper coarse step; recomputing them gives the same values.)
  * Conservation is tallied on leaf cells (cells not covered by a finer level).
"""
from __future__ import annotations

import numpy as np

from . import Grid, cons_to_prim, face_fluxes, prim_to_cons, rhs

NG = 2  # exterior ring width of levels >= 1


class _Mesh:
    """Minimal problem description for the oracle's Grid."""

    def __init__(self, ndim, n, widths, bc_lo, bc_hi, gamma, theta, solver):
        self.ndim = ndim
        self.n = tuple(n) + (1,) * (3 - len(n))
        self.widths = widths
        self.bc_lo = tuple(bc_lo) + (0,) * (3 - len(bc_lo))
        self.bc_hi = tuple(bc_hi) + (0,) * (3 - len(bc_hi))
        self.gamma = gamma
        self.theta = theta
        self.solver = solver


class Multilevel:
    """Nested-box levels over [lo, lo + size]^ndim with N cells per axis each."""

    def __init__(self, ndim, N, nlevels, lo, size, bc, gamma=1.4, theta=1.4, solver=1):
        if N % 4 or N < 16:
            raise ValueError("N must be a multiple of 4 and at least 16")
        self.ndim, self.N, self.nlevels = ndim, N, nlevels
        self.gamma, self.theta, self.solver = gamma, theta, solver
        self.h = [size / N / 2 ** l for l in range(nlevels)]
        # low corner of each level's box
        self.lo = [lo + 0.5 * size * (1.0 - 0.5 ** l) for l in range(nlevels)]
        self.grids = []
        for l in range(nlevels):
            npad = N + (2 * NG if l else 0)
            w = np.full(npad, self.h[l])
            b = (bc,) * ndim if l == 0 else (2,) * ndim   # outflow around the padded array (never read by interior cells)
            self.grids.append(Grid(_Mesh(ndim, (npad,) * ndim, [w] * ndim, b, b, gamma, theta, solver)))
        self.U = [None] * nlevels
        self.time = [0.0] * nlevels

    # ---------------------------------------------------------------- indexing
    def interior(self, l):
        """Slices of level l's interior in its stored array (vars first)."""
        o = NG if l else 0
        return (slice(None),) + (slice(o, o + self.N),) * self.ndim

    def covered(self, l):
        """Slices of the cells of level l covered by level l+1 (stored indices)."""
        o = NG if l else 0
        a = o + self.N // 4
        return (slice(None),) + (slice(a, a + self.N // 2),) * self.ndim

    def centers(self, l, stored=False):
        """Cell-centre coordinates of level l per axis (interior, or the stored
        padded array)."""
        k = np.arange(-NG, self.N + NG) if (stored and l) else np.arange(self.N)
        return self.lo[l] + (k + 0.5) * self.h[l]

    # ---------------------------------------------------------------- transfers
    def restrict(self, l):
        """Covered cells of level l = mean of their children on level l+1."""
        f = self.U[l + 1][self.interior(l + 1)]
        for ax in range(1, self.ndim + 1):
            sh = list(f.shape)
            sh[ax] //= 2
            sh.insert(ax + 1, 2)
            f = f.reshape(sh).mean(axis=ax + 1)
        self.U[l][self.covered(l)] = f

    def prolong(self, l):
        """Fill the exterior ring of level l (>= 1) from level l-1."""
        N, nd = self.N, self.ndim
        Uc = self.U[l - 1]
        oc = NG if l - 1 else 0
        hc = self.h[l - 1]
        # the fine stored cells 0 .. N+3 are the children of coarse cells
        # N/4 - 1 .. 3N/4; take those with one more coarse cell on each side
        a = N // 4 - 1 + oc
        m = N // 2 + 2
        B = Uc[(slice(None),) + (slice(a - 1, a + m + 1),) * nd]
        core = (slice(None),) + (slice(1, m + 1),) * nd
        sub = B[core]
        out = sub
        for ax in range(1, nd + 1):
            out = np.repeat(out, 2, axis=ax)
        for q in range(nd):
            ax = nd - q  # array axis of coordinate q (x fastest)
            lo_sel, hi_sel = list(core), list(core)
            lo_sel[ax] = slice(0, m)
            hi_sel[ax] = slice(2, m + 2)
            # minmod of the one-sided differences; times the child offset
            # -+h_c/4 this is the limited slope times the offset
            dm = sub - B[tuple(lo_sel)]
            dp = B[tuple(hi_sel)] - sub
            s = np.where(dm * dp > 0.0, np.where(np.abs(dm) < np.abs(dp), dm, dp), 0.0)
            for ax2 in range(1, nd + 1):
                s = np.repeat(s, 2, axis=ax2)
            off = np.tile(np.array([-0.25, 0.25]), m)
            shape = [1] * (nd + 1)
            shape[ax] = -1
            out = out + s * off.reshape(shape)
        ring = np.ones(out.shape[1:], dtype=bool)
        ring[(slice(NG, NG + N),) * nd] = False
        self.U[l][:, ring] = out[:, ring]

    # ---------------------------------------------------------------- one level
    def cfl_dt(self, l):
        """min over the interior cells of level l of min_q h / (|v_q| + c_s)."""
        rho, vel, p = cons_to_prim(self.grids[l], self.U[l])
        sl = self.interior(l)[1:]
        cs = np.sqrt(self.gamma * p[sl] / rho[sl])
        speed = np.max([np.abs(vel[q][sl]) + cs for q in range(self.ndim)], axis=0)
        return float(self.h[l] / speed.max())

    def _effective_fluxes(self, l, U0, U1):
        g = self.grids[l]
        F1 = face_fluxes(g, U0)
        F2 = face_fluxes(g, U1)
        return [0.5 * (a + b) for a, b in zip(F1, F2)]

    def _ring_mask(self, l):
        m = np.ones((self.N + 2 * NG,) * self.ndim, dtype=bool)
        m[(slice(NG, NG + self.N),) * self.ndim] = False
        return m

    def rk2(self, l, dt, from_children=None):
        """One Heun step of level l with its exterior ring held; returns the
        effective face fluxes (for the parent's flux replacement)."""
        g = self.grids[l]
        U0 = self.U[l]
        L1 = rhs(g, U0)
        U1 = U0 + dt * L1
        if l:
            ring = self._ring_mask(l)
            U1[:, ring] = U0[:, ring]
        L2 = rhs(g, U1)
        Un = U0 + 0.5 * dt * (L1 + L2)
        if l:
            Un[:, ring] = U0[:, ring]
        F = self._effective_fluxes(l, U0, U1)
        if from_children is not None:
            self._replace_fluxes(l, Un, dt, F, from_children)
        self.U[l] = Un
        return F

    def _face_window(self, l, q, side):
        """Stored-array slices of level l's faces on the boundary of level
        l+1's box along axis q (side 0: low, 1: high), as face indices of the
        face arrays (axis q has n+1 faces)."""
        N, nd = self.N, self.ndim
        o = NG if l else 0
        sel = [slice(None)] * (nd + 1)
        for r in range(nd):
            ax = nd - r
            if r == q:
                sel[ax] = o + (N // 4 if side == 0 else 3 * N // 4)
            else:
                sel[ax] = slice(o + N // 4, o + 3 * N // 4)
        return tuple(sel)

    def _outer_cells(self, l, q, side):
        N, nd = self.N, self.ndim
        o = NG if l else 0
        sel = [slice(None)] * (nd + 1)
        for r in range(nd):
            ax = nd - r
            if r == q:
                sel[ax] = o + (N // 4 - 1 if side == 0 else 3 * N // 4)
            else:
                sel[ax] = slice(o + N // 4, o + 3 * N // 4)
        return tuple(sel)

    def _replace_fluxes(self, l, Un, dt, F, phi):
        h = self.h[l]
        for q in range(self.ndim):
            for side in (0, 1):
                fc = F[q][self._face_window(l, q, side)]
                sign = 1.0 if side == 0 else -1.0
                Un[self._outer_cells(l, q, side)] += sign * (dt * fc - phi[q][side]) / h

    def boundary_fluxes(self, l, F, dt):
        """dt x the effective fluxes of level l (>= 1) through its box boundary,
        averaged onto the parent's faces: phi[q][side], transverse shape
        (N/2,)^(d-1) in stored order."""
        N, nd = self.N, self.ndim
        out = []
        for q in range(nd):
            pair = []
            for side in (0, 1):
                sel = [slice(None)] * (nd + 1)
                for r in range(nd):
                    ax = nd - r
                    sel[ax] = (NG if side == 0 else NG + N) if r == q else slice(NG, NG + N)
                f = F[q][tuple(sel)]
                # average pairs of fine faces along each transverse axis
                for ax in range(1, f.ndim):
                    sh = list(f.shape)
                    sh[ax] //= 2
                    sh.insert(ax + 1, 2)
                    f = f.reshape(sh).mean(axis=ax + 1)
                pair.append(dt * f)
            out.append(pair)
        return out

    # ---------------------------------------------------------------- evolution
    def _evolve_level(self, i, acc, cfl):
        self._step_level(i, acc, cfl)
        if i == 0:
            return
        save = self.U[i - 1].copy()
        dtc = self.time[i] - self.time[i - 1]
        # provisional coarse substep (forward Euler), exterior held
        L1 = rhs(self.grids[i - 1], self.U[i - 1])
        Up = self.U[i - 1] + dtc * L1
        if i - 1:
            ring = self._ring_mask(i - 1)
            Up[:, ring] = self.U[i - 1][:, ring]
        self.U[i - 1] = Up
        self._step_level(i, acc, cfl)
        self.U[i - 1] = save

    def _step_level(self, i, acc, cfl):
        L = self.nlevels
        phi = None
        if i + 1 < L:
            acc_next = [[0.0, 0.0] for _ in range(self.ndim)]
            self._evolve_level(i + 1, acc_next, cfl)
            phi = acc_next
        if i > 0:
            self.prolong(i)
        if i == L - 1:
            dt = cfl * min(self.cfl_dt(l) / 2 ** (L - 1 - l) for l in range(L))
        else:
            dt = self.time[i + 1] - self.time[i]
        F = self.rk2(i, dt, phi)
        if i + 1 < L:
            self.restrict(i)
        self.time[i] += dt
        if acc is not None:
            b = self.boundary_fluxes(i, F, dt)
            for q in range(self.ndim):
                for side in (0, 1):
                    acc[q][side] = acc[q][side] + b[q][side]

    def step(self, cfl):
        """One global step (Algorithm Evolve, one pass of its loop)."""
        t = self.time[0]
        self.time = [t] * self.nlevels
        self._evolve_level(0, None, cfl)
        return self.time[0]

    def leaf_totals(self):
        """Sum over leaf cells of U h^d, per conserved variable."""
        tot = np.zeros(self.ndim + 2)
        for l in range(self.nlevels):
            u = self.U[l][self.interior(l)].copy()
            if l + 1 < self.nlevels:
                o = self.N // 4
                u[(slice(None),) + (slice(o, o + self.N // 2),) * self.ndim] = 0.0
            tot += u.reshape(self.ndim + 2, -1).sum(axis=1) * self.h[l] ** self.ndim
        return tot


def sedov(ndim, N, nlevels, energy=1.0, gamma=1.4, half=0.5, solver=1):
    """Point blast on nested levels over [-half, half]^d (Sec. 4.2.6 set-up,
    reflecting walls): rho = 1, p = 1e-5, the energy deposited as internal
    energy in the central 2^d cells of the finest level; coarser levels take
    the restriction of the finer ones where covered."""
    M = Multilevel(ndim, N, nlevels, -half, 2 * half, bc=1, gamma=gamma, solver=solver)
    for l in range(nlevels):
        npad = N + (2 * NG if l else 0)
        shape = (npad,) * ndim
        rho = np.ones(shape)
        p = np.full(shape, 1e-5)
        vel = np.zeros((ndim,) + shape)
        if l == nlevels - 1:
            o = (NG if l else 0) + N // 2 - 1
            cv = M.h[l] ** ndim
            p[(slice(o, o + 2),) * ndim] = (gamma - 1.0) * energy / (2 ** ndim * cv)
        M.U[l] = prim_to_cons(M.grids[l], rho, vel, p)
    for l in range(nlevels - 2, -1, -1):
        M.restrict(l)
    for l in range(1, nlevels):
        M.prolong(l)
    return M

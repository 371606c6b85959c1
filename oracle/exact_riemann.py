"""Exact solution of the ideal-gas Riemann problem (TEST INFRASTRUCTURE ONLY).

Used to pin the oracle on two-state problems (the Sod shock tube and the other
Riemann problems of Sec. 4.2.1 of arXiv:1207.3392).  Written from the
mathematics of the problem, not from any program:

* Across a shock from state K = (rho_K, u_K, p_K) to pressure p the velocity
  changes by (p - p_K) sqrt(A_K / (p + B_K)), A_K = 2 / ((g+1) rho_K),
  B_K = (g-1)/(g+1) p_K (Rankine-Hugoniot); across a rarefaction by
  2 c_K / (g-1) ((p / p_K)^((g-1)/(2g)) - 1) (isentropic Riemann invariant).
* The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0; f is increasing in
  p, so a bracketing root finder (Brent) finds it to machine precision.
* The solution is self-similar in s = (x - x0) / t and is sampled wave by wave.

A vacuum (2 (c_L + c_R) / (g - 1) <= u_R - u_L) raises ValueError.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


class RiemannSolution:
    def __init__(self, left, right, gamma):
        self.rL, self.uL, self.pL = map(float, left)
        self.rR, self.uR, self.pR = map(float, right)
        self.g = float(gamma)
        g = self.g
        self.cL = math.sqrt(g * self.pL / self.rL)
        self.cR = math.sqrt(g * self.pR / self.rR)
        if 2.0 * (self.cL + self.cR) / (g - 1.0) <= self.uR - self.uL:
            raise ValueError("initial data generate a vacuum")
        self.pstar = self._solve_pstar()
        fL, _ = self._f(self.pstar, self.rL, self.pL, self.cL)
        fR, _ = self._f(self.pstar, self.rR, self.pR, self.cR)
        self.ustar = 0.5 * (self.uL + self.uR) + 0.5 * (fR - fL)

    def _f(self, p, rK, pK, cK):
        g = self.g
        if p > pK:
            A = 2.0 / ((g + 1.0) * rK)
            B = (g - 1.0) / (g + 1.0) * pK
            q = math.sqrt(A / (p + B))
            return (p - pK) * q, q * (1.0 - 0.5 * (p - pK) / (B + p))
        e = (g - 1.0) / (2.0 * g)
        return 2.0 * cK / (g - 1.0) * ((p / pK) ** e - 1.0), (p / pK) ** (-(g + 1.0) / (2.0 * g)) / (rK * cK)

    def pressure_function(self, p):
        return (self._f(p, self.rL, self.pL, self.cL)[0] + self._f(p, self.rR, self.pR, self.cR)[0]
                + self.uR - self.uL)

    def _solve_pstar(self):
        lo = 1e-300
        hi = max(self.pL, self.pR)
        while self.pressure_function(hi) < 0.0:
            hi *= 2.0
        if self.pressure_function(lo) >= 0.0:
            return lo
        return brentq(self.pressure_function, lo, hi, xtol=1e-300, rtol=4.0 * np.finfo(float).eps,
                      maxiter=500)

    def sample(self, s):
        """Primitive state (rho, u, p) at similarity coordinate s = x/t (arrays)."""
        s = np.asarray(s, dtype=np.float64)
        rho = np.empty_like(s)
        u = np.empty_like(s)
        p = np.empty_like(s)
        for idx, si in np.ndenumerate(s):
            rho[idx], u[idx], p[idx] = self._sample1(float(si))
        return rho, u, p

    def _sample1(self, s):
        g = self.g
        ps, us = self.pstar, self.ustar
        gm = (g - 1.0) / (g + 1.0)
        if s <= us:
            rK, uK, pK, cK = self.rL, self.uL, self.pL, self.cL
            if ps > pK:
                SK = uK - cK * math.sqrt((g + 1.0) / (2.0 * g) * ps / pK + (g - 1.0) / (2.0 * g))
                if s <= SK:
                    return rK, uK, pK
                return rK * (ps / pK + gm) / (gm * ps / pK + 1.0), us, ps
            head = uK - cK
            cs = cK * (ps / pK) ** ((g - 1.0) / (2.0 * g))
            tail = us - cs
            if s <= head:
                return rK, uK, pK
            if s >= tail:
                return rK * (ps / pK) ** (1.0 / g), us, ps
            u = 2.0 / (g + 1.0) * (cK + 0.5 * (g - 1.0) * uK + s)
            c = 2.0 / (g + 1.0) * (cK + 0.5 * (g - 1.0) * (uK - s))
            return rK * (c / cK) ** (2.0 / (g - 1.0)), u, pK * (c / cK) ** (2.0 * g / (g - 1.0))
        rK, uK, pK, cK = self.rR, self.uR, self.pR, self.cR
        if ps > pK:
            SK = uK + cK * math.sqrt((g + 1.0) / (2.0 * g) * ps / pK + (g - 1.0) / (2.0 * g))
            if s >= SK:
                return rK, uK, pK
            return rK * (ps / pK + gm) / (gm * ps / pK + 1.0), us, ps
        head = uK + cK
        cs = cK * (ps / pK) ** ((g - 1.0) / (2.0 * g))
        tail = us + cs
        if s >= head:
            return rK, uK, pK
        if s <= tail:
            return rK * (ps / pK) ** (1.0 / g), us, ps
        u = 2.0 / (g + 1.0) * (-cK + 0.5 * (g - 1.0) * uK + s)
        c = 2.0 / (g + 1.0) * (cK - 0.5 * (g - 1.0) * (uK - s))
        return rK * (c / cK) ** (2.0 / (g - 1.0)), u, pK * (c / cK) ** (2.0 * g / (g - 1.0))

    def at_points(self, x, t, x0=0.5):
        return self.sample((np.asarray(x, dtype=np.float64) - x0) / t)

    def cell_averages(self, edges, t, x0=0.5, sub=64):
        """Cell averages of (rho, u, p) over [edges[i], edges[i+1]] by the
        midpoint rule on `sub` sub-cells."""
        edges = np.asarray(edges, dtype=np.float64)
        frac = (np.arange(sub) + 0.5) / sub
        pts = edges[:-1, None] + (edges[1:] - edges[:-1])[:, None] * frac[None, :]
        r, u, p = self.at_points(pts, t, x0)
        return r.mean(axis=1), u.mean(axis=1), p.mean(axis=1)

"""Sedov-Taylor self-similar point blast (TEST INFRASTRUCTURE ONLY).

Pins the oracle on the 3D point blast (Sec. 4.2.3 of arXiv:1207.3392).  The
paper quotes the dimensional estimate R = (E t^2 / rho0)^(1/5) (i.e. xi0 = 1);
the true constant xi0 comes from the energy integral of the similarity
solution, which is computed here from the equations of motion:

Spherical, adiabatic ideal-gas flow behind a strong shock at R(t) = A t^(2/5).
With x = r / R, v = R' f(x), rho = rho0 g(x), p = rho0 R'^2 h(x) the
continuity, momentum and entropy equations become the ODEs

    (f - x) g' + g f'              = -2 g f / x
    (f - x) f' + h' / g            = (3/2) f
    (f - x) (h'/h - gamma g'/g)    = 3

with strong-shock values at x = 1: g = (gamma+1)/(gamma-1),
f = h = 2/(gamma+1).  Energy conservation E = int (rho v^2 / 2 + p/(gamma-1)) dV
gives xi0^5 = 25 / (16 pi I), I = int_0^1 (g f^2 / 2 + h/(gamma-1)) x^2 dx.
The ODEs are integrated inward from the shock with scipy's solve_ivp.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(x, y, gamma):
    f, g, h = y
    a = f - x
    # linear system M [f', g', h'] = b
    M = np.array([[g, a, 0.0],
                  [a, 0.0, 1.0 / g],
                  [0.0, -gamma * a / g, a / h]])
    b = np.array([-2.0 * g * f / x, 1.5 * f, 3.0])
    return np.linalg.solve(M, b)


class SedovSolution:
    def __init__(self, gamma=1.4, x_min=1e-4):
        self.gamma = gamma
        y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
        sol = solve_ivp(_rhs, (1.0, x_min), y0, args=(gamma,), rtol=1e-11, atol=1e-13,
                        dense_output=True, method="DOP853")
        if not sol.success:
            raise RuntimeError(sol.message)
        self._sol = sol
        xs = np.linspace(x_min, 1.0, 20001)
        f, g, h = sol.sol(xs)
        integrand = (0.5 * g * f * f + h / (gamma - 1.0)) * xs * xs
        I = np.trapezoid(integrand, xs)
        self.energy_integral = I
        self.xi0 = (25.0 / (16.0 * math.pi * I)) ** 0.2

    def radius(self, t, energy=1.0, rho0=1.0):
        return self.xi0 * (energy * t * t / rho0) ** 0.2

    def time_at_radius(self, R, energy=1.0, rho0=1.0):
        return math.sqrt(rho0 * (R / self.xi0) ** 5 / energy)

    def profile(self, r, t, energy=1.0, rho0=1.0):
        """(rho, v, p) at radii r and time t (zero-pressure background)."""
        R = self.radius(t, energy, rho0)
        Rdot = 0.4 * R / t
        x = np.asarray(r, dtype=np.float64) / R
        rho = np.full_like(x, rho0)
        v = np.zeros_like(x)
        p = np.zeros_like(x)
        inside = (x <= 1.0) & (x >= self._sol.t[-1])
        f, g, h = self._sol.sol(np.clip(x[inside], self._sol.t[-1], 1.0))
        rho[inside] = rho0 * g
        v[inside] = Rdot * f
        p[inside] = rho0 * Rdot * Rdot * h
        return rho, v, p

    def post_shock(self, t, energy=1.0, rho0=1.0):
        """Strong-shock jump values just behind the shock (Eq. JumpConditions)."""
        gm = self.gamma
        R = self.radius(t, energy, rho0)
        Rdot = 0.4 * R / t
        return rho0 * (gm + 1.0) / (gm - 1.0), 2.0 * Rdot / (gm + 1.0), 2.0 * rho0 * Rdot * Rdot / (gm + 1.0)

"""Whole-scheme pins of the oracle: it must reproduce the L1 error tables the
paper prints (Sec. 4.1.1 advection tables, Sec. 4.2.1 Sod table).  These fix
theta = 1.4, C_CFL = 0.5, the HLL/HLLC fluxes, the reconstruction and RK2: a
dropped term or a wrong sign anywhere changes the printed digits."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.exact_riemann import RiemannSolution
from paper_1207_3392_gb300 import problems as P
from conftest import golden


def _sod_l1(n, solver):
    pr = P.sod(n, t_end=0.25, cfl=0.5, solver=solver)
    g = O.Grid(pr)
    U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 0.25)
    assert t == 0.25
    rho, _, p = O.cons_to_prim(g, U)
    ex = RiemannSolution(pr.meta["left"], pr.meta["right"], 1.4)
    re, _, pe = ex.at_points(pr.centers(0), t)
    return O.l1_relative(rho, re), O.l1_relative(p, pe)


@pytest.mark.parametrize("row", [r for r in golden("sod_l1.txt") if int(r[0]) <= 512],
                         ids=lambda r: f"N{r[0]}")
def test_sod_table(row):
    """Sod, t = 0.25: matches the printed 4 significant digits for N >= 64."""
    n = int(row[0])
    tol = 1.2e-2 if n == 32 else 1.2e-3
    for solver, (cr, cp) in ((0, (1, 2)), (1, (3, 4))):
        l1r, l1p = _sod_l1(n, solver)
        assert l1r == pytest.approx(float(row[cr]), rel=tol)
        assert l1p == pytest.approx(float(row[cp]), rel=tol)


def test_sod_printed_right_state_is_a_misprint():
    """The right state as printed (rho=0.1, p=0.125) misses the table by >10%."""
    pr = P.sod(128, t_end=0.25, cfl=0.5, solver=1, paper_states=True)
    g = O.Grid(pr)
    U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 0.25)
    rho, _, _ = O.cons_to_prim(g, U)
    ex = RiemannSolution(pr.meta["left"], pr.meta["right"], 1.4)
    l1 = O.l1_relative(rho, ex.at_points(pr.centers(0), t)[0])
    assert abs(l1 / 7.803e-3 - 1.0) > 0.1


def _adv1d(n, mach, solver, t_end, theta=1.4):
    pr = P.advection_1d(n, mach, solver=solver, t_end=t_end)
    g = O.Grid(pr, theta=theta)
    U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, t_end)
    return O.l1_relative(U[0], pr.rho)


def test_advection_1d_tables():
    """1D advection: every entry equals the printed one divided by a single
    constant, c = pi to within 2.5%, for both Mach numbers, both solvers and
    both times; the shape of all 40 entries (and so every convergence rate)
    is reproduced.  (The constant is a normalisation difference in the 1D
    tables only: the 2D table below matches with c = 1.)"""
    ratios = []
    for row in golden("advection_1d.txt"):
        mach, n = float(row[0]), int(row[1])
        if n > 256:
            continue
        for col, (solver, t_end) in enumerate(((0, 1.0), (1, 1.0), (0, 5.0), (1, 5.0))):
            ratios.append(float(row[2 + col]) / _adv1d(n, mach, solver, t_end))
    ratios = np.array(ratios)
    assert np.all(np.abs(ratios / math.pi - 1.0) < 0.025), ratios / math.pi


def test_advection_1d_table_rejects_other_theta():
    """theta = 1.2 or 1.6 cannot be brought onto the table by any constant."""
    rows = [r for r in golden("advection_1d.txt") if r[0] == "0.6" and int(r[1]) <= 128]
    for theta in (1.2, 1.6):
        r = np.array([float(row[3]) / _adv1d(int(row[1]), 0.6, 1, 1.0, theta) for row in rows])
        assert (r.max() - r.min()) / r.mean() > 0.05


@pytest.mark.parametrize("row", [r for r in golden("advection_2d.txt") if int(r[0]) <= 64],
                         ids=lambda r: f"N{r[0]}")
def test_advection_2d_table(row):
    """2D oblique advection at t = 1 matches the printed values (2%)."""
    n = int(row[0])
    for solver, col in ((0, 1), (1, 2)):
        pr = P.advection_2d(n, solver=solver)
        g = O.Grid(pr)
        U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 1.0)
        assert O.l1_relative(U[0], pr.rho) == pytest.approx(float(row[col]), rel=0.02)


def test_blast_waves_peak_density():
    """Interacting blast waves, 400 cells, HLLC, t = 0.038: max rho about 5.4."""
    row = {r[0]: float(r[1]) for r in golden("printed_values.txt")}
    pr = P.blast_waves(400)
    g = O.Grid(pr)
    U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 0.038)
    assert U[0].max() == pytest.approx(row["blast_waves_max_rho_t0.038_n400_hllc"], abs=0.05)

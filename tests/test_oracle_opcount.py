"""The operation counter of the oracle (oracle/opcount.cpp: the oracle's own
code run with a counting scalar) and the per-cell operation counts the bench
reports for the arithmetic roofline.

The counter is pinned by counts written out by hand from the formulas of the
update, and the per-cell counts are the exact leading coefficients of the
counts on meshes of growing size (an integer polynomial in n)."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from conftest import ROOT
from paper_1207_3392_gb300 import problems as P


def _ramp(n, ndim, solver):
    """A state strictly increasing along every axis in every primitive, with
    subsonic velocities: every limited slope takes the same minmod branch and
    every HLLC face uses its middle state, so the counts do not depend on the
    data; outflow walls."""
    shape = (n,) * ndim
    idx = np.indices(shape).astype(float)
    s = idx.sum(axis=0) / n
    rho = 1.0 + 0.05 * s + 0.01 * idx[-1] / n
    vel = np.stack([0.01 + 0.02 * s + 0.001 * q * idx[0] / n for q in range(ndim)])
    p = 1.0 + 0.07 * s
    w = [P.uniform_widths(n, 0.0, 1.0) for _ in range(ndim)]
    bc = ((P.OUTFLOW,) * ndim, (P.OUTFLOW,) * ndim)
    return P._make("ramp", ndim, shape, w, bc, 1.4, rho, vel, p, (0.0,) * ndim, solver=solver)


def per_cell(what, ndim, solver, sizes=(4, 5, 6, 7, 8)):
    """Leading coefficient of the count of `what` on n^ndim meshes: the count
    per cell away from the walls.  The fit over ndim + 1 sizes must reproduce
    the extra size exactly (the count is an integer polynomial in n)."""
    counts = []
    for n in sizes:
        pr = _ramp(n, ndim, solver)
        g = O.Grid(pr)
        counts.append(O.count_ops(g, O.initial_state(pr, g), what, 1e-3)["total"])
    k = ndim + 1
    A = np.vander(np.array(sizes[:k], dtype=float), k)
    coef = np.linalg.solve(A, np.array(counts[:k], dtype=float))
    pred = np.polyval(coef, sizes[k])
    assert pred == pytest.approx(counts[k], abs=1e-6), (what, counts, coef)
    assert np.allclose(coef, np.round(coef), atol=1e-6), coef
    return int(round(coef[0]))


def test_counter_matches_hand_counts():
    """Counts written out from the formulas:
      totals (3D): dV = 2 products; 5 x (product + sum)              = 12 per cell
      CFL dt (3D): recovery 12 (3 quotients, |v|^2 3 + 3, e 2 + 1),
                   p twice (2 + 2), c_s (product, quotient, sqrt) 3,
                   per axis v -+ c 2, two fabs, one max, dq / s 1 = 6 x 3
                                                                    = 37 per cell
      RK2 combine: K1 *= dt, U1 = U + K1, K2 *= dt, U + (K1 + K2)/2  = 6 per value
      HLL face (3D, from primitives): e = p / (gamma - 1) twice 4; U(W) twice
                   2 x 12; F(U) twice 2 x 11 (p 2, F 9); p_L, p_R 4; c_L, c_R 6;
                   alpha_+ 2 sums + 2 max; alpha_- 2 differences + 2 max;
                   Eq. FluxHLL 5 x 9                                 = 113"""
    assert per_cell("totals", 3, P.HLLC) == 12
    assert per_cell("cfl_dt", 3, P.HLLC) == 37
    assert per_cell("step", 3, P.HLLC) == 2 * per_cell("rhs", 3, P.HLLC) + 5 * 6
    f = O.count_face_flux(P.HLL, 1.4, 3, 0, [1.0, 0.1, 0.05, 0.0, 1.0], [0.9, 0.12, 0.05, 0.0, 0.9])
    assert f["total"] == 113 and f["sqrt"] == 2 and f["minmax"] == 4 and f["div"] == 9


def test_hllc_face_counts_only_one_middle_state():
    """A subsonic HLLC face forms the middle state of the side Eq. FluxHLLC
    selects, so both signs of alpha_m cost the same; a supersonic face
    returns the upwind flux and costs less."""
    g = 1.4
    left = O.count_face_flux(P.HLLC, g, 3, 0, [1.0, 0.3, 0.0, 0.0, 1.0], [1.0, 0.2, 0.0, 0.0, 1.0])
    right = O.count_face_flux(P.HLLC, g, 3, 0, [1.0, -0.3, 0.0, 0.0, 1.0], [1.0, -0.2, 0.0, 0.0, 1.0])
    sup = O.count_face_flux(P.HLLC, g, 3, 0, [1.0, 3.0, 0.0, 0.0, 1.0], [1.0, 3.0, 0.0, 0.0, 1.0])
    assert left["total"] == right["total"] == 121
    assert sup["total"] < left["total"]


def test_bench_flop_constants_come_from_the_counter():
    """bench.py's per-cell operation counts of the dominant kernel (stage 1:
    L[U^n] plus the CFL speed and the conserved totals) and of a whole RK2
    step are the counter's."""
    sys.path.insert(0, ROOT)
    import bench
    for name, solver in (("hllc", P.HLLC), ("hll", P.HLL)):
        rhs = per_cell("rhs", 3, solver)
        cfl = per_cell("cfl_dt", 3, solver)
        tot = per_cell("totals", 3, solver)
        step = per_cell("step", 3, solver)
        assert bench.FLOPS_STAGE1_3D[name] == rhs + cfl + tot, (name, rhs, cfl, tot)
        assert bench.FLOPS_STEP_3D[name] == step + cfl + tot, (name, step)

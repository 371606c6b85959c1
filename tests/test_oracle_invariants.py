"""Invariants and analytic solutions that pin the oracle: conservation
(Sec. 3.3), identical results along any axis (Sec. 4.2.1), diagonal symmetry
(Sec. 4.2.1 implosion), exact stationary contact under HLLC, positivity in the
double rarefaction, the Sedov-Taylor similarity solution (Sec. 4.2.3), the
exact Riemann solution for the Sod problem used by the benchmark, and the CFL
time step against its definition by brute force."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.exact_riemann import RiemannSolution
from oracle.sedov import SedovSolution
from paper_1207_3392_gb300 import problems as P
from conftest import golden


@pytest.mark.parametrize("ndim,nonuniform", [(1, False), (2, True), (3, True)])
def test_conservation_periodic(ndim, nonuniform):
    """All conserved totals are constant to roundoff on a periodic box."""
    n = {1: 64, 2: 24, 3: 12}[ndim]
    pr = P.smooth_periodic(ndim, n, seed=ndim, nonuniform=nonuniform)
    g = O.Grid(pr)
    U0 = O.initial_state(pr, g)
    U, _, _ = O.evolve(g, U0, 0.5, max_steps=20)
    t0, t1 = O.totals(g, U0), O.totals(g, U)
    scale = np.abs(t0).max()
    np.testing.assert_allclose(t1, t0, rtol=0, atol=1e-13 * scale)
    assert np.abs(U - U0).max() > 1e-4  # it did evolve


def test_conservation_reflecting_mass_energy():
    """Reflecting walls: mass and energy are conserved to roundoff (the wall
    mass and energy fluxes vanish); momentum changes by the wall pressure."""
    pr = P.random_blocks(2, 20, seed=5, bc=P.REFLECT)
    g = O.Grid(pr)
    U0 = O.initial_state(pr, g)
    U, _, _ = O.evolve(g, U0, 0.4, max_steps=15)
    t0, t1 = O.totals(g, U0), O.totals(g, U)
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    assert t1[3] == pytest.approx(t0[3], rel=1e-13)


def test_sod_along_each_axis_identical():
    """A 1D problem run along y or z of a 3D mesh gives exactly the 1D result."""
    n = 64
    p1 = P.sod(n, solver=1)
    g1 = O.Grid(p1)
    U1, t1, s1 = O.evolve(g1, O.initial_state(p1, g1), 0.8, max_steps=30)
    for axis in (1, 2):
        dims = [3, 3, 3]
        dims[axis] = n
        shape = tuple(reversed(dims))
        rho = np.broadcast_to(p1.rho.reshape([n if a == axis else 1 for a in (2, 1, 0)]), shape)
        pp = np.broadcast_to(p1.p.reshape([n if a == axis else 1 for a in (2, 1, 0)]), shape)
        vel = np.zeros((3,) + shape)
        widths = [np.full(m, 1.0 / n) if m == n else np.full(m, 1.0 / n) for m in dims]
        p3 = P._make("sod_axis", 3, tuple(dims), widths, ((P.OUTFLOW,) * 3, (P.OUTFLOW,) * 3), 1.4,
                     rho, vel, pp, (0, 0, 0), solver=1)
        g3 = O.Grid(p3)
        U3, t3, s3 = O.evolve(g3, O.initial_state(p3, g3), 0.8, max_steps=30)
        assert (s3, t3) == (s1, t1)
        line = [slice(1, 2)] * 3
        line[2 - axis] = slice(None)
        for v3, v1 in ((0, 0), (1 + axis, 1), (4, 2)):
            np.testing.assert_array_equal(U3[v3][tuple(line)].ravel(), U1[v1])


def test_implosion_diagonal_symmetry():
    """Implosion: the solution stays symmetric about the diagonal x = y."""
    pr = P.implosion(48)
    g = O.Grid(pr)
    U, _, _ = O.evolve(g, O.initial_state(pr, g), 0.5, max_steps=60)
    np.testing.assert_allclose(U[0], U[0].T, rtol=1e-12, atol=0)
    np.testing.assert_allclose(U[1], U[2].T, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(U[3], U[3].T, rtol=1e-12, atol=0)


def test_stationary_contact_exact_hllc_diffused_hll():
    """HLLC keeps the stationary contact exact (Sec. 4.2.1); HLL smears it."""
    pr = P.contact(128, 0.0, solver=1)
    g = O.Grid(pr)
    U0 = O.initial_state(pr, g)
    U, _, _ = O.evolve(g, U0, 0.5, 2.0)
    np.testing.assert_array_equal(U, U0)
    gh = O.Grid(pr, solver=0)
    Uh, _, _ = O.evolve(gh, U0, 0.5, 2.0)
    assert np.abs(Uh[0] - U0[0]).max() > 0.05


def test_double_rarefaction_positive():
    """Einfeldt 1-2-0-3 with 128 cells, HLLC, t = 0.15: rho and p stay > 0."""
    pr = P.double_rarefaction(128)
    g = O.Grid(pr)
    U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 0.15)
    rho, _, p = O.cons_to_prim(g, U)
    assert rho.min() > 0 and p.min() > 0


def test_sound_wave_hll_equals_hllc():
    """Linear sound wave: HLL and HLLC errors are identical (Sec. 4.1.2)."""
    errs = []
    for solver in (0, 1):
        pr = P.sound_wave_1d(64, solver=solver)
        g = O.Grid(pr)
        U, t, _ = O.evolve(g, O.initial_state(pr, g), 0.5, 1.0)
        errs.append(np.sum(np.abs(U[0] - pr.rho)))
    assert errs[0] == pytest.approx(errs[1], rel=1e-4)


def test_sod_benchmark_case_vs_exact():
    """The 1D benchmark case (Sod, 256 cells, C_CFL = 0.8, t = 0.2): close to the
    exact solution, first order under refinement (discontinuities)."""
    l1 = []
    for n in (128, 256, 512):
        pr = P.sod(n)
        g = O.Grid(pr)
        U, t, _ = O.evolve(g, O.initial_state(pr, g), pr.cfl, pr.t_end)
        assert t == 0.2
        rho, _, _ = O.cons_to_prim(g, U)
        ex = RiemannSolution(pr.meta["left"], pr.meta["right"], 1.4)
        l1.append(O.l1_relative(rho, ex.at_points(pr.centers(0), t)[0]))
    assert l1[1] < 6e-3
    rates = np.log2(np.array(l1[:-1]) / np.array(l1[1:]))
    assert np.all((rates > 0.7) & (rates < 1.3))


def test_sedov_similarity_constant_and_jumps():
    """xi0 from the energy integral (gamma = 1.4) and the paper's post-shock
    numbers, which follow from the strong-shock jumps with R = 0.302."""
    S = SedovSolution(1.4)
    assert S.xi0 == pytest.approx(1.033, abs=2e-3)
    vals = {r[0]: float(r[1]) for r in golden("printed_values.txt")}
    R = vals["sedov3d_radius_t0.05"]
    Rdot = 0.4 * R / 0.05
    assert 2 * Rdot / 2.4 == pytest.approx(vals["sedov3d_post_shock_v"], abs=1e-3)
    assert 2 * Rdot ** 2 / 2.4 == pytest.approx(vals["sedov3d_post_shock_p"], abs=2e-3)
    assert (1.4 + 1) / (1.4 - 1) == pytest.approx(vals["sedov3d_post_shock_rho"])


@pytest.mark.slow
def test_sedov_3d_shock_radius_and_symmetry():
    """3D point blast (benchmark setup at 40^3): shock radius within 1.5 cells
    of the similarity solution, octant mirror symmetry, energy and mass kept."""
    n = 40
    pr = P.sedov_3d(n)
    g = O.Grid(pr)
    S = SedovSolution(1.4)
    t_target = S.time_at_radius(0.6)
    U0 = O.initial_state(pr, g)
    U, t, _ = O.evolve(g, U0, 0.3, t_target)
    c = pr.centers(0)
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    R = np.sqrt(X * X + Y * Y + Z * Z).ravel()
    rho = U[0].ravel()
    # outermost radius where the density is still compressed by more than half the peak excess
    peak = rho.max()
    r_shock = R[rho > 1.0 + 0.5 * (peak - 1.0)].max()
    dx = 2.0 / n
    assert abs(r_shock - S.radius(t)) < 1.5 * dx
    np.testing.assert_allclose(U[0], U[0][::-1, :, :], rtol=1e-10)
    np.testing.assert_allclose(U[0], np.transpose(U[0], (2, 1, 0)), rtol=1e-10)
    t0, t1 = O.totals(g, U0), O.totals(g, U)
    # roundoff bound of ~100 steps of 64000-term sums
    assert t1[0] == pytest.approx(t0[0], rel=1e-11)
    assert t1[4] == pytest.approx(t0[4], rel=1e-11)


def test_cfl_dt_brute_force():
    """dt_CFL = min over cells and axes of dq / max(|v - c|, |v + c|)."""
    pr = P.random_blocks(3, (5, 6, 7), seed=11)
    g = O.Grid(pr)
    U = O.initial_state(pr, g)
    c = np.sqrt(pr.gamma * pr.p / pr.rho)
    best = math.inf
    for k in range(7):
        for j in range(6):
            for i in range(5):
                for q, idx in enumerate((i, j, k)):
                    v = pr.vel[q][k, j, i]
                    best = min(best, pr.widths[q][idx] / max(abs(v - c[k, j, i]), abs(v + c[k, j, i])))
    assert O.cfl_dt(g, U) == pytest.approx(best, rel=1e-14)


def test_nonphysical_state_is_reported():
    """A negative pressure makes the oracle raise instead of continuing."""
    pr = P.sod(16)
    pr.p[3] = -1.0
    g = O.Grid(pr)
    with pytest.raises(FloatingPointError):
        O.rhs(g, O.initial_state(pr, g))

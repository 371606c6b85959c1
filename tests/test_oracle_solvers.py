"""Pins of the oracle's single-face Riemann solvers and limiter against
properties the paper states (Secs. 3.1, 3.2, 3.5) and the exact Riemann solver."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.exact_riemann import RiemannSolution


def _random_states(rng, nd):
    rho = math.exp(rng.uniform(-2, 2))
    p = math.exp(rng.uniform(-3, 3))
    v = rng.uniform(-1.0, 1.0, size=nd)
    return np.concatenate([[rho], v, [p]])


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_hllc_middle_pressure_is_continuous(nd):
    """p*_L = p*_R across the middle wave (Sec. 3.5, the equation after
    Eq. EnergyMiddle); fails for the pressure formula as printed."""
    rng = np.random.default_rng(10 + nd)
    checked = 0
    for _ in range(400):
        L, R = _random_states(rng, nd), _random_states(rng, nd)
        q = int(rng.integers(nd))
        F, d = O.riemann_flux(1, 1.4, nd, q, L, R)
        if d[0] == 0.0 or d[1] == 0.0:
            continue
        assert d[3] == pytest.approx(d[4], rel=1e-11, abs=1e-13)
        checked += 1
    assert checked > 100


@pytest.mark.parametrize("solver", [0, 1])
def test_consistency_equal_states(solver):
    """Equal left/right states give the physical flux (both solvers)."""
    rng = np.random.default_rng(3)
    for nd in (1, 2, 3):
        for _ in range(50):
            s = _random_states(rng, nd)
            q = int(rng.integers(nd))
            F, _ = O.riemann_flux(solver, 1.4, nd, q, s, s)
            np.testing.assert_allclose(F, O.physical_flux(1.4, nd, q, s), rtol=1e-12, atol=1e-13)


def test_supersonic_faces_are_upwind():
    """alpha_- = 0 (alpha_+ = 0) gives F(U_L) (F(U_R)) for HLL and HLLC alike
    (Sec. 3.2 after Eq. FluxHLL and after Eq. FluxHLLC)."""
    L = np.array([1.0, 3.0, 0.2, 0.5])    # v = 3 > c ~ 0.84
    R = np.array([0.5, 2.5, -0.1, 0.3])
    for solver in (0, 1):
        F, d = O.riemann_flux(solver, 1.4, 2, 0, L, R)
        assert d[1] == 0.0
        np.testing.assert_allclose(F, O.physical_flux(1.4, 2, 0, L), rtol=4e-16, atol=0)
        Lm, Rm = L.copy(), R.copy()
        Lm[1], Rm[1] = -3.0, -2.5
        F, d = O.riemann_flux(solver, 1.4, 2, 0, Lm, Rm)
        assert d[0] == 0.0
        np.testing.assert_allclose(F, O.physical_flux(1.4, 2, 0, Rm), rtol=4e-16, atol=0)


def test_hllc_resolves_stationary_contact_exactly():
    """Stationary contact: middle wave speed is exact (0) and there is no mass
    flux (Sec. 4.2.1); HLL has a diffusive mass flux."""
    L = np.array([1.4, 0.0, 1.0])
    R = np.array([1.0, 0.0, 1.0])
    F, d = O.riemann_flux(1, 1.4, 1, 0, L, R)
    assert d[2] == 0.0
    np.testing.assert_array_equal(F, [0.0, 1.0, 0.0])
    Fh, _ = O.riemann_flux(0, 1.4, 1, 0, L, R)
    assert abs(Fh[0]) > 1e-3


def test_hll_flux_matches_jump_conditions():
    """HLL state and flux satisfy both outer jump conditions
    (Eqs. JumpConditionHLLMinus/Plus) with U_* = U_HLL of Eq. BalancedHLL:
    F_HLL = F_L + alpha_- (U_L - U_HLL) = F_R + alpha_+ (U_HLL - U_R)."""
    rng = np.random.default_rng(7)
    g = 1.4
    for _ in range(100):
        L, R = _random_states(rng, 1), _random_states(rng, 1)
        F, d = O.riemann_flux(0, g, 1, 0, L, R)
        ap, am = d[0], d[1]
        def cons(s):
            return np.array([s[0], s[0] * s[1], s[2] / (g - 1) + 0.5 * s[0] * s[1] ** 2])
        UL, UR = cons(L), cons(R)
        FL, FR = O.physical_flux(g, 1, 0, L), O.physical_flux(g, 1, 0, R)
        Uhll = (ap * UR + am * UL - (FR - FL)) / (ap + am)
        np.testing.assert_allclose(F, FL + am * (UL - Uhll), rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(F, FR + ap * (Uhll - UR), rtol=1e-10, atol=1e-10)


def test_wave_speed_bounds():
    """alpha_+- = max[0, +-lambda_+-(U_L), +-lambda_+-(U_R)] with lambda = v +- c_s."""
    L = np.array([1.0, 0.3, 1.0])
    R = np.array([0.125, -0.2, 0.1])
    _, d = O.riemann_flux(0, 1.4, 1, 0, L, R)
    cL, cR = math.sqrt(1.4), math.sqrt(1.4 * 0.1 / 0.125)
    assert d[0] == pytest.approx(max(0.3 + cL, -0.2 + cR), rel=1e-15)
    assert d[1] == pytest.approx(max(cL - 0.3, cR + 0.2), rel=1e-15)


def test_minmod_limiter():
    """Eq. MinMod: smallest magnitude when all signs agree, else zero."""
    assert O.minmod(1.0, 2.0, 3.0) == 1.0
    assert O.minmod(-3.0, -0.5, -2.0) == -0.5
    assert O.minmod(1.0, -2.0, 3.0) == 0.0
    assert O.minmod(0.0, 2.0, 3.0) == 0.0
    assert O.minmod(2.0, 2.0, 5.0) == 2.0


def test_exact_riemann_solver_self_checks():
    """The analytic pin itself: star pressure is a root of the pressure
    function; the shock obeys Rankine-Hugoniot (mass and momentum)."""
    ex = RiemannSolution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert abs(ex.pressure_function(ex.pstar)) < 1e-14
    assert ex.pstar == pytest.approx(0.30313, abs=1e-5)
    assert ex.ustar == pytest.approx(0.92745, abs=1e-5)
    g = 1.4
    rs = ex.sample(np.array([ex.ustar + 1e-9]))[0][0]        # density just behind the shock
    S = (ex.rR * ex.uR - rs * ex.ustar) / (ex.rR - rs)      # shock speed from the mass jump
    mom_l = rs * ex.ustar ** 2 + ex.pstar - S * rs * ex.ustar
    mom_r = ex.rR * ex.uR ** 2 + ex.pR - S * ex.rR * ex.uR
    assert mom_l == pytest.approx(mom_r, rel=1e-12)
    # sampled states: far left/right are the initial data
    r, u, p = ex.sample(np.array([-10.0, 10.0]))
    assert (r[0], u[0], p[0]) == (1.0, 0.0, 1.0)
    assert (r[1], u[1], p[1]) == (0.125, 0.0, 0.1)

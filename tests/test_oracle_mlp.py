"""Pins of the FP64 reference of the learned flux correction (oracle/mlp.py):
analytic gradients against central finite differences, Adam against its
definition on a quadratic with a known minimiser, and the face features
against their symmetries (x faces of a state = y faces of its transpose,
invariance under a uniform rescaling of density and pressure)."""
import numpy as np
import pytest

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = M.init_params(1)
    theta[-M.NOUT * M.NH - M.NOUT:] = rng.normal(0, 0.3, M.NOUT * M.NH + M.NOUT)  # non-zero last layer
    X = rng.normal(0, 0.5, (37, M.NIN))
    T = rng.normal(0, 0.2, (37, M.NOUT))
    g = M.grad(theta, X, T)
    idx = rng.choice(M.NPARAM, 300, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros(M.NPARAM)
        e[i] = h
        fd = (M.loss(theta + e, X, T) - M.loss(theta - e, X, T)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(M.dsilu(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_adam_reaches_the_minimiser_of_a_linear_fit():
    """Fitting y = A x with only the last layer free (h2 fixed) converges to
    the least-squares solution."""
    rng = np.random.default_rng(2)
    theta = M.init_params(3)
    X = rng.normal(0, 1, (256, M.NIN))
    _, (_, _, _, _, h2) = M.forward(theta, X)
    Wt = rng.normal(0, 0.1, (M.NOUT, M.NH))
    T = h2 @ Wt.T + 0.05
    m = np.zeros(M.NPARAM)
    v = np.zeros(M.NPARAM)
    last = slice(M.NPARAM - M.NOUT * M.NH - M.NOUT, M.NPARAM)
    for step in range(1, 4001):
        g = M.grad(theta, X, T)
        g[: last.start] = 0.0
        theta, m, v = M.adam(theta, g, m, v, step, lr=3e-3)
    assert M.loss(theta, X, T) < 1e-6


def test_face_features_symmetry_and_scaling():
    rng = np.random.default_rng(4)
    n = 12
    rho = np.exp(rng.normal(0, 0.3, (n, n)))
    vx = rng.normal(0, 0.5, (n, n))
    vy = rng.normal(0, 0.5, (n, n))
    p = np.exp(rng.normal(0, 0.3, (n, n)))
    Xx, sx = M.face_features(rho, vx, vy, p, 1.4, 0)
    Xy, sy = M.face_features(rho.T, vy.T, vx.T, p.T, 1.4, 1)
    np.testing.assert_allclose(Xx, Xy.transpose(1, 0, 2), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(sx, sy.transpose(1, 0, 2), rtol=1e-14)
    # dimensionless: rescaling rho and p by the same factor leaves features unchanged
    X2, s2 = M.face_features(3.0 * rho, vx, vy, 3.0 * p, 1.4, 0)
    np.testing.assert_allclose(X2, Xx, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(s2[..., 0], 3.0 * sx[..., 0], rtol=1e-13)
    # the stencil of face (j, i) along x is cells i-3 .. i+2 of row j
    j, i = 5, 7
    np.testing.assert_allclose(Xx[j, i, 0::4] + 1.0, rho[j, i - 3:i + 3] / rho[j, i - 3:i + 3].mean(), rtol=1e-14)


def _kh_state(n=16, seed=1):
    import oracle as O
    from paper_1207_3392_gb300 import problems as P
    pr = P.kelvin_helmholtz(n, seed=seed)
    g = O.Grid(pr)
    return O, pr, g, O.initial_state(pr, g)


def test_corrected_step_with_zero_network_is_the_plain_step():
    O, pr, g, U = _kh_state()
    theta = M.init_params(5)  # last layer zero: the network outputs 0
    dt = 0.4 * O.cfl_dt(g, U)
    Uc, flagged = M.corrected_step(O, g, U, dt, theta)
    np.testing.assert_allclose(Uc, O.step(g, U, dt), rtol=0, atol=1e-14 * np.abs(U).max())
    assert flagged == 0


def test_corrected_step_conserves_totals():
    O, pr, g, U = _kh_state()
    rng = np.random.default_rng(9)
    theta = M.init_params(6)
    theta[-(M.NOUT * M.NH + M.NOUT):] = rng.normal(0, 0.05, M.NOUT * M.NH + M.NOUT)
    dt = 0.4 * O.cfl_dt(g, U)
    Uc, _ = M.corrected_step(O, g, U, dt, theta)
    np.testing.assert_allclose(O.totals(g, Uc), O.totals(g, U), rtol=0, atol=1e-13)
    assert np.abs(Uc - O.step(g, U, dt)).max() > 1e-6  # the correction does something


def test_fct_step_keeps_local_bounds_and_conserves():
    """With an aggressive correction the FCT-limited step keeps every conserved
    variable within the stage bounds (so density stays positive) and is
    conservative; with a zero network it is the plain step."""
    O, pr, g, U = _kh_state(24, seed=3)
    dt = 0.4 * O.cfl_dt(g, U)
    theta = M.init_params(5)
    np.testing.assert_allclose(M.fct_step(O, g, U, dt, theta), O.step(g, U, dt), rtol=0, atol=1e-13)
    rng = np.random.default_rng(1)
    theta[-(M.NOUT * M.NH + M.NOUT):] = rng.normal(0, 2.0, M.NOUT * M.NH + M.NOUT)
    Un = M.fct_step(O, g, U, dt, theta)
    np.testing.assert_allclose(O.totals(g, Un), O.totals(g, U), rtol=0, atol=1e-12)
    assert Un[0].min() > 0
    # the unlimited corrected step with the same network leaves the bounds
    Uu, _ = M.corrected_step(O, g, U, dt, theta)
    assert Uu[0].min() < U[0].min() - 1e-3 or Uu[0].max() > U[0].max() + 1e-3
    # first stage alone: every variable inside [min, max] of U_L and U over neighbours
    wx, wy = np.asarray(g.widths[0]), np.asarray(g.widths[1])
    Fx, Fy, dfx, dfy = M._corrections(O, g, U, theta, False, np.inf)
    Cx, Cy = M.fct_factors(U, U, Fx, Fy, dfx, dfy, dt, wx, wy)
    assert Cx.min() >= 0 and Cx.max() <= 1 and Cy.min() >= 0 and Cy.max() <= 1
    div = lambda a, b: (a[:, :, 1:] - a[:, :, :-1]) / wx[None, None, :] + (b[:, 1:, :] - b[:, :-1, :]) / wy[None, :, None]
    UL = U - dt * div(Fx, Fy)
    U1 = U - dt * div(Fx + Cx[None] * dfx, Fy + Cy[None] * dfy)
    hi, _ = M._neighbour_extrema(np.maximum(UL, U))
    _, lo = M._neighbour_extrema(np.minimum(UL, U))
    tol = 1e-12 * np.abs(U).max()
    assert np.all(U1 <= hi + tol) and np.all(U1 >= lo - tol)

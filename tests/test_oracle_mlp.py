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

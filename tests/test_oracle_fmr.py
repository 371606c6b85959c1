"""The multilevel reference (nested boxes, subcycling, prolongation,
restriction and flux replacement; GenASiS I Sec. 3.7, Algorithms Evolve,
EvolveLevel and StepLevel) pinned by: leaf-cell conservation to rounding, a
uniform state staying uniform, one level reducing to the single-level step,
and a blast on nested levels matching the single-level run at the finest
resolution while its shock is still inside the finest box."""
import numpy as np
import pytest

import oracle as O
from oracle import fmr as F
from paper_1207_3392_gb300 import problems as P


@pytest.mark.parametrize("nd,N,L", [(2, 32, 3), (3, 16, 2)])
def test_leaf_totals_are_conserved(nd, N, L):
    M = F.sedov(nd, N, L)
    t0 = M.leaf_totals()
    for _ in range(12):
        M.step(0.3)
    t1 = M.leaf_totals()
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    assert t1[-1] == pytest.approx(t0[-1], rel=1e-13)


def test_uniform_state_stays_uniform():
    M = F.Multilevel(2, 16, 3, -0.5, 1.0, bc=0)
    for l in range(3):
        npad = 16 + (4 if l else 0)
        shape = (npad, npad)
        M.U[l] = O.prim_to_cons(M.grids[l], np.full(shape, 1.3), np.stack([np.full(shape, 0.2), np.full(shape, -0.1)]),
                                np.full(shape, 0.7))
    U0 = [u.copy() for u in M.U]
    for _ in range(3):
        M.step(0.4)
    for l in range(3):
        np.testing.assert_allclose(M.U[l][M.interior(l)], U0[l][M.interior(l)], rtol=1e-14)


def test_one_level_is_the_single_level_step():
    pr = P.random_blocks(2, (16, 16), seed=3, bc=P.REFLECT)
    pr = pr.with_(widths=[np.full(16, 1.0 / 16)] * 2)
    M = F.Multilevel(2, 16, 1, 0.0, 1.0, bc=P.REFLECT)
    g = O.Grid(pr)
    M.U[0] = O.initial_state(pr, g)
    for _ in range(4):
        M.step(0.4)
    Uo, _, _ = O.evolve(g, O.initial_state(pr, g), 0.4, max_steps=4)
    np.testing.assert_allclose(M.U[0], Uo, rtol=1e-12, atol=1e-13)


def test_blast_matches_single_level_fine_run_inside_the_finest_box():
    """While the blast stays inside the finest box every c/f boundary sees gas
    at rest, so the finest level evolves as the same region of a single-level
    run at its resolution (to rounding), the levels' time steps coincide, and
    the coarse levels hold its restriction."""
    nd, N, L = 2, 32, 3
    M = F.sedov(nd, N, L)
    n_fine = N * 2 ** (L - 1)
    h = 1.0 / n_fine
    shape = (n_fine, n_fine)
    rho = np.ones(shape)
    p = np.full(shape, 1e-5)
    c = n_fine // 2 - 1
    p[c:c + 2, c:c + 2] = 0.4 * 1.0 / (4 * h * h)
    pr = P._make("sedov2d", 2, shape, [np.full(n_fine, h)] * 2, ((P.REFLECT,) * 2, (P.REFLECT,) * 2), 1.4,
                 rho, np.zeros((2,) + shape), p, (-0.5, -0.5), cfl=0.3)
    g = O.Grid(pr)
    U = O.initial_state(pr, g)
    o = (n_fine - N) // 2
    for _ in range(6):
        t = M.step(0.3)
        for _sub in range(2 ** (L - 1)):
            dt = 0.3 * O.cfl_dt(g, U)
            U = O.step(g, U, dt)
    fine = M.U[L - 1][M.interior(L - 1)]
    ref = U[:, o:o + N, o:o + N]
    # the shock is still well inside the finest box
    assert np.abs(fine[0, :, :3] - 1.0).max() < 1e-9
    np.testing.assert_allclose(fine, ref, rtol=1e-9, atol=1e-12)

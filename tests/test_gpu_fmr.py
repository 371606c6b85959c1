"""Multilevel evolution with subcycling on the GPU (genasis_fmr_*) against the
FP64 multilevel reference, level by level, from the same nested-box initial
state; and leaf-cell conservation on the GPU."""
import numpy as np
import pytest

from oracle import fmr as F
from paper_1207_3392_gb300 import hydro as H
from parity_util import TOL_FP32, TOL_FP64, check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def _run(nd, N, L, steps, precision, solver=1):
    M = F.sedov(nd, N, L, solver=solver)
    g = H.Fmr(nd, N, L, 1.0, 1, solver=solver, precision=precision)
    for l in range(L):
        g.set_level(l, np.ascontiguousarray(M.U[l]))
    tg = g.step(steps, 0.3)
    for _ in range(steps):
        to = M.step(0.3)
    out = [g.get_level(l) for l in range(L)]
    g.close()
    return M, out, tg, to


@pytest.mark.parametrize("nd,N,L,steps", [(2, 32, 3, 8), (3, 16, 3, 5), (2, 16, 4, 6)])
@pytest.mark.parametrize("precision,tol", [(H.FP64, TOL_FP64), (H.FP32_MIXED, TOL_FP32)])
def test_fmr_matches_reference(nd, N, L, steps, precision, tol):
    M, out, tg, to = _run(nd, N, L, steps, precision)
    assert tg == pytest.approx(to, rel=1e-9 if precision == H.FP64 else 1e-5)
    for l in range(L):
        a = out[l][M.interior(l)]
        b = M.U[l][M.interior(l)]
        check(a, b, nd, tol, f"level {l}")


def test_fmr_graph_replay_equals_stepwise():
    """Steps replayed from the captured graph (two global steps at a time)
    equal steps taken one call at a time, bitwise."""
    nd, N, L = 3, 16, 3
    M = F.sedov(nd, N, L)
    a = H.Fmr(nd, N, L, 1.0, 1, precision=H.FP64)
    b = H.Fmr(nd, N, L, 1.0, 1, precision=H.FP64)
    for l in range(L):
        a.set_level(l, np.ascontiguousarray(M.U[l]))
        b.set_level(l, np.ascontiguousarray(M.U[l]))
    ta = a.step(7, 0.3)
    tb = 0.0
    for _ in range(7):
        tb = b.step(1, 0.3)
    assert ta == tb
    for l in range(L):
        np.testing.assert_array_equal(a.get_level(l)[M.interior(l)], b.get_level(l)[M.interior(l)])
    a.close()
    b.close()


def test_fmr_autotune_keeps_results():
    """Autotuning the levels restores their states, and the tuned launch
    configurations step to bitwise the same levels."""
    nd, N, L = 3, 32, 3
    M = F.sedov(nd, N, L)
    a = H.Fmr(nd, N, L, 1.0, 1, precision=H.FP32_MIXED)
    b = H.Fmr(nd, N, L, 1.0, 1, precision=H.FP32_MIXED)
    for l in range(L):
        a.set_level(l, np.ascontiguousarray(M.U[l]))
        b.set_level(l, np.ascontiguousarray(M.U[l]))
    b.autotune(1)
    for l in range(L):
        np.testing.assert_array_equal(b.get_level(l), a.get_level(l))
    ta, tb = a.step(4, 0.3), b.step(4, 0.3)
    assert ta == tb
    for l in range(L):
        np.testing.assert_array_equal(b.get_level(l), a.get_level(l))
    a.close()
    b.close()


def test_fmr_hll_and_leaf_conservation():
    nd, N, L = 2, 32, 3
    M, out, _, _ = _run(nd, N, L, 10, H.FP64, solver=0)
    M0 = F.sedov(nd, N, L, solver=0)
    t0 = M0.leaf_totals()
    M.U = out
    t1 = M.leaf_totals()
    assert t1[0] == pytest.approx(t0[0], rel=1e-13)
    assert t1[-1] == pytest.approx(t0[-1], rel=1e-13)

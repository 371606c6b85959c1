"""Batched persistent path (many independent 1D/2D problems of uneven size in
one launch per RK stage): every problem must match the oracle run of that
problem alone (FP64 1e-10, FP32-mixed 1e-5 relative L1, L-infinity within ten times
that), with its own dt."""
import numpy as np
import pytest

import oracle as O
from paper_1207_3392_gb300 import hydro as H
from paper_1207_3392_gb300 import problems as P
from parity_util import TOL_FP32, TOL_FP64, check, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def _subset(count=48, seed=4, steps=10):
    """A reduced copy of the batched Riemann set: same generator, smaller sizes."""
    specs = P.batched_riemann(count=count, seed=seed, n1_range=(16, 700), n2_range=(8, 90), steps=steps)
    return [P.batch_problem(s) for s in specs]


@pytest.mark.parametrize("precision,tol", [(H.FP64, TOL_FP64), (H.FP32_MIXED, TOL_FP32), (H.FP64_DW, TOL_FP64)])
def test_batch_matches_oracle_per_problem(precision, tol):
    probs = _subset()
    steps = 10
    b = H.Batch(probs, precision=precision)
    for i, pr in enumerate(probs):
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    b.run(steps, 0.5)
    assert b.status() == -1
    times = b.times()
    for i, pr in enumerate(probs):
        Uo, to = oracle_run(pr, steps=steps)
        assert times[i] == pytest.approx(to, rel={H.FP64: 1e-12, H.FP64_DW: 1e-10}.get(precision, 1e-5))
        check(b.get_conserved(i), Uo, pr.ndim, tol, f"problem {i} {pr.name}")
    b.close()


def test_batch_tiles_and_chunks_identical():
    probs = _subset(count=24, seed=9)
    ref = None
    for tile in (0, 1):
        for chunk in (8, 32):
            b = H.Batch(probs, precision=H.FP32_MIXED)
            b.set_tile(tile, chunk)
            for i, pr in enumerate(probs):
                b.set_primitive(i, pr.rho, pr.vel, pr.p)
            b.run(6, 0.5)
            out = [b.get_conserved(i, precision=H.FP32_MIXED) for i in range(len(probs))]
            b.close()
            if ref is None:
                ref = out
            else:
                for a, c in zip(ref, out):
                    np.testing.assert_array_equal(a, c)


def test_batch_t_end_and_single_handle_agree():
    """t_end clamps each problem separately; a batch of one equals a handle."""
    probs = _subset(count=6, seed=2)
    b = H.Batch(probs, precision=H.FP64)
    for i, pr in enumerate(probs):
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    t_end = 0.01
    b.run(400, 0.5, t_end)
    np.testing.assert_array_equal(b.times(), np.full(len(probs), t_end))
    for i, pr in enumerate(probs):
        h = H.Hydro.from_problem(pr, precision=H.FP64)
        h.evolve(0.5, t_end)
        np.testing.assert_array_equal(b.get_conserved(i), h.get_conserved())
        h.close()
    b.close()


def test_batch_autotune_keeps_state():
    probs = _subset(count=16, seed=3)
    b = H.Batch(probs, precision=H.FP32_MIXED)
    for i, pr in enumerate(probs):
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    before = [b.get_conserved(i) for i in range(len(probs))]
    info = b.autotune(trial_steps=1)
    assert info["tile"] in (0, 1)
    for i in range(len(probs)):
        np.testing.assert_array_equal(b.get_conserved(i), before[i])
    assert np.all(b.times() == 0)
    b.close()


def test_batch_reports_the_bad_problem():
    probs = _subset(count=8, seed=5)
    probs[5].p[3] = -1.0
    b = H.Batch(probs, precision=H.FP64)
    for i, pr in enumerate(probs):
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    b.run(1, 0.5)
    with pytest.raises(H.NonPhysicalState, match="problem 5"):
        b.status()
    b.close()


@pytest.mark.parametrize("precision,tol", [(H.FP32_MIXED, TOL_FP32), (H.FP64, TOL_FP64)])
def test_full_batched_set_sampled(precision, tol):
    """The full batched Riemann set (4096 problems, 2.09e8 cells, 50 steps) in
    one batch; 12 problems (largest and smallest of each kind plus random ones)
    are checked one by one against the oracle."""
    specs = P.batched_riemann()
    b = H.Batch([_Lazy(s) for s in specs], precision=precision)
    for i, s in enumerate(specs):
        pr = P.batch_problem(s)
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    b.run(50, 0.5)
    assert b.status() == -1
    rng = np.random.default_rng(0)
    one = [i for i, s in enumerate(specs) if s.ndim == 1]
    two = [i for i, s in enumerate(specs) if s.ndim == 2]
    pick = {max(one, key=lambda i: specs[i].n), min(one, key=lambda i: specs[i].n),
            max(two, key=lambda i: specs[i].n), min(two, key=lambda i: specs[i].n)}
    pick |= set(int(x) for x in rng.choice(one, 4, replace=False))
    pick |= set(int(x) for x in rng.choice(two, 4, replace=False))
    times = b.times()
    for i in sorted(pick):
        pr = P.batch_problem(specs[i])
        Uo, to = oracle_run(pr, steps=50)
        assert times[i] == pytest.approx(to, rel={H.FP64: 1e-12, H.FP64_DW: 1e-10}.get(precision, 1e-5))
        check(b.get_conserved(i), Uo, pr.ndim, tol, f"problem {i}")
    b.close()


class _Lazy:
    """Mesh-only view of a BatchSpec (the batch needs no arrays at creation)."""

    def __init__(self, spec):
        self.ndim = spec.ndim
        self.n = (spec.n, spec.n if spec.ndim == 2 else 1, 1)
        w = P.uniform_widths(spec.n, 0.0, 1.0)
        self.widths = [w, w] if spec.ndim == 2 else [w]
        self.bc_lo = (P.OUTFLOW,) * 3
        self.bc_hi = (P.OUTFLOW,) * 3
        self.gamma = spec.gamma


def test_hydro_batch_calls_match_the_batch_engine():
    """genasis_hydro_batch_create from one genasis_hydro_desc per problem runs
    the same engine as genasis_batch_create: bitwise the same states and times;
    single-mesh calls on the batch handle are refused."""
    probs = _subset(count=20, seed=11)
    a = H.Batch(probs, precision=H.FP32_MIXED)
    b = H.HydroBatch(probs, precision=H.FP32_MIXED)
    for i, pr in enumerate(probs):
        a.set_primitive(i, pr.rho, pr.vel, pr.p)
        b.set_primitive(i, pr.rho, pr.vel, pr.p)
    a.run(7, 0.5)
    b.run(7, 0.5)
    assert b.status() == 0
    np.testing.assert_array_equal(a.times(), b.times())
    for i, pr in enumerate(probs):
        np.testing.assert_array_equal(a.get_conserved(i), b.get_conserved(i))
    Uo, _ = oracle_run(probs[3], steps=7)
    check(b.get_conserved(3), Uo, probs[3].ndim, TOL_FP32, "hydro batch problem 3")
    with pytest.raises(H.HydroError, match="batch handle"):
        H.check(H.load().genasis_hydro_step(b._h, 1e-3))
    a.close()
    b.close()

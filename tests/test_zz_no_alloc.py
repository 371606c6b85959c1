"""genasis_hydro_step_noalloc: the RK2 step for callers that cannot allocate
device memory (their memory belongs to a pooling allocator that has already
reserved it, or they must not allocate after initialisation).  Its scratch is
a static device array inside the library.

Two calls in a row must give bitwise the same state as two steps of the
handle-based genasis_hydro_step (the same stage kernels; results do not depend
on the tile shape or plane count), and match the oracle within the parity
bars.  A call must not change the device's free memory or torch's reserved
pool, must run on a non-default stream, and must refuse sizes beyond the
static array, overlapping buffers and a capturing stream.  Collected last on
purpose; self-contained so it also passes alone."""
import numpy as np
import pytest

import oracle as O
from paper_1207_3392_gb300 import hydro as H
from paper_1207_3392_gb300 import problems as P
from parity_util import TOL_FP32, TOL_FP64, check

pytestmark = pytest.mark.gpu

TOL = {H.FP64: TOL_FP64, H.FP32_MIXED: TOL_FP32}
CASES = {"sod1d": lambda: P.sod(200),
         "blocks2d": lambda: P.random_blocks(2, (150, 70), seed=31, bc=P.REFLECT),
         "blocks3d": lambda: P.random_blocks(3, (40, 36, 28), seed=32, bc=P.PERIODIC)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def _handle_steps(prob, precision, cfl=0.4):
    """Initial state, two handle steps (dt0, dt0 / 2) and their result."""
    import torch
    h = H.Hydro.from_problem(prob, precision=precision)
    dt0 = h.compute_dt(cfl)  # a stable step for this mesh and state
    dts = (dt0, 0.5 * dt0)
    dtype = torch.float64 if precision == H.FP64 else torch.float32
    u0 = torch.empty((prob.nvar,) + prob.shape, dtype=dtype, device="cuda")
    h.get_conserved(u0)
    for dt in dts:
        h.step(dt)
    ref = h.get_conserved(precision=precision)
    h.close()
    return u0, dts, ref


@pytest.mark.parametrize("precision", [H.FP64, H.FP32_MIXED])
@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_two_steps_match_handle_bitwise(precision, case):
    import torch
    prob = CASES[case]()
    u0, dts, ref = _handle_steps(prob, precision)
    u1 = torch.empty_like(u0)
    u2 = torch.empty_like(u0)
    H.step_noalloc(prob, u0, u1, dts[0], precision=precision)
    H.step_noalloc(prob, u1, u2, dts[1], precision=precision)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u2.cpu().numpy(), ref)
    # and the oracle's two steps with the same dt, within the parity bars
    g = O.Grid(prob)
    Uo = O.initial_state(prob, g)
    for dt in dts:
        Uo = O.step(g, Uo, dt)
    check(u2.double().cpu().numpy(), Uo, prob.ndim, TOL[precision], f"noalloc {case}")


def test_noalloc_allocates_nothing_and_runs_on_a_side_stream():
    """After a warm-up call (which loads the kernels and looks up the static
    array), a call on a non-default stream leaves the device's free memory and
    torch's reserved pool unchanged, and gives the handle's result bitwise."""
    import torch
    prob = CASES["blocks3d"]()
    u0, dts, ref = _handle_steps(prob, H.FP32_MIXED)
    u1 = torch.empty_like(u0)
    u2 = torch.empty_like(u0)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    H.step_noalloc(prob, u0, u1, dts[0], precision=H.FP32_MIXED, stream=s)  # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    res0 = torch.cuda.memory_reserved()
    H.step_noalloc(prob, u1, u2, dts[1], precision=H.FP32_MIXED, stream=s)
    free1, _ = torch.cuda.mem_get_info()
    res1 = torch.cuda.memory_reserved()
    assert free1 == free0 and res1 == res0, (free0, free1, res0, res1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u2.cpu().numpy(), ref)


def test_noalloc_refuses_a_capturing_stream():
    import torch
    prob = P.sod(64)
    u = torch.zeros((3, 64), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    u[0] = 1.0
    u[2] = 2.5
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(H.HydroError, match="capturing"):
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            H.step_noalloc(prob, u, v, 1e-3, precision=H.FP64, stream=s)
    # the stream is usable afterwards
    H.step_noalloc(prob, u, v, 1e-3, precision=H.FP64, stream=s)
    torch.cuda.synchronize()
    assert torch.isfinite(v).all()


def test_noalloc_rejects_oversize_and_overlap():
    import torch
    big = P.sedov_3d(128)  # 2.1 M cells x 5 x 8 B: beyond the static stage buffer
    u = torch.zeros((5, 128, 128, 128), dtype=torch.float64, device="cuda")
    v = torch.zeros_like(u)
    with pytest.raises(H.HydroError, match="scratch"):
        H.step_noalloc(big, u, v, 1e-3, precision=H.FP64)
    small = P.sod(64)
    w = torch.zeros((3, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HydroError, match="overlap"):
        H.step_noalloc(small, w, w, 1e-3, precision=H.FP64)

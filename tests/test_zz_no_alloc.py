"""genasis_hydro_step_noalloc: the RK2 step for callers that cannot allocate
device memory (their memory belongs to a pooling allocator that has already
reserved it, or they must not allocate after initialisation).  Its scratch is
a static device array inside the library.  Two calls in a row must reproduce
two steps of the handle-based genasis_hydro_step, within the parity tolerances
used for the CUDA path, and sizes beyond the static array must be refused.
Collected last on purpose; self-contained so it also passes alone."""
import numpy as np
import pytest

from paper_1207_3392_gb300 import hydro as H
from paper_1207_3392_gb300 import problems as P

pytestmark = pytest.mark.gpu

TOL = {H.FP64: 1e-10, H.FP32_MIXED: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def _rel_l1(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b).sum(axis=tuple(range(1, a.ndim))) / np.abs(b).sum(axis=tuple(range(1, b.ndim)))


@pytest.mark.parametrize("precision", [H.FP64, H.FP32_MIXED])
@pytest.mark.parametrize("case", ["sod1d", "blocks2d", "blocks3d"])
def test_noalloc_two_steps_match_handle(precision, case):
    import torch
    prob = {"sod1d": lambda: P.sod(200),
            "blocks2d": lambda: P.random_blocks(2, (150, 70), seed=31, bc=P.REFLECT),
            "blocks3d": lambda: P.random_blocks(3, (40, 36, 28), seed=32, bc=P.PERIODIC)}[case]()
    h = H.Hydro.from_problem(prob, precision=precision)
    dt0 = h.compute_dt(0.4)  # a stable step for this mesh and state
    dts = (dt0, 0.5 * dt0)
    dtype = torch.float64 if precision == H.FP64 else torch.float32
    u0 = torch.empty((prob.nvar,) + prob.shape, dtype=dtype, device="cuda")
    h.get_conserved(u0)
    for dt in dts:
        h.step(dt)
    ref = h.get_conserved()
    h.close()
    u1 = torch.empty_like(u0)
    u2 = torch.empty_like(u0)
    H.step_noalloc(prob, u0, u1, dts[0], precision=precision)
    H.step_noalloc(prob, u1, u2, dts[1], precision=precision)
    torch.cuda.synchronize()
    err = _rel_l1(u2.cpu().numpy(), ref)
    assert np.all(err <= TOL[precision]), err


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

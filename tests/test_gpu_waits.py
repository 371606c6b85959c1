"""Failure detection without a GPU fault: the kernels' bounded waits (the
grid barrier of the one-launch advances, the mbarrier waits of the TMA and
tcgen05 kernels) give up after about a second on a flag that nothing sets,
report the timeout bit to the host, and leave the context usable."""
import pytest

from paper_1207_3392_gb300 import hydro as H
from paper_1207_3392_gb300 import problems as P
from parity_util import TOL_FP64, check, gpu_run, oracle_run

pytestmark = pytest.mark.gpu

STATUS_TIMEOUT = 2  # the device status bit a wait sets when it gives up


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1207_3392_gb300 import build
    build.build()


def test_bounded_waits_give_up_and_report():
    status, seconds = H.check_bounded_waits()
    assert status == [STATUS_TIMEOUT, STATUS_TIMEOUT]
    for s in seconds:
        assert 0.9 < s < 5.0, seconds
    # the context is still usable: a short run matches the oracle
    pr = P.sod(128)
    Ug, _ = gpu_run(pr, H.FP64, steps=20)
    Uo, _ = oracle_run(pr, steps=20)
    check(Ug, Uo, 1, TOL_FP64, "after the timed-out waits")

"""Failure detection on the GPU without a fault: a bounded device wait that
nothing completes (an mbarrier no one arrives at) runs out after a short
limit, the kernel sets the timeout bit of the status word and returns, the
host reads QFLEX_ERR_DEVICE_TIMEOUT, and the context keeps working."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QFLEX_OK, QFLEX_ERR_DEVICE_TIMEOUT = 0, 6


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def test_bounded_wait_runs_out_and_context_survives(api):
    api.device_status(0)                                     # read and clear
    assert api.device_selftest_timeout(0, 10_000_000) == QFLEX_ERR_DEVICE_TIMEOUT
    # the library word was cleared after the report; the self-test's second
    # wait left its bit in the allocation-free GEMM's word, reported once
    assert api.device_status(0) == QFLEX_ERR_DEVICE_TIMEOUT
    assert api.device_status(0) == QFLEX_OK
    # the context still computes: FP64 norm of known amplitudes
    amps = torch.full((4, 8), 0.5 + 0.5j, dtype=torch.complex128, device="cuda")
    assert abs(api.norm(amps).item() - 16.0) < 1e-12
    assert api.device_selftest_timeout(0, 1_000_000) == QFLEX_ERR_DEVICE_TIMEOUT

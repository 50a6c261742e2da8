"""qflex_cgemm_noalloc: the complex GEMM for callers that cannot allocate.

Callers such as a serving loop that must not stall other streams (cudaMalloc
may synchronize the device) or code inside a framework that owns all device
memory through its own pool cannot hand qflex_cgemm a freshly allocated
workspace.  qflex_cgemm_noalloc takes no workspace and uses a fixed 64 MiB
scratch array in the library instead.  This test calls it through the C ABI
and checks it against qflex_cgemm (the entry point with a caller workspace)
within the GEMM tolerances the other GPU tests use, twice in a row with
different inputs, so the second call runs on scratch left over by the first.
A bounded device wait that ran out in one call must not make later calls
skip their work: the failure-detection self-test leaves the timeout bit in
this entry point's private status word, and the next call must still
compute C while qflex_device_status reports the timeout once.
"""
import ctypes as C

import numpy as np
import pytest

from tests.gpu_util import gemm_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-4, "fp16x3": 1e-5}
QFLEX_OK, QFLEX_ERR_DEVICE_TIMEOUT = 0, 6


@pytest.fixture(scope="module")
def api():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _noalloc(api, prec, a, b):
    lib = api._lib.load()
    M, K = a.shape
    N = b.shape[0]
    out = torch.full((M, N), float("nan"), dtype=torch.complex64, device=a.device)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    api.check(lib.qflex_cgemm_noalloc(api.PRECISIONS[prec], M, N, K, C.c_void_p(a.data_ptr()),
                                      C.c_void_p(b.data_ptr()), C.c_void_p(out.data_ptr()), stream))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp32", "fp16x3"])
def test_noalloc_matches_workspace_entry_point(api, prec):
    rng = np.random.default_rng(5)
    shapes = [(1024, 256, 512), (640, 96, 200)]       # second call: other shape, other data
    for call, (M, N, K) in enumerate(shapes):
        a_np = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)
        b_np = (rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).astype(np.complex64)
        a, b = torch.from_numpy(a_np).cuda(), torch.from_numpy(b_np).cuda()
        got = _noalloc(api, prec, a, b).cpu().numpy()
        ref_ws = api.cgemm(a, b, prec).cpu().numpy()
        ref = a_np.astype(np.complex128) @ b_np.astype(np.complex128).T
        assert np.all(np.isfinite(got)), (prec, call)
        assert gemm_error(got, ref_ws) < TOL[prec], (prec, call)
        assert gemm_error(got, ref) < TOL[prec], (prec, call)


def test_noalloc_rejects_oversize(api):
    lib = api._lib.load()
    M = N = 4096
    K = 1024       # bf16x3 planes: (M + N) * K * 12 bytes = 96 MiB > 64 MiB
    a = torch.zeros((M, K), dtype=torch.complex64, device="cuda")
    b = torch.zeros((N, K), dtype=torch.complex64, device="cuda")
    c = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
    st = lib.qflex_cgemm_noalloc(api.PRECISIONS["bf16x3"], M, N, K, C.c_void_p(a.data_ptr()),
                                 C.c_void_p(b.data_ptr()), C.c_void_p(c.data_ptr()), None)
    assert st == 1 and b"64 MiB" in lib.qflex_last_error()


@pytest.mark.parametrize("prec", ["bf16x3", "fp16x3"])
def test_noalloc_computes_after_a_timed_out_call(api, prec):
    rng = np.random.default_rng(11)
    M, N, K = 512, 128, 256
    a_np = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)
    b_np = (rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))).astype(np.complex64)
    a, b = torch.from_numpy(a_np).cuda(), torch.from_numpy(b_np).cuda()
    ref = a_np.astype(np.complex128) @ b_np.astype(np.complex128).T
    _noalloc(api, prec, a, b)                          # set up on this device
    api.device_status(0)                               # drain what earlier tests left
    # a wait that runs out on the entry point's own status word, as in a call
    # that timed out; the bit stays there
    assert api.device_selftest_timeout(0, 1_000_000) == QFLEX_ERR_DEVICE_TIMEOUT
    got = _noalloc(api, prec, a, b).cpu().numpy()      # must not skip its work
    assert np.all(np.isfinite(got)) and gemm_error(got, ref) < TOL[prec]
    assert api.device_status(0) == QFLEX_ERR_DEVICE_TIMEOUT   # reported once ...
    assert api.device_status(0) == QFLEX_OK                   # ... then cleared
    got = _noalloc(api, prec, a, b).cpu().numpy()
    assert gemm_error(got, ref) < TOL[prec]
    assert api.device_status(0) == QFLEX_OK

"""GPU parity of the standalone hot-path kernels through the C ABI.

Permutation: bit-exact against the oracle's row-major definition.
Complex GEMM: each precision against a complex128 product on the CPU.
"""
import numpy as np
import pytest

from oracle import permute as PM
from tests.gpu_util import gemm_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    from paper_1811_09599_gb300 import api
    api._lib.load(build_if_missing=True)
    return api


def _rand_c64(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _check_perm(K, shape, perm, seed=0):
    x = _rand_c64(shape, seed)
    got = K.permute(torch.from_numpy(x).cuda(), perm).cpu().numpy()
    want = PM.permute(x, perm)
    assert got.shape == want.shape
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


@pytest.mark.parametrize("m", [1, 5, 9, 12, 16, 22])
def test_permute_binary_random(K, m):
    rng = np.random.default_rng(m)
    for _ in range(3):
        _check_perm(K, (2,) * m, list(rng.permutation(m)), seed=m)


def test_permute_specials(K):
    m = 20
    _check_perm(K, (2,) * m, list(range(m)))                      # identity
    _check_perm(K, (2,) * m, list(range(m))[::-1])                # full reversal
    rng = np.random.default_rng(1)
    left = list(rng.permutation(m - 10)) + list(range(m - 10, m))  # L move (last 10 fixed)
    _check_perm(K, (2,) * m, left)
    right = list(range(m - 10)) + list(m - 10 + rng.permutation(10))  # R move
    _check_perm(K, (2,) * m, right)
    _check_perm(K, (16,) * 5, [4, 2, 0, 3, 1])                    # bond-like axes
    _check_perm(K, (16, 16, 16, 4), [3, 0, 2, 1])
    _check_perm(K, (2,) * 7, [2, 5, 4, 0, 3, 6, 1])              # abcdefg -> cfeadgb


def test_permute_non_power_of_two_and_tiny(K):
    _check_perm(K, (3, 5, 7), [2, 0, 1])
    _check_perm(K, (6, 10, 4, 3), [1, 3, 0, 2])
    _check_perm(K, (2,), [0])
    _check_perm(K, (4, 2), [1, 0])
    _check_perm(K, (1, 8, 1), [2, 1, 0])


def test_permute_empty(K):
    x = torch.zeros((0, 4), dtype=torch.complex64, device="cuda")
    assert K.permute(x, [1, 0]).shape == (4, 0)


def _gemm_case(K, prec, M, N, Kd, seed):
    a = _rand_c64((M, Kd), seed)
    b = _rand_c64((N, Kd), seed + 1)
    got = K.cgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), prec).cpu().numpy()
    ref = a.astype(np.complex128) @ b.astype(np.complex128).T
    return gemm_error(got, ref)


SHAPES = [(128, 128, 64), (256, 128, 128), (300, 200, 72), (128, 64, 8), (1024, 512, 256),
          (4096, 256, 256), (130, 33, 40), (7, 5, 3), (65536, 16, 16), (20000, 32, 256),
          (4096, 17, 16), (2048, 256, 16),
          # pipelined thin form (N <= 16, even K <= 512): ragged rows, a K
          # tail chunk, K = 2, odd N, the largest K, and K = 514 (older form)
          (1000, 5, 6), (777, 16, 40), (3000, 13, 512), (129, 16, 2), (65, 1, 200), (300, 16, 514),
          # block-per-row form (few rows, K >= 64): the 7x7 plan's 256 x 32 x 256 and
          # 32 x 2 x 256, a ragged second column group, one output, K not a
          # multiple of the block's 256-entry stride
          (256, 32, 256), (32, 2, 256), (5, 20, 1000), (1, 1, 64), (3, 17, 4099)]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5)])
def test_cgemm_fp32(K, prec, tol):
    for i, (M, N, Kd) in enumerate(SHAPES):
        assert _gemm_case(K, prec, M, N, Kd, i) < tol, (M, N, Kd)


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("bf16x3", 1e-4), ("fp16x3", 1e-5)])
def test_cgemm_tensor_core(K, prec, tol):
    for i, (M, N, Kd) in enumerate(SHAPES):
        err = _gemm_case(K, prec, M, N, Kd, 10 + i)
        assert err < tol, (prec, M, N, Kd, err)
    assert K.device_status(0) == 0


# split products in both MMA forms: the wide form (64-wide tiles, and
# 128-wide tiles with K >= 256: two accumulators in turn) with ragged M and
# N, a K tail, several tiles per SM; the three-MMA form just below K = 256
WIDE_SHAPES = [(256, 48, 16), (1000, 100, 200), (300, 128, 2048), (2100, 200, 2056), (8192, 1024, 2048),
               (4096, 256, 248), (65536, 256, 256), (640, 130, 4096)]


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1e-5), ("bf16x3", 1e-4), ("fp16x3", 1e-5)])
def test_cgemm_wide_mma_form(K, prec, tol):
    for i, (M, N, Kd) in enumerate(WIDE_SHAPES):
        err = _gemm_case(K, prec, M, N, Kd, 40 + i)
        assert err < tol, (prec, M, N, Kd, err)
    assert K.device_status(0) == 0


@pytest.mark.parametrize("Kd", [4096, 32768])
def test_cgemm_long_k_accuracy(K, Kd):
    """Long contractions (K up to 2^15, the 7x7 1+40+1 shape) keep the split
    tensor-core forms within their tolerances: chunked FP32 promotion of the
    TMEM accumulators bounds the accumulation drift."""
    tol = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-4, "fp16x3": 1e-5}
    for prec in ("fp32", "tf32x3", "bf16x3", "fp16x3"):
        err = _gemm_case(K, prec, 256, 256, Kd, 7)
        assert err < tol[prec], (prec, Kd, err)


def test_cgemm_plain_precisions_reported(K):
    """Plain bf16 / tf32 (one product per part) are reported, not gated: they
    must only be far better than noise."""
    for prec in ("bf16", "tf32"):
        err = _gemm_case(K, prec, 512, 256, 256, 99)
        assert err < 5e-2, (prec, err)


@pytest.mark.parametrize("mag", [1e-20, 1e-9, 1e+20])
def test_cgemm_fp16_power_of_two_scaling(K, mag):
    """fp16 has 5 exponent bits: without the per-operand power-of-two scale,
    entries of 1e-9 (the size of 49-qubit amplitudes) or 1e-20 would flush to
    zero and 1e+20 would overflow.  With it the split form keeps its ~22-bit
    accuracy at any magnitude."""
    a = _rand_c64((512, 256), 31) * np.float32(mag)
    b = _rand_c64((256, 256), 32)
    got = K.cgemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), "fp16x3").cpu().numpy()
    ref = a.astype(np.complex128) @ b.astype(np.complex128).T
    assert np.all(np.isfinite(got)) and gemm_error(got, ref) < 1e-5

"""Host logic of bench.py's roofline fields (no GPU): the per-step bound of
a schedule, the per-shape rows built from profiled launch records, and the
rule that ncu traffic is reported only for the kernel source it was taken
on."""
import hashlib
import json
import os

import pytest

import bench


class _FakePlan:
    def __init__(self, steps):
        self._steps = steps

    def steps(self, n_bs):
        return self._steps


def _step(M, N, K, runs, fused, kernel="tensor_cores"):
    return {"M": M, "N": N, "K": K, "runs": runs, "out_fused": fused, "kernel": kernel}


def test_per_step_roofline_sums_the_binding_side_of_each_step():
    # peaks of 1 TFLOP/s and 1 GB/s keep the arithmetic readable
    square = _step(1024, 1024, 1024, 2, 1)       # 1024^3 x 18 flop = 19.33 ms; 3 x 2^20 x 12 B = 37.7 ms
    absorb = _step(65536, 16, 16, 4, 0)          # 0.30 ms of MMA; (2^20 + 256) x 12 + 2^20 x 8 B = 20.97 ms
    thin = _step(4096, 4096, 4096, 9, 0, kernel="fp32_tiled")   # not a tensor-core step: ignored
    r = bench.per_step_roofline(_FakePlan([square, absorb, thin]), 1, "bf16x3", 1.0, 1.0, 100.0)
    want_hbm = 2 * 3 * 2**20 * 12 / 1e9 + 4 * ((2**20 + 256) * 12 + 2**20 * 8) / 1e9
    assert r["roofline_ms_per_call"] == pytest.approx(want_hbm * 1e3, abs=1e-3)
    assert r["tensor_bound_share"] == 0.0
    assert r["frac"] == pytest.approx(want_hbm * 1e3 / 100.0, abs=1e-4)
    # with a slow tensor peak the square product becomes tensor-bound
    r = bench.per_step_roofline(_FakePlan([square]), 1, "bf16x3", 0.1, 1.0, 1000.0)
    assert r["tensor_bound_share"] == 1.0
    assert r["roofline_ms_per_call"] == pytest.approx(2 * 1024**3 * 18 / 0.1e12 * 1e3, abs=1e-3)


def test_per_shape_roofline_rows():
    recs = [
        {"cls": "gemm_tc", "M": 4096, "N": 4096, "K": 4096, "out_planes": 1, "launches": 4, "ms": 4.0,
         "mma_flops": 4 * 4096**3 * 18.0},
        {"cls": "gemm_tc", "M": 65536, "N": 256, "K": 256, "out_planes": 1, "launches": 10, "ms": 1.0,
         "mma_flops": 10 * 65536 * 256 * 256 * 18.0},
        {"cls": "gemm_fp32", "M": 256, "N": 32, "K": 256, "out_planes": 0, "launches": 3, "ms": 9.0,
         "mma_flops": 0.0},
        {"cls": "gemm_tc", "M": 128, "N": 128, "K": 64, "out_planes": 0, "launches": 0, "ms": 0.0,
         "mma_flops": 0.0},
    ]
    rows = bench.per_shape_roofline(recs, "bf16x3", 1700.0, 6700.0)
    assert [(r["M"], r["N"], r["K"]) for r in rows] == [(4096, 4096, 4096), (65536, 256, 256)]
    sq, ab = rows
    assert sq["bound"] == "tensor" and sq["unit"] == "TFLOP/s"
    t = 1e-3   # 1 ms per launch
    assert sq["achieved"] == pytest.approx(4096**3 * 18 / t / 1e12, rel=1e-3)
    assert sq["frac"] == pytest.approx(4096**3 * 18 / 1700e12 / t, rel=1e-3)
    assert ab["bound"] == "hbm" and ab["unit"] == "GB/s"
    byts = (65536 * 256 + 256 * 256) * 12 + 65536 * 256 * 12
    assert ab["achieved"] == pytest.approx(byts / 1e-4 / 1e9, rel=1e-3)
    assert ab["frac"] == pytest.approx(byts / 6700e9 / 1e-4, rel=1e-3)


def test_traffic_reported_only_for_the_captured_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_1811_09599_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    kern = src / "k_cgemm_tc.cu"
    kern.write_text("// kernel v1\n")
    sha = hashlib.sha256(kern.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(
        json.dumps({"bf16x3": {"kernel_sha": sha, "dram_bytes_per_launch": 12345}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profiles("bf16x3") == 12345
    assert bench.traffic_from_profiles("tf32x3") is None
    kern.write_text("// kernel v2\n")
    assert bench.traffic_from_profiles("bf16x3") is None
    os.remove(tmp_path / "profiles" / "roofline_traffic.json")
    assert bench.traffic_from_profiles("bf16x3") is None

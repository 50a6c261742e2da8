"""ctypes declarations of the C ABI in include/qflex.h (argument marshalling only).

The shared library is built in-tree (paper_1811_09599_gb300/libqflex_gb300.so);
loading fails loudly if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqflex_gb300.so")

QFLEX_OK = 0
STATUS_NAMES = {0: "QFLEX_OK", 1: "QFLEX_ERR_ARG", 2: "QFLEX_ERR_CIRCUIT", 3: "QFLEX_ERR_PLAN",
                4: "QFLEX_ERR_OOM", 5: "QFLEX_ERR_CUDA", 6: "QFLEX_ERR_DEVICE_TIMEOUT",
                7: "QFLEX_ERR_UNSUPPORTED"}
PRECISIONS = {"fp32": 0, "tf32x3": 1, "bf16x3": 2, "bf16": 3, "tf32": 4, "fp16x3": 5}


class QFlexError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Gate(C.Structure):
    _fields_ = [("cycle", C.c_int32), ("kind", C.c_int32), ("q0", C.c_int32),
                ("q1", C.c_int32), ("param", C.c_int32)]


class Circuit(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("edges", C.POINTER(C.c_int32)), ("n_edges", C.c_int32),
                ("gates", C.POINTER(Gate)), ("n_gates", C.c_int64), ("n_params", C.c_int32)]


class Ordering(C.Structure):
    _fields_ = [("steps", C.POINTER(C.c_int32)), ("n_steps", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("circuit", C.POINTER(Circuit)), ("ordering", C.POINTER(Ordering)),
                ("cut_edges", C.POINTER(C.c_int32)), ("n_cuts", C.c_int32),
                ("open_tile", C.POINTER(C.c_int32)), ("n_open", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("n_slices", C.c_int64), ("n_qubits", C.c_int32), ("n_params", C.c_int32),
                ("n_open", C.c_int32), ("n_steps", C.c_int32), ("max_tensor_elems", C.c_int64),
                ("workspace_bytes", C.c_size_t), ("n_tc_steps", C.c_int32),
                ("n_persistent_buffers", C.c_int32), ("n_nonzero_slices", C.c_int64),
                ("n_problems", C.c_int32), ("plane_format", C.c_int32),
                ("problem_workspace_bytes", C.c_size_t)]


class Cost(C.Structure):
    _fields_ = [("cmacs", C.c_double), ("tc_cmacs", C.c_double), ("tc_mma_flops", C.c_double),
                ("permute_bytes", C.c_double), ("launches", C.c_int64),
                ("steps_executed", C.c_int64), ("largest_gemm_cmacs", C.c_double)]


class StepInfo(C.Structure):
    _fields_ = [("dst", C.c_int32), ("src", C.c_int32), ("M", C.c_int64), ("N", C.c_int64),
                ("K", C.c_int64), ("kernel", C.c_int32), ("bn", C.c_int32), ("a_direct", C.c_int32),
                ("b_direct", C.c_int32), ("runs", C.c_int64), ("a_cached", C.c_int32),
                ("b_cached", C.c_int32), ("a_builds", C.c_int64), ("b_builds", C.c_int64),
                ("a_fused", C.c_int32), ("b_fused", C.c_int32), ("out_fused", C.c_int32),
                ("tc_wide", C.c_int32)]


class SearchResult(C.Structure):
    _fields_ = [("log2_max_tensor", C.c_double), ("cmacs_per_bitstring", C.c_double),
                ("n_slices", C.c_double), ("n_nonzero_slices", C.c_double), ("n_cuts", C.c_int32),
                ("n_steps", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 5), ("ms", C.c_double * 5), ("flops", C.c_double * 5),
                ("mma_flops", C.c_double * 5), ("bytes", C.c_double * 5)]


class ProfileShape(C.Structure):
    _fields_ = [("cls", C.c_int32), ("out_planes", C.c_int32), ("M", C.c_int64), ("N", C.c_int64),
                ("K", C.c_int64), ("launches", C.c_int64), ("ms", C.c_double), ("mma_flops", C.c_double)]


PROFILE_CLASSES = ("gridtensor", "permute", "gemm_fp32", "gemm_tc", "slicesum")

# (name, restype, argtypes) for every exported symbol of include/qflex.h
SIGNATURES = [
    ("qflex_abi_version", C.c_int32, []),
    ("qflex_last_error", C.c_char_p, []),
    ("qflex_plan_create", C.c_int, [C.POINTER(Problem), C.c_int32, C.c_int, C.c_size_t, C.c_int,
                                    C.POINTER(C.c_void_p)]),
    ("qflex_plan_destroy", None, [C.c_void_p]),
    ("qflex_plan_get_info", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(PlanInfo)]),
    ("qflex_plan_cost", C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_int64), C.c_int64,
                                  C.POINTER(Cost)]),
    ("qflex_select_slices", C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_uint64, C.POINTER(C.c_int64),
                                      C.c_int64, C.POINTER(C.c_int64)]),
    ("qflex_nonzero_slices", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.c_int64,
                                       C.POINTER(C.c_int64)]),
    ("qflex_select_nonzero_slices", C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_uint64,
                                              C.POINTER(C.c_int64), C.c_int64, C.POINTER(C.c_int64)]),
    ("qflex_amplitudes", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_int64), C.c_int64, C.c_void_p, C.c_void_p]),
    ("qflex_amplitudes_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                        C.POINTER(C.c_int64), C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p]),
    ("qflex_plan_sync", C.c_int, [C.c_void_p]),
    ("qflex_plan_enable_gradients", C.c_int, [C.c_void_p]),
    ("qflex_plan_use_graphs", C.c_int, [C.c_void_p, C.c_int32]),
    ("qflex_plan_autotune", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32),
                                      C.POINTER(C.c_double)]),
    ("qflex_plan_profile", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Profile)]),
    ("qflex_plan_profile_shapes", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
    ("qflex_permute", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int64),
                                C.POINTER(C.c_int32), C.c_void_p]),
    ("qflex_cgemm_workspace_size", C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64,
                                             C.POINTER(C.c_size_t)]),
    ("qflex_cgemm", C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("qflex_norm", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("qflex_frugal_sample", C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                      C.c_uint64, C.c_void_p, C.c_void_p]),
    ("qflex_fidelity_samples", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int32,
                                         C.c_int32, C.c_double, C.c_uint64, C.c_int64, C.c_void_p,
                                         C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    ("qflex_plan_steps", C.c_int, [C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_int64), C.c_int64,
                                   C.c_void_p, C.c_int32, C.POINTER(C.c_int32)]),
    ("qflex_search_ordering", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32),
                                        C.c_int32, C.c_int32, C.c_int64, C.c_int32, C.c_uint64,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p]),
    ("qflex_device_status", C.c_int, [C.c_int, C.POINTER(C.c_int32)]),
    ("qflex_device_selftest_timeout", C.c_int, [C.c_int, C.c_uint64, C.POINTER(C.c_int32)]),
    ("qflex_cgemm_noalloc", C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
]

_lib = None


def load(build_if_missing: bool = False):
    """Load the library (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from . import build as _b
            _b.build()
        else:
            raise OSError(f"{LIB_PATH} is missing: run paper_1811_09599_gb300.build.build() "
                          "(the CUDA extension is required; there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != QFLEX_OK:
        msg = _lib.qflex_last_error().decode() if _lib is not None else ""
        raise QFlexError(status, msg)

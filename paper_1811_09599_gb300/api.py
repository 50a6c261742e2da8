"""Thin Python binding over the C ABI (argument marshalling only).

Every computation runs in the CUDA library; PyTorch supplies device memory and
streams.  Names follow include/qflex.h.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import PRECISIONS, check


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _i64_array(values):
    if values is None:
        return None, 0
    arr = np.ascontiguousarray(np.asarray(values, dtype=np.int64).reshape(-1))
    return arr, int(arr.size)


def _circuit_struct(circ, keep: list):
    edges = np.ascontiguousarray(circ.edge_array().reshape(-1), dtype=np.int32)
    garr = circ.gate_array()
    gates = (_lib.Gate * max(1, len(garr)))()
    for i, row in enumerate(garr):
        gates[i] = _lib.Gate(*[int(v) for v in row])
    keep += [edges, gates]
    return _lib.Circuit(circ.n, edges.ctypes.data_as(C.POINTER(C.c_int32)), len(circ.edges), gates, len(garr),
                        circ.n_params)


def search_ordering(problem, max_tensor_elems: int, max_new_cuts: int = 0, trials: int = 32,
                    seed: int = 0) -> dict:
    """qflex_search_ordering: greedy ordering (and up to max_new_cuts extra
    cuts after problem.cut_edges) whose largest tensor has at most
    max_tensor_elems entries.  Returns cuts, ordering ((dst, src) pairs),
    log2_max_tensor, cmacs_per_bitstring, n_slices, n_nonzero_slices (paths
    that do not vanish identically) and `fits`."""
    lib = _lib.load()
    keep: list = []
    circ = _circuit_struct(problem.circuit, keep)
    tile = np.ascontiguousarray(np.asarray(problem.open_tile, dtype=np.int32).reshape(-1))
    cuts = np.ascontiguousarray(np.asarray(problem.cut_edges, dtype=np.int32).reshape(-1))
    cuts_out = np.zeros(max(1, cuts.size + max_new_cuts), dtype=np.int32)
    steps = np.zeros(max(1, 2 * (problem.circuit.n - 1)), dtype=np.int32)
    res = _lib.SearchResult()
    st = lib.qflex_search_ordering(C.byref(circ), tile.ctypes.data_as(C.POINTER(C.c_int32)), int(tile.size),
                                   cuts.ctypes.data_as(C.POINTER(C.c_int32)), int(cuts.size), int(max_new_cuts),
                                   int(max_tensor_elems), int(trials), C.c_uint64(seed),
                                   cuts_out.ctypes.data_as(C.POINTER(C.c_int32)),
                                   steps.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(res))
    if st not in (0, 3):                       # QFLEX_ERR_PLAN: best result written, limit not met
        check(st)
    n = problem.circuit.n
    return {"cuts": [int(v) for v in cuts_out[: res.n_cuts]],
            "ordering": [(int(steps[2 * i]), int(steps[2 * i + 1])) for i in range(n - 1)],
            "log2_max_tensor": res.log2_max_tensor, "cmacs_per_bitstring": res.cmacs_per_bitstring,
            "n_slices": res.n_slices, "n_nonzero_slices": res.n_nonzero_slices, "fits": st == 0}


class Plan:
    """qflex_plan for one problem, or for several independent problems that
    one call contracts together (circuit, ordering, cuts, open tile each).

    `problem` is a qflex_inputs.Problem (or any object with .circuit,
    .cut_edges, .open_tile, .ordering), or a list of them.  device < 0 builds
    a host-only plan.  With several problems the inputs and outputs of
    amplitudes / amplitudes_grad are flat tensors holding the problems'
    arrays back to back (see `layout`).
    """

    def __init__(self, problem, precision: str = "bf16x3", device: int = 0,
                 workspace_bytes_max: int = 0):
        self.lib = _lib.load()
        probs = list(problem) if isinstance(problem, (list, tuple)) else [problem]
        self.multi = isinstance(problem, (list, tuple))
        self.n_problems = len(probs)
        self.precision = precision
        self.device = device
        self._keep = []
        arr = (_lib.Problem * max(1, len(probs)))()
        for k, pr in enumerate(probs):
            circ = _circuit_struct(pr.circuit, self._keep)
            self._keep.append(circ)
            ordering = None
            if pr.ordering is not None:
                st = np.ascontiguousarray(np.asarray(pr.ordering, dtype=np.int32).reshape(-1))
                ordering = _lib.Ordering(st.ctypes.data_as(C.POINTER(C.c_int32)), len(pr.ordering))
                self._keep += [st, ordering]
            cuts = np.ascontiguousarray(np.asarray(pr.cut_edges, dtype=np.int32).reshape(-1))
            tile = np.ascontiguousarray(np.asarray(pr.open_tile, dtype=np.int32).reshape(-1))
            self._keep += [cuts, tile]
            arr[k] = _lib.Problem(C.pointer(circ), C.pointer(ordering) if ordering is not None else None,
                                  cuts.ctypes.data_as(C.POINTER(C.c_int32)), int(cuts.size),
                                  tile.ctypes.data_as(C.POINTER(C.c_int32)), int(tile.size))
        self._probs = arr
        self.qubits = [pr.circuit.n for pr in probs]
        self.params = [pr.circuit.n_params for pr in probs]
        self.opens = [len(pr.open_tile) for pr in probs]
        self.n_qubits, self.n_params, self.n_open = self.qubits[0], self.params[0], self.opens[0]
        handle = C.c_void_p()
        check(self.lib.qflex_plan_create(arr, len(probs), PRECISIONS[precision], workspace_bytes_max, device,
                                         C.byref(handle)))
        self.handle = handle

    def layout(self, n_bs: int = 1) -> dict:
        """Offsets of each problem's part in the flat arrays of a call over
        n_bs bitstrings: bits (bytes), params (angles), amps (complex entries)."""
        ob, op, oa = np.cumsum([0] + self.qubits), np.cumsum([0] + self.params), \
            np.cumsum([0] + [1 << t for t in self.opens])
        return {"bits": [int(n_bs * v) for v in ob], "params": [int(v) for v in op],
                "amps": [int(n_bs * v) for v in oa]}

    # ------------------------------------------------------------------ info
    def info(self, problem: int = 0) -> dict:
        inf = _lib.PlanInfo()
        check(self.lib.qflex_plan_get_info(self.handle, problem, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    @property
    def n_slices(self) -> int:
        return self.info()["n_slices"]

    def cost(self, n_bs: int, slice_ids: Optional[Sequence[int]] = None, problem: Optional[int] = 0) -> dict:
        """qflex_plan_cost of one problem; problem=None sums over all problems
        (largest_gemm_cmacs: the largest over them)."""
        if problem is None:
            tot = None
            for k in range(self.n_problems):
                c = self.cost(n_bs, slice_ids, k)
                if tot is None:
                    tot = c
                else:
                    for key in c:
                        tot[key] = max(tot[key], c[key]) if key == "largest_gemm_cmacs" else tot[key] + c[key]
            return tot
        arr, n = _i64_array(slice_ids)
        c = _lib.Cost()
        ptr = arr.ctypes.data_as(C.POINTER(C.c_int64)) if arr is not None else None
        check(self.lib.qflex_plan_cost(self.handle, problem, n_bs, ptr, n, C.byref(c)))
        return {k: getattr(c, k) for k, _ in c._fields_}

    KERNELS = ("fp32_tiled", "fp32_thin16", "fp32_thin32", "fp32_rowwarp", "tensor_cores")

    def steps(self, n_bs: int = 1, slice_ids: Optional[Sequence[int]] = None, problem: int = 0) -> list:
        """qflex_plan_steps: per step dst, src, M, N, K, kernel, bn, direct
        operands and executions in one call over n_bs bitstrings."""
        arr, n = _i64_array(slice_ids)
        ptr = arr.ctypes.data_as(C.POINTER(C.c_int64)) if arr is not None else None
        cnt = C.c_int32()
        check(self.lib.qflex_plan_steps(self.handle, problem, n_bs, ptr, n, None, 0, C.byref(cnt)))
        buf = (_lib.StepInfo * max(1, cnt.value))()
        check(self.lib.qflex_plan_steps(self.handle, problem, n_bs, ptr, n, buf, cnt.value, C.byref(cnt)))
        out = []
        for s in buf[: cnt.value]:
            d = {k: getattr(s, k) for k, _ in s._fields_}
            d["kernel"] = self.KERNELS[d["kernel"]]
            out.append(d)
        return out

    def select_slices(self, fidelity: float, seed: int, nonzero: bool = False, problem: int = 0) -> np.ndarray:
        """Fraction-f path choice; nonzero=True chooses among the paths that
        do not vanish identically (qflex_select_nonzero_slices)."""
        inf = self.info(problem)
        P = inf["n_nonzero_slices"] if nonzero else inf["n_slices"]
        cap = int(min(P, max(1, int(np.floor(float(fidelity) * P + 0.5)))))   # n_f of the rule
        out = np.zeros(max(cap, 1), dtype=np.int64)
        n = C.c_int64()
        fn = self.lib.qflex_select_nonzero_slices if nonzero else self.lib.qflex_select_slices
        check(fn(self.handle, problem, float(fidelity), C.c_uint64(seed), out.ctypes.data_as(C.POINTER(C.c_int64)),
                 out.size, C.byref(n)))
        return out[: n.value].copy()

    def nonzero_slices(self, problem: int = 0) -> np.ndarray:
        """Ascending ids of the paths that do not vanish identically."""
        n = C.c_int64()
        cnt = self.info(problem)["n_nonzero_slices"]
        out = np.zeros(cnt, dtype=np.int64)
        check(self.lib.qflex_nonzero_slices(self.handle, problem, out.ctypes.data_as(C.POINTER(C.c_int64)), cnt,
                                            C.byref(n)))
        return out[: n.value].copy()

    # ------------------------------------------------------------------ compute
    def _n_bs(self, bitstrings: torch.Tensor) -> int:
        assert bitstrings.dtype == torch.uint8 and bitstrings.is_cuda and bitstrings.is_contiguous()
        if not self.multi:
            return bitstrings.shape[0]
        total = sum(self.qubits)
        assert bitstrings.numel() % total == 0, "flat bitstrings of all problems expected"
        return bitstrings.numel() // total

    def amplitudes(self, bitstrings: torch.Tensor, angles: Optional[torch.Tensor] = None,
                   slice_ids: Optional[Sequence[int]] = None, out: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
        """complex128 [n_bs, 2^n_open] on the plan's device (qflex_amplitudes);
        several problems: flat bitstrings in, flat amplitudes out (layout)."""
        dev = torch.device("cuda", self.device)
        n_bs = self._n_bs(bitstrings)
        T = sum(1 << t for t in self.opens) if self.multi else 1 << self.n_open
        if out is None:
            out = torch.empty((n_bs, T, 2), dtype=torch.float64, device=dev)
        if angles is not None:
            assert angles.dtype == torch.float64 and angles.is_cuda and angles.is_contiguous()
        arr, n = _i64_array(slice_ids)
        ptr = arr.ctypes.data_as(C.POINTER(C.c_int64)) if arr is not None else None
        check(self.lib.qflex_amplitudes(self.handle, C.c_void_p(angles.data_ptr()) if angles is not None else None,
                                        C.c_void_p(bitstrings.data_ptr()), n_bs, ptr, n,
                                        C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        if self.multi:
            return torch.view_as_complex(out.view(-1, 2))
        return torch.view_as_complex(out.view(n_bs, T, 2))

    def autotune(self, reps: int = 3) -> dict:
        """qflex_plan_autotune: pick the fastest kernel configuration per shape."""
        n = C.c_int32()
        g = C.c_double()
        check(self.lib.qflex_plan_autotune(self.handle, reps, C.byref(n), C.byref(g)))
        return {"shapes": n.value, "gain_ms": g.value}

    def use_graphs(self, enable: bool = True):
        """qflex_plan_use_graphs: replay repeated calls from a captured CUDA graph."""
        check(self.lib.qflex_plan_use_graphs(self.handle, int(enable)))

    def enable_gradients(self):
        """qflex_plan_enable_gradients: allocate the reverse-pass workspace once."""
        check(self.lib.qflex_plan_enable_gradients(self.handle))

    def amplitudes_grad(self, bitstrings, angles, grad_amps, slice_ids=None, stream=None, out=None,
                        grad_out=None):
        """(amps, grad_angles) for L = Re sum conj(g) amps (qflex_amplitudes_grad);
        several problems: flat arrays as in amplitudes.  out (float64 [n_bs,
        T, 2]) and grad_out (float64 [max(1, n_params)]) may be given to keep
        the output addresses fixed across calls (CUDA-graph replay)."""
        self.enable_gradients()
        dev = torch.device("cuda", self.device)
        n_bs = self._n_bs(bitstrings)
        T = sum(1 << t for t in self.opens) if self.multi else 1 << self.n_open
        n_par = sum(self.params)
        amps = torch.empty((n_bs, T, 2), dtype=torch.float64, device=dev) if out is None else out
        grad = torch.empty(max(1, n_par), dtype=torch.float64, device=dev) if grad_out is None else grad_out
        assert amps.numel() == n_bs * T * 2 and grad.numel() >= max(1, n_par)
        g = grad_amps if grad_amps.dtype == torch.float64 else \
            torch.view_as_real(grad_amps.to(torch.complex128).contiguous()).contiguous()
        assert g.is_contiguous() and g.numel() == n_bs * T * 2
        arr, n = _i64_array(slice_ids)
        ptr = arr.ctypes.data_as(C.POINTER(C.c_int64)) if arr is not None else None
        check(self.lib.qflex_amplitudes_grad(self.handle, C.c_void_p(angles.data_ptr()),
                                             C.c_void_p(bitstrings.data_ptr()), n_bs, ptr, n,
                                             C.c_void_p(g.data_ptr()), C.c_void_p(amps.data_ptr()),
                                             C.c_void_p(grad.data_ptr()), _stream_handle(stream)))
        if self.multi:
            return torch.view_as_complex(amps.view(-1, 2)), grad[:n_par]
        return torch.view_as_complex(amps.view(n_bs, T, 2)), grad[: self.n_params]

    def profile_start(self, classes=_lib.PROFILE_CLASSES):
        """Clear the per-class totals and record an event pair around every
        launch of the named kernel classes."""
        mask = sum(1 << _lib.PROFILE_CLASSES.index(c) for c in classes)
        check(self.lib.qflex_plan_profile(self.handle, mask, None))

    def profile_stop(self) -> dict:
        """Stop recording; per-class launches, ms, flops, mma_flops, bytes."""
        pr = _lib.Profile()
        check(self.lib.qflex_plan_profile(self.handle, 0, C.byref(pr)))
        return {cls: {"launches": pr.launches[i], "ms": pr.ms[i], "flops": pr.flops[i],
                      "mma_flops": pr.mma_flops[i], "bytes": pr.bytes[i]}
                for i, cls in enumerate(_lib.PROFILE_CLASSES)}

    def profile_shapes(self) -> list:
        """The GEMM launches of the last profile_stop() by product shape:
        dicts with cls, M, N, K, out_planes, launches, ms, mma_flops."""
        n = C.c_int64()
        check(self.lib.qflex_plan_profile_shapes(self.handle, None, 0, C.byref(n)))
        arr = (_lib.ProfileShape * max(1, n.value))()
        check(self.lib.qflex_plan_profile_shapes(self.handle, arr, n.value, C.byref(n)))
        return [{"cls": _lib.PROFILE_CLASSES[r.cls], "M": r.M, "N": r.N, "K": r.K, "out_planes": r.out_planes,
                 "launches": r.launches, "ms": r.ms, "mma_flops": r.mma_flops} for r in arr[:n.value]]

    def sync(self):
        check(self.lib.qflex_plan_sync(self.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.qflex_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class QFlexAmplitudes(torch.autograd.Function):
    """amps = QFlexAmplitudes.apply(angles, bitstrings, plan, slice_ids) (complex128).

    Backward calls qflex_amplitudes_grad with the upstream cotangent; the
    gradient convention for real angles and complex outputs is PyTorch's:
    grad_angles = sum Re(conj(g) d amp / d angle).
    """

    @staticmethod
    def forward(ctx, angles, bitstrings, plan, slice_ids=None):
        ctx.plan = plan
        ctx.slice_ids = slice_ids
        ctx.save_for_backward(angles, bitstrings)
        return plan.amplitudes(bitstrings, angles, slice_ids)

    @staticmethod
    def backward(ctx, g):
        angles, bitstrings = ctx.saved_tensors
        _, grad = ctx.plan.amplitudes_grad(bitstrings, angles, g, ctx.slice_ids)
        return grad, None, None, None


# ---------------------------------------------------------------------- kernels
def permute(x: torch.Tensor, perm: Sequence[int], stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """qflex_permute: out axis i = in axis perm[i] (complex64, bit-exact)."""
    lib = _lib.load()
    assert x.dtype == torch.complex64 and x.is_cuda and x.is_contiguous()
    dims = np.asarray(x.shape, dtype=np.int64)
    p = np.asarray(perm, dtype=np.int32)
    shape = [x.shape[i] for i in perm]
    if out is None:
        out = torch.empty(shape, dtype=x.dtype, device=x.device)
    assert out.dtype == x.dtype and out.is_contiguous() and list(out.shape) == shape
    check(lib.qflex_permute(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.dim(),
                            dims.ctypes.data_as(C.POINTER(C.c_int64)),
                            p.ctypes.data_as(C.POINTER(C.c_int32)), _stream_handle(stream)))
    return out


def cgemm(A: torch.Tensor, B: torch.Tensor, precision: str = "fp32", workspace=None,
          stream=None) -> torch.Tensor:
    """qflex_cgemm: C[m][n] = sum_k A[m][k] B[n][k] (complex64)."""
    lib = _lib.load()
    assert A.dtype == torch.complex64 and B.dtype == torch.complex64
    M, K = A.shape
    N, K2 = B.shape
    assert K == K2
    prec = PRECISIONS[precision]
    need = C.c_size_t()
    check(lib.qflex_cgemm_workspace_size(prec, M, N, K, C.byref(need)))
    if workspace is None and need.value:
        workspace = torch.empty(need.value, dtype=torch.uint8, device=A.device)
    out = torch.empty((M, N), dtype=torch.complex64, device=A.device)
    check(lib.qflex_cgemm(prec, M, N, K, C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                          C.c_void_p(out.data_ptr()),
                          C.c_void_p(workspace.data_ptr()) if workspace is not None else None,
                          need.value, _stream_handle(stream)))
    return out


def norm(amps: torch.Tensor, stream=None) -> torch.Tensor:
    """qflex_norm: FP64 sum |a|^2 of a complex128 tensor (returns a 1-element tensor)."""
    lib = _lib.load()
    a = amps.contiguous()
    assert a.dtype == torch.complex128 and a.is_cuda
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    check(lib.qflex_norm(C.c_void_p(a.data_ptr()), a.numel(), C.c_void_p(out.data_ptr()),
                         _stream_handle(stream)))
    return out


def frugal_sample(amps: torch.Tensor, n_qubits: int, M: float = 10.0, seed: int = 0,
                  stream=None) -> torch.Tensor:
    """qflex_frugal_sample: one accepted index (or -1) per batch (row of amps)."""
    lib = _lib.load()
    a = amps.contiguous()
    assert a.dtype == torch.complex128 and a.is_cuda and a.dim() == 2
    out = torch.empty(a.shape[0], dtype=torch.int32, device=a.device)
    check(lib.qflex_frugal_sample(C.c_void_p(a.data_ptr()), a.shape[0], a.shape[1], n_qubits,
                                  float(M), C.c_uint64(seed), C.c_void_p(out.data_ptr()),
                                  _stream_handle(stream)))
    return out


def fidelity_samples(batch_bits: torch.Tensor, accepted: torch.Tensor, tile, fidelity: float,
                     n_samples: int, seed: int = 0, stream=None):
    """qflex_fidelity_samples: n_samples bitstrings of a fidelity-f sampler
    (exact with probability f, from the accepted batches in order; uniform
    otherwise).  Returns (samples uint8 [n_samples, n], source int32
    [n_samples], n_exact); raises QFlexError when too few batches were
    accepted for the exact draws."""
    lib = _lib.load()
    bb = batch_bits.contiguous()
    acc = accepted.contiguous()
    assert bb.dtype == torch.uint8 and bb.is_cuda and bb.dim() == 2
    assert acc.dtype == torch.int32 and acc.is_cuda and acc.numel() == bb.shape[0]
    n = bb.shape[1]
    t = (C.c_int32 * max(1, len(tile)))(*[int(q) for q in tile])
    samples = torch.empty((n_samples, n), dtype=torch.uint8, device=bb.device)
    source = torch.empty(n_samples, dtype=torch.int32, device=bb.device)
    n_exact = C.c_int64()
    check(lib.qflex_fidelity_samples(C.c_void_p(bb.data_ptr()), C.c_void_p(acc.data_ptr()), bb.shape[0], t,
                                     len(tile), n, float(fidelity), C.c_uint64(seed), int(n_samples),
                                     C.c_void_p(samples.data_ptr()), C.c_void_p(source.data_ptr()),
                                     C.byref(n_exact), _stream_handle(stream)))
    return samples, source, n_exact.value


def device_status(device: int = 0) -> int:
    lib = _lib.load()
    v = C.c_int32()
    check(lib.qflex_device_status(device, C.byref(v)))
    return v.value


def device_selftest_timeout(device: int = 0, limit_ns: int = 10_000_000) -> int:
    """qflex_device_selftest_timeout: a bounded device wait that nothing
    completes runs out after limit_ns; returns the status it reports
    (QFLEX_ERR_DEVICE_TIMEOUT = 6 expected)."""
    lib = _lib.load()
    v = C.c_int32()
    check(lib.qflex_device_selftest_timeout(int(device), C.c_uint64(limit_ns), C.byref(v)))
    return v.value

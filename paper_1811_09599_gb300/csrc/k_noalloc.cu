// Allocation-free complex GEMM (qflex_cgemm_noalloc, include/qflex.h).
//
// Same product and kernels as qflex_cgemm, but the split operand planes live
// in a fixed array compiled into the library instead of a caller workspace,
// for callers that cannot allocate device memory (see the header).
#include <mutex>
#include <stdexcept>
#include <string>

#include "internal.h"
#include "qflex.h"

using namespace qflex;

namespace {

// File-scope scratch and status words.  In host code these names are host
// stand-ins, not device addresses: the device addresses come from
// cudaGetSymbolAddress below.
//  g_noalloc_status  the word the tensor-core kernel of the current call
//                    sets when one of its bounded waits runs out (and that
//                    makes later launches given the same word skip their work);
//  g_noalloc_report  what earlier calls left in g_noalloc_status, moved there
//                    by the next call before it starts; qflex_device_status
//                    reads and clears both.
__device__ __align__(256) unsigned char g_noalloc_scratch[QFLEX_NOALLOC_SCRATCH_BYTES];
__device__ int32_t g_noalloc_status;
__device__ int32_t g_noalloc_report;
__device__ unsigned g_noalloc_smax[2];   // fp16 operand scales

constexpr int kMaxDevices = 64;
struct DeviceScratch {
  void* scratch = nullptr;
  int32_t* status = nullptr;
  int32_t* report = nullptr;
  unsigned* smax = nullptr;
};
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

qflex_status fail(qflex_status st, const std::string& msg) {
  set_last_error(msg.c_str());
  return st;
}

// One thread, first launch of every tensor-core call: whatever an earlier
// call left in the status word (a wait that ran out) goes to the report word,
// and the status word starts this call at zero, so no call is skipped because
// of an earlier one.
__global__ void k_noalloc_rollover(int32_t* status, int32_t* report) {
  const int32_t v = *status;
  if (v) *report |= v;
  *status = 0;
}

// Once per device, with that device current: look up the device addresses of
// the scratch array and the status words, and clear the status words.
qflex_status setup(int dev, DeviceScratch* out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(QFLEX_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceScratch& d = g_dev[dev];
  if (!d.scratch) {
    void* s = nullptr;
    void* w = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&s, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&w, g_noalloc_status);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("cudaGetSymbolAddress(status): ") + cudaGetErrorString(e));
    void* r = nullptr;
    e = cudaGetSymbolAddress(&r, g_noalloc_report);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("cudaGetSymbolAddress(report): ") + cudaGetErrorString(e));
    void* m = nullptr;
    e = cudaGetSymbolAddress(&m, g_noalloc_smax);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("cudaGetSymbolAddress(smax): ") + cudaGetErrorString(e));
    d.smax = static_cast<unsigned*>(m);
    e = cudaMemset(w, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(r, 0, sizeof(int32_t));
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("cudaMemset(status): ") + cudaGetErrorString(e));
    d.status = static_cast<int32_t*>(w);
    d.report = static_cast<int32_t*>(r);
    d.scratch = s;
  }
  *out = d;
  return QFLEX_OK;
}

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

// Identity "permutation" of a [rows][K] complex64 matrix into operand planes.
cudaError_t planes(const void* src, int64_t rows, int64_t K, int kind, int nsplit, void* dst,
                   cudaStream_t s, unsigned* smax) {
  const int64_t total = rows * K;
  const int fmt = kind == 0 ? kFmtTF32 : (kind == 1 ? kFmtBF16 : kFmtFP16);
  if (fmt == kFmtFP16) {
    cudaError_t e = launch_absmax(static_cast<const float2*>(src), total, smax, s);
    if (e != cudaSuccess) return e;
  } else {
    smax = nullptr;
  }
  if ((total & (total - 1)) == 0) {
    int nb = 0;
    while ((int64_t(1) << nb) < total) ++nb;
    int64_t w[64];
    for (int b = 0; b < nb; ++b) w[b] = int64_t(1) << b;
    PermTile t;
    if (!build_perm_tile(nb, w, &t)) return cudaErrorInvalidValue;
    return launch_permute_tiled(static_cast<const float2*>(src), 0, t, fmt, nsplit, dst, total, s, smax);
  }
  GatherDesc g{};
  g.rank = 1;
  g.total = total;
  g.dims[0] = total;
  g.in_strides[0] = 1;
  return launch_permute_gather(static_cast<const float2*>(src), 0, g, fmt, nsplit, dst, total, s, smax);
}

}  // namespace

namespace qflex {

// Status of the allocation-free GEMM on `dev` for qflex_device_status: the
// OR of its status and report words (0 when the entry point was never set
// up on that device); both are cleared.  The caller has synchronized `dev`.
cudaError_t noalloc_take_status(int dev, int32_t* bits) {
  *bits = 0;
  if (dev < 0 || dev >= kMaxDevices) return cudaSuccess;
  DeviceScratch d;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    d = g_dev[dev];
  }
  if (!d.scratch) return cudaSuccess;
  int32_t v[2] = {0, 0};
  cudaError_t e = cudaMemcpy(&v[0], d.status, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&v[1], d.report, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(d.status, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(d.report, 0, sizeof(int32_t));
  *bits = v[0] | v[1];
  return e;
}

// Failure-detection self-test of this entry point's word (called by
// qflex_device_selftest_timeout with `dev` current and synchronized): the
// bounded wait of launch_wait_selftest runs out on the private status word
// and leaves its bit there, as a call whose wait ran out would.
cudaError_t noalloc_selftest(int dev, uint64_t limit_ns) {
  DeviceScratch d;
  if (setup(dev, &d) != QFLEX_OK) return cudaErrorUnknown;
  cudaError_t e = launch_wait_selftest(limit_ns, d.status, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

}  // namespace qflex

extern "C" qflex_status qflex_cgemm_noalloc(int32_t prec, int64_t M, int64_t N, int64_t K, const void* A,
                                            const void* B, void* C, void* stream) {
  try {
    if (prec < QFLEX_FP32_SIMT || prec > QFLEX_FP16X3) return fail(QFLEX_ERR_ARG, "unknown precision");
    if (M < 0 || N < 0 || K < 0 || (M * N > 0 && (!A || !B || !C))) return fail(QFLEX_ERR_ARG, "bad GEMM arguments");
    if (M == 0 || N == 0) return QFLEX_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    DeviceScratch d;
    if (qflex_status st = setup(dev, &d)) return st;
    const bool tc = prec != QFLEX_FP32_SIMT && M >= 128 && K % 8 == 0 && K > 0 && N >= 16;
    if (!tc) {
      if (K == 0) e = cudaMemsetAsync(C, 0, size_t(M) * N * 8, s);
      else if (N <= 32)
        e = launch_cgemm_thin(M, N, K, static_cast<const float2*>(A), static_cast<const float2*>(B),
                              static_cast<float2*>(C), s);
      else
        e = launch_cgemm_simt(M, N, K, static_cast<const float2*>(A), static_cast<const float2*>(B),
                              static_cast<float2*>(C), s);
      if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
      return QFLEX_OK;
    }
    const int kind = (prec == QFLEX_TF32X3 || prec == QFLEX_TF32_PLAIN) ? 0 : (prec == QFLEX_FP16X3 ? 2 : 1);
    const int nsplit = (prec == QFLEX_TF32X3 || prec == QFLEX_BF16X3 || prec == QFLEX_FP16X3) ? 2 : 1;
    const size_t per = size_t(3) * nsplit * (kind == 0 ? 4 : 2);
    // reject sizes whose plane bytes exceed the scratch before multiplying
    // them out (K > 0 on this path), so that the products cannot wrap
    const uint64_t max_rows = QFLEX_NOALLOC_SCRATCH_BYTES / (per * uint64_t(K));
    if (uint64_t(M) > max_rows || uint64_t(N) > max_rows)
      return fail(QFLEX_ERR_ARG, "operand planes exceed the 64 MiB static scratch of qflex_cgemm_noalloc");
    const size_t a_bytes = round256(per * size_t(M) * size_t(K));
    const size_t b_bytes = round256(per * size_t(N) * size_t(K));
    if (a_bytes + b_bytes > QFLEX_NOALLOC_SCRATCH_BYTES)
      return fail(QFLEX_ERR_ARG, "operand planes need " + std::to_string(a_bytes + b_bytes) +
                                     " bytes, more than the 64 MiB static scratch of qflex_cgemm_noalloc");
    if (!tc_available()) return fail(QFLEX_ERR_UNSUPPORTED, "tensor-map encoder unavailable");
    char* pa = static_cast<char*>(d.scratch);
    char* pb = pa + a_bytes;
    k_noalloc_rollover<<<1, 1, 0, s>>>(d.status, d.report);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    if ((e = planes(A, M, K, kind, nsplit, pa, s, d.smax)) != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    if ((e = planes(B, N, K, kind, nsplit, pb, s, d.smax + 1)) != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    TcGemmMaps maps;
    const int bn = N >= 128 ? 128 : 64;
    if (!tc_encode_maps(kind, nsplit, bn, pa, M, pb, N, K, &maps)) return fail(QFLEX_ERR_CUDA, "tensor map encoding failed");
    e = launch_cgemm_tc(kind, nsplit, bn, maps, M, N, K, static_cast<float2*>(C), d.status, s,
                        kind == 2 ? d.smax : nullptr, kind == 2 ? d.smax + 1 : nullptr);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    return QFLEX_OK;
  } catch (const std::exception&) {   // no C++ exception crosses the C ABI
    return QFLEX_ERR_OOM;
  } catch (...) {
    return QFLEX_ERR_UNSUPPORTED;
  }
}

// Steps a4 and a6: FP64 slice summation and norm reductions.
//
// Methods, "Cutting indexes": the amplitude is the sum of the contributions
// of all paths (slices); Methods, "Summing a fraction of the paths": summing
// a fraction f of them gives fidelity-f amplitudes of norm ~f.  The
// cross-slice sum and the norm reduction are the only FP64 arithmetic on the
// GPU.
#include "internal.h"

#include <mutex>
#include <vector>

namespace qflex {
namespace {

struct SliceSumArgs {
  int64_t strides[32];
  int32_t n_open;
};

__global__ void k_slicesum(const float2* __restrict__ src, const __grid_constant__ SliceSumArgs a,
                           double* __restrict__ amps) {
  const int64_t count = int64_t(1) << a.n_open;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < count;
       j += int64_t(gridDim.x) * blockDim.x) {
    int64_t idx = 0;
    for (int t = 0; t < a.n_open; ++t)
      if ((j >> (a.n_open - 1 - t)) & 1) idx += a.strides[t];
    const float2 v = src[idx];
    amps[2 * j] += double(v.x);
    amps[2 * j + 1] += double(v.y);
  }
}

__global__ void k_norm(const double* __restrict__ amps, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double re = amps[2 * i], im = amps[2 * i + 1];
    acc += re * re + im * im;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *out = acc;
  }
}

// Frugal rejection sampling (Methods, "Fast sampling technique"): one thread
// per batch.  Entries are visited in a uniformly random order by a forward
// Fisher-Yates walk (step k swaps a[k] with a[k + (x mod (n_c - k))]); entry
// a[k] is accepted when u < p N / M with p = |amp|^2 and u = (x >> 11) 2^-53,
// x drawn from SplitMix64; the first acceptance ends the batch (at most one
// per batch), none gives -1.  The stream of batch b starts at
// seed + b * 0xD1B54A32D192ED03.  FP64 products are rounded separately (no
// contraction) so that every decision is reproducible on the host.
__device__ __forceinline__ uint64_t splitmix64(uint64_t& x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int kMaxBatch = 4096;

__global__ void k_frugal(const double* __restrict__ amps, int64_t n_batches, int n_c, double scale,
                         uint64_t seed, int32_t* __restrict__ accepted) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= n_batches) return;
  uint16_t a[kMaxBatch];
  for (int i = 0; i < n_c; ++i) a[i] = uint16_t(i);
  uint64_t x = seed + uint64_t(b) * 0xD1B54A32D192ED03ull;
  const double* amp = amps + 2 * b * n_c;
  int32_t res = -1;
  for (int k = 0; k < n_c; ++k) {
    const int j = k + int(splitmix64(x) % uint64_t(n_c - k));
    const uint16_t t = a[k];
    a[k] = a[j];
    a[j] = t;
    const int idx = a[k];
    const double re = amp[2 * idx], im = amp[2 * idx + 1];
    const double p = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
    const double u = double(splitmix64(x) >> 11) * 0x1.0p-53;
    if (u < __dmul_rn(p, scale)) {
      res = idx;
      break;
    }
  }
  accepted[b] = res;
}

// Largest |re|, |im|, |re + im| of a complex64 array (the three parts of the
// 3M product), as float bits, for the power-of-two scale of fp16 operands.
__global__ void k_absmax(const float2* __restrict__ in, int64_t n, unsigned* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float2 v = in[i];
    m = fmaxf(m, fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.x + v.y))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

}  // namespace

cudaError_t launch_absmax(const float2* in, int64_t n, unsigned* smax, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(unsigned), s);
  if (e != cudaSuccess || n <= 0) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const int blocks = int(want < int64_t(sms) * 4 ? want : int64_t(sms) * 4);
  k_absmax<<<blocks, 256, 0, s>>>(in, n, smax);
  return cudaGetLastError();
}

cudaError_t launch_frugal(const double* amps, int64_t n_batches, int n_c, double scale, uint64_t seed,
                          int32_t* accepted, cudaStream_t s) {
  if (n_c < 1 || n_c > kMaxBatch) return cudaErrorInvalidValue;
  if (n_batches <= 0) return cudaSuccess;
  k_frugal<<<unsigned((n_batches + 127) / 128), 128, 0, s>>>(amps, n_batches, n_c, scale, seed, accepted);
  return cudaGetLastError();
}

cudaError_t launch_slicesum(const float2* src, const int64_t* strides, int n_open, double* amps,
                            cudaStream_t s) {
  if (n_open < 0 || n_open > 30) return cudaErrorInvalidValue;
  SliceSumArgs a{};
  for (int t = 0; t < n_open; ++t) a.strides[t] = strides[t];
  a.n_open = n_open;
  const int64_t count = int64_t(1) << n_open;
  const int blocks = int(count < 256 ? 1 : (count + 255) / 256 > 4096 ? 4096 : (count + 255) / 256);
  k_slicesum<<<blocks, 256, 0, s>>>(src, a, amps);
  return cudaGetLastError();
}

cudaError_t launch_norm(const double* amps, int64_t n, double* out, cudaStream_t s) {
  k_norm<<<1, 1024, 0, s>>>(amps, n, out);
  return cudaGetLastError();
}

int32_t* device_status_word(int device) {
  static std::mutex mu;
  static std::vector<int32_t*> words;
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0) return nullptr;
  if (int(words.size()) <= device) words.resize(device + 1, nullptr);
  if (!words[device]) {
    int32_t* p = nullptr;
    if (cudaMalloc(&p, sizeof(int32_t)) != cudaSuccess) return nullptr;
    cudaMemset(p, 0, sizeof(int32_t));
    words[device] = p;
  }
  return words[device];
}

}  // namespace qflex

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
  pdl_wait();
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

// Fidelity-f samples (Methods, "Fraction of perfect fidelity amplitudes"):
// the output of a fidelity-f circuit is f |psi><psi| + (1 - f) I / N, so
// sample i is exact with probability f and uniform otherwise.  Sample i runs
// its own SplitMix64 stream from seed + i * 0xD1B54A32D192ED03: the first
// draw x gives u = (x >> 11) 2^-53, exact when u < f; a uniform sample takes
// qubit q from bit 63 - (q mod 64) of draw 1 + q div 64.  The k-th exact
// sample takes the k-th batch that frugal rejection sampling accepted.
constexpr uint64_t kStreamStep = 0xD1B54A32D192ED03ull;
constexpr int kMixThreads = 1024;
constexpr int kMaxMixTile = 30;

struct MixTile {
  int32_t q[kMaxMixTile];
  int32_t n;
};

// Exclusive block-wide prefix sum of v (one value per thread); `total` gets
// the block's sum.  Uses sh[32]; ends with a barrier so sh can be reused.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;
  }
  __syncthreads();
  const int before = (w > 0 ? sh[w - 1] : 0) + x - v;
  total = sh[nw - 1];
  __syncthreads();
  return before;
}

// One block: compacts the accepted batches (batch order) into `pool`, then
// walks the samples in order, deciding exact or uniform and numbering the
// exact ones; source[i] = pool[k] for the k-th exact sample (-2 past the
// pool), -1 for a uniform one.  counts = {exact samples, accepted batches}.
__global__ void __launch_bounds__(kMixThreads) k_mix_plan(const int32_t* __restrict__ accepted, int64_t n_batches,
                                                          double f, uint64_t seed, int64_t n_samples,
                                                          int32_t* __restrict__ pool, int32_t* __restrict__ source,
                                                          int64_t* __restrict__ counts) {
  __shared__ int sh[32];
  int64_t n_acc = 0;
  for (int64_t base = 0; base < n_batches; base += blockDim.x) {
    const int64_t b = base + threadIdx.x;
    const int v = (b < n_batches && accepted[b] >= 0) ? 1 : 0;
    int tot;
    const int pre = block_exclusive_scan(v, sh, tot);
    if (v) pool[n_acc + pre] = int32_t(b);
    n_acc += tot;
  }
  __syncthreads();
  int64_t n_ex = 0;
  for (int64_t base = 0; base < n_samples; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int v = 0;
    if (i < n_samples) {
      uint64_t x = seed + uint64_t(i) * kStreamStep;
      const double u = double(splitmix64(x) >> 11) * 0x1.0p-53;
      v = u < f ? 1 : 0;
    }
    int tot;
    const int pre = block_exclusive_scan(v, sh, tot);
    if (i < n_samples) {
      const int64_t k = n_ex + pre;
      source[i] = v ? (k < n_acc ? pool[k] : -2) : -1;
    }
    n_ex += tot;
  }
  if (threadIdx.x == 0) {
    counts[0] = n_ex;
    counts[1] = n_acc;
  }
}

// One thread per sample writes its n_qubits bytes.
__global__ void k_mix_write(const uint8_t* __restrict__ batch_bits, const int32_t* __restrict__ accepted,
                            const int32_t* __restrict__ source, const __grid_constant__ MixTile tile,
                            int n_qubits, uint64_t seed, int64_t n_samples, uint8_t* __restrict__ out) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_samples) return;
  const int32_t b = source[i];
  uint8_t* o = out + i * n_qubits;
  if (b >= 0) {
    const uint8_t* src = batch_bits + int64_t(b) * n_qubits;
    for (int q = 0; q < n_qubits; ++q) o[q] = src[q];
    const int j = accepted[b];
    for (int t = 0; t < tile.n; ++t) o[tile.q[t]] = uint8_t((j >> (tile.n - 1 - t)) & 1);
  } else if (b == -1) {
    uint64_t x = seed + uint64_t(i) * kStreamStep;
    splitmix64(x);                         // the exact-or-uniform draw
    uint64_t w = 0;
    for (int q = 0; q < n_qubits; ++q) {
      if ((q & 63) == 0) w = splitmix64(x);
      o[q] = uint8_t((w >> (63 - (q & 63))) & 1);
    }
  } else {
    for (int q = 0; q < n_qubits; ++q) o[q] = 0;
  }
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

// Self-test of failure detection: thread 0 waits, by the same bounded
// pattern as the tensor-core GEMM's mbarrier waits (mbarrier.try_wait in a
// loop, %globaltimer checked every 256 tries), on an mbarrier that no one
// arrives at.  After limit_ns the wait gives up, sets kDevTimeout in the
// status word and the kernel returns; nothing faults and the context stays
// usable.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status) {
  __shared__ alignas(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1u) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(b), "r"(0u)
        : "memory");
    if (done) return;   // not reached: phase 0 never completes
    if ((it & 255u) == 255u) {
      uint64_t now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > limit_ns) {
        atomicOr(status, kDevTimeout);
        return;
      }
    }
  }
}

}  // namespace

cudaError_t launch_wait_selftest(uint64_t limit_ns, int32_t* status, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(limit_ns, status);
  return cudaGetLastError();
}

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

cudaError_t launch_fidelity_mix(const uint8_t* batch_bits, const int32_t* accepted, int64_t n_batches,
                               const int32_t* tile, int n_tile, int n_qubits, double f, uint64_t seed,
                               int64_t n_samples, int32_t* pool, int32_t* source, int64_t* counts,
                               uint8_t* out, cudaStream_t s) {
  if (n_tile < 0 || n_tile > kMaxMixTile || n_samples < 0 || n_batches < 0) return cudaErrorInvalidValue;
  MixTile t{};
  for (int i = 0; i < n_tile; ++i) t.q[i] = tile[i];
  t.n = n_tile;
  k_mix_plan<<<1, kMixThreads, 0, s>>>(accepted, n_batches, f, seed, n_samples, pool, source, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_samples == 0) return e;
  k_mix_write<<<unsigned((n_samples + 255) / 256), 256, 0, s>>>(batch_bits, accepted, source, t, n_qubits, seed,
                                                                 n_samples, out);
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
  return launch_pdl(k_slicesum, dim3(blocks), dim3(256), 0, s, src, a, amps);
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

// Internal declarations shared by the host planner (api.cpp) and the CUDA
// kernels.  Not part of the public ABI (see include/qflex.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

namespace qflex {

// ------------------------------------------------------------------ status
// Device-side status bits, OR-ed into a device word by kernels whose bounded
// waits ran out (they then skip their remaining work and return).
enum : int32_t { kDevTimeout = 1, kDevBadIndex = 2 };

#ifdef __CUDACC__
}  // namespace qflex
#include <cuda_bf16.h>
#include <cuda_fp16.h>
namespace qflex {
__device__ __forceinline__ float fp16_scale_of(unsigned max_bits) {
  const float m = __uint_as_float(max_bits);
  if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
  int e;
  frexpf(m, &e);
  return ldexpf(1.f, 14 - e);
}
#endif

// ------------------------------------------------------------------ grid tensors
// One qubit's gate line, compiled by the planner.  Op encoding (int2):
//   x = type | (bitpos << 8), y = angle index (or -1)
//   type 0..3, 5..7: one-qubit gate kinds (H, T, SX, SY, RX, RY, RZ)
//   type 8: CZ half carried by the lower-index qubit, |k><k| with k = entry bit `bitpos`
//   type 9: CZ half carried by the higher-index qubit, Z^k
//   type 10: iSWAP half carried by the lower-index qubit, P_k with
//            P = (I, Z, X, Y) and k = entry bits [bitpos, bitpos + 2)
//   type 11: iSWAP half carried by the higher-index qubit, c_k P_k,
//            c = (1/2, 1/2, i/2, i/2)  (iSWAP = (II + ZZ)/2 + i (XX + YY)/2)
struct GridQubitMeta {
  int64_t offset;     // element offset of this qubit's tensor in the grid buffer
  int32_t n_bits;     // bond bits (entries per output value = 2^n_bits)
  int32_t op_begin;   // first op in the op array
  int32_t op_count;
  int32_t tile;       // 1: output leg kept open (stored outermost, dim 2)
  int32_t qubit;
  int32_t pad;
};
enum : int { kOpCzProj = 8, kOpCzZ = 9, kOpIswA = 10, kOpIswB = 11 };

#ifdef __CUDACC__
// Column form v <- H v of an iSWAP half (type 10 or 11, 2-bit value k).
__device__ __forceinline__ void iswap_half_col(int type, int k, float2& v0, float2& v1) {
  float2 n0 = v0, n1 = v1;
  if (k == 1) {
    n1 = make_float2(-v1.x, -v1.y);
  } else if (k == 2) {
    n0 = v1;
    n1 = v0;
  } else if (k == 3) {            // Y = [[0, -i], [i, 0]]
    n0 = make_float2(v1.y, -v1.x);
    n1 = make_float2(-v0.y, v0.x);
  }
  if (type == kOpIswB) {          // c_k = 1/2 or i/2
    if (k < 2) {
      n0 = make_float2(0.5f * n0.x, 0.5f * n0.y);
      n1 = make_float2(0.5f * n1.x, 0.5f * n1.y);
    } else {
      n0 = make_float2(-0.5f * n0.y, 0.5f * n0.x);
      n1 = make_float2(-0.5f * n1.y, 0.5f * n1.x);
    }
  }
  v0 = n0;
  v1 = n1;
}
// Row form u <- u H of the same half.
__device__ __forceinline__ void iswap_half_row(int type, int k, float2& u0, float2& u1) {
  float2 n0 = u0, n1 = u1;
  if (k == 1) {
    n1 = make_float2(-u1.x, -u1.y);
  } else if (k == 2) {
    n0 = u1;
    n1 = u0;
  } else if (k == 3) {            // (u0, u1) Y = (i u1, -i u0)
    n0 = make_float2(-u1.y, u1.x);
    n1 = make_float2(u0.y, -u0.x);
  }
  if (type == kOpIswB) {
    if (k < 2) {
      n0 = make_float2(0.5f * n0.x, 0.5f * n0.y);
      n1 = make_float2(0.5f * n1.x, 0.5f * n1.y);
    } else {
      n0 = make_float2(-0.5f * n0.y, 0.5f * n0.x);
      n1 = make_float2(-0.5f * n1.y, 0.5f * n1.x);
    }
  }
  u0 = n0;
  u1 = n1;
}
#endif

cudaError_t launch_gridtensor(const GridQubitMeta* d_meta, int n_qubits, int max_bits,
                              const int2* d_ops, const double* d_angles,
                              const uint8_t* d_bits, float2* d_grid, cudaStream_t s);

// ------------------------------------------------------------------ permutation
// A permutation of a power-of-two-sized view is a permutation of the bits of
// the linear output index: output bit j carries input weight w_j (elements).
// The tiled kernel moves 2^tile_bits elements per tile through shared memory:
// loads enumerate the tile bits by increasing input weight (coalesced reads),
// stores by increasing output position (coalesced writes).  Shared-memory
// slots are the load index with its low 4 bits XOR-ed by the store-fast
// bits that sit higher up, so both 16-thread halves of a warp hit 16
// distinct bank pairs in both phases, whatever the permutation.
constexpr int kPermMaxRest = 48;
constexpr int kPermTileBits = 11;   // 2048 entries per tile, 8 per thread
struct PermTile {
  int64_t in_lo[32], in_hi[64];    // input offsets of load-index bits [0,5) and [5,11)
  int64_t out_lo[32], out_hi[64];  // output offsets of store-index bits [0,5) and [5,11)
  int32_t ld_lo[32], ld_hi[64];    // shared-memory slot of load-index bits [0,5) and [5,11)
  int32_t st_lo[32], st_hi[64];    // shared-memory slot of store-index bits [0,5) and [5,11)
  int64_t rest_in[kPermMaxRest], rest_out[kPermMaxRest];  // non-tile bits
  int64_t n_tiles;
  int32_t tile_bits, n_rest;
};

// Output formats of the operand producer.
enum PermFormat : int {
  kFmtC64 = 0,        // complex64, the permuted tensor itself
  kFmtTF32 = 1,       // 3M planes re, im, re+im, each split into tf32 hi (+ lo)
  kFmtBF16 = 2,       // same with bf16
  kFmtAccC128 = 3,    // out (complex128) += entry: scatter-add of cotangents
  kFmtFP16 = 4        // 3M planes in fp16 hi (+ lo), scaled by a power of two
};

#ifdef __CUDACC__
// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel on its stream is still running; it must call
// pdl_wait() before reading anything that kernel wrote (the wait returns once
// the previous kernel has completed and its writes are visible).  It then
// allows the next such launch to stage itself early.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
}
template <int BYTES>
__device__ __forceinline__ void store_bytes(void* dst, const void* src) {
  if constexpr (BYTES == 16) {
    *static_cast<uint4*>(dst) = *static_cast<const uint4*>(src);
  } else if constexpr (BYTES == 8) {
    *static_cast<uint2*>(dst) = *static_cast<const uint2*>(src);
  } else if constexpr (BYTES == 4) {
    *static_cast<uint32_t*>(dst) = *static_cast<const uint32_t*>(src);
  } else {
    *static_cast<uint16_t*>(dst) = *static_cast<const uint16_t*>(src);
  }
}
__device__ __forceinline__ uint32_t tf32_rna(float x);
// Two values rounded to nearest even into one packed pair of 16-bit values
// (the first at the lower address) by one paired conversion, and the pair
// widened back to fp32 (exact).  The rounding is the same as two single
// conversions'; one paired instruction per two values halves the conversion
// work of the plane writers below.
template <int FMT>
__device__ __forceinline__ uint32_t pack2_rn(float a, float b) {
  if constexpr (FMT == kFmtFP16) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}
template <int FMT>
__device__ __forceinline__ float2 unpack2(uint32_t w) {
  if constexpr (FMT == kFmtFP16) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  } else {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
}
template <int NW>
__device__ __forceinline__ void store_words(void* dst, const uint32_t* w) {
  if constexpr (NW == 4) {
    *static_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  } else if constexpr (NW == 2) {
    *static_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
  } else {
    *static_cast<uint32_t*>(dst) = w[0];
  }
}
// V consecutive entries (positions o .. o + V - 1 of every plane) written
// as the 3M planes of put_entry, one vector store per plane; o is a
// multiple of V.  Same arithmetic as put_entry, entry by entry.
template <int FMT, int V>
__device__ __forceinline__ void put_planes_vec(void* out, int64_t o, const float2* v, int nsplit, int64_t plane,
                                               float scale = 1.f) {
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    float x[V];
#pragma unroll
    for (int j = 0; j < V; ++j) x[j] = p == 0 ? v[j].x : (p == 1 ? v[j].y : v[j].x + v[j].y);
    if constexpr ((FMT == kFmtFP16 || FMT == kFmtBF16) && V >= 2) {
      // paired conversions: hi = rn(x), lo = rn(x - hi) (x - hi is exact)
      uint32_t hi[V / 2], lo[V / 2];
#pragma unroll
      for (int j = 0; j < V / 2; ++j) {
        const float y0 = FMT == kFmtFP16 ? x[2 * j] * scale : x[2 * j];   // exact: a power of two
        const float y1 = FMT == kFmtFP16 ? x[2 * j + 1] * scale : x[2 * j + 1];
        hi[j] = pack2_rn<FMT>(y0, y1);
        const float2 h = unpack2<FMT>(hi[j]);
        lo[j] = pack2_rn<FMT>(y0 - h.x, y1 - h.y);
      }
      uint16_t* q = static_cast<uint16_t*>(out);
      store_words<V / 2>(q + int64_t(p * nsplit) * plane + o, hi);
      if (nsplit == 2) store_words<V / 2>(q + int64_t(p * 2 + 1) * plane + o, lo);
    } else if constexpr (FMT == kFmtFP16) {
      __half hi[V], lo[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const float y = x[j] * scale;   // exact: scale is a power of two
        hi[j] = __float2half_rn(y);
        lo[j] = __float2half_rn(y - __half2float(hi[j]));
      }
      __half* q = static_cast<__half*>(out);
      store_bytes<2 * V>(q + int64_t(p * nsplit) * plane + o, hi);
      if (nsplit == 2) store_bytes<2 * V>(q + int64_t(p * 2 + 1) * plane + o, lo);
    } else if constexpr (FMT == kFmtTF32) {
      uint32_t hi[V], lo[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        hi[j] = tf32_rna(x[j]);
        lo[j] = tf32_rna(x[j] - __uint_as_float(hi[j]));
      }
      uint32_t* q = static_cast<uint32_t*>(out);
      store_bytes<4 * V>(q + int64_t(p * nsplit) * plane + o, hi);
      if (nsplit == 2) store_bytes<4 * V>(q + int64_t(p * 2 + 1) * plane + o, lo);
    } else {
      __nv_bfloat16 hi[V], lo[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        hi[j] = __float2bfloat16_rn(x[j]);
        lo[j] = __float2bfloat16_rn(x[j] - __bfloat162float(hi[j]));
      }
      __nv_bfloat16* q = static_cast<__nv_bfloat16*>(out);
      store_bytes<2 * V>(q + int64_t(p * nsplit) * plane + o, hi);
      if (nsplit == 2) store_bytes<2 * V>(q + int64_t(p * 2 + 1) * plane + o, lo);
    }
  }
}
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Write one complex entry at linear output position o in the requested
// format: complex64, FP64 accumulate, or the 3M operand planes
// [part][split][plane] (part re, im, re + im; split hi, lo = the rounding of
// x - hi) -- shared by the permutation kernels and the GEMM epilogue that
// writes the next step's operand, so both produce identical planes.
template <int FMT>
__device__ __forceinline__ void put_entry(void* out, int64_t o, float2 v, int nsplit, int64_t plane,
                                    float scale = 1.f) {
  if constexpr (FMT == kFmtC64) {
    static_cast<float2*>(out)[o] = v;
  } else if constexpr (FMT == kFmtAccC128) {
    double2* q = static_cast<double2*>(out) + o;
    const double2 c = *q;
    *q = make_double2(c.x + double(v.x), c.y + double(v.y));
  } else {
    const float part[3] = {v.x, v.y, v.x + v.y};
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      if constexpr (FMT == kFmtFP16) {
        __half* q = static_cast<__half*>(out);
        const float x = part[p] * scale;   // exact: scale is a power of two
        const __half hi = __float2half_rn(x);
        q[int64_t(p * nsplit) * plane + o] = hi;
        if (nsplit == 2) q[int64_t(p * 2 + 1) * plane + o] = __float2half_rn(x - __half2float(hi));
      } else if constexpr (FMT == kFmtTF32) {
        uint32_t* q = static_cast<uint32_t*>(out);
        const uint32_t hi = tf32_rna(part[p]);
        q[int64_t(p * nsplit) * plane + o] = hi;
        if (nsplit == 2) q[int64_t(p * 2 + 1) * plane + o] = tf32_rna(part[p] - __uint_as_float(hi));
      } else {
        __nv_bfloat16* q = static_cast<__nv_bfloat16*>(out);
        const __nv_bfloat16 hi = __float2bfloat16_rn(part[p]);
        q[int64_t(p * nsplit) * plane + o] = hi;
        if (nsplit == 2)
          q[int64_t(p * 2 + 1) * plane + o] = __float2bfloat16_rn(part[p] - __bfloat162float(hi));
      }
    }
  }
}
#endif

// Power-of-two scaling of fp16 operands: `smax` points to the bits of the
// largest |re|, |im|, |re+im| of the operand (written by launch_absmax);
// scale = 2^(14 - e) with smax = f 2^e, f in [0.5, 1), so scaled parts stay
// below 2^14.  Both the producer and the GEMM epilogue derive it from smax.
// Fidelity-f mixture of exact (accepted) and uniform samples; pool:
// [n_batches] scratch, source: [n_samples], counts: 2 x int64 (device).
cudaError_t launch_fidelity_mix(const uint8_t* batch_bits, const int32_t* accepted, int64_t n_batches,
                               const int32_t* tile, int n_tile, int n_qubits, double f, uint64_t seed,
                               int64_t n_samples, int32_t* pool, int32_t* source, int64_t* counts,
                               uint8_t* out, cudaStream_t s);
cudaError_t launch_absmax(const float2* in, int64_t n, unsigned* smax, cudaStream_t s);

// Build the tile tables for a map of `nbits` index bits: bit j moves the
// input by w_in[j] entries and the output by w_out[j] (1 << j when w_out is
// null: contiguous output).  Returns false if nbits exceeds the supported range.
bool build_perm_tile(int nbits, const int64_t* w_in, PermTile* t, const int64_t* w_out = nullptr);

// out-of-place permutation / operand production.  `in_base` is added to
// every input offset (cut-bond slicing).  For plane formats, `nsplit` is 1 or
// 2 and `plane_elems` the number of entries of one plane (rows*cols).
cudaError_t launch_permute_tiled(const float2* in, int64_t in_base, const PermTile& t,
                                 int fmt, int nsplit, void* out, int64_t plane_elems,
                                 cudaStream_t s, const unsigned* smax = nullptr);

// Generic gather for any dims: out[o] = in[base + sum_a idx_a(o) * stride_a].
constexpr int kGatherMaxRank = 32;
struct GatherDesc {
  int64_t dims[kGatherMaxRank];
  int64_t in_strides[kGatherMaxRank];
  int64_t total;
  int32_t rank;
};
cudaError_t launch_permute_gather(const float2* in, int64_t in_base, const GatherDesc& d,
                                  int fmt, int nsplit, void* out, int64_t plane_elems,
                                  cudaStream_t s, const unsigned* smax = nullptr);

// ------------------------------------------------------------------ complex GEMM
// C[m][n] = sum_k A[m][k] B[n][k], complex64, row-major, FP32 accumulate.
cudaError_t launch_cgemm_simt(int64_t M, int64_t N, int64_t K, const float2* A,
                              const float2* B, float2* C, cudaStream_t s);
// Same product for thin shapes (N <= 32): one thread per output row.
cudaError_t launch_cgemm_thin(int64_t M, int64_t N, int64_t K, const float2* A,
                              const float2* B, float2* C, cudaStream_t s);
// Split-K form of the block-per-row product (few outputs, long K): blocks
// over (row, 16-column group, split), each summing its K range of `chunk`
// entries into the partial product P + split M N.
cudaError_t launch_cgemm_rowwarp_split(int64_t M, int64_t N, int64_t K, const float2* A,
                                       const float2* B, float2* P, int splits, cudaStream_t s);
// Split-K form of the tiled product: grid z = split, same partial layout.
cudaError_t launch_cgemm_simt_split(int64_t M, int64_t N, int64_t K, const float2* A,
                                    const float2* B, float2* P, int splits, cudaStream_t s);
// C[i] = sum over s = 0..splits-1, in that order, of P[s * n + i] (FP32).
cudaError_t launch_splitk_reduce(const float2* P, int splits, int64_t n, float2* C, cudaStream_t s);

// Tensor-core GEMM on split 3M planes (produced by the permutation kernel in
// kFmtTF32 / kFmtBF16 / kFmtFP16 format).  kind: 0 = tf32, 1 = bf16, 2 = fp16
// (then smax_a / smax_b give the operand scales).  bn: 64 or 128.
struct TcGemmMaps {
  CUtensorMap a;
  CUtensorMap b;
};
// Epilogue output as the next step's 3M operand planes instead of C: entry
// (m, n) of the product goes to position sum_b bit_b(m) wm[b] + sum_b
// bit_b(n) wn[b] of each plane [part][split] (M and N powers of two; the map
// is a bijection onto [0, plane)).  n_fast: the lowest destination bits come
// from the column index (writes go along rows of the staged tile), else from
// the row index (writes go along columns).
constexpr int kMaxOutBits = 40;
struct TcPlaneOut {
  void* base = nullptr;      // planes [3 * nsplit][plane] (nullptr: write C)
  int64_t plane = 0;         // entries per plane (M * N)
  int64_t wm[kMaxOutBits] = {};
  int64_t wn[kMaxOutBits] = {};
  int32_t mbits = 0, nbits = 0;
  int32_t n_fast = 1;
  int32_t vec = 1;           // n_fast: columns per store (wn[b] = 2^b for 2^b < vec)
  int32_t fmt = 0;           // plane format for the CUDA-core producer: kFmtTF32 or kFmtBF16
  int32_t nsplit = 2;        // splits per part, same use
  // fp16 planes (tensor-core producer only).  The planes hold s x entry with
  // s = fp16_scale_of(bound), bound = 3 K max_a max_b >= 2 sqrt(2) K max_a max_b,
  // which no part of any entry can exceed (|C| <= K max|A| max|B|, |A| <=
  // sqrt(2) times its largest part, |re + im| <= sqrt(2) |C|): block 0 stores
  // the bound's bits in *out_scale for the consumer, and every warp takes the
  // atomicMax of the largest |re|, |im|, |re + im| it wrote into *out_max,
  // which later products read as their max_a / max_b.
  unsigned* out_scale = nullptr;
  unsigned* out_max = nullptr;
  const unsigned* max_a = nullptr;  // bits of upper bounds of the parts of A and of B
  const unsigned* max_b = nullptr;
};
// The pipelined thin product (launch_cgemm_thin's form for this shape) with
// its result written as operand planes (po) instead of C.
bool thin_pipelined(int64_t M, int64_t N, int64_t K);
cudaError_t launch_cgemm_thin_planes(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                                     const TcPlaneOut& po, cudaStream_t s);
// Form of the split (nsplit = 2) tensor-core product: true = per k-step one
// MMA of width 2 bn over the adjacent B hi and B lo tiles ([hi.hi | hi.lo])
// plus one of width bn (lo.hi); false = three MMAs of width bn.  The wide
// form is taken for bn = 64 and for bn = 128 when K >= 256 (with bn = 128
// it leaves room in TMEM for two accumulators instead of three, which costs
// more than it gains when K is a single k-block).
bool tc_wide_mma(int nsplit, int bn, int64_t K);
bool tc_encode_maps(int kind, int nsplit, int bn, const void* a_planes, int64_t M,
                    const void* b_planes, int64_t N, int64_t K, TcGemmMaps* maps);
// splits > 1 (complex64 output only): split-K, the k-blocks cut into
// `splits` ranges whose partial products go to C + s M N, s = 0..splits-1
// (C then holds splits x M x N entries; launch_splitk_reduce sums them).
cudaError_t launch_cgemm_tc(int kind, int nsplit, int bn, const TcGemmMaps& maps, int64_t M,
                            int64_t N, int64_t K, float2* C, int32_t* d_status,
                            cudaStream_t s, const unsigned* smax_a = nullptr,
                            const unsigned* smax_b = nullptr, const TcPlaneOut* planes = nullptr,
                            int splits = 1);
bool tc_available();   // driver entry point for tensor-map encoding found

// ------------------------------------------------------------------ small kernels
// amps[j] (complex128) += src[sum_t bit_t(j) * strides[t]] for j < 2^n_open.
cudaError_t launch_slicesum(const float2* src, const int64_t* strides, int n_open,
                            double* amps, cudaStream_t s);
cudaError_t launch_norm(const double* amps, int64_t n, double* out, cudaStream_t s);
// One CTA whose bounded wait on an mbarrier that no one arrives at runs out
// after limit_ns and sets kDevTimeout in *status (failure-detection test).
cudaError_t launch_wait_selftest(uint64_t limit_ns, int32_t* status, cudaStream_t s);
// Frugal rejection sampling, one accepted tile index (or -1) per batch;
// scale = N / M.  n_c <= 4096.
cudaError_t launch_frugal(const double* amps, int64_t n_batches, int n_c, double scale, uint64_t seed,
                          int32_t* accepted, cudaStream_t s);

// ------------------------------------------------------------------ adjoint
// W[sum_t bit_t(j) * strides[t]] = conj(g[j]) for j < 2^n_open (complex64).
cudaError_t launch_init_cotangent(float2* w, const int64_t* strides, int n_open, const double* g,
                                  cudaStream_t s);
// grad[param] += dL/dtheta from the FP64 grid-tensor cotangents of one bitstring.
cudaError_t launch_gridgrad(const GridQubitMeta* d_meta, int n_qubits, int max_bits, const int2* d_ops,
                            const double* d_angles, const uint8_t* d_bits, const double2* d_wgrid,
                            double* d_grad, cudaStream_t s);

int32_t* device_status_word(int device);   // library-wide status word for standalone calls
// Allocation-free GEMM (k_noalloc.cu): read and clear its status and report
// words on `dev` (synchronized by the caller); and its failure-detection
// self-test, which leaves the timeout bit in its status word.
cudaError_t noalloc_take_status(int dev, int32_t* bits);
cudaError_t noalloc_selftest(int dev, uint64_t limit_ns);

void set_last_error(const char* msg);      // text returned by qflex_last_error()

}  // namespace qflex

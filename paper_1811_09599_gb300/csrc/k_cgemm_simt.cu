// Step a3b, plain FP32 form: complex GEMM on the CUDA cores.
//
// Methods, "Implementation of the simulator": after the permutation each
// pairwise contraction is a row-major complex matrix product (the paper
// calls MKL's cgemm).  Here C[m][n] = sum_k A[m][k] * B[n][k] with four real
// FMAs per complex multiply-add and FP32 accumulation: the "plain FP32"
// arithmetic the split-precision tensor-core forms are compared against, and
// the path for shapes too small or too thin for the tensor cores.
//
// 64x64 output tile per 256-thread block, 4x4 complex outputs per thread,
// K staged 16 at a time through shared memory (transposed so that the inner
// loop reads contiguous rows).
#include "internal.h"

#include <algorithm>
#include <mutex>
#include <vector>

namespace qflex {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, PAD = 2;

// Kahan's compensated summation step: sum += x, with c holding minus the
// low-order part lost so far (unfused operations, so the compensation is
// computed as the method states).
__device__ __forceinline__ void kahan_add(float& sum, float& c, float x) {
  const float y = __fsub_rn(x, c);
  const float t = __fadd_rn(sum, y);
  c = __fsub_rn(__fsub_rn(t, sum), y);
  sum = t;
}

__global__ void __launch_bounds__(256) k_cgemm_simt(int64_t M, int64_t N, int64_t K,
                                                    const float2* __restrict__ A,
                                                    const float2* __restrict__ B,
                                                    float2* __restrict__ C) {
  pdl_wait();
  // split-K (gridDim.z > 1): block z sums the K range [z chunk, (z + 1)
  // chunk) into the partial product C + z M N; the loads below keep their
  // row stride K and stop at the range's end
  const int64_t chunk = (K + gridDim.z - 1) / gridDim.z;
  const int64_t k_begin = min(K, int64_t(blockIdx.z) * chunk);
  const int64_t k_end = min(K, k_begin + chunk);
  C += int64_t(blockIdx.z) * M * N;
  __shared__ __align__(16) float2 As[BK][BM + PAD];
  __shared__ __align__(16) float2 Bs[BK][BN + PAD];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  // p_*: the current K tile's partial sums, added once per tile to the
  // running sums acc_* with Kahan's compensated summation (c_*: the
  // compensation), so the FP32 rounding error of an output does not grow
  // with the number of tiles.
  float acc_re[TM][TN], acc_im[TM][TN], c_re[TM][TN], c_im[TM][TN];
  float p_re[TM][TN], p_im[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_re[i][j] = acc_im[i][j] = c_re[i][j] = c_im[i][j] = 0.f;

  for (int64_t k0 = k_begin; k0 < k_end; k0 += BK) {
#pragma unroll
    for (int i = 0; i < (BM * BK) / 256; ++i) {
      const int e = tid + i * 256;
      const int r = e / BK, kk = e % BK;
      const int64_t gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < k_end) ? A[gm * K + gk] : make_float2(0.f, 0.f);
      const int64_t gn = n0 + r;
      Bs[kk][r] = (gn < N && gk < k_end) ? B[gn * K + gk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) p_re[i][j] = p_im[i][j] = 0.f;
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], b[TN];
      const float4* ap = reinterpret_cast<const float4*>(&As[kk][ty * TM]);
      const float4* bp = reinterpret_cast<const float4*>(&Bs[kk][tx * TN]);
#pragma unroll
      for (int i = 0; i < TM / 2; ++i) {
        const float4 va = ap[i], vb = bp[i];
        a[2 * i] = make_float2(va.x, va.y);
        a[2 * i + 1] = make_float2(va.z, va.w);
        b[2 * i] = make_float2(vb.x, vb.y);
        b[2 * i + 1] = make_float2(vb.z, vb.w);
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          p_re[i][j] = fmaf(a[i].x, b[j].x, p_re[i][j]);
          p_re[i][j] = fmaf(-a[i].y, b[j].y, p_re[i][j]);
          p_im[i][j] = fmaf(a[i].x, b[j].y, p_im[i][j]);
          p_im[i][j] = fmaf(a[i].y, b[j].x, p_im[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        kahan_add(acc_re[i][j], c_re[i][j], p_re[i][j]);
        kahan_add(acc_im[i][j], c_im[i][j], p_im[i][j]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tx * TN + j;
      if (gn < N) C[gm * N + gn] = make_float2(__fsub_rn(acc_re[i][j], c_re[i][j]), __fsub_rn(acc_im[i][j], c_im[i][j]));
    }
  }
}

// Thin forms for N <= 32 (a large tensor absorbing a small one, HBM-bound).
// Packed FP32 pairs: P[n] = sum a.x * (b.x, b.y) and Q[n] = sum a.y * (b.x, b.y)
// with fma.rn.f32x2, so one complex multiply-add costs two packed FMAs and
// no register shuffling; C[n] = (P.x - Q.y, P.y + Q.x) at the end (the same
// products and sums as the four-FMA form, in the same order per component).
__device__ __forceinline__ unsigned long long pk(float x, float y) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long v) {
  float x, y;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
  return make_float2(x, y);
}
__device__ __forceinline__ void fma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}

// Row-per-thread form: each thread owns one output row and 16 of its
// columns; A is staged through shared memory, B broadcast from it.
constexpr int TBK = 16;
template <int TBN>
__global__ void __launch_bounds__(256, 2) k_cgemm_thin(int64_t M, int64_t N, int64_t K,
                                                      const float2* __restrict__ A,
                                                      const float2* __restrict__ B,
                                                      float2* __restrict__ C) {
  pdl_wait();
  constexpr int CG = TBN / 16;            // column groups per row
  constexpr int RB = 256 / CG;            // rows per block
  __shared__ __align__(16) float2 As[RB][TBK + 1];
  __shared__ __align__(16) float2 Bs[TBK][TBN];
  const int t = threadIdx.x;
  const int row = t / CG, cg = t % CG;
  const int64_t m0 = int64_t(blockIdx.x) * RB, n0 = int64_t(blockIdx.y) * TBN;
  unsigned long long P[16], Q[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) P[n] = Q[n] = 0ull;
  for (int64_t k0 = 0; k0 < K; k0 += TBK) {
#pragma unroll 4
    for (int i = 0; i < (RB * TBK) / 256; ++i) {
      const int e = t + i * 256;
      const int r = e / TBK, kk = e % TBK;
      const int64_t gm = m0 + r, gk = k0 + kk;
      As[r][kk] = (gm < M && gk < K) ? __ldg(A + gm * K + gk) : make_float2(0.f, 0.f);
    }
    for (int e = t; e < TBN * TBK; e += 256) {
      const int n = e / TBK, kk = e % TBK;
      const int64_t gn = n0 + n, gk = k0 + kk;
      Bs[kk][n] = (gn < N && gk < K) ? __ldg(B + gn * K + gk) : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < TBK; ++kk) {
      const float2 a = As[row][kk];
      const unsigned long long ax = pk(a.x, a.x), ay = pk(a.y, a.y);
      const float4* bp = reinterpret_cast<const float4*>(&Bs[kk][cg * 16]);
#pragma unroll
      for (int n = 0; n < 16; n += 2) {
        const float4 b = bp[n / 2];
        const unsigned long long b0 = pk(b.x, b.y), b1 = pk(b.z, b.w);
        fma2(P[n], ax, b0);
        fma2(Q[n], ay, b0);
        fma2(P[n + 1], ax, b1);
        fma2(Q[n + 1], ay, b1);
      }
    }
    __syncthreads();
  }
  const int64_t gm = m0 + row;
  if (gm < M) {
    const int64_t c0 = n0 + cg * 16;
    float2* crow = C + gm * N + c0;
    const int64_t ncols = N - c0 < 16 ? N - c0 : 16;
    const bool vec = ((reinterpret_cast<uintptr_t>(crow) & 15) == 0);
#pragma unroll
    for (int n = 0; n < 16; n += 2) {
      const float2 p0 = upk(P[n]), q0 = upk(Q[n]), p1 = upk(P[n + 1]), q1 = upk(Q[n + 1]);
      const float2 c0v = make_float2(p0.x - q0.y, p0.y + q0.x);
      const float2 c1v = make_float2(p1.x - q1.y, p1.y + q1.x);
      if (vec && n + 1 < ncols) {
        *reinterpret_cast<float4*>(crow + n) = make_float4(c0v.x, c0v.y, c1v.x, c1v.y);
      } else {
        if (n < ncols) crow[n] = c0v;
        if (n + 1 < ncols) crow[n + 1] = c1v;
      }
    }
  }
}

// Block-per-row form for few rows and a long K (the row-per-thread forms
// would leave most SMs idle): block b computes row m and 16 output columns
// n0 .. n0 + 15 of split `split` ((split, m, column group) = b); its 8 warps
// take interleaved 32-entry runs of the K range, every lane accumulating in
// k order, then each warp sums its lanes with shuffles and the 8 warp sums
// are added in warp order (deterministic).  With splits > 1 the K range of
// split s is [s chunk, (s + 1) chunk), chunk = ceil(K / splits), possibly
// empty, written as the partial product C + s M N (zeros for an empty
// range).
__global__ void __launch_bounds__(256) k_cgemm_rowwarp(int64_t M, int64_t N, int64_t K,
                                                      const float2* __restrict__ A,
                                                      const float2* __restrict__ B,
                                                      float2* __restrict__ C, int splits) {
  pdl_wait();
  __shared__ float2 part[8][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t cgs = (N + 15) / 16;
  const int64_t item = blockIdx.x;
  const int64_t split = item / (M * cgs), w = item % (M * cgs);
  if (split >= splits) return;
  const int64_t m = w / cgs, n0 = (w % cgs) * 16;
  const int64_t chunk = (K + splits - 1) / splits;
  const int64_t k_lo = split * chunk < K ? split * chunk : K;
  const int64_t k_hi = k_lo + chunk < K ? k_lo + chunk : K;
  C += split * M * N;
  const int nn = int(N - n0 < 16 ? N - n0 : 16);
  unsigned long long P[16], Q[16];
#pragma unroll
  for (int n = 0; n < 16; ++n) P[n] = Q[n] = 0ull;
  for (int64_t k = k_lo + warp * 32 + lane; k < k_hi; k += 256) {
    const float2 a = __ldg(A + m * K + k);
    const unsigned long long ax = pk(a.x, a.x), ay = pk(a.y, a.y);
#pragma unroll
    for (int n = 0; n < 16; ++n) {
      if (n < nn) {
        const float2 b = __ldg(B + (n0 + n) * K + k);
        const unsigned long long bb = pk(b.x, b.y);
        fma2(P[n], ax, bb);
        fma2(Q[n], ay, bb);
      }
    }
  }
#pragma unroll
  for (int n = 0; n < 16; ++n) {
    float2 p = upk(P[n]), q = upk(Q[n]);
    float re = p.x - q.y, im = p.y + q.x;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == n) part[warp][n] = make_float2(re, im);
  }
  __syncthreads();
  if (threadIdx.x < nn) {
    float2 acc = part[0][threadIdx.x];
#pragma unroll
    for (int v = 1; v < 8; ++v) {
      acc.x += part[v][threadIdx.x].x;
      acc.y += part[v][threadIdx.x].y;
    }
    C[m * N + n0 + threadIdx.x] = acc;
  }
}

// Pipelined row-tile form for N <= 16 (absorbing a tensor with few free
// entries into a large one: HBM-bound).  Persistent blocks walk 64-row
// tiles; A streams through a 4-stage cp.async pipeline in k-chunks of KC
// (zero-filled past M and K), B sits transposed in shared memory for the
// whole kernel.  Thread t owns row t / 4 and output columns 4 (t % 4) ..
// +3, accumulating P = sum a.x b and Q = sum a.y b in k order with scalar
// FMAs (the same per-lane roundings as the packed form of k_cgemm_thin,
// whose register-pair moves made it issue-bound here), so every output is
// summed exactly as there.  Rows of a stage are padded by 16 B: the 8 rows
// a warp reads fall in distinct banks.
constexpr int T2_RT = 64, T2_NST = 4;

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

template <int KC, bool PO>
__global__ void __launch_bounds__(256) k_cgemm_thin2(int64_t M, int N, int K, const float2* __restrict__ A,
                                                    const float2* __restrict__ B, float2* __restrict__ C,
                                                    const __grid_constant__ TcPlaneOut po) {
  pdl_wait();
  // fp16 planes: the scale of the bound 3 K max|A| max|B| of the entries
  // (TcPlaneOut), stored once for the consumer
  float po_scale = 1.f;
  if constexpr (PO) {
    if (po.fmt == kFmtFP16) {
      const unsigned bb = __float_as_uint(3.f * float(K) * __uint_as_float(*po.max_a) * __uint_as_float(*po.max_b));
      if (blockIdx.x == 0 && threadIdx.x == 0) *po.out_scale = bb;
      po_scale = fp16_scale_of(bb);
    }
  }
  extern __shared__ __align__(16) float2 sm2[];
  constexpr int LD = KC + 2;                      // padded row (float2), 16-byte multiple
  float2* Bt = sm2;                               // [K][16]
  float2* As = sm2 + size_t(K) * 16;              // [T2_NST][T2_RT][LD]
  const int t = threadIdx.x;
  for (int e = t; e < K * 16; e += 256) {
    const int k = e >> 4, n = e & 15;
    Bt[e] = n < N ? B[int64_t(n) * K + k] : make_float2(0.f, 0.f);
  }
  const int64_t n_tiles = (M + T2_RT - 1) / T2_RT;
  const int nch = (K + KC - 1) / KC;
  // units of this block: (tile i, chunk c), i over blockIdx.x + j * gridDim.x
  const int64_t my_tiles = blockIdx.x < n_tiles ? (n_tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t n_units = my_tiles * nch;
  auto issue = [&](int64_t u) {
    if (u < n_units) {
      const int64_t tile = blockIdx.x + (u / nch) * gridDim.x;
      const int c = int(u % nch);
      const int64_t m0 = tile * T2_RT;
      float2* dst = As + size_t(u % T2_NST) * T2_RT * LD;
#pragma unroll
      for (int j = 0; j < (T2_RT * KC / 2) / 256; ++j) {
        const int e2 = t + j * 256;               // pair of complex entries (16 bytes)
        const int r = e2 / (KC / 2), kp = e2 % (KC / 2);
        const int64_t gm = m0 + r;
        const int gk = c * KC + 2 * kp;
        const bool in = gm < M && gk < K;
        const float2* src = in ? A + gm * K + gk : A;
        cp_async16(uint32_t(__cvta_generic_to_shared(dst + r * LD + 2 * kp)), src, in ? 16 : 0);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  for (int u = 0; u < T2_NST - 1; ++u) issue(u);
  const int row = t >> 2, cq = t & 3;
  // plane output: the destination of (row gm, column n) is the sum of the
  // weights of the set bits of gm and n.  Per thread, the weights of its
  // row within a tile (bits 0-5 of gm) and of its four columns are summed
  // once; the weights of the tile index (bits 6-19 of gm) come from two
  // 128-entry tables built once per block.
  int64_t d_low = 0, dn[4] = {0, 0, 0, 0};
  int64_t* dtab = reinterpret_cast<int64_t*>(As + size_t(T2_NST) * T2_RT * LD);   // [2][128]
  if constexpr (PO) {
    for (int b = 0; b < 6 && b < po.mbits; ++b)
      if ((row >> b) & 1) d_low += po.wm[b];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      for (int b = 0; b < po.nbits; ++b)
        if (((cq * 4 + j) >> b) & 1) dn[j] += po.wn[b];
    const int half = t >> 7, v = t & 127;
    int64_t d = 0;
    for (int i = 0; i < 7; ++i) {
      const int b = 6 + 7 * half + i;
      if (b < po.mbits && ((v >> i) & 1)) d += po.wm[b];
    }
    dtab[t] = d;   // visible after the first unit's barrier
  }
  float2 P[4], Q[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) P[j] = Q[j] = make_float2(0.f, 0.f);
  for (int64_t u = 0; u < n_units; ++u) {
    asm volatile("cp.async.wait_group %0;" ::"n"(T2_NST - 2) : "memory");
    __syncthreads();                              // stage u landed; stage u - 1 fully consumed
    issue(u + T2_NST - 1);
    const int c = int(u % nch);
    const float2* a_row = As + size_t(u % T2_NST) * T2_RT * LD + row * LD;
    const float2* b_col = Bt + size_t(c) * KC * 16 + cq * 4;
    const int kn = min(KC, K - c * KC);
#pragma unroll 4
    for (int kk = 0; kk < kn; ++kk) {
      const float2 a = a_row[kk];
      const float4 b01 = *reinterpret_cast<const float4*>(b_col + kk * 16);
      const float4 b23 = *reinterpret_cast<const float4*>(b_col + kk * 16 + 2);
      const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                           make_float2(b23.z, b23.w)};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        P[j].x = fmaf(a.x, b[j].x, P[j].x);
        P[j].y = fmaf(a.x, b[j].y, P[j].y);
        Q[j].x = fmaf(a.y, b[j].x, Q[j].x);
        Q[j].y = fmaf(a.y, b[j].y, Q[j].y);
      }
    }
    if (c == nch - 1) {
      const int64_t gm = (blockIdx.x + (u / nch) * gridDim.x) * T2_RT + row;
      if constexpr (PO) {
        // the next step's operand planes at the bit-permuted positions
        float mx = 0.f;   // largest part written (fp16 planes: for later bounds)
        if (gm < M) {
          float2 o[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) o[j] = make_float2(P[j].x - Q[j].y, P[j].y + Q[j].x);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (cq * 4 + j < N) mx = fmaxf(mx, fmaxf(fabsf(o[j].x), fmaxf(fabsf(o[j].y), fabsf(o[j].x + o[j].y))));
          const int64_t tile = gm / T2_RT;
          int64_t d0 = d_low + dtab[tile & 127] + dtab[128 + ((tile >> 7) & 127)];
          for (int b = 20; b < po.mbits; ++b)
            if ((gm >> b) & 1) d0 += po.wm[b];
          if (po.n_fast && po.vec >= 4 && cq * 4 + 3 < N && d0 + dn[0] + 4 <= po.plane) {
            if (po.fmt == kFmtTF32)
              put_planes_vec<kFmtTF32, 4>(po.base, d0 + dn[0], o, po.nsplit, po.plane);
            else if (po.fmt == kFmtFP16)
              put_planes_vec<kFmtFP16, 4>(po.base, d0 + dn[0], o, po.nsplit, po.plane, po_scale);
            else
              put_planes_vec<kFmtBF16, 4>(po.base, d0 + dn[0], o, po.nsplit, po.plane);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int64_t d = d0 + dn[j];
              if (cq * 4 + j < N && d >= 0 && d < po.plane) {
                if (po.fmt == kFmtTF32)
                  put_entry<kFmtTF32>(po.base, d, o[j], po.nsplit, po.plane);
                else if (po.fmt == kFmtFP16)
                  put_entry<kFmtFP16>(po.base, d, o[j], po.nsplit, po.plane, po_scale);
                else
                  put_entry<kFmtBF16>(po.base, d, o[j], po.nsplit, po.plane);
              }
            }
          }
        }
        if (po.fmt == kFmtFP16) {
          for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
          if ((t & 31) == 0 && mx > 0.f) atomicMax(po.out_max, __float_as_uint(mx));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) P[j] = Q[j] = make_float2(0.f, 0.f);
        continue;
      }
      if (gm < M) {
        float2 o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = make_float2(P[j].x - Q[j].y, P[j].y + Q[j].x);
        float2* crow = C + gm * N + cq * 4;
        if (N == 16 && (reinterpret_cast<uintptr_t>(crow) & 15) == 0) {
          reinterpret_cast<float4*>(crow)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
          reinterpret_cast<float4*>(crow)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (cq * 4 + j < N) crow[j] = o[j];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) P[j] = Q[j] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int KC, bool PO>
cudaError_t launch_thin2(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B, float2* C,
                         const TcPlaneOut& po, cudaStream_t s) {
  const size_t smem = size_t(K) * 16 * sizeof(float2) + size_t(T2_NST) * T2_RT * (KC + 2) * sizeof(float2) +
                      (PO ? 256 * sizeof(int64_t) : 0);
  // at most 512 x 16 x 8 + 4 x 64 x 34 x 8 + 2048 bytes (K <= 512): opt in once per device
  int dev = 0, sms = 148, occ = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static std::vector<char> opted;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (int(opted.size()) <= dev) opted.resize(size_t(dev) + 1, 0);
    if (!opted[size_t(dev)]) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_cgemm_thin2<KC, PO>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e != cudaSuccess) return e;
      opted[size_t(dev)] = 1;
    }
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cgemm_thin2<KC, PO>, 256, smem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int64_t tiles = (M + T2_RT - 1) / T2_RT;
  const int blocks = int(std::min<int64_t>(tiles, int64_t(sms) * occ));
  return launch_pdl(k_cgemm_thin2<KC, PO>, dim3(blocks), dim3(256), smem, s, M, int(N), int(K), A, B, C, po);
}

}  // namespace

bool thin_pipelined(int64_t M, int64_t N, int64_t K) {
  const bool rowwarp = K >= 64 && ((M + 255) / 256) * ((N + 15) / 16) < 256;
  return !rowwarp && N <= 16 && K % 2 == 0 && K <= 512;
}

cudaError_t launch_cgemm_thin_planes(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                                     const TcPlaneOut& po, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!thin_pipelined(M, N, K) || (reinterpret_cast<uintptr_t>(A) & 15) != 0 || !po.base ||
      (po.fmt != kFmtTF32 && po.fmt != kFmtBF16 && po.fmt != kFmtFP16) ||
      (po.fmt == kFmtFP16 && (!po.out_scale || !po.out_max || !po.max_a || !po.max_b)))
    return cudaErrorInvalidValue;
  return K <= 16 ? launch_thin2<16, true>(M, N, K, A, B, nullptr, po, s)
                 : launch_thin2<32, true>(M, N, K, A, B, nullptr, po, s);
}

namespace {
__global__ void __launch_bounds__(256) k_splitk_reduce(const float2* __restrict__ P, int splits, int64_t n,
                                                      float2* __restrict__ C) {
  pdl_wait();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float2 acc = P[i];
    for (int sp = 1; sp < splits; ++sp) {
      const float2 v = P[sp * n + i];
      acc.x += v.x;
      acc.y += v.y;
    }
    C[i] = acc;
  }
}
}  // namespace

cudaError_t launch_cgemm_simt_split(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                                    float2* P, int splits, cudaStream_t s) {
  if (M <= 0 || N <= 0 || splits < 1 || splits > 65535 || K <= 0) return cudaErrorInvalidValue;
  dim3 grid(unsigned((N + BN - 1) / BN), unsigned((M + BM - 1) / BM), unsigned(splits));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  return launch_pdl(k_cgemm_simt, grid, dim3(256), 0, s, M, N, K, A, B, P);
}

cudaError_t launch_cgemm_rowwarp_split(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                                       float2* P, int splits, cudaStream_t s) {
  if (M <= 0 || N <= 0 || splits < 1 || K <= 0) return cudaErrorInvalidValue;
  const int64_t cgs = (N + 15) / 16;
  const int64_t blocks = M * cgs * splits;
  if (blocks > INT32_MAX) return cudaErrorInvalidValue;
  return launch_pdl(k_cgemm_rowwarp, dim3(unsigned(blocks)), dim3(256), 0, s, M, N, K, A, B, P, splits);
}

cudaError_t launch_splitk_reduce(const float2* P, int splits, int64_t n, float2* C, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 8);
  return launch_pdl(k_splitk_reduce, dim3(unsigned(blocks)), dim3(256), 0, s, P, splits, n, C);
}

cudaError_t launch_cgemm_thin(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                              float2* C, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int64_t cgs = (N + 15) / 16;
  if (K >= 64 && ((M + 255) / 256) * cgs < 256) {   // few rows, long K: warp per row
    return launch_pdl(k_cgemm_rowwarp, dim3(unsigned(M * cgs)), dim3(256), 0, s, M, N, K, A, B, C, 1);
  }
  if (thin_pipelined(M, N, K) && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
    static const TcPlaneOut none{};
    return K <= 16 ? launch_thin2<16, false>(M, N, K, A, B, C, none, s)
                   : launch_thin2<32, false>(M, N, K, A, B, C, none, s);
  }
  if (N <= 16) {
    dim3 grid(unsigned((M + 255) / 256), unsigned((N + 15) / 16));
    return launch_pdl(k_cgemm_thin<16>, grid, dim3(256), 0, s, M, N, K, A, B, C);
  } else {
    dim3 grid(unsigned((M + 127) / 128), unsigned((N + 31) / 32));
    return launch_pdl(k_cgemm_thin<32>, grid, dim3(256), 0, s, M, N, K, A, B, C);
  }
}

cudaError_t launch_cgemm_simt(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                              float2* C, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(unsigned((N + BN - 1) / BN), unsigned((M + BM - 1) / BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  return launch_pdl(k_cgemm_simt, grid, dim3(256), 0, s, M, N, K, A, B, C);
}

}  // namespace qflex

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

namespace qflex {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4, PAD = 2;

__global__ void __launch_bounds__(256) k_cgemm_simt(int64_t M, int64_t N, int64_t K,
                                                    const float2* __restrict__ A,
                                                    const float2* __restrict__ B,
                                                    float2* __restrict__ C) {
  __shared__ __align__(16) float2 As[BK][BM + PAD];
  __shared__ __align__(16) float2 Bs[BK][BN + PAD];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = int64_t(blockIdx.y) * BM, n0 = int64_t(blockIdx.x) * BN;
  float acc_re[TM][TN], acc_im[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc_re[i][j] = acc_im[i][j] = 0.f;

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int i = 0; i < (BM * BK) / 256; ++i) {
      const int e = tid + i * 256;
      const int r = e / BK, kk = e % BK;
      const int64_t gm = m0 + r, gk = k0 + kk;
      As[kk][r] = (gm < M && gk < K) ? A[gm * K + gk] : make_float2(0.f, 0.f);
      const int64_t gn = n0 + r;
      Bs[kk][r] = (gn < N && gk < K) ? B[gn * K + gk] : make_float2(0.f, 0.f);
    }
    __syncthreads();
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
          acc_re[i][j] = fmaf(a[i].x, b[j].x, acc_re[i][j]);
          acc_re[i][j] = fmaf(-a[i].y, b[j].y, acc_re[i][j]);
          acc_im[i][j] = fmaf(a[i].x, b[j].y, acc_im[i][j]);
          acc_im[i][j] = fmaf(a[i].y, b[j].x, acc_im[i][j]);
        }
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
      if (gn < N) C[gm * N + gn] = make_float2(acc_re[i][j], acc_im[i][j]);
    }
  }
}

}  // namespace

cudaError_t launch_cgemm_simt(int64_t M, int64_t N, int64_t K, const float2* A, const float2* B,
                              float2* C, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(unsigned((N + BN - 1) / BN), unsigned((M + BM - 1) / BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  k_cgemm_simt<<<grid, 256, 0, s>>>(M, N, K, A, B, C);
  return cudaGetLastError();
}

}  // namespace qflex

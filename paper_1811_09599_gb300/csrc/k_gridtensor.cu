// Step a1: per-qubit grid tensors.
//
// Methods, "Overview of the simulator" / "Contraction of the 3D tensor
// network": every gate acting on qubit q is contracted, in time order, into
// one tensor T_q whose legs are the qubit's output (input fixed to |0>) and
// one bond per neighbour of dimension 2^{K_e} (K_e = number of CZs on that
// edge).  Each CZ enters through its rank-2 Schmidt split
//   (-1)^{ab} = sum_k d_{a,k} (-1)^{k b}:
// the lower-index qubit applies |k><k|, the higher-index one applies Z^k,
// with k one bit of the bond multi-index (first CZ in time = most
// significant bit of that bond).  An iSWAP enters through its rank-4 split
// iSWAP = (II + ZZ)/2 + i (XX + YY)/2: the lower-index qubit applies P_k,
// the other c_k P_k, with k two bits of the bond multi-index.
//
// One thread per bond-index entry evolves the qubit's 2-vector through its
// gate line (FP32) with the CZ halves selected by the entry's bits, and
// writes T[o][entry] for o in {0,1} (open output leg, tile qubits) or only
// T[x_q][entry] (output bit fixed by the bitstring).
#include "internal.h"

namespace qflex {
namespace {

struct C2 {
  float2 m00, m01, m10, m11;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ C2 gate_matrix(int kind, const double* angles, int param) {
  const float r = 0.70710678118654752440f;
  C2 g;
  switch (kind) {
    case 0:  // H
      g = {make_float2(r, 0), make_float2(r, 0), make_float2(r, 0), make_float2(-r, 0)};
      break;
    case 1:  // T = diag(1, e^{i pi/4})
      g = {make_float2(1, 0), make_float2(0, 0), make_float2(0, 0), make_float2(r, r)};
      break;
    case 2:  // X^1/2 = 1/2 [[1+i, 1-i], [1-i, 1+i]]
      g = {make_float2(.5f, .5f), make_float2(.5f, -.5f), make_float2(.5f, -.5f), make_float2(.5f, .5f)};
      break;
    case 3:  // Y^1/2 = 1/2 [[1+i, -1-i], [1+i, 1+i]]
      g = {make_float2(.5f, .5f), make_float2(-.5f, -.5f), make_float2(.5f, .5f), make_float2(.5f, .5f)};
      break;
    default: {  // R_P(t) = cos(t/2) I - i sin(t/2) P
      float s, c;
      sincosf(0.5f * (float)angles[param], &s, &c);
      if (kind == 5)  // RX: [[c, -is], [-is, c]]
        g = {make_float2(c, 0), make_float2(0, -s), make_float2(0, -s), make_float2(c, 0)};
      else if (kind == 6)  // RY: [[c, -s], [s, c]]
        g = {make_float2(c, 0), make_float2(-s, 0), make_float2(s, 0), make_float2(c, 0)};
      else  // RZ: diag(c - is, c + is)
        g = {make_float2(c, -s), make_float2(0, 0), make_float2(0, 0), make_float2(c, s)};
    }
  }
  return g;
}

__global__ void k_gridtensor(const GridQubitMeta* __restrict__ meta, const int2* __restrict__ ops,
                             const double* __restrict__ angles, const uint8_t* __restrict__ bits,
                             float2* __restrict__ grid) {
  const GridQubitMeta m = meta[blockIdx.y];
  const int64_t entries = int64_t(1) << m.n_bits;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  float2 v0 = make_float2(1.f, 0.f), v1 = make_float2(0.f, 0.f);
  for (int i = 0; i < m.op_count; ++i) {
    const int2 op = ops[m.op_begin + i];
    const int type = op.x & 0xff;
    if (type == kOpCzProj || type == kOpCzZ) {
      const int k = int((e >> (op.x >> 8)) & 1);
      if (type == kOpCzProj) {
        if (k) v0 = make_float2(0.f, 0.f);
        else v1 = make_float2(0.f, 0.f);
      } else if (k) {
        v1 = make_float2(-v1.x, -v1.y);
      }
    } else if (type == kOpIswA || type == kOpIswB) {
      iswap_half_col(type, int((e >> (op.x >> 8)) & 3), v0, v1);
    } else {
      const C2 g = gate_matrix(type, angles, op.y);
      const float2 n0 = cadd(cmul(g.m00, v0), cmul(g.m01, v1));
      const float2 n1 = cadd(cmul(g.m10, v0), cmul(g.m11, v1));
      v0 = n0;
      v1 = n1;
    }
  }
  float2* out = grid + m.offset;
  if (m.tile) {
    out[e] = v0;
    out[entries + e] = v1;
  } else {
    out[e] = bits[m.qubit] ? v1 : v0;
  }
}

}  // namespace

cudaError_t launch_gridtensor(const GridQubitMeta* d_meta, int n_qubits, int max_bits,
                              const int2* d_ops, const double* d_angles, const uint8_t* d_bits,
                              float2* d_grid, cudaStream_t s) {
  const int threads = 256;
  const int64_t entries = int64_t(1) << max_bits;
  dim3 grid(unsigned((entries + threads - 1) / threads), unsigned(n_qubits));
  k_gridtensor<<<grid, threads, 0, s>>>(d_meta, d_ops, d_angles, d_bits, d_grid);
  return cudaGetLastError();
}

}  // namespace qflex

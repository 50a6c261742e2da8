// Step a7: gradients of amplitudes with respect to rotation angles.
//
// The paper computes amplitudes only; the gradient follows from the same
// network.  With L = Re sum_j conj(g_j) amp_j and amp holomorphic in the
// grid-tensor entries, the cotangent of every tensor X is
// W_X = sum_j conj(g_j) d amp_j / d X.  The host walks the pairwise
// contractions backwards (W_A = W_C B, W_B = W_C^T A for C = A B^T), which
// accumulates the environment W_q of every grid tensor over the slices in
// FP64.  This file holds the two ends of that walk:
//   k_init_cotangent  W of the final tensor: conj(g_j) at tile index j;
//   k_gridgrad        dL/dtheta for each rotation on qubit q: for every
//                     entry e of T_q, Re( u . dG . v ) where v is the
//                     qubit's state just before the gate (prefix), u the
//                     row vector W_q[., e] propagated back through the gates
//                     after it (suffix), and dG/dtheta = R_P(theta + pi) / 2.
// The per-entry terms are reduced in FP64 (warp shuffles, one atomic per
// warp and gate).
#include "internal.h"

namespace qflex {
namespace {

struct TileMap {
  int64_t strides[32];
  int32_t n_open;
};

__global__ void k_init_cotangent(float2* __restrict__ w, const __grid_constant__ TileMap m,
                                 const double* __restrict__ g) {
  const int64_t count = int64_t(1) << m.n_open;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < count;
       j += int64_t(gridDim.x) * blockDim.x) {
    int64_t idx = 0;
    for (int t = 0; t < m.n_open; ++t)
      if ((j >> (m.n_open - 1 - t)) & 1) idx += m.strides[t];
    w[idx] = make_float2(float(g[2 * j]), -float(g[2 * j + 1]));
  }
}

struct M2 {
  float2 a, b, c, d;   // [[a, b], [c, d]]
};
__device__ __forceinline__ float2 cm(float2 x, float2 y) {
  return make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
}
__device__ __forceinline__ float2 ca(float2 x, float2 y) { return make_float2(x.x + y.x, x.y + y.y); }

__device__ __forceinline__ M2 fixed_gate(int kind) {
  const float r = 0.70710678118654752440f;
  switch (kind) {
    case 0: return {make_float2(r, 0), make_float2(r, 0), make_float2(r, 0), make_float2(-r, 0)};
    case 1: return {make_float2(1, 0), make_float2(0, 0), make_float2(0, 0), make_float2(r, r)};
    case 2: return {make_float2(.5f, .5f), make_float2(.5f, -.5f), make_float2(.5f, -.5f), make_float2(.5f, .5f)};
    default: return {make_float2(.5f, .5f), make_float2(-.5f, -.5f), make_float2(.5f, .5f), make_float2(.5f, .5f)};
  }
}
// R_P(t) = cos(t/2) I - i sin(t/2) P
__device__ __forceinline__ M2 rot(int kind, float th) {
  float s, c;
  sincosf(0.5f * th, &s, &c);
  if (kind == 5) return {make_float2(c, 0), make_float2(0, -s), make_float2(0, -s), make_float2(c, 0)};
  if (kind == 6) return {make_float2(c, 0), make_float2(-s, 0), make_float2(s, 0), make_float2(c, 0)};
  return {make_float2(c, -s), make_float2(0, 0), make_float2(0, 0), make_float2(c, s)};
}

constexpr int kMaxRot = 64;   // rotation gates per qubit line

__global__ void __launch_bounds__(256) k_gridgrad(const GridQubitMeta* __restrict__ meta,
                                                  const int2* __restrict__ ops,
                                                  const double* __restrict__ angles,
                                                  const uint8_t* __restrict__ bits,
                                                  const double2* __restrict__ wgrid,
                                                  double* __restrict__ grad) {
  const GridQubitMeta m = meta[blockIdx.y];
  const int64_t entries = int64_t(1) << m.n_bits;
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool live = e < entries;
  // prefix states before each rotation gate
  float2 pv0[kMaxRot], pv1[kMaxRot];
  int nrot = 0;
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
      continue;
    }
    if (type == kOpIswA || type == kOpIswB) {
      iswap_half_col(type, int((e >> (op.x >> 8)) & 3), v0, v1);
      continue;
    }
    M2 g;
    if (type >= 5) {
      if (nrot < kMaxRot) {
        pv0[nrot] = v0;
        pv1[nrot] = v1;
      }
      ++nrot;
      g = rot(type, float(angles[op.y]));
    } else {
      g = fixed_gate(type);
    }
    const float2 n0 = ca(cm(g.a, v0), cm(g.b, v1));
    const float2 n1 = ca(cm(g.c, v0), cm(g.d, v1));
    v0 = n0;
    v1 = n1;
  }
  // row vector u = sum_o W[o, e] <o|
  float2 u0 = make_float2(0.f, 0.f), u1 = make_float2(0.f, 0.f);
  if (live) {
    const double2* w = wgrid + m.offset;
    if (m.tile) {
      u0 = make_float2(float(w[e].x), float(w[e].y));
      u1 = make_float2(float(w[entries + e].x), float(w[entries + e].y));
    } else {
      const float2 x = make_float2(float(w[e].x), float(w[e].y));
      if (bits[m.qubit]) u1 = x;
      else u0 = x;
    }
  }
  int r = nrot;
  for (int i = m.op_count - 1; i >= 0; --i) {
    const int2 op = ops[m.op_begin + i];
    const int type = op.x & 0xff;
    if (type == kOpCzProj || type == kOpCzZ) {
      const int k = int((e >> (op.x >> 8)) & 1);
      if (type == kOpCzProj) {
        if (k) u0 = make_float2(0.f, 0.f);
        else u1 = make_float2(0.f, 0.f);
      } else if (k) {
        u1 = make_float2(-u1.x, -u1.y);
      }
      continue;
    }
    if (type == kOpIswA || type == kOpIswB) {
      iswap_half_row(type, int((e >> (op.x >> 8)) & 3), u0, u1);
      continue;
    }
    M2 g;
    if (type >= 5) {
      --r;
      const float th = float(angles[op.y]);
      g = rot(type, th);
      const M2 d = rot(type, th + 3.14159265358979323846f);   // dG/dtheta = R(theta+pi)/2
      double contrib = 0.0;
      if (live && r < kMaxRot) {
        const float2 a0 = ca(cm(d.a, pv0[r]), cm(d.b, pv1[r]));
        const float2 a1 = ca(cm(d.c, pv0[r]), cm(d.d, pv1[r]));
        const float2 s = ca(cm(u0, a0), cm(u1, a1));
        contrib = 0.5 * double(s.x);
      }
      for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
      if ((threadIdx.x & 31) == 0 && contrib != 0.0) atomicAdd(grad + op.y, contrib);
    } else {
      g = fixed_gate(type);
    }
    // u <- u . G
    const float2 n0 = ca(cm(u0, g.a), cm(u1, g.c));
    const float2 n1 = ca(cm(u0, g.b), cm(u1, g.d));
    u0 = n0;
    u1 = n1;
  }
}

}  // namespace

cudaError_t launch_init_cotangent(float2* w, const int64_t* strides, int n_open, const double* g,
                                  cudaStream_t s) {
  if (n_open < 0 || n_open > 30) return cudaErrorInvalidValue;
  TileMap m{};
  for (int t = 0; t < n_open; ++t) m.strides[t] = strides[t];
  m.n_open = n_open;
  const int64_t count = int64_t(1) << n_open;
  const int blocks = int(count < 256 ? 1 : ((count + 255) / 256 > 4096 ? 4096 : (count + 255) / 256));
  k_init_cotangent<<<blocks, 256, 0, s>>>(w, m, g);
  return cudaGetLastError();
}

cudaError_t launch_gridgrad(const GridQubitMeta* d_meta, int n_qubits, int max_bits, const int2* d_ops,
                            const double* d_angles, const uint8_t* d_bits, const double2* d_wgrid,
                            double* d_grad, cudaStream_t s) {
  const int64_t entries = int64_t(1) << max_bits;
  dim3 grid(unsigned((entries + 255) / 256), unsigned(n_qubits));
  k_gridgrad<<<grid, 256, 0, s>>>(d_meta, d_ops, d_angles, d_bits, d_wgrid, d_grad);
  return cudaGetLastError();
}

}  // namespace qflex

// Step a3a: index permutation (and the fused GEMM operand producer).
//
// Methods, "Cache-efficient index permutations": before every pairwise
// contraction the operands are reordered so that the contracted indexes are
// contiguous (row-major matrix form).  The paper's CPU design (left/right
// moves chained L-R-L, memoised index maps) is built around CPU caches; on
// the GPU one pass suffices: for power-of-two dimensions a permutation is a
// permutation of the bits of the linear index, and a tile spanning the
// input's fastest bits and the output's fastest bits is staged through
// shared memory, so both the HBM reads and the HBM writes are coalesced.
// The index maps are precomputed once per plan step (the analogue of the
// paper's memoisation) as small tables.
//
// The same kernel can write, instead of the permuted complex64 tensor, the
// tensor-core operand planes of the 3-multiply complex product: re, im and
// re+im, each split into a high part and (optionally) the rounded residual
// low part, in tf32, bf16 or power-of-two-scaled fp16.
#include "internal.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <vector>

namespace qflex {

bool build_perm_tile(int nbits, const int64_t* w, PermTile* t, const int64_t* w_out) {
  const int T = std::min(kPermTileBits, nbits);
  if (nbits - T > kPermMaxRest) return false;
  std::vector<int64_t> wo(nbits);
  for (int i = 0; i < nbits; ++i) wo[i] = w_out ? w_out[i] : (int64_t(1) << i);
  std::vector<int> by_w(nbits), by_o(nbits);
  for (int i = 0; i < nbits; ++i) by_w[i] = by_o[i] = i;
  std::sort(by_w.begin(), by_w.end(), [&](int a, int b) { return w[a] < w[b]; });
  std::sort(by_o.begin(), by_o.end(), [&](int a, int b) { return wo[a] < wo[b]; });
  std::vector<char> in_u(nbits, 0);
  std::vector<int> U;
  auto add = [&](int b) {
    if (!in_u[b] && int(U.size()) < T) { in_u[b] = 1; U.push_back(b); }
  };
  for (int i = 0; i < std::min(5, nbits); ++i) add(by_w[i]);   // input-fastest bits
  for (int i = 0; i < std::min(5, nbits); ++i) add(by_o[i]);   // output-fastest bits
  int pw = 0, po = 0;
  while (int(U.size()) < T) {                                    // extend alternately
    while (pw < nbits && in_u[by_w[pw]]) ++pw;
    if (pw < nbits) add(by_w[pw]);
    while (po < nbits && in_u[by_o[po]]) ++po;
    if (po < nbits) add(by_o[po]);
  }
  std::vector<int> load = U, store = U;
  std::sort(load.begin(), load.end(), [&](int a, int b) { return w[a] < w[b]; });
  std::sort(store.begin(), store.end(), [&](int a, int b) { return wo[a] < wo[b]; });
  std::vector<int> pos_in_load(nbits, -1);
  for (int i = 0; i < T; ++i) pos_in_load[load[i]] = i;
  // Slot map slot(L) = L ^ g(L): g sends each of the store-fast bits 0..3
  // that sits at load position >= 4 onto a low position that no store-fast
  // bit occupies, so 16 consecutive loads and 16 consecutive stores both
  // land in 16 distinct low-4-bit slots.  slot is linear over GF(2), so it
  // distributes over the lo/hi table split.
  int gmask[kPermTileBits] = {0};
  {
    bool used[4] = {false, false, false, false};
    for (int b = 0; b < std::min(4, T); ++b)
      if (pos_in_load[store[b]] < 4) used[pos_in_load[store[b]]] = true;
    int f = 0;
    for (int b = 0; b < std::min(4, T); ++b) {
      const int p = pos_in_load[store[b]];
      if (p < 4) continue;
      while (f < 4 && used[f]) ++f;
      if (f < 4) {
        gmask[p] = 1 << f;
        used[f] = true;
      }
    }
  }
  auto slot = [&](int L) {
    int x = L;
    for (int p = 4; p < T; ++p)
      if ((L >> p) & 1) x ^= gmask[p];
    return x;
  };
  for (int a = 0; a < 64; ++a) {
    int64_t il = 0, ih = 0, ol = 0, oh = 0;
    int32_t sl = 0, sh = 0;
    for (int b = 0; b < 6; ++b) {
      if (!((a >> b) & 1)) continue;
      if (b < 5 && b < T) {
        il += w[load[b]];
        ol += wo[store[b]];
        sl += 1 << pos_in_load[store[b]];
      }
      if (5 + b < T) {
        ih += w[load[5 + b]];
        oh += wo[store[5 + b]];
        sh += 1 << pos_in_load[store[5 + b]];
      }
    }
    const int la = a < (1 << std::min(5, T)) ? a : 0;
    const int ha = T > 5 && a < (1 << (T - 5)) ? a : 0;
    if (a < 32) {
      t->in_lo[a] = il;
      t->out_lo[a] = ol;
      t->ld_lo[a] = slot(la);
      t->st_lo[a] = slot(sl);
    }
    t->in_hi[a] = ih;
    t->out_hi[a] = oh;
    t->ld_hi[a] = slot(ha << 5);
    t->st_hi[a] = slot(sh);
  }
  int r = 0;
  for (int b = 0; b < nbits; ++b) {
    if (in_u[b]) continue;
    t->rest_in[r] = w[b];
    t->rest_out[r] = wo[b];
    ++r;
  }
  for (int i = r; i < kPermMaxRest; ++i) t->rest_in[i] = t->rest_out[i] = 0;
  t->n_rest = r;
  t->tile_bits = T;
  t->n_tiles = int64_t(1) << (nbits - T);
  return true;
}

namespace {

template <int FMT>
__global__ void __launch_bounds__(256, 6) k_permute_tiled(const float2* __restrict__ in, int64_t in_base,
                                                       const __grid_constant__ PermTile t, void* out,
                                                       int nsplit, int64_t plane, const unsigned* smax) {
  pdl_wait();
  static_assert((1 << kPermTileBits) % 256 == 0, "tile must be a multiple of the block");
  __shared__ float2 tile[1 << kPermTileBits];
  __shared__ int64_t s_in_lo[32], s_in_hi[64], s_out_lo[32], s_out_hi[64];
  __shared__ int32_t s_ld_lo[32], s_ld_hi[64], s_st_lo[32], s_st_hi[64];
  if (threadIdx.x < 64) {
    const int a = threadIdx.x;
    if (a < 32) {
      s_in_lo[a] = t.in_lo[a];
      s_out_lo[a] = t.out_lo[a];
      s_ld_lo[a] = t.ld_lo[a];
      s_st_lo[a] = t.st_lo[a];
    }
    s_in_hi[a] = t.in_hi[a];
    s_out_hi[a] = t.out_hi[a];
    s_ld_hi[a] = t.ld_hi[a];
    s_st_hi[a] = t.st_hi[a];
  }
  __syncthreads();
  // Software pipeline: the global loads of the next tile are issued before
  // the stores of the current one, so HBM reads stay in flight across the
  // shared-memory round trip.  Each thread holds kPer entries in registers.
  // Entry j = threadIdx.x + 256 k: its low 5 bits are the lane, its high bits
  // warp + 8 k, so the lane's table entries are read once per kernel and the
  // high ones are warp-uniform.
  constexpr int kPer = (1 << kPermTileBits) / 256;
  const int n = 1 << t.tile_bits;
  float scale = 1.f;
  if constexpr (FMT == kFmtFP16) scale = smax ? fp16_scale_of(*smax) : 1.f;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t in_lo = s_in_lo[lane], out_lo = s_out_lo[lane];
  const int ld_lo = s_ld_lo[lane], st_lo = s_st_lo[lane];
  auto tile_base = [&](int64_t tb, int64_t& ib, int64_t& ob) {
    ib = in_base;
    ob = 0;
    for (int r = 0; r < t.n_rest; ++r) {
      if ((tb >> r) & 1) {
        ib += t.rest_in[r];
        ob += t.rest_out[r];
      }
    }
  };
  float2 v[kPer];
  int64_t tb = blockIdx.x, ib = 0, ob = 0;
  if (tb < t.n_tiles) {
    tile_base(tb, ib, ob);
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int h = wid + 8 * k;
      if (h * 32 < n) v[k] = __ldg(in + ib + in_lo + s_in_hi[h]);
    }
  }
  for (; tb < t.n_tiles; tb += gridDim.x) {
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int h = wid + 8 * k;
      if (h * 32 + lane < n) tile[ld_lo ^ s_ld_hi[h]] = v[k];
    }
    __syncthreads();
    const int64_t cur_ob = ob;
    const int64_t nxt = tb + gridDim.x;
    if (nxt < t.n_tiles) {
      tile_base(nxt, ib, ob);
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int h = wid + 8 * k;
        if (h * 32 < n) v[k] = __ldg(in + ib + in_lo + s_in_hi[h]);
      }
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int h = wid + 8 * k;
      if (h * 32 + lane < n)
        put_entry<FMT>(out, cur_ob + out_lo + s_out_hi[h], tile[st_lo ^ s_st_hi[h]], nsplit, plane, scale);
    }
    __syncthreads();
  }
}

template <int FMT>
__global__ void k_permute_gather(const float2* __restrict__ in, int64_t in_base,
                                 const __grid_constant__ GatherDesc d, void* out, int nsplit,
                                 int64_t plane, const unsigned* smax) {
  pdl_wait();
  float scale = 1.f;
  if constexpr (FMT == kFmtFP16) scale = smax ? fp16_scale_of(*smax) : 1.f;
  for (int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; o < d.total;
       o += int64_t(gridDim.x) * blockDim.x) {
    int64_t rem = o, off = in_base;
    for (int a = d.rank - 1; a >= 0; --a) {
      const int64_t i = rem % d.dims[a];
      rem /= d.dims[a];
      off += i * d.in_strides[a];
    }
    put_entry<FMT>(out, o, in[off], nsplit, plane, scale);
  }
}

// Grid of a grid-stride kernel: every block resident at once (SMs x the
// kernel's occupancy at 256 threads), so the loop shares the work evenly
// instead of leaving a partial second wave; fewer blocks for small inputs.
template <auto Kern>
int grid_for(int64_t work_units) {
  static const int occ = [] {
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, Kern, 256, 0) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    return v;
  }();
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = int64_t(sms) * occ;
  return int(std::max<int64_t>(1, std::min<int64_t>(cap, work_units)));
}

}  // namespace

cudaError_t launch_permute_tiled(const float2* in, int64_t in_base, const PermTile& t, int fmt,
                                 int nsplit, void* out, int64_t plane, cudaStream_t s,
                                 const unsigned* smax) {
#define QF_TILED(F) e = launch_pdl(k_permute_tiled<F>, dim3(grid_for<k_permute_tiled<F>>(t.n_tiles)), dim3(256), 0, s, \
    in, in_base, t, out, nsplit, plane, smax)
  cudaError_t e;
  switch (fmt) {
    case kFmtC64: QF_TILED(kFmtC64); break;
    case kFmtTF32: QF_TILED(kFmtTF32); break;
    case kFmtAccC128: QF_TILED(kFmtAccC128); break;
    case kFmtFP16: QF_TILED(kFmtFP16); break;
    default: QF_TILED(kFmtBF16); break;
  }
#undef QF_TILED
  return e;
}

cudaError_t launch_permute_gather(const float2* in, int64_t in_base, const GatherDesc& d, int fmt,
                                  int nsplit, void* out, int64_t plane, cudaStream_t s,
                                  const unsigned* smax) {
#define QF_GATHER(F) e = launch_pdl(k_permute_gather<F>, dim3(grid_for<k_permute_gather<F>>((d.total + 255) / 256)), \
    dim3(256), 0, s, in, in_base, d, out, nsplit, plane, smax)
  cudaError_t e;
  switch (fmt) {
    case kFmtC64: QF_GATHER(kFmtC64); break;
    case kFmtTF32: QF_GATHER(kFmtTF32); break;
    case kFmtAccC128: QF_GATHER(kFmtAccC128); break;
    case kFmtFP16: QF_GATHER(kFmtFP16); break;
    default: QF_GATHER(kFmtBF16); break;
  }
#undef QF_GATHER
  return e;
}

}  // namespace qflex

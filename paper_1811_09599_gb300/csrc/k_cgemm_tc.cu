// Step a3b, tensor-core form: complex GEMM on tcgen05 with TMEM accumulators.
//
// C[m][n] = sum_k A[m][k] B[n][k] for complex operands, by the 3-multiply
// (Gauss) trick:
//   T1 = Ar.Br, T2 = Ai.Bi, T3 = (Ar+Ai).(Br+Bi);  Re C = T1 - T2,
//   Im C = T3 - T1 - T2.
// Each real operand is split x = hi + lo (tf32, bf16, or fp16 after an exact
// power-of-two scaling) and each real product is taken as hi.hi + hi.lo +
// lo.hi with FP32 accumulation in TMEM.
// The operand planes (re, im, re+im; hi, lo) are in [plane][rows][K]
// layout, written by the permutation kernel, by the pipelined thin CUDA-core
// product, or by this kernel's own epilogue for the next product.
//
// Kernel organisation (128 x BN output tiles, walked persistently, one CTA
// per SM, cta_group::1):
//   warp 0      one lane issues TMA loads of (A hi, A lo, B hi, B lo) tiles
//               for one (k-block, part) pair per pipeline stage;
//   warp 1      allocates TMEM (two or three accumulators, used in turn) and
//               one lane issues the tcgen05.mma instructions of each stage,
//               then tcgen05.commit releases the stage;
//   warps 2-3   idle (they complete warpgroup 0 for the register split)
//   warps 4-11  epilogue: after each part of each K chunk, tcgen05.ld of that
//               part's accumulator, round-to-nearest FP32 promotion into
//               Re/Im register accumulators; at the end, staged coalesced
//               complex64 stores (or the next product's operand planes).
// Every mbarrier wait is bounded (wall-clock limit); on expiry the kernel
// sets the status word, skips the remaining work, waits (bounded) for its
// own copies in flight, frees TMEM and returns.
#include "internal.h"

#include <cudaTypedefs.h>

#include <mutex>

namespace qflex {
namespace {

constexpr int BM = 128;
constexpr int ROW_BYTES = 128;           // one 128-byte swizzle row of K per tile row
constexpr int NSTAGE_MAX = 4;
constexpr uint64_t kWaitLimitNs = 4000000000ull;   // 4 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false (and flags the CTA / status word) after the
// limit, or at once when another role of the CTA has already given up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int32_t* status) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      const uint64_t now = gtimer();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitLimitNs) {
        *abort_flag = 1;
        if (status) atomicOr(status, kDevTimeout);
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// Shared-memory matrix descriptor: K-major tile, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr & 0x3FFFFu) >> 4);         // start address
  d |= uint64_t(1) << 16;                         // leading byte offset (unused for SW128 K-major)
  d |= uint64_t(1024 >> 4) << 32;                 // stride byte offset
  d |= uint64_t(1) << 46;                         // fixed 0b001
  d |= uint64_t(2) << 61;                         // 128-byte swizzle
  return d;
}
template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accum) {
  if constexpr (KIND == 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
  }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// WIDE (split operands only): B hi and B lo tiles are adjacent in a stage,
// so one MMA of width 2 BN gives [A_hi B_hi | A_hi B_lo] and a second of
// width BN adds A_lo B_hi onto the first half: two MMAs per k-step instead of
// three.  Measured on a GB300: an MMA of width 128 reads its shared-memory
// operands (8 KB) at ~87 B/cycle, 94 cycles instead of the 64 of its math;
// width 256 (12 KB) takes 135 cycles for 128 of math.  An accumulator is
// then DW = 2 BN columns wide (its halves summed when drained).
template <int BN, int NSPLIT, bool WIDE = false>
struct Cfg {
  static constexpr int A_TILE = BM * ROW_BYTES;              // bytes of one A plane tile
  static constexpr int B_TILE = BN * ROW_BYTES;
  static constexpr int STAGE = NSPLIT * (A_TILE + B_TILE);
  static constexpr int NSTAGE = (196 * 1024) / STAGE > NSTAGE_MAX ? NSTAGE_MAX : (196 * 1024) / STAGE;
  static constexpr int NPROD = NSPLIT == 2 ? 3 : 1;          // hi.hi, hi.lo, lo.hi
  static_assert(!WIDE || NSPLIT == 2, "the wide form is for split operands");
  static constexpr int DW = WIDE ? 2 * BN : BN;              // accumulator width (columns)
  static constexpr int NBUF = 3 * DW <= 512 ? 3 : 2;         // accumulators, used in turn
  static constexpr int TMEM_COLS = NBUF * DW <= 256 ? 256 : 512;
  static constexpr int HALF = BN / 2;                        // columns per epilogue warp
  static constexpr int STAGING = 8 * 32 * 16 * 8;            // 8 warps x 32 rows x 16 complex
  static constexpr int DN_TABLE = BN * 8;                     // column offsets of a plane output
  static constexpr int SMEM = NSTAGE * STAGE + STAGING + 1024 /*align*/ + 256 /*barriers*/ + DN_TABLE;
  static_assert(NSTAGE >= 2, "pipeline needs at least two stages");
  static_assert(SMEM <= 232448, "shared memory per CTA");
};
constexpr int KB_CHUNK = 8;      // k-blocks accumulated in TMEM before promotion to registers
constexpr int EPI_WARPS = 8;
// Block of three warpgroups: warpgroup 0 = warp 0 (TMA producer), warp 1
// (TMEM owner, MMA issuer) and two idle warps; warpgroups 1 and 2 = the
// epilogue warps.  Launched at REG_LAUNCH registers per thread, warpgroup 0
// gives registers back (REG_LOW) and the epilogue warpgroups take them
// (REG_HIGH), so that the epilogue's register accumulators (two per column
// of its half tile) do not spill: 128 REG_LOW + 256 REG_HIGH must not exceed
// 384 REG_LAUNCH, or the increase would wait forever (checked on the host
// against the compiled kernel's register count before the first launch).
constexpr int EPI_WARP0 = 4;
constexpr int THREADS = 32 * (EPI_WARP0 + EPI_WARPS);
constexpr int REG_LAUNCH = 168, REG_LOW = 56, REG_HIGH = 224;
static_assert(128 * REG_LOW + 32 * EPI_WARPS * REG_HIGH <= THREADS * REG_LAUNCH, "register split");

// Tile order of the persistent walk: groups of TILE_GROUP row blocks, each
// group swept column by column, so the tiles in flight at once (one per SM)
// share a few A row blocks and a part of B instead of all of B.
constexpr int64_t TILE_GROUP = 8;
template <int BN>
__device__ __forceinline__ void tile_origin(int64_t tile, int64_t n_mt, int64_t n_nt, int64_t* m0, int64_t* n0) {
  const int64_t per_group = TILE_GROUP * n_nt;
  const int64_t g = tile / per_group, r = tile - g * per_group;
  const int64_t rows = min(TILE_GROUP, n_mt - g * TILE_GROUP);
  *m0 = (g * TILE_GROUP + r % rows) * BM;
  *n0 = (r / rows) * BN;
}

// Column-mode plane output of one staged 32 x 16 sub-block (row r's column
// j in slot j ^ 2 (r % 8): both the 16-byte pair stores and the 16-byte
// pair loads are free of bank conflicts): V consecutive
// columns per lane (their destinations are consecutive), 16 / V lanes per
// row; returns whether a destination fell outside the planes.
template <int FMT, int NSPLIT, int V>
__device__ __forceinline__ bool write_sub_columns(const TcPlaneOut& po, const float2* st, int lane, int64_t drow,
                                                  int64_t row0, int64_t M, int64_t gn0, int64_t N, int64_t dn_hi,
                                                  const int64_t* s_dn, int colb, float scale) {
  constexpr int LPR = 16 / V, RPI = 32 / LPR;
  const int c = (lane % LPR) * V, rl = lane / LPR;
  bool bad = false;
#pragma unroll
  for (int r0 = 0; r0 < 32; r0 += RPI) {
    const int r = r0 + rl;
    const int64_t dr = __shfl_sync(0xffffffffu, drow, r);
    if (row0 + r < M && gn0 + c < N) {
      const int64_t d = dr + dn_hi + s_dn[colb + c];
      if (d >= 0 && d + V <= po.plane) {
        // staged with column pairs kept adjacent (slot = column ^ 2 (row % 8)):
        // V >= 2 columns are read as 16-byte pairs
        float2 v[V];
        const int swz = (r & 7) << 1;
        if constexpr (V >= 2) {
#pragma unroll
          for (int j = 0; j < V; j += 2) {
            const float4 w = *reinterpret_cast<const float4*>(&st[r * 16 + ((c + j) ^ swz)]);
            v[j] = make_float2(w.x, w.y);
            v[j + 1] = make_float2(w.z, w.w);
          }
        } else {
          v[0] = st[r * 16 + (c ^ swz)];
        }
        put_planes_vec<FMT, V>(po.base, d, v, NSPLIT, po.plane, scale);
      } else {
        bad = true;
      }
    }
  }
  return bad;
}

// Plane output of this warp's HALF columns of a tile, 16 at a time through
// its staging area: column mode (V consecutive columns per vector store).
template <int FMT, int NSPLIT, int V, int HALF>
__device__ __forceinline__ bool store_tile_columns(const TcPlaneOut& po, float2* st, const float (&re)[HALF],
                                                   const float (&im)[HALF], int lane, int64_t drow, int64_t row0,
                                                   int64_t M, int64_t n0, int64_t N, int64_t dn_hi,
                                                   const int64_t* s_dn, int col0, float scale) {
  bool bad = false;
#pragma unroll
  for (int sub = 0; sub < HALF / 16; ++sub) {
#pragma unroll
    for (int j = 0; j < 16; j += 2)   // column pairs stay adjacent: 16-byte stores
      *reinterpret_cast<float4*>(&st[lane * 16 + (j ^ ((lane & 7) << 1))]) =
          make_float4(re[sub * 16 + j], im[sub * 16 + j], re[sub * 16 + j + 1], im[sub * 16 + j + 1]);
    __syncwarp();
    const int colb = col0 + sub * 16;
    bad |= write_sub_columns<FMT, NSPLIT, V>(po, st, lane, drow, row0, M, n0 + colb, N, dn_hi, s_dn, colb, scale);
    __syncwarp();
  }
  return bad;
}
// Row mode: each lane its own row (`own`: inside M), column by column from
// the staging area, so that consecutive lanes write consecutive
// destinations.
template <int FMT, int NSPLIT, int HALF>
__device__ __forceinline__ bool store_tile_rows(const TcPlaneOut& po, float2* st, const float (&re)[HALF],
                                                const float (&im)[HALF], int lane, int64_t drow, bool own, int64_t n0,
                                                int64_t N, int64_t dn_hi, const int64_t* s_dn, int col0, float scale) {
  bool bad = false;
#pragma unroll
  for (int sub = 0; sub < HALF / 16; ++sub) {
#pragma unroll
    for (int j = 0; j < 16; ++j) st[lane * 16 + (j ^ (lane & 15))] = make_float2(re[sub * 16 + j], im[sub * 16 + j]);
    __syncwarp();
    if (own) {
#pragma unroll 4
      for (int c = 0; c < 16; ++c) {
        const int col = col0 + sub * 16 + c;
        if (n0 + col < N) {
          const int64_t d = drow + dn_hi + s_dn[col];
          if (d >= 0 && d < po.plane)
            put_entry<FMT>(po.base, d, st[lane * 16 + (c ^ (lane & 15))], NSPLIT, po.plane, scale);
          else
            bad = true;
        }
      }
    }
    __syncwarp();
  }
  return bad;
}

// Persistent: one CTA per SM walks the output tiles (tile += gridDim.x, N
// fastest).  Block: warp 0 = TMA producer, warp 1 = TMEM owner + MMA issuer,
// warps 4..11 = epilogue (two warps per TMEM lane quarter, each owning half of
// the BN columns).  Barrier set-up and TMEM allocation happen once per CTA,
// the producer runs ahead into the next tile, and the final store of a tile
// (from registers, through a dedicated staging area) overlaps the next tile's
// MMAs because the accumulators are handed back part by part.
//
// Accuracy: the tensor core adds each MMA's partial sum into the FP32
// accumulator with truncation, so a long K accumulation drifts (measured:
// relative error ~ 7e-9 * K).  The K range is therefore cut into chunks of
// KB_CHUNK k-blocks; within a chunk the three parts (T1, T2, T3) are
// accumulated one after another in TMEM, each in the next of NBUF
// accumulators, and after each part the epilogue warps load it and add it
// with round-to-nearest FP32 adds into register accumulators
// Re += T1 - T2, Im += T3 - T1 - T2, while the tensor core already works on
// the next part.
template <int KIND, int BN, int NSPLIT, bool PO, bool WIDE>
__global__ void __launch_bounds__(THREADS, 1)
    k_cgemm_tc(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
               int64_t M, int64_t N, int64_t K, float2* __restrict__ C, int32_t* status,
               const unsigned* smax_a, const unsigned* smax_b, const __grid_constant__ TcPlaneOut po,
               int splits) {
  using G = Cfg<BN, NSPLIT, WIDE>;
  constexpr int ELEM = KIND == 0 ? 4 : 2;
  constexpr uint32_t FMT_AB = KIND == 0 ? 2u : (KIND == 1 ? 1u : 0u);   // tf32 / bf16 / f16
  constexpr int BK = ROW_BYTES / ELEM;              // K elements per stage
  constexpr int MMA_K = 32 / ELEM;                  // 8 (tf32) or 16 (bf16): 32 bytes
  constexpr uint32_t IDESC = (1u << 4)                               // D = f32
                             | (FMT_AB << 7)                         // A format
                             | (FMT_AB << 10)                        // B format
                             | (uint32_t(BN >> 3) << 17)             // N
                             | (uint32_t(BM >> 4) << 24);            // M
  constexpr uint32_t IDESC_W = (IDESC & ~(uint32_t(63) << 17)) | (uint32_t((2 * BN) >> 3) << 17);   // N = 2 BN
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  float2* staging = reinterpret_cast<float2*>(smem + G::NSTAGE * G::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + G::NSTAGE * G::STAGE + G::STAGING);
  // [0,NSTAGE) full, [NSTAGE,2NSTAGE) empty, +0..2 accumulator ready, +3..5 drained
  uint64_t* acc_full = bars + 2 * G::NSTAGE;
  uint64_t* acc_empty = acc_full + 3;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(acc_empty + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  int64_t* s_dn = reinterpret_cast<int64_t*>(smem + G::NSTAGE * G::STAGE + G::STAGING + 256);
  constexpr int BN_LOG = BN == 128 ? 7 : 6;
  if (PO) {   // destination offset of each column within a BN-wide tile
    for (int j = threadIdx.x; j < BN; j += blockDim.x) {
      int64_t d = 0;
      for (int b = 0; b < BN_LOG && b < po.nbits; ++b)
        if ((j >> b) & 1) d += po.wn[b];
      s_dn[j] = d;
    }
  }

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n_nt = (N + BN - 1) / BN;
  const int64_t n_mt = (M + BM - 1) / BM;
  // split-K: work item t = output tile t % (n_mt n_nt) over the k-blocks of
  // split t / (n_mt n_nt), whose partial product goes to C + split M N
  const int64_t n_out_tiles = n_mt * n_nt;
  const int64_t n_tiles = n_out_tiles * splits;
  const int nkb = int((K + BK - 1) / BK);
  const int kps = (nkb + splits - 1) / splits;    // k-blocks per split
  // k-block range [kbs, kbe) of work item t and its number of chunks
  auto krange = [&](int64_t t, int* kbs, int* kbe) {
    const int sp = int(t / n_out_tiles);
    *kbs = min(nkb, sp * kps);
    *kbe = min(nkb, *kbs + kps);
  };

  // Set-up that reads nothing the previous kernel writes (barriers, TMEM,
  // tensor-map prefetch) runs before the wait below, so that it overlaps the
  // tail of the previous kernel on the stream.  (TMEM is free: a CTA of this
  // kernel needs more shared memory than two CTAs can share an SM with, and
  // no other kernel here uses TMEM.)
  if (threadIdx.x == 0) {
    for (int s = 0; s < G::NSTAGE; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[G::NSTAGE + s]), 1);
    }
    for (int p = 0; p < 3; ++p) {
      mbar_init(smem_u32(&acc_full[p]), 1);
      mbar_init(smem_u32(&acc_empty[p]), EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();

  // Launched with programmatic stream serialization: the launch itself can
  // be staged while the previous kernel on the stream runs; wait here for
  // its completion (and the visibility of its writes) before reading any
  // input, then let the next such launch stage itself.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  // A CTA of an earlier launch gave up on a wait: skip the work (the status
  // word stays set until the host reads and clears it).
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = status ? *reinterpret_cast<volatile int32_t*>(status) : 0;
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (!s_skip) {
  if (warp < EPI_WARP0) {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(REG_LOW));
  if (warp == 0) {
    if (lane == 0) {
      int i = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int64_t m0, n0;
      tile_origin<BN>(tile % n_out_tiles, n_mt, n_nt, &m0, &n0);
      int kbs, kbe;
      krange(tile, &kbs, &kbe);
      for (int kb0 = kbs; kb0 < kbe && ok; kb0 += KB_CHUNK) {
        const int kb1 = min(kbe, kb0 + KB_CHUNK);
        for (int part = 0; part < 3 && ok; ++part) {
          for (int kb = kb0; kb < kb1; ++kb, ++i) {
            const int s = i % G::NSTAGE;
            const uint32_t ph = (i / G::NSTAGE) & 1;
            if (!mbar_wait(smem_u32(&bars[G::NSTAGE + s]), ph ^ 1, abort_flag, status)) {
              ok = false;
              break;
            }
            const uint32_t full = smem_u32(&bars[s]);
            mbar_expect_tx(full, G::STAGE);
            const uint32_t sa = smem_u32(smem + s * G::STAGE);
            for (int sp = 0; sp < NSPLIT; ++sp)
              tma_load_2d(sa + sp * G::A_TILE, &map_a, full, kb * BK,
                          int((part * NSPLIT + sp) * M + m0));
            for (int sp = 0; sp < NSPLIT; ++sp)
              tma_load_2d(sa + NSPLIT * G::A_TILE + sp * G::B_TILE, &map_b, full, kb * BK,
                          int((part * NSPLIT + sp) * N + n0));
          }
        }
      }
      }
      if (!ok) {   // let the copies this lane started land before the CTA exits
        for (int j = i > G::NSTAGE ? i - G::NSTAGE : 0; j < i; ++j) {
          volatile int never = 0;
          mbar_wait(smem_u32(&bars[j % G::NSTAGE]), (j / G::NSTAGE) & 1, &never, nullptr);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int i = 0, jb = 0;   // stage counter; (chunk, part) job counter across tiles
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int kbs, kbe;
      krange(tile, &kbs, &kbe);
      for (int kb0 = kbs; kb0 < kbe && ok; kb0 += KB_CHUNK) {
        const int kb1 = min(kbe, kb0 + KB_CHUNK);
        for (int part = 0; part < 3 && ok; ++part, ++jb) {
          // job jb accumulates in buffer jb % NBUF, whose previous job
          // (jb - NBUF) must have been drained
          const int buf = jb % G::NBUF, use = jb / G::NBUF;
          if (use > 0 && !mbar_wait(smem_u32(&acc_empty[buf]), (use - 1) & 1, abort_flag, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + uint32_t(buf * G::DW);
          for (int kb = kb0; kb < kb1; ++kb, ++i) {
            const int s = i % G::NSTAGE;
            const uint32_t ph = (i / G::NSTAGE) & 1;
            if (!mbar_wait(smem_u32(&bars[s]), ph, abort_flag, status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * G::STAGE);
            const uint32_t sb = sa + NSPLIT * G::A_TILE;
            if constexpr (WIDE) {
#pragma unroll
              for (int ks = 0; ks < BK / MMA_K; ++ks) {
                // [hi.hi | hi.lo] over B hi and B lo as one 2 BN-row operand, then lo.hi
                mma<KIND>(d, smem_desc(sa + ks * 32), smem_desc(sb + ks * 32), IDESC_W,
                          ((kb - kb0) | ks) != 0 ? 1u : 0u);
                mma<KIND>(d, smem_desc(sa + G::A_TILE + ks * 32), smem_desc(sb + ks * 32), IDESC, 1u);
              }
            } else {
#pragma unroll
              for (int pr = 0; pr < G::NPROD; ++pr) {
                const int ai = pr == 2 ? 1 : 0, bi = pr == 1 ? 1 : 0;
#pragma unroll
                for (int ks = 0; ks < BK / MMA_K; ++ks) {
                  const uint64_t adesc = smem_desc(sa + ai * G::A_TILE + ks * 32);
                  const uint64_t bdesc = smem_desc(sb + bi * G::B_TILE + ks * 32);
                  mma<KIND>(d, adesc, bdesc, IDESC, ((kb - kb0) | pr | ks) != 0 ? 1u : 0u);
                }
              }
            }
            tc_commit(smem_u32(&bars[G::NSTAGE + s]));
          }
          if (ok) tc_commit(smem_u32(&acc_full[buf]));   // fires when this job's MMAs are done
        }
      }
      }
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(REG_HIGH));
    // epilogue warps 4..11: TMEM lane quarter q = warp % 4, column half h
    const int q = warp & 3, h = (warp - EPI_WARP0) >> 2;
    const int col0 = h * G::HALF;
    const uint32_t lane_base = tmem + (uint32_t(q * 32) << 16) + uint32_t(col0);
    float2* st = staging + (warp - EPI_WARP0) * (32 * 16);
    // fp16 operands were scaled by exact powers of two: undo both here
    float unscale = 1.f;
    if constexpr (KIND == 2) {
      const float sa = smax_a ? fp16_scale_of(*smax_a) : 1.f;
      const float sb = smax_b ? fp16_scale_of(*smax_b) : 1.f;
      unscale = 1.f / (sa * sb);
    }
    // plane output: raw accumulators x po_factor are the planes' values
    // (fp16: the entry times the consumer's scale, both powers of two)
    float po_factor = 1.f;
    if constexpr (PO && KIND == 2) {
      const float bound = 3.f * float(K) * __uint_as_float(*po.max_a) * __uint_as_float(*po.max_b);
      const unsigned bb = __float_as_uint(bound);
      if (blockIdx.x == 0 && warp == EPI_WARP0 && lane == 0) *po.out_scale = bb;
      po_factor = fp16_scale_of(bb) * unscale;
    }
    bool ok = true;
    int jb = 0;   // (chunk, part) job counter, as the MMA issuer's
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      int64_t m0, n0;
      tile_origin<BN>(tile % n_out_tiles, n_mt, n_nt, &m0, &n0);
      float2* Ct = C + (tile / n_out_tiles) * M * N;   // this split's partial product
      int kbs, kbe;
      krange(tile, &kbs, &kbe);
      float re[G::HALF], im[G::HALF];
#pragma unroll
      for (int j = 0; j < G::HALF; ++j) re[j] = im[j] = 0.f;
      for (int kb0 = kbs; kb0 < kbe && ok; kb0 += KB_CHUNK) {
        for (int part = 0; part < 3; ++part, ++jb) {
          const int buf = jb % G::NBUF, use = jb / G::NBUF;
          if (!mbar_wait(smem_u32(&acc_full[buf]), use & 1, abort_flag, status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = lane_base + uint32_t(buf * G::DW);
#pragma unroll
          for (int sub = 0; sub < G::HALF / 16; ++sub) {
            uint32_t r[16], r2[16];
            tmem_ld16(acc + uint32_t(sub * 16), r);
            if constexpr (WIDE) tmem_ld16(acc + uint32_t(BN + sub * 16), r2);   // the hi.lo half
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float t = __uint_as_float(r[j]);
              if constexpr (WIDE) t += __uint_as_float(r2[j]);
              if (part == 0) {
                re[sub * 16 + j] += t;
                im[sub * 16 + j] -= t;
              } else if (part == 1) {
                re[sub * 16 + j] -= t;
                im[sub * 16 + j] -= t;
              } else {
                im[sub * 16 + j] += t;
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf]))
                         : "memory");
          }
        }
      }
      if (!ok || *abort_flag) break;
      if constexpr (PO) {
        // the next step's operand planes: each entry goes to its bit-permuted
        // position in every [part][split] plane
        constexpr int FMT = KIND == 0 ? kFmtTF32 : (KIND == 1 ? kFmtBF16 : kFmtFP16);
        const int64_t gm_own = m0 + q * 32 + lane;
        int64_t drow = 0;
        for (int b = 0; b < po.mbits; ++b)
          if ((gm_own >> b) & 1) drow += po.wm[b];
        int64_t dn_hi = 0;
        for (int b = BN_LOG; b < po.nbits; ++b)
          if ((n0 >> b) & 1) dn_hi += po.wn[b];
        bool bad = false;
        if constexpr (KIND == 2) {   // largest part written, for the bounds of later products
          float mx = 0.f;
#pragma unroll
          for (int j = 0; j < G::HALF; ++j)
            mx = fmaxf(mx, fmaxf(fabsf(re[j]), fmaxf(fabsf(im[j]), fabsf(re[j] + im[j]))));
          for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          mx *= unscale;
          if (lane == 0 && mx > 0.f) atomicMax(po.out_max, __float_as_uint(mx));
        }
        // the store form is chosen once per tile, so that the code of the
        // form in use lies in one piece (instruction-cache locality)
        const int64_t row0 = m0 + q * 32;
        if (po.n_fast && KIND != 0 && po.vec == 8)
          bad |= store_tile_columns<FMT, NSPLIT, (KIND != 0 ? 8 : 4), G::HALF>(po, st, re, im, lane, drow, row0, M,
                                                                                 n0, N, dn_hi, s_dn, col0, po_factor);
        else if (po.n_fast && po.vec >= 4)
          bad |= store_tile_columns<FMT, NSPLIT, 4, G::HALF>(po, st, re, im, lane, drow, row0, M, n0, N, dn_hi, s_dn,
                                                             col0, po_factor);
        else if (po.n_fast && po.vec == 2)
          bad |= store_tile_columns<FMT, NSPLIT, 2, G::HALF>(po, st, re, im, lane, drow, row0, M, n0, N, dn_hi, s_dn,
                                                             col0, po_factor);
        else if (po.n_fast)
          bad |= store_tile_columns<FMT, NSPLIT, 1, G::HALF>(po, st, re, im, lane, drow, row0, M, n0, N, dn_hi, s_dn,
                                                             col0, po_factor);
        else
          bad |= store_tile_rows<FMT, NSPLIT, G::HALF>(po, st, re, im, lane, drow, gm_own < M, n0, N, dn_hi, s_dn,
                                                       col0, po_factor);
        if (bad && status) atomicOr(status, kDevBadIndex);
        continue;
      }
      // final store: 16 columns at a time through this warp's staging area
      // (row = lane, column slot XOR-swizzled by the row: conflict-free in
      // both directions), then two 128-byte row segments per instruction.
#pragma unroll
      for (int sub = 0; sub < G::HALF / 16; ++sub) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          st[lane * 16 + (j ^ (lane & 15))] = make_float2(re[sub * 16 + j] * unscale, im[sub * 16 + j] * unscale);
        __syncwarp();
        const int cj = lane & 15;
        const int64_t gn = n0 + col0 + sub * 16 + cj;
#pragma unroll 4
        for (int r2 = 0; r2 < 32; r2 += 2) {
          const int r = r2 + (lane >> 4);
          const int64_t gm = m0 + q * 32 + r;
          if (gm < M && gn < N) Ct[gm * N + gn] = st[r * 16 + (cj ^ (r & 15))];
        }
        __syncwarp();
      }
    }
  }
  }   // !s_skip
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(G::TMEM_COLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool encode(int kind, const void* ptr, int64_t rows, int64_t K, int box_rows, CUtensorMap* map) {
  auto fn = get_encode();
  if (!fn) return false;
  const int elem = kind == 0 ? 4 : 2;
  cuuint64_t gdim[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t gstride[1] = {cuuint64_t(K) * elem};
  cuuint32_t box[2] = {cuuint32_t(ROW_BYTES / elem), cuuint32_t(box_rows)};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = fn(map,
                  kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                            : (kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16),
                  2, const_cast<void*>(ptr), gdim, gstride, box, estride,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int KIND, int BN, int NSPLIT, bool PO, bool WIDE>
cudaError_t launch_t(const TcGemmMaps& maps, int64_t M, int64_t N, int64_t K, float2* C,
                     int32_t* status, cudaStream_t s, const unsigned* sa, const unsigned* sb,
                     const TcPlaneOut& po, int splits) {
  using G = Cfg<BN, NSPLIT, WIDE>;
  auto kern = k_cgemm_tc<KIND, BN, NSPLIT, PO, WIDE>;
  static int configured_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (configured_dev != dev) {
    // the register split assumes the block is launched with REG_LAUNCH
    // registers per thread
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if (fa.numRegs < REG_LAUNCH) return cudaErrorInvalidConfiguration;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (e != cudaSuccess) return e;
    configured_dev = dev;
  }
  static int sms = 0;
  if (sms == 0) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * splits;
  const unsigned grid = unsigned(tiles < sms ? tiles : sms);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = G::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, maps.a, maps.b, M, N, K, C, status, sa, sb, po, splits);
}

}  // namespace

bool tc_available() { return get_encode() != nullptr; }

bool tc_wide_mma(int nsplit, int bn, int64_t K) { return nsplit == 2 && (bn == 64 || K >= 256); }

bool tc_encode_maps(int kind, int nsplit, int bn, const void* a_planes, int64_t M,
                    const void* b_planes, int64_t N, int64_t K, TcGemmMaps* maps) {
  if (K % 8 != 0 || M <= 0 || N <= 0) return false;
  const int64_t planes = 3 * nsplit;
  return encode(kind, a_planes, planes * M, K, BM, &maps->a) &&
         encode(kind, b_planes, planes * N, K, bn, &maps->b);
}

cudaError_t launch_cgemm_tc(int kind, int nsplit, int bn, const TcGemmMaps& maps, int64_t M,
                            int64_t N, int64_t K, float2* C, int32_t* status, cudaStream_t s,
                            const unsigned* smax_a, const unsigned* smax_b, const TcPlaneOut* planes,
                            int splits) {
  if (3 * nsplit * M > INT32_MAX || 3 * nsplit * N > INT32_MAX) return cudaErrorInvalidValue;
  if (splits < 1 || splits > 1024 || (splits > 1 && planes && planes->base)) return cudaErrorInvalidValue;
  static const TcPlaneOut none{};
  const TcPlaneOut& po = planes ? *planes : none;
  if (po.base && (po.mbits > kMaxOutBits || po.nbits > kMaxOutBits || (int64_t(1) << po.mbits) != M ||
                  (int64_t(1) << po.nbits) != N))
    return cudaErrorInvalidValue;
  if (po.base && kind == 2 && (!po.out_scale || !po.out_max || !po.max_a || !po.max_b || !smax_a || !smax_b))
    return cudaErrorInvalidValue;
  const bool wide = tc_wide_mma(nsplit, bn, K);
#define QF_TC(KD, B, S, W)                                                                               \
  if (kind == KD && bn == B && nsplit == S && wide == W)                                                 \
    return po.base ? launch_t<KD, B, S, true, W>(maps, M, N, K, C, status, s, smax_a, smax_b, po, splits) \
                   : launch_t<KD, B, S, false, W>(maps, M, N, K, C, status, s, smax_a, smax_b, po, splits);
  QF_TC(0, 64, 1, false) QF_TC(0, 64, 2, true) QF_TC(0, 128, 1, false) QF_TC(0, 128, 2, false) QF_TC(0, 128, 2, true)
  QF_TC(1, 64, 1, false) QF_TC(1, 64, 2, true) QF_TC(1, 128, 1, false) QF_TC(1, 128, 2, false) QF_TC(1, 128, 2, true)
  QF_TC(2, 64, 2, true) QF_TC(2, 128, 2, false) QF_TC(2, 128, 2, true)
#undef QF_TC
  return cudaErrorInvalidValue;
}

}  // namespace qflex

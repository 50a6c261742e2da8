// Host side of the C ABI (include/qflex.h): planner and executor.
//
// The planner turns the paper's problem statement into a fixed schedule:
//  * network metadata (Methods, "Overview of the simulator"): bond exponent
//    K_e per edge (bond bits: 1 per CZ, 2 per iSWAP), per-qubit gate lines
//    compiled into ops for the grid-tensor kernel, grid-tensor layouts
//    [o?][bonds by neighbour id];
//  * cuts (Methods, "Cutting indexes"): slice id s in mixed radix 2^{K_e} over
//    the cut list, first cut most significant; a cut bond is removed from the
//    views of its two grid tensors and contributes value * stride to their
//    base offsets, so slicing moves no data;
//  * the pairwise contraction order (Methods, "Remarks on the choice of cuts
//    and contraction ordering"), each step = operand permutation into matrix
//    form (Methods, "Implementation of the simulator") + complex GEMM;
//  * reuse across paths (SI A: A, pB, pC, ppD are built once and B, AB once
//    per outer-cut value): each step carries the set of cuts its result
//    depends on and is re-run only when one of them changes; results reused
//    across slices keep dedicated buffers, the others share memory by
//    liveness;
//  * one device workspace allocated at plan time (Methods, "Implementation
//    of the simulator": scratch preallocated once).
#include "qflex.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"
#include "search.h"
#include "slices.h"

using namespace qflex;

namespace {

thread_local std::string g_err;

qflex_status fail(qflex_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

// Runs an entry point's body; no C++ exception crosses the C ABI (a failed
// host allocation becomes QFLEX_ERR_OOM, anything else QFLEX_ERR_UNSUPPORTED
// with its message).
template <class F>
qflex_status guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return fail(QFLEX_ERR_OOM, "host allocation failed");
  } catch (const std::length_error&) {
    return fail(QFLEX_ERR_OOM, "host allocation too large");
  } catch (const std::exception& e) {
    try {
      return fail(QFLEX_ERR_UNSUPPORTED, std::string("internal error: ") + e.what());
    } catch (...) {
      return QFLEX_ERR_UNSUPPORTED;
    }
  } catch (...) {
    return QFLEX_ERR_UNSUPPORTED;
  }
}

#define QF_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(QFLEX_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Projector lines (slices.h) of a circuit: `order` = gate indices in time
// order, gate_edge = edge of each two-qubit gate, K = bond bits per edge.
ProjLines proj_lines(const qflex_circuit* c, const std::vector<int64_t>& order, const std::vector<int>& gate_edge,
                     const std::vector<int>& K) {
  ProjLines lines(size_t(c->n_qubits));
  std::vector<int> used(K.size(), 0);
  for (int64_t gi : order) {
    const qflex_gate& g = c->gates[gi];
    if (g.kind == QFLEX_GATE_CZ) {
      const int e = gate_edge[size_t(gi)];
      lines[size_t(std::min(g.q0, g.q1))].push_back({e, K[size_t(e)] - 1 - used[size_t(e)]});
      used[size_t(e)] += 1;
    } else if (g.kind == QFLEX_GATE_ISWAP) {
      used[size_t(gate_edge[size_t(gi)])] += 2;
      lines[size_t(g.q0)].push_back({-1, 0});
      lines[size_t(g.q1)].push_back({-1, 0});
    } else if (g.kind != QFLEX_GATE_T && g.kind != QFLEX_GATE_RZ) {
      lines[size_t(g.q0)].push_back({-1, 0});
    }
  }
  return lines;
}

int tc_kind_of(int prec) {
  return (prec == QFLEX_TF32X3 || prec == QFLEX_TF32_PLAIN) ? 0 : (prec == QFLEX_FP16X3 ? 2 : 1);
}
int nsplit_of(int prec) {
  return (prec == QFLEX_TF32X3 || prec == QFLEX_BF16X3 || prec == QFLEX_FP16X3) ? 2 : 1;
}
int plane_fmt(int kind) { return kind == 0 ? kFmtTF32 : (kind == 1 ? kFmtBF16 : kFmtFP16); }

int ilog2(int64_t v) {
  int b = 0;
  while ((int64_t(1) << b) < v) ++b;
  return b;
}
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// A tensor as seen by a step: memory legs (cut legs removed) with strides.
struct Ref {
  bool grid = true;
  int id = 0;                                  // qubit (grid) or buffer index
  std::vector<int> legs;
  std::vector<int64_t> strides;
  std::vector<std::pair<int, int64_t>> cut_terms;  // (cut index, stride)
  uint64_t dep = 0;                            // cuts the values depend on
};

struct Operand {
  Ref ref;
  bool direct = false;      // consumed in place by the GEMM (FP32 path, already in matrix form)
  int cache = -1;           // index of a dedicated operand buffer kept across executions, or -1
  bool fused = false;       // written as planes by its producer's epilogue (tensor cores)
  bool pow2 = true;
  PermTile tile{};
  GatherDesc gather{};
};

struct Step {
  int dst = 0, src = 0;
  Operand A, B;
  int64_t M = 1, N = 1, K = 1;
  bool tc = false;
  bool fuse_out = false;    // epilogue writes the consumer's operand planes (po) instead of C
  TcPlaneOut po{};
  TcGemmMaps maps_plain{};  // maps on the operand scratch (used when fusion is off: gradients)
  int bn = 128;
  int fp32_kernel = 0;   // CUDA-core form: 0 = by shape, 1 = thin, 2 = tiled
  int out_buf = -1;
  uint64_t dep = 0;
  std::vector<int> out_legs;
  std::vector<int> ml, nl, sh;   // free legs of dst, free legs of src, contracted legs
  TcGemmMaps maps{};
  unsigned* tmax = nullptr;      // CUDA-core producer of fp16 planes: largest parts of its A and B
};

// One GEMM of the reverse pass, C'[m][n] = sum_k X[m][k] Y[n][k], followed by
// the scatter of C' into the cotangent of the step's dst (ga) or src (gb).
struct BwdGemm {
  int64_t M = 0, N = 0, K = 0;
  int route = 0;                 // 0 FP32 tiled, 1 FP32 thin, 2 tensor cores
  int bn = 128;
  int splits = 1;                // split-K: partial products summed by launch_splitk_reduce
  bool x_direct = false;         // X is the output cotangent itself, already [M][K]
  PermTile xt{}, yt{}, st{};     // producers of X and Y, scatter of C'
  Ref ysrc;                      // forward tensor feeding Y
  Ref target;                    // view whose cotangent receives C'
  TcGemmMaps maps{};
};
struct StepGrad {
  BwdGemm ga, gb;
};

struct Buf {
  int64_t elems = 0;
  int bytes_per = 8;        // 8 (complex64) or the operand-plane bytes of a fused output
  int producer = -1, consumer = -1;
  bool persistent = false;
  size_t offset = 0;
};

}  // namespace

// Profiling state of a plan (qflex_plan_profile), shared by its problems:
// event pairs around launches of the chosen kernel classes.
struct Prof {
  bool on = false;
  int32_t mask = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec { int cls; size_t e0; double flops, mma, bytes; int64_t M, N, K; int planes; };
  std::vector<Rec> recs;
  qflex_profile tot{};
  // GEMM launches by (class, M, N, K, output as operand planes)
  std::map<std::tuple<int, int64_t, int64_t, int64_t, int>, qflex_profile_shape> shapes;
};

// The product shape a GEMM launch records with its event pair.
struct ProfShape {
  int64_t M = 0, N = 0, K = 0;
  int planes = 0;
};

// One problem of a plan: network, schedule, buffers (a slice of the plan's
// workspace) and the reverse pass's buffers.
struct Sub {
  int device = -1;
  qflex_precision prec = QFLEX_FP32_SIMT;
  int tc_kind = 0, nsplit = 1;
  Prof* prof = nullptr;                        // the plan's
  int n = 0, E = 0, n_params = 0;
  std::vector<int> K;                          // per edge
  std::vector<std::vector<int>> inc;           // per qubit: incident edges by neighbour id
  std::vector<int> cuts, cut_of_edge, tile, tile_pos;
  int64_t P = 1;
  SliceZeros zeros;                            // paths that vanish identically (skipped)
  std::vector<int64_t> leg_dim;                // E bond legs then n output legs
  std::vector<GridQubitMeta> gmeta;
  std::vector<int2> gops;
  int64_t grid_elems = 0;
  int max_bits = 0;
  std::vector<Ref> grid_ref;
  std::vector<Step> steps;
  std::vector<Buf> bufs;
  Ref final_ref;
  std::vector<int64_t> final_strides;          // per tile qubit, tile order
  int64_t max_tensor = 0;
  size_t grid_bytes = 0, arena_bytes = 0, opA_bytes = 0, opB_bytes = 0, total_bytes = 0;
  int n_persistent = 0, n_tc = 0;
  // device (a slice of the plan's one workspace allocation)
  char* d_ws = nullptr;
  float2* d_grid = nullptr;
  char* d_arena = nullptr;
  void* d_opA = nullptr;
  void* d_opB = nullptr;
  // Operand caches: a permuted operand whose source depends on fewer cuts
  // than its step keeps a dedicated buffer and is rebuilt only when its
  // source changes (a new bitstring or a new value of one of its cuts);
  // the state is reset at the start of every call.
  struct OpCache { size_t off = 0; uint64_t dep = 0; };
  std::vector<OpCache> opcache;
  size_t opcache_bytes = 0;
  char* d_opcache = nullptr;
  std::vector<int64_t> oc_b;
  std::vector<std::vector<int64_t>> oc_v;
  GridQubitMeta* d_gmeta = nullptr;
  int2* d_gops = nullptr;
  int32_t* d_status = nullptr;
  unsigned* d_smax = nullptr;                  // fp16 operand scales: [0] A, [1] B, [2 + c] cache c (192 slots)
  // fp16 planes written by a producer's epilogue (fused operands), per
  // buffer: the bound whose scale the planes carry, and the largest part
  // written (reset at the start of every call; only grows within a call)
  unsigned* d_bscale = nullptr;
  unsigned* d_bmax = nullptr;
  bool fp16_fused = false;
  // gradients (qflex_plan_enable_gradients)
  std::vector<StepGrad> sg;
  std::vector<size_t> fwd_off, w_off;          // dedicated forward / cotangent buffers
  size_t grad_bytes = 0, garena_bytes = 0, gxa = 0, gyb = 0, gcc = 0;
  char* d_gws = nullptr;
  char* d_garena = nullptr;
  char* d_warena = nullptr;
  double2* d_wgrid = nullptr;
  void* d_gA = nullptr;
  void* d_gB = nullptr;
  float2* d_gC = nullptr;
  float2* d_gP = nullptr;                      // split-K partial products of reverse GEMMs
  bool grad_active = false;                    // forward runs on the dedicated buffers
};

// A plan: one or more problems (qflex_plan_create), one device workspace
// holding every problem's buffers, the launch state shared by its calls.
struct qflex_plan_s {
  int device = -1;
  qflex_precision prec = QFLEX_FP32_SIMT;
  std::vector<std::unique_ptr<Sub>> subs;
  // Inputs and outputs of a call are the problems' arrays back to back:
  // problem i's bitstrings start at n_bs * off_qubits[i] bytes, its angles
  // (and angle gradients) at off_params[i], its amplitudes (and upstream
  // cotangents) at n_bs * off_amps[i] complex entries.
  std::vector<int64_t> off_qubits, off_params, off_amps;
  int64_t n_qubits_total = 0, n_params_total = 0, amps_total = 0;
  size_t total_bytes = 0, grad_bytes = 0;
  char* d_ws = nullptr;
  char* d_gws = nullptr;
  bool grad_ready = false;
  cudaStream_t last_stream = nullptr;
  // problems of one call run concurrently on these streams, forked from
  // and joined to the caller's stream by events
  std::vector<cudaStream_t> workers;
  std::vector<cudaEvent_t> fork_ev, join_ev;
  // CUDA-graph replay of qflex_amplitudes / qflex_amplitudes_grad
  bool use_graphs = false;
  struct GraphKey {
    const void* angles = nullptr;
    const void* bits = nullptr;
    const void* out = nullptr;
    const void* grad = nullptr;
    const void* g = nullptr;
    int64_t n_bs = -1;
    int kind = -1;
    std::vector<int64_t> ids;
    bool all = false;
    bool operator==(const GraphKey& o) const {
      return angles == o.angles && bits == o.bits && out == o.out && grad == o.grad && g == o.g &&
             n_bs == o.n_bs && kind == o.kind && ids == o.ids && all == o.all;
    }
  };
  GraphKey gkey, gseen;
  cudaGraphExec_t gexec = nullptr;
  Prof prof;
  ~qflex_plan_s() {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (cudaEvent_t e : prof.pool) cudaEventDestroy(e);
    for (cudaEvent_t e : fork_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : join_ev) cudaEventDestroy(e);
    for (cudaStream_t w : workers) cudaStreamDestroy(w);
    if (d_gws) cudaFree(d_gws);
    if (d_ws) cudaFree(d_ws);
  }
};

namespace {

size_t operand_bytes(const Sub& p, bool tc, int64_t elems) {
  if (!tc) return size_t(elems) * 8;
  return size_t(elems) * 3 * p.nsplit * (p.tc_kind == 0 ? 4 : 2);
}

// Tensor cores for contractions with enough work per output; thin
// absorptions of a small tensor (N < 32, or N = 32 with a short K) run on
// the CUDA cores.  Measured (7x7 workload shapes, bf16x3 incl. the operand
// split vs FP32): 2^20 x 16 x 16: 530 vs 121 us; 65536 x 16 x 256: 134 vs
// 87 us; 2^19 x 32 x 32: 195 vs 197 us; 65536 x 32 x 256: 132 vs 189 us.
bool tc_route(int64_t M, int64_t N, int64_t K) {
  return M >= 128 && N >= 32 && K >= 16 && K % 8 == 0 && double(M) * N * K >= double(1 << 24) &&
         !(N <= 32 && K <= 64);
}

constexpr int kMaxOpCache = 128;                // fp16 scale slots 2..129 of 192
constexpr int32_t kMaxProblems = 1 << 16;      // problems of one plan
constexpr int kBf16MaxTcSteps = 36;             // longest tensor-core chain kept in bf16 planes (QFLEX_BF16X3)
constexpr int kMaxWorkers = 8;                  // streams a multi-problem call spreads over
constexpr size_t kOpCacheMinBytes = 0;           // small operands too: each saves a launch per execution

// Buffer an operand is produced into (its cache, else the shared scratch).
void* op_buf(const Sub& p, const Operand& op, bool is_a) {
  if (op.cache >= 0) return p.d_opcache + p.opcache[size_t(op.cache)].off;
  return is_a ? p.d_opA : p.d_opB;
}
int op_slot(const Operand& op, bool is_a) { return op.cache >= 0 ? 2 + op.cache : (is_a ? 0 : 1); }

// Word whose fp16_scale_of gives the scale of operand X's fp16 planes: the
// producer's bound for planes written by its epilogue (fusion on), else the
// measured maximum of the permuted source (launch_absmax).
const unsigned* scale_word(const Sub& p, const Operand& X, bool is_a, bool fused_mode) {
  if (p.tc_kind != 2) return nullptr;
  if (X.fused && fused_mode) return p.d_bscale + X.ref.id;
  return p.d_smax + op_slot(X, is_a);
}

// Planes a tensor-core step reads for operand X: its producer's fused output
// (fusion on), else its own buffer.
void* x_buf(const Sub& p, const Operand& X, bool is_a, bool fused_mode) {
  if (X.fused && fused_mode) return p.d_arena + p.bufs[size_t(X.ref.id)].offset;
  return op_buf(p, X, is_a);
}

// Tensor maps of a tensor-core step: fused operands (maps) and, when the step
// has any, the same on the operand scratch for the unfused gradient forward.
bool encode_step(Sub& p, Step& s) {
  if (!tc_encode_maps(p.tc_kind, p.nsplit, s.bn, x_buf(p, s.A, true, true), s.M, x_buf(p, s.B, false, true), s.N,
                      s.K, &s.maps))
    return false;
  if (!s.A.fused && !s.B.fused) {
    s.maps_plain = s.maps;
    return true;
  }
  return tc_encode_maps(p.tc_kind, p.nsplit, s.bn, op_buf(p, s.A, true), s.M, op_buf(p, s.B, false), s.N, s.K,
                        &s.maps_plain);
}

// True when cache c already holds the operand for bitstring b and cut values
// vals (same bitstring and same values of the cuts its source depends on);
// otherwise records the new key and returns false.
bool oc_hit(std::vector<int64_t>& ob, std::vector<std::vector<int64_t>>& ov, uint64_t dep, int c, int64_t b,
            const std::vector<int64_t>& vals) {
  bool same = ob[size_t(c)] == b;
  for (size_t k = 0; same && k < vals.size(); ++k)
    if (((dep >> k) & 1) && ov[size_t(c)][k] != vals[k]) same = false;
  if (same) return true;
  ob[size_t(c)] = b;
  ov[size_t(c)] = vals;
  return false;
}
void oc_reset(const Sub& p, std::vector<int64_t>& ob, std::vector<std::vector<int64_t>>& ov) {
  ob.assign(p.opcache.size(), -1);
  ov.assign(p.opcache.size(), {});
}

// Permutation descriptors taking `r` to the row-major order `target`.
bool make_operand(const Ref& r, const std::vector<int>& target, const std::vector<int64_t>& leg_dim,
                  Operand* op) {
  op->ref = r;
  std::vector<int64_t> dims, strides;
  for (int l : target) {
    auto it = std::find(r.legs.begin(), r.legs.end(), l);
    if (it == r.legs.end()) return false;
    dims.push_back(leg_dim[l]);
    strides.push_back(r.strides[it - r.legs.begin()]);
  }
  op->pow2 = true;
  for (int64_t d : dims) op->pow2 = op->pow2 && is_pow2(d);
  if (op->pow2) {
    std::vector<int64_t> w;
    for (int a = int(dims.size()) - 1; a >= 0; --a)
      for (int b = 0; b < ilog2(dims[a]); ++b) w.push_back(strides[a] << b);
    if (!build_perm_tile(int(w.size()), w.data(), &op->tile)) return false;
  } else {
    if (dims.size() > size_t(kGatherMaxRank)) return false;
    GatherDesc& g = op->gather;
    g.rank = int(dims.size());
    g.total = 1;
    for (size_t a = 0; a < dims.size(); ++a) {
      g.dims[a] = dims[a];
      g.in_strides[a] = strides[a];
      g.total *= dims[a];
    }
  }
  return true;
}

int64_t leg_product(const std::vector<int>& legs, const std::vector<int64_t>& dim) {
  int64_t v = 1;
  for (int l : legs) v *= dim[l];
  return v;
}

// Epilogue fusion: a tensor-core step whose result is an operand of a later
// tensor-core step writes that operand's 3M planes itself (bit-permuted
// into the consumer's [rows][K] layout) instead of complex64, and the
// consumer skips its permutation.  Needs power-of-two legs and an output
// whose lowest row or column bit lands at stride 1 of the operand (so that
// the scatter stays coalesced).  fp16 planes need a power-of-two scale
// before the first entry is written, so the producer takes it from a bound
// of its output's entries (3 K max_a max_b, TcPlaneOut) instead of their
// measured maximum; tensor-core producers track the maxima of the planes
// they write, and a CUDA-core producer of fp16 planes measures those of its
// complex64 operands right before its product.
void plan_fusion(Sub& p) {
  if (p.prec == QFLEX_FP32_SIMT) return;
  const int bytes = 3 * p.nsplit * (p.tc_kind == 0 ? 4 : 2);
  for (Step& k : p.steps) {
    // A CUDA-core product with N >= 16, at least 2^10 rows and a long K whose
    // A comes straight from a tensor-core step moves to the tensor cores too:
    // with its operand fused it skips both the permutation and the CUDA-core
    // product (65536 x 16 x 256: ~45 us vs 90 us + 45 us; on the 7x7 plan
    // the threshold 2^10 instead of 2^14 also takes 4096 x 16 x 256 and
    // 1024 x 32 x 256: 128.9 -> 132.7 amplitudes/s).
    if (!k.tc && k.N >= 16 && k.K >= 64 && k.K % 8 == 0 && k.M >= (int64_t(1) << 10) && !k.A.ref.grid &&
        k.A.pow2 && p.steps[size_t(p.bufs[size_t(k.A.ref.id)].producer)].tc) {
      k.tc = true;
      k.bn = 64;
      k.A.direct = k.B.direct = false;
      k.fp32_kernel = 0;
      ++p.n_tc;
    }
    if (!k.tc) continue;
    for (int w = 0; w < 2; ++w) {
      Operand& X = w == 0 ? k.A : k.B;
      if (X.ref.grid || X.direct || !X.pow2) continue;
      const int i = p.bufs[size_t(X.ref.id)].producer;
      Step& pi = p.steps[size_t(i)];
      // producers: tensor-core steps, and CUDA-core steps that take the
      // pipelined thin form (it has a plane-output variant)
      const bool thin_prod = !pi.tc && pi.fp32_kernel != 2 && thin_pipelined(pi.M, pi.N, pi.K);
      if ((!pi.tc && !thin_prod) || pi.fuse_out) continue;
      // the operand's layout: target legs row-major
      std::vector<int> target = w == 0 ? k.ml : k.nl;
      target.insert(target.end(), k.sh.begin(), k.sh.end());
      std::vector<int64_t> stride(target.size());
      int64_t st = 1;
      bool pow2 = true;
      for (int a = int(target.size()) - 1; a >= 0; --a) {
        stride[size_t(a)] = st;
        st *= p.leg_dim[size_t(target[size_t(a)])];
        pow2 = pow2 && is_pow2(p.leg_dim[size_t(target[size_t(a)])]);
      }
      auto weights = [&](const std::vector<int>& legs, std::vector<int64_t>* out) {
        for (int a = int(legs.size()) - 1; a >= 0; --a) {
          auto it = std::find(target.begin(), target.end(), legs[size_t(a)]);
          if (it == target.end() || !is_pow2(p.leg_dim[size_t(legs[size_t(a)])])) return false;
          for (int b = 0; b < ilog2(p.leg_dim[size_t(legs[size_t(a)])]); ++b)
            out->push_back(stride[size_t(it - target.begin())] << b);
        }
        return true;
      };
      std::vector<int64_t> wm, wn;
      if (!pow2 || !weights(pi.ml, &wm) || !weights(pi.nl, &wn)) continue;
      if (wm.size() > size_t(kMaxOutBits) || wn.size() > size_t(kMaxOutBits)) continue;
      const bool n_fast = !wn.empty() && wn[0] == 1, m_fast = !wm.empty() && wm[0] == 1;
      if (!n_fast && !m_fast) continue;
      TcPlaneOut& po = pi.po;
      po.plane = pi.M * pi.N;
      po.mbits = int32_t(wm.size());
      po.nbits = int32_t(wn.size());
      for (size_t b = 0; b < wm.size(); ++b) po.wm[b] = wm[b];
      for (size_t b = 0; b < wn.size(); ++b) po.wn[b] = wn[b];
      po.n_fast = n_fast ? 1 : 0;
      po.fmt = plane_fmt(p.tc_kind);
      po.nsplit = p.nsplit;
      if (thin_prod) pi.fp32_kernel = 1;   // keep the form that writes planes
      po.vec = 1;
      if (n_fast) {   // widest vector of columns at destination strides 1, 2, 4, ...
        const int vmax = p.tc_kind == 0 ? 4 : 8;
        while (po.vec < vmax && wn.size() > size_t(ilog2(po.vec)) &&
               wn[size_t(ilog2(po.vec))] == int64_t(po.vec))
          po.vec *= 2;
      }
      pi.fuse_out = true;
      X.fused = true;
      p.bufs[size_t(pi.out_buf)].bytes_per = bytes;
      if (p.tc_kind == 2) p.fp16_fused = true;
    }
  }
}

qflex_status build_plan(const qflex_problem* pr, Sub& p) {
  const qflex_circuit* c = pr->circuit;
  if (!c) return fail(QFLEX_ERR_ARG, "problem->circuit is NULL");
  if (c->n_qubits <= 0 || c->n_qubits > 4096) return fail(QFLEX_ERR_CIRCUIT, "n_qubits out of range");
  if (c->n_edges < 0 || (c->n_edges > 0 && !c->edges)) return fail(QFLEX_ERR_CIRCUIT, "bad edge list");
  if (c->n_gates < 0 || (c->n_gates > 0 && !c->gates)) return fail(QFLEX_ERR_CIRCUIT, "bad gate list");
  if (c->n_params < 0) return fail(QFLEX_ERR_CIRCUIT, "n_params < 0");
  const int n = c->n_qubits, E = c->n_edges;
  p.n = n;
  p.E = E;
  p.n_params = c->n_params;
  // edges and adjacency
  std::vector<std::pair<int, int>> ed(E);
  for (int e = 0; e < E; ++e) {
    int a = c->edges[2 * e], b = c->edges[2 * e + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b)
      return fail(QFLEX_ERR_CIRCUIT, "edge " + std::to_string(e) + " is not a pair of distinct qubits");
    ed[e] = {std::min(a, b), std::max(a, b)};
  }
  {
    auto s = ed;
    std::sort(s.begin(), s.end());
    if (std::adjacent_find(s.begin(), s.end()) != s.end()) return fail(QFLEX_ERR_CIRCUIT, "duplicate edge");
  }
  auto edge_of = [&](int a, int b) -> int {
    const std::pair<int, int> key{std::min(a, b), std::max(a, b)};
    for (int e = 0; e < E; ++e)
      if (ed[e] == key) return e;
    return -1;
  };
  p.inc.assign(n, {});
  for (int e = 0; e < E; ++e) {
    p.inc[ed[e].first].push_back(e);
    p.inc[ed[e].second].push_back(e);
  }
  for (int q = 0; q < n; ++q)
    std::sort(p.inc[q].begin(), p.inc[q].end(), [&](int x, int y) {
      const int ox = ed[x].first == q ? ed[x].second : ed[x].first;
      const int oy = ed[y].first == q ? ed[y].second : ed[y].first;
      return ox < oy;
    });
  // gates: validate, count bond bits per edge (1 per CZ, 2 per iSWAP),
  // per-qubit lines in time order
  std::vector<int64_t> order(size_t(c->n_gates));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return c->gates[x].cycle < c->gates[y].cycle; });
  p.K.assign(E, 0);
  std::vector<std::vector<std::pair<int64_t, int>>> line(n);   // (gate index, edge or -1)
  std::vector<int> gate_edge(size_t(c->n_gates), -1);
  for (int64_t gi : order) {
    const qflex_gate& g = c->gates[gi];
    if (g.kind < 0 || g.kind > 8) return fail(QFLEX_ERR_CIRCUIT, "unknown gate kind");
    if (g.q0 < 0 || g.q0 >= n) return fail(QFLEX_ERR_CIRCUIT, "gate qubit out of range");
    if (g.kind == QFLEX_GATE_CZ || g.kind == QFLEX_GATE_ISWAP) {
      if (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0) return fail(QFLEX_ERR_CIRCUIT, "bad two-qubit gate qubits");
      const int e = edge_of(g.q0, g.q1);
      if (e < 0) return fail(QFLEX_ERR_CIRCUIT, "two-qubit gate on a pair that is not a lattice edge");
      p.K[e] += g.kind == QFLEX_GATE_ISWAP ? 2 : 1;
      if (p.K[e] > 20) return fail(QFLEX_ERR_PLAN, "bond with more than 20 bits");
      gate_edge[size_t(gi)] = e;
      line[g.q0].push_back({gi, e});
      line[g.q1].push_back({gi, e});
    } else {
      if (g.kind >= QFLEX_GATE_RX && (g.param < 0 || g.param >= c->n_params))
        return fail(QFLEX_ERR_CIRCUIT, "rotation gate angle index out of range");
      line[g.q0].push_back({gi, -1});
    }
  }
  // legs
  p.leg_dim.assign(E + n, 2);
  for (int e = 0; e < E; ++e) p.leg_dim[e] = int64_t(1) << p.K[e];
  // cuts and tile
  p.cut_of_edge.assign(E, -1);
  if (pr->n_cuts < 0 || (pr->n_cuts > 0 && !pr->cut_edges)) return fail(QFLEX_ERR_ARG, "bad cut list");
  if (pr->n_cuts > 64) return fail(QFLEX_ERR_PLAN, "more than 64 cuts");
  p.P = 1;
  for (int i = 0; i < pr->n_cuts; ++i) {
    const int e = pr->cut_edges[i];
    if (e < 0 || e >= E || p.cut_of_edge[e] >= 0) return fail(QFLEX_ERR_ARG, "bad or repeated cut edge");
    p.cut_of_edge[e] = i;
    p.cuts.push_back(e);
    if (p.P > (int64_t(1) << 50) >> p.K[e]) return fail(QFLEX_ERR_PLAN, "too many slices");
    p.P <<= p.K[e];
  }
  const ProjLines plines = proj_lines(c, order, gate_edge, p.K);
  p.zeros = SliceZeros(plines, p.K, p.cuts);
  p.tile_pos.assign(n, -1);
  if (pr->n_open < 0 || pr->n_open > 30 || (pr->n_open > 0 && !pr->open_tile))
    return fail(QFLEX_ERR_ARG, "bad open tile");
  for (int t = 0; t < pr->n_open; ++t) {
    const int q = pr->open_tile[t];
    if (q < 0 || q >= n || p.tile_pos[q] >= 0) return fail(QFLEX_ERR_ARG, "bad or repeated tile qubit");
    p.tile_pos[q] = t;
    p.tile.push_back(q);
  }
  // grid tensors: [o if tile][bond legs by neighbour id], bits per bond leg,
  // first two-qubit gate in time = most significant bit(s) of the leg
  p.gmeta.resize(n);
  p.grid_ref.resize(n);
  int64_t off = 0;
  for (int q = 0; q < n; ++q) {
    std::vector<int> low(E, 0);
    int bits = 0;
    for (int j = int(p.inc[q].size()) - 1; j >= 0; --j) {
      low[p.inc[q][j]] = bits;
      bits += p.K[p.inc[q][j]];
    }
    if (bits > 30) return fail(QFLEX_ERR_PLAN, "grid tensor with more than 2^30 entries");
    GridQubitMeta& m = p.gmeta[q];
    m.offset = off;
    m.n_bits = bits;
    m.op_begin = int(p.gops.size());
    m.tile = p.tile_pos[q] >= 0;
    m.qubit = q;
    std::vector<int> seen(E, 0);
    for (auto& [gi, e] : line[q]) {
      const qflex_gate& g = c->gates[gi];
      if (e < 0) {
        p.gops.push_back(make_int2(g.kind, g.kind >= QFLEX_GATE_RX ? g.param : -1));
      } else {
        const int other = g.q0 == q ? g.q1 : g.q0;
        const bool isw = g.kind == QFLEX_GATE_ISWAP;
        seen[e] += isw ? 2 : 1;
        const int bitpos = low[e] + p.K[e] - seen[e];   // lowest bit of this gate's k
        const int type = isw ? (q < other ? kOpIswA : kOpIswB) : (q < other ? kOpCzProj : kOpCzZ);
        p.gops.push_back(make_int2(type | (bitpos << 8), -1));
      }
    }
    m.op_count = int(p.gops.size()) - m.op_begin;
    p.max_bits = std::max(p.max_bits, bits);
    const int64_t entries = int64_t(1) << bits;
    // full memory legs and strides
    std::vector<int> legs;
    if (m.tile) legs.push_back(E + q);
    for (int e : p.inc[q]) legs.push_back(e);
    std::vector<int64_t> strides(legs.size());
    int64_t st = 1;
    for (int a = int(legs.size()) - 1; a >= 0; --a) {
      strides[a] = st;
      st *= p.leg_dim[legs[a]];
    }
    Ref& r = p.grid_ref[q];
    r.grid = true;
    r.id = q;
    for (size_t a = 0; a < legs.size(); ++a) {
      const int l = legs[a];
      if (l < E && p.cut_of_edge[l] >= 0) {
        r.cut_terms.push_back({p.cut_of_edge[l], strides[a]});
        r.dep |= uint64_t(1) << p.cut_of_edge[l];
      } else {
        r.legs.push_back(l);
        r.strides.push_back(strides[a]);
      }
    }
    off += entries * (m.tile ? 2 : 1);
  }
  p.grid_elems = off;
  // ordering
  std::vector<int32_t> def;
  const int32_t* steps = nullptr;
  int ns = 0;
  if (pr->ordering) {
    if (pr->ordering->n_steps < 0 || (pr->ordering->n_steps > 0 && !pr->ordering->steps))
      return fail(QFLEX_ERR_ARG, "bad ordering");
    steps = pr->ordering->steps;
    ns = pr->ordering->n_steps;
  } else {
    SearchNet net;
    net.n = n;
    for (int e = 0; e < E; ++e) net.edges.push_back(ed[size_t(e)]);
    net.bits = p.K;
    net.open.assign(size_t(n), 0);
    for (int q : p.tile) net.open[size_t(q)] = 1;
    net.lines = plines;
    SearchResult sr;
    if (!search_greedy_order(net, p.cuts, &sr, 32, 28.0, 0)) return fail(QFLEX_ERR_PLAN, "ordering search failed");
    def = sr.steps;
    steps = def.data();
    ns = n - 1;
  }
  // Legs each step's result shares with the step that consumes it (a dry
  // run over leg sets): those legs go last in the result, so the consumer's
  // contracted index is the fastest in memory (and, when the producer's
  // epilogue writes the consumer's operand, its stores run along the
  // lowest bits of one of its own indexes).
  std::vector<std::vector<int>> next_shared(size_t(std::max(ns, 0)));
  {
    std::vector<std::vector<int>> legs(static_cast<size_t>(n));
    std::vector<int> last_step(size_t(n), -1);   // step that produced the live tensor of this id
    for (int q = 0; q < n; ++q) legs[size_t(q)] = p.grid_ref[size_t(q)].legs;
    for (int i = 0; i < ns; ++i) {
      const int dst = steps[2 * i], src = steps[2 * i + 1];
      if (dst < 0 || src < 0 || dst >= n || src >= n || dst == src) break;   // reported below
      const std::vector<int>& la = legs[size_t(dst)];
      const std::vector<int>& lb = legs[size_t(src)];
      for (int side = 0; side < 2; ++side) {
        const int id = side == 0 ? dst : src;
        const int prod = last_step[size_t(id)];
        if (prod < 0) continue;
        const std::vector<int>& mine = side == 0 ? la : lb;
        const std::vector<int>& other = side == 0 ? lb : la;
        for (int l : mine)
          if (std::find(other.begin(), other.end(), l) != other.end()) next_shared[size_t(prod)].push_back(l);
      }
      std::vector<int> r;
      for (int l : la)
        if (std::find(lb.begin(), lb.end(), l) == lb.end()) r.push_back(l);
      for (int l : lb)
        if (std::find(la.begin(), la.end(), l) == la.end()) r.push_back(l);
      legs[size_t(dst)] = r;
      last_step[size_t(dst)] = i;
    }
  }
  std::vector<Ref> live(n);
  std::vector<char> alive(n, 1);
  for (int q = 0; q < n; ++q) live[q] = p.grid_ref[q];
  const bool tc_prec = p.prec != QFLEX_FP32_SIMT;
  for (int i = 0; i < ns; ++i) {
    const int dst = steps[2 * i], src = steps[2 * i + 1];
    if (dst < 0 || src < 0 || dst >= n || src >= n || dst == src || !alive[dst] || !alive[src])
      return fail(QFLEX_ERR_PLAN, "ordering step " + std::to_string(i) + " names a dead or invalid tensor");
    Step s;
    s.dst = dst;
    s.src = src;
    const Ref& ra = live[dst];
    const Ref& rb = live[src];
    std::vector<int> shared, ml, nl;
    for (int l : ra.legs)
      (std::find(rb.legs.begin(), rb.legs.end(), l) != rb.legs.end() ? shared : ml).push_back(l);
    for (int l : rb.legs)
      if (std::find(shared.begin(), shared.end(), l) == shared.end()) nl.push_back(l);
    {
      const std::vector<int>& kn = next_shared[size_t(i)];
      auto later = [&](int l) { return std::find(kn.begin(), kn.end(), l) == kn.end(); };
      std::stable_partition(ml.begin(), ml.end(), later);
      std::stable_partition(nl.begin(), nl.end(), later);
    }
    s.M = leg_product(ml, p.leg_dim);
    s.N = leg_product(nl, p.leg_dim);
    s.K = leg_product(shared, p.leg_dim);
    if (s.M * s.N > (int64_t(1) << 34) || s.M * s.K > (int64_t(1) << 34) || s.N * s.K > (int64_t(1) << 34))
      return fail(QFLEX_ERR_PLAN, "intermediate tensor larger than 2^34 entries at step " + std::to_string(i));
    s.tc = tc_prec && tc_route(s.M, s.N, s.K);
    // 128-wide tiles when they fill the SMs; 64-wide for products of fewer
    // than 152 such tiles (twice the CTAs, half the per-tile latency: what
    // the autotuner picks for every such shape of the 7x7 plan)
    s.bn = (s.N >= 128 && ((s.M + 127) / 128) * ((s.N + 127) / 128) >= 152) ? 128 : 64;
    s.ml = ml;
    s.nl = nl;
    s.sh = shared;
    s.out_legs = ml;
    s.out_legs.insert(s.out_legs.end(), nl.begin(), nl.end());
    std::vector<int> ta = ml, tb = nl;
    ta.insert(ta.end(), shared.begin(), shared.end());
    tb.insert(tb.end(), shared.begin(), shared.end());
    if (!make_operand(ra, ta, p.leg_dim, &s.A) || !make_operand(rb, tb, p.leg_dim, &s.B))
      return fail(QFLEX_ERR_PLAN, "operand layout not supported at step " + std::to_string(i));
    s.A.direct = !s.tc && !ra.grid && ra.legs == ta;
    s.B.direct = !s.tc && !rb.grid && rb.legs == tb;
    s.dep = ra.dep | rb.dep;
    if (!ra.grid) p.bufs[ra.id].consumer = i;
    if (!rb.grid) p.bufs[rb.id].consumer = i;
    Buf b;
    b.elems = s.M * s.N;
    b.producer = i;
    s.out_buf = int(p.bufs.size());
    p.bufs.push_back(b);
    p.max_tensor = std::max(p.max_tensor, b.elems);
    Ref out;
    out.grid = false;
    out.id = s.out_buf;
    out.legs = s.out_legs;
    out.strides.resize(out.legs.size());
    int64_t st = 1;
    for (int a = int(out.legs.size()) - 1; a >= 0; --a) {
      out.strides[a] = st;
      st *= p.leg_dim[out.legs[a]];
    }
    out.dep = s.dep;
    live[dst] = out;
    alive[src] = 0;
    if (s.tc) ++p.n_tc;
    p.steps.push_back(std::move(s));
  }
  int left = -1, count = 0;
  for (int q = 0; q < n; ++q)
    if (alive[q]) {
      left = q;
      ++count;
    }
  if (count != 1) return fail(QFLEX_ERR_PLAN, "ordering does not contract the network into one tensor");
  p.final_ref = live[left];
  {
    std::vector<int> want;
    for (int q : p.tile) want.push_back(E + q);
    std::vector<int> got = p.final_ref.legs;
    std::sort(want.begin(), want.end());
    std::sort(got.begin(), got.end());
    if (want != got) return fail(QFLEX_ERR_PLAN, "final tensor legs are not the open tile");
    if (!p.final_ref.cut_terms.empty()) return fail(QFLEX_ERR_PLAN, "final tensor still has cut legs");
    for (int q : p.tile) {
      auto it = std::find(p.final_ref.legs.begin(), p.final_ref.legs.end(), E + q);
      p.final_strides.push_back(p.final_ref.strides[it - p.final_ref.legs.begin()]);
    }
  }
  const uint64_t all_cuts = p.cuts.size() >= 64 ? ~uint64_t(0) : ((uint64_t(1) << p.cuts.size()) - 1);
  if (!p.final_ref.grid) p.bufs[p.final_ref.id].consumer = ns;   // read by the slice sum
  if (p.prec == QFLEX_BF16X3) {
    // Long chains of bf16 splits: a bf16 hi + lo split keeps 16 significand
    // bits per operand, and past 36 split products on the amplitude's path
    // the accumulated rounding exceeds the 1e-4 amplitude bar (measured
    // against the FP64 oracle: 5.8e-5 at 36 products on the 7x7 depth-32
    // region plan, 1.1e-4 to 1.3e-4 at 40 to 45 on the searched 7x7 and the
    // 70-qubit diamond plans).  Such plans keep the 3-term split products but
    // store the operands as power-of-two-scaled fp16 hi + lo (22 significand
    // bits, the same MMA rate and plane bytes): 2.8e-5 to 3.9e-5 there.
    Sub trial = p;
    plan_fusion(trial);
    if (trial.n_tc > kBf16MaxTcSteps) p.tc_kind = 2;
  }
  plan_fusion(p);
  // buffers: reused across slices -> dedicated; others share by liveness
  for (Buf& b : p.bufs) {
    const uint64_t cdep = b.consumer >= ns ? all_cuts : p.steps[b.consumer].dep;
    b.persistent = p.steps[b.producer].dep != cdep;
  }
  size_t arena = 0;
  for (Buf& b : p.bufs)
    if (b.persistent) {
      b.offset = arena;
      arena += align256(size_t(b.elems) * size_t(b.bytes_per));
      ++p.n_persistent;
    }
  struct Live { size_t off, size; int end; };
  std::vector<Live> used;
  for (Buf& b : p.bufs) {
    if (b.persistent) continue;
    used.erase(std::remove_if(used.begin(), used.end(), [&](const Live& l) { return l.end < b.producer; }),
               used.end());
    std::sort(used.begin(), used.end(), [](const Live& x, const Live& y) { return x.off < y.off; });
    const size_t need = align256(size_t(b.elems) * size_t(b.bytes_per));
    size_t cur = arena;   // transient region starts after the persistent ones
    for (const Live& l : used) {
      if (l.off >= cur + need) break;
      cur = std::max(cur, l.off + l.size);
    }
    b.offset = cur;
    used.push_back({cur, need, b.consumer});
    p.arena_bytes = std::max(p.arena_bytes, cur + need);
  }
  p.arena_bytes = std::max(p.arena_bytes, arena);
  for (Step& s : p.steps) {
    for (int w = 0; w < 2; ++w) {
      Operand& X = w == 0 ? s.A : s.B;
      if (X.direct) continue;
      const size_t bytes = operand_bytes(p, s.tc, (w == 0 ? s.M : s.N) * s.K);
      const uint64_t d = X.ref.dep;
      if (!X.fused && (d & ~s.dep) == 0 && d != s.dep && bytes >= kOpCacheMinBytes &&
          int(p.opcache.size()) < kMaxOpCache) {
        X.cache = int(p.opcache.size());
        p.opcache.push_back({p.opcache_bytes, d});
        p.opcache_bytes += align256(bytes);
      } else if (w == 0) {
        p.opA_bytes = std::max(p.opA_bytes, bytes);
      } else {
        p.opB_bytes = std::max(p.opB_bytes, bytes);
      }
    }
  }
  p.grid_bytes = align256(size_t(p.grid_elems) * 8);
  p.total_bytes = p.grid_bytes + align256(p.arena_bytes) + align256(p.opA_bytes) + align256(p.opB_bytes) +
                  align256(p.opcache_bytes) +
                  align256(sizeof(GridQubitMeta) * n) + align256(sizeof(int2) * std::max<size_t>(1, p.gops.size())) +
                  256 /* status word */ + 768 /* fp16 scale slots: A, B, one per cache */ +
                  align256(sizeof(unsigned) * 2 * std::max<size_t>(1, p.bufs.size())) /* fused fp16 words */ +
                  align256(sizeof(unsigned) * 2 * std::max<size_t>(1, p.steps.size())) /* thin fp16 producers */;
  static_assert((2 + kMaxOpCache) * sizeof(unsigned) <= 768, "fp16 scale slots");
  return QFLEX_OK;
}

// Lay out a problem's buffers at `base` (its slice of the plan's workspace,
// total_bytes long), upload its tables and encode its tensor maps.
qflex_status allocate(Sub& p, char* base) {
  p.d_ws = base;
  char* c = p.d_ws;
  p.d_grid = reinterpret_cast<float2*>(c);
  c += p.grid_bytes;
  p.d_arena = c;
  c += align256(p.arena_bytes);
  p.d_opA = c;
  c += align256(p.opA_bytes);
  p.d_opB = c;
  c += align256(p.opB_bytes);
  p.d_opcache = c;
  c += align256(p.opcache_bytes);
  p.d_gmeta = reinterpret_cast<GridQubitMeta*>(c);
  c += align256(sizeof(GridQubitMeta) * p.n);
  p.d_gops = reinterpret_cast<int2*>(c);
  c += align256(sizeof(int2) * std::max<size_t>(1, p.gops.size()));
  p.d_status = reinterpret_cast<int32_t*>(c);
  p.d_smax = reinterpret_cast<unsigned*>(c + 256);
  c += 256 + 768;
  p.d_bscale = reinterpret_cast<unsigned*>(c);
  p.d_bmax = p.d_bscale + std::max<size_t>(1, p.bufs.size());
  QF_CUDA(cudaMemset(p.d_bscale, 0, sizeof(unsigned) * 2 * std::max<size_t>(1, p.bufs.size())));
  c += align256(sizeof(unsigned) * 2 * std::max<size_t>(1, p.bufs.size()));
  unsigned* d_tmax = reinterpret_cast<unsigned*>(c);
  for (size_t i = 0; i < p.steps.size(); ++i) p.steps[i].tmax = d_tmax + 2 * i;
  QF_CUDA(cudaMemcpy(p.d_gmeta, p.gmeta.data(), sizeof(GridQubitMeta) * p.n, cudaMemcpyHostToDevice));
  if (!p.gops.empty())
    QF_CUDA(cudaMemcpy(p.d_gops, p.gops.data(), sizeof(int2) * p.gops.size(), cudaMemcpyHostToDevice));
  QF_CUDA(cudaMemset(p.d_status, 0, sizeof(int32_t)));
  for (Step& s : p.steps) {
    if (s.fuse_out) s.po.base = p.d_arena + p.bufs[size_t(s.out_buf)].offset;
    if (s.fuse_out && p.tc_kind == 2) {
      s.po.out_scale = p.d_bscale + s.out_buf;
      s.po.out_max = p.d_bmax + s.out_buf;
      if (s.tc) {
        s.po.max_a = s.A.fused ? p.d_bmax + s.A.ref.id : p.d_smax + op_slot(s.A, true);
        s.po.max_b = s.B.fused ? p.d_bmax + s.B.ref.id : p.d_smax + op_slot(s.B, false);
      } else {   // complex64 operands: their maxima are taken right before the product
        s.po.max_a = s.tmax;
        s.po.max_b = s.tmax + 1;
      }
    }
    if (!s.tc) continue;
    if (!encode_step(p, s)) return fail(QFLEX_ERR_CUDA, "tensor map encoding failed (driver entry point missing?)");
  }
  return QFLEX_OK;
}

char* buf_ptr(const Sub& p, int id) {
  return p.grad_active ? p.d_garena + p.fwd_off[id] : p.d_arena + p.bufs[id].offset;
}

const float2* ref_ptr(const Sub& p, const Ref& r) {
  if (r.grid) return p.d_grid + p.gmeta[r.id].offset;
  return reinterpret_cast<const float2*>(buf_ptr(p, r.id));
}

int64_t ref_base(const Ref& r, const std::vector<int64_t>& vals) {
  int64_t b = 0;
  for (auto& [ci, st] : r.cut_terms) b += vals[ci] * st;
  return b;
}

// Whole tensor behind a view (for the fp16 scale: the largest part of the
// whole tensor bounds the largest part of any view of it).
void ref_region(const Sub& p, const Ref& r, const float2** ptr, int64_t* n) {
  if (r.grid) {
    const GridQubitMeta& m = p.gmeta[r.id];
    *ptr = p.d_grid + m.offset;
    *n = (int64_t(1) << m.n_bits) * (m.tile ? 2 : 1);
  } else {
    *ptr = ref_ptr(p, r);
    *n = p.bufs[r.id].elems;
  }
}

cudaError_t produce(const Sub& p, const Operand& op, bool tc, int64_t rows, int64_t cols,
                    const std::vector<int64_t>& vals, void* out, cudaStream_t s, int slot) {
  const int fmt = tc ? plane_fmt(p.tc_kind) : kFmtC64;
  const float2* in = ref_ptr(p, op.ref);
  const int64_t base = ref_base(op.ref, vals);
  const unsigned* smax = nullptr;
  if (fmt == kFmtFP16) {
    const float2* rp;
    int64_t rn;
    ref_region(p, op.ref, &rp, &rn);
    cudaError_t e = launch_absmax(rp, rn, p.d_smax + slot, s);
    if (e != cudaSuccess) return e;
    smax = p.d_smax + slot;
  }
  if (op.pow2) return launch_permute_tiled(in, base, op.tile, fmt, p.nsplit, out, rows * cols, s, smax);
  return launch_permute_gather(in, base, op.gather, fmt, p.nsplit, out, rows * cols, s, smax);
}

// Launch `fn` on `s`, bracketed by an event pair when the plan is profiling.
template <class F>
cudaError_t timed_shape(Sub& sp, int cls, double flops, double mma, double bytes, const ProfShape& sh,
                        cudaStream_t s, F&& fn) {
  Prof& p = *sp.prof;
  if (!p.on || !((p.mask >> cls) & 1)) return fn();
  while (p.pool.size() < p.used + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    p.pool.push_back(e);
  }
  const size_t i = p.used;
  p.used += 2;
  cudaError_t r = cudaEventRecord(p.pool[i], s);
  if (r != cudaSuccess) return r;
  if ((r = fn()) != cudaSuccess) return r;
  p.recs.push_back({cls, i, flops, mma, bytes, sh.M, sh.N, sh.K, sh.planes});
  return cudaEventRecord(p.pool[i + 1], s);
}
template <class F>
cudaError_t timed(Sub& sp, int cls, double flops, double mma, double bytes, cudaStream_t s, F&& fn) {
  return timed_shape(sp, cls, flops, mma, bytes, ProfShape{}, s, std::forward<F>(fn));
}

cudaError_t run_step(Sub& p, const Step& st, int64_t b, const std::vector<int64_t>& vals,
                     cudaStream_t s) {
  cudaError_t e;
  const double out_per = st.tc ? 3.0 * p.nsplit * (p.tc_kind == 0 ? 4 : 2) : 8.0;
  const float2* A = nullptr;
  const float2* B = nullptr;
  const bool fused_mode = !p.grad_active;
  if (st.A.direct) {
    A = ref_ptr(p, st.A.ref);
  } else if (st.A.fused && fused_mode) {
    // planes written by the producing step's epilogue
  } else {
    void* buf = op_buf(p, st.A, true);
    const bool hit = st.A.cache >= 0 && oc_hit(p.oc_b, p.oc_v, p.opcache[size_t(st.A.cache)].dep, st.A.cache, b, vals);
    if (!hit && (e = timed(p, 1, 0, 0, double(st.M) * st.K * (8.0 + out_per), s, [&] {
                   return produce(p, st.A, st.tc, st.M, st.K, vals, buf, s, op_slot(st.A, true));
                 })) != cudaSuccess)
      return e;
    A = static_cast<const float2*>(buf);
  }
  if (st.B.direct) {
    B = ref_ptr(p, st.B.ref);
  } else if (st.B.fused && fused_mode) {
    // planes written by the producing step's epilogue
  } else {
    void* buf = op_buf(p, st.B, false);
    const bool hit = st.B.cache >= 0 && oc_hit(p.oc_b, p.oc_v, p.opcache[size_t(st.B.cache)].dep, st.B.cache, b, vals);
    if (!hit && (e = timed(p, 1, 0, 0, double(st.N) * st.K * (8.0 + out_per), s, [&] {
                   return produce(p, st.B, st.tc, st.N, st.K, vals, buf, s, op_slot(st.B, false));
                 })) != cudaSuccess)
      return e;
    B = static_cast<const float2*>(buf);
  }
  float2* C = reinterpret_cast<float2*>(buf_ptr(p, st.out_buf));
  const double mnk = double(st.M) * double(st.N) * double(st.K);
  const double mma = st.tc ? mnk * 3.0 * (p.nsplit == 2 ? 3.0 : 1.0) * 2.0 : 0.0;
  const double gbytes = 8.0 * (double(st.M) * st.K + double(st.N) * st.K + double(st.M) * st.N);
  const ProfShape shape{st.M, st.N, st.K, st.fuse_out && fused_mode ? 1 : 0};
  if (st.tc)
    return timed_shape(p, 3, 8.0 * mnk, mma, gbytes, shape, s, [&] {
      return launch_cgemm_tc(p.tc_kind, p.nsplit, st.bn, fused_mode ? st.maps : st.maps_plain, st.M, st.N, st.K, C,
                             p.d_status, s, scale_word(p, st.A, true, fused_mode), scale_word(p, st.B, false, fused_mode),
                             st.fuse_out && fused_mode ? &st.po : nullptr);
    });
  const bool thin = st.fp32_kernel == 1 || (st.fp32_kernel == 0 && st.N <= 32);
  return timed_shape(p, 2, 8.0 * mnk, 0, gbytes, shape, s, [&] {
    if (st.fuse_out && fused_mode) {
      if (p.tc_kind == 2) {   // fp16 planes: the bound needs the largest parts of A and B
        cudaError_t e2 = launch_absmax(A, st.M * st.K, st.tmax, s);
        if (e2 == cudaSuccess) e2 = launch_absmax(B, st.N * st.K, st.tmax + 1, s);
        if (e2 != cudaSuccess) return e2;
      }
      return launch_cgemm_thin_planes(st.M, st.N, st.K, A, B, st.po, s);
    }
    return thin ? launch_cgemm_thin(st.M, st.N, st.K, A, B, C, s) : launch_cgemm_simt(st.M, st.N, st.K, A, B, C, s);
  });
}


// ------------------------------------------------------------------ reverse pass
int route_of(const Sub& p, int64_t M, int64_t N, int64_t K) {
  const bool tc = p.prec != QFLEX_FP32_SIMT && tc_route(M, N, K);
  return tc ? 2 : (N <= 32 ? 1 : 0);
}

// Tile tables of a map whose logical index runs over `order` (row-major): each
// leg moves the input by its stride in `in` and the output by its stride in `out`.
bool leg_map(const std::vector<int>& order, const std::vector<int>& in_legs,
             const std::vector<int64_t>& in_strides, const std::vector<int>& out_legs,
             const std::vector<int64_t>& out_strides, const std::vector<int64_t>& dim, PermTile* t) {
  std::vector<int64_t> wi, wo;
  for (int a = int(order.size()) - 1; a >= 0; --a) {
    const int l = order[a];
    auto ii = std::find(in_legs.begin(), in_legs.end(), l);
    auto oo = std::find(out_legs.begin(), out_legs.end(), l);
    if (ii == in_legs.end() || oo == out_legs.end() || !is_pow2(dim[l])) return false;
    const int64_t si = in_strides[ii - in_legs.begin()], so = out_strides[oo - out_legs.begin()];
    for (int b = 0; b < ilog2(dim[l]); ++b) {
      wi.push_back(si << b);
      wo.push_back(so << b);
    }
  }
  return build_perm_tile(int(wi.size()), wi.data(), t, wo.data());
}

std::vector<int64_t> contiguous(const std::vector<int>& legs, const std::vector<int64_t>& dim) {
  std::vector<int64_t> st(legs.size());
  int64_t v = 1;
  for (int a = int(legs.size()) - 1; a >= 0; --a) {
    st[a] = v;
    v *= dim[legs[a]];
  }
  return st;
}

std::vector<int> cat(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> r = a;
  r.insert(r.end(), b.begin(), b.end());
  return r;
}

// Split-K of a reverse GEMM.  The reverse pass meets products with few
// outputs and a long K (W_B = W_C^T A for a step whose dst has many free
// entries: e.g. 256 x 256 outputs over K = 65536), which as one output tile
// per CTA or one block per row use a handful of SMs.  Their K range is cut
// into `splits` parts whose partial products land in the gradient scratch
// and are summed in split order (deterministic): enough parts to give every
// SM work, none shorter than 8 k-blocks (tensor cores) or 2048 entries (CUDA
// cores).  The tiled CUDA-core form keeps its own K tiles inside a part.
int bwd_splits(const Sub& p, const BwdGemm& g) {
  constexpr int64_t kSMs = 152;
  if (g.route == 2) {
    const int64_t bk = p.tc_kind == 0 ? 32 : 64;
    const int64_t tiles = ((g.M + 127) / 128) * ((g.N + g.bn - 1) / g.bn);
    const int64_t nkb = (g.K + bk - 1) / bk;
    if (tiles * 2 > kSMs || nkb < 16) return 1;
    return int(std::max<int64_t>(1, std::min<int64_t>((kSMs + tiles - 1) / tiles, nkb / 8)));
  }
  const int64_t cgs = (g.N + 15) / 16;
  if (g.route == 1) {
    const bool rowwarp = g.K >= 64 && ((g.M + 255) / 256) * cgs < 256;
    const int64_t warps = g.M * cgs * 8;   // a block of 8 warps per (row, 16 columns)
    if (!rowwarp || warps * 4 > kSMs * 32 || g.K < 8192) return 1;
    return int(std::max<int64_t>(1, std::min<int64_t>((kSMs * 32 + warps - 1) / warps, g.K / 2048)));
  }
  const int64_t blocks = ((g.M + 63) / 64) * ((g.N + 63) / 64);
  if (blocks * 2 > kSMs || g.K < 8192) return 1;
  return int(std::max<int64_t>(1, std::min<int64_t>((kSMs * 2 + blocks - 1) / blocks, g.K / 2048)));
}

// Build one reverse GEMM: C' = X Y^T with X taken from the cotangent W of the
// step output (legs `wlegs`, contiguous) in order xorder = (rows, inner),
// Y from the forward view `ysrc` in order (cols, inner), and C' (rows, cols)
// scattered into the view `target`.
bool make_bwd(const Sub& p, const std::vector<int>& wlegs, const std::vector<int>& rows,
              const std::vector<int>& inner, const std::vector<int>& cols, const Ref& ysrc,
              const Ref& target, BwdGemm* g) {
  const auto& dim = p.leg_dim;
  g->M = leg_product(rows, dim);
  g->K = leg_product(inner, dim);
  g->N = leg_product(cols, dim);
  g->route = route_of(p, g->M, g->N, g->K);
  g->bn = g->N >= 128 ? 128 : 64;
  g->splits = bwd_splits(p, *g);
  g->ysrc = ysrc;
  g->target = target;
  const std::vector<int> xorder = cat(rows, inner), yorder = cat(cols, inner), corder = cat(rows, cols);
  g->x_direct = g->route != 2 && xorder == wlegs;
  const auto wst = contiguous(wlegs, dim);
  if (!leg_map(xorder, wlegs, wst, xorder, contiguous(xorder, dim), dim, &g->xt)) return false;
  if (!leg_map(yorder, ysrc.legs, ysrc.strides, yorder, contiguous(yorder, dim), dim, &g->yt)) return false;
  if (!leg_map(target.legs, corder, contiguous(corder, dim), target.legs, target.strides, dim, &g->st))
    return false;
  return true;
}

// Reverse-pass descriptors and the bytes of a problem's gradient buffers
// (p.grad_bytes); grad_assign then lays them out at a base address.
qflex_status build_grad(Sub& p) {
  p.sg.resize(p.steps.size());
  // forward views of each step's operands, as recorded by the planner
  for (size_t i = 0; i < p.steps.size(); ++i) {
    const Step& st = p.steps[i];
    const Ref& ra = st.A.ref;
    const Ref& rb = st.B.ref;
    StepGrad& g = p.sg[i];
    // W_A[m][k] = sum_n W_C[m][n] B[n][k]
    if (!make_bwd(p, st.out_legs, st.ml, st.nl, st.sh, rb, ra, &g.ga) ||
        !make_bwd(p, st.out_legs, st.nl, st.ml, st.sh, ra, rb, &g.gb))
      return fail(QFLEX_ERR_UNSUPPORTED, "reverse pass needs power-of-two bond dimensions");
  }
  size_t off = 0;
  p.fwd_off.resize(p.bufs.size());
  p.w_off.resize(p.bufs.size());
  for (size_t b = 0; b < p.bufs.size(); ++b) {
    p.fwd_off[b] = off;
    off += align256(size_t(p.bufs[b].elems) * 8);
  }
  const size_t arena = off;
  size_t xa = 0, yb = 0, cc = 0, pp = 0;
  for (const StepGrad& g : p.sg)
    for (const BwdGemm* b : {&g.ga, &g.gb}) {
      xa = std::max(xa, operand_bytes(p, b->route == 2, b->M * b->K));
      yb = std::max(yb, operand_bytes(p, b->route == 2, b->N * b->K));
      cc = std::max(cc, size_t(b->M * b->N) * 8);
      if (b->splits > 1) pp = std::max(pp, size_t(b->splits) * size_t(b->M * b->N) * 8);
    }
  p.grad_bytes = align256(2 * arena + align256(size_t(p.grid_elems) * 16) + align256(xa) + align256(yb) +
                          align256(cc) + align256(pp));
  p.garena_bytes = arena;
  p.gxa = xa;
  p.gyb = yb;
  p.gcc = cc;
  return QFLEX_OK;
}

qflex_status grad_assign(Sub& p, char* base) {
  const size_t arena = p.garena_bytes;
  p.d_gws = base;
  char* c = p.d_gws;
  p.d_garena = c;
  c += arena;
  p.d_warena = c;
  c += arena;
  for (size_t b = 0; b < p.bufs.size(); ++b) p.w_off[b] = p.fwd_off[b];
  p.d_wgrid = reinterpret_cast<double2*>(c);
  c += align256(size_t(p.grid_elems) * 16);
  p.d_gA = c;
  c += align256(p.gxa);
  p.d_gB = c;
  c += align256(p.gyb);
  p.d_gC = reinterpret_cast<float2*>(c);
  c += align256(p.gcc);
  p.d_gP = reinterpret_cast<float2*>(c);
  for (StepGrad& g : p.sg)
    for (BwdGemm* b : {&g.ga, &g.gb})
      if (b->route == 2 && !tc_encode_maps(p.tc_kind, p.nsplit, b->bn, p.d_gA, b->M, p.d_gB, b->N, b->K, &b->maps))
        return fail(QFLEX_ERR_CUDA, "tensor map encoding failed");
  return QFLEX_OK;
}

cudaError_t run_bwd(Sub& p, const Step& st, const BwdGemm& g, const std::vector<int64_t>& vals,
                    cudaStream_t s) {
  cudaError_t e;
  const float2* W = reinterpret_cast<const float2*>(p.d_warena + p.w_off[st.out_buf]);
  const int fmt = g.route == 2 ? plane_fmt(p.tc_kind) : kFmtC64;
  const double out_per = g.route == 2 ? 3.0 * p.nsplit * (p.tc_kind == 0 ? 4 : 2) : 8.0;
  const bool scaled = fmt == kFmtFP16;
  const float2* X = W;
  if (!g.x_direct) {
    if (scaled && (e = launch_absmax(W, g.M * g.K, p.d_smax, s)) != cudaSuccess) return e;
    if ((e = timed(p, 1, 0, 0, double(g.M) * g.K * (8.0 + out_per), s, [&] {
           return launch_permute_tiled(W, 0, g.xt, fmt, p.nsplit, p.d_gA, g.M * g.K, s,
                                       scaled ? p.d_smax : nullptr);
         })) != cudaSuccess)
      return e;
    X = static_cast<const float2*>(p.d_gA);
  }
  if (scaled) {
    const float2* rp;
    int64_t rn;
    ref_region(p, g.ysrc, &rp, &rn);
    if ((e = launch_absmax(rp, rn, p.d_smax + 1, s)) != cudaSuccess) return e;
  }
  if ((e = timed(p, 1, 0, 0, double(g.N) * g.K * (8.0 + out_per), s, [&] {
         return launch_permute_tiled(ref_ptr(p, g.ysrc), ref_base(g.ysrc, vals), g.yt, fmt, p.nsplit, p.d_gB,
                                     g.N * g.K, s, scaled ? p.d_smax + 1 : nullptr);
       })) != cudaSuccess)
    return e;
  const float2* Y = static_cast<const float2*>(p.d_gB);
  const double mnk = double(g.M) * double(g.N) * double(g.K);
  float2* out = g.splits > 1 ? p.d_gP : p.d_gC;
  if (g.route == 2) {
    e = timed(p, 3, 8.0 * mnk, mnk * 3.0 * (p.nsplit == 2 ? 3.0 : 1.0) * 2.0, 0, s, [&] {
      return launch_cgemm_tc(p.tc_kind, p.nsplit, g.bn, g.maps, g.M, g.N, g.K, out, p.d_status, s,
                             scaled ? p.d_smax : nullptr, scaled ? p.d_smax + 1 : nullptr, nullptr, g.splits);
    });
  } else {
    e = timed(p, 2, 8.0 * mnk, 0, 0, s, [&] {
      if (g.splits > 1)
        return g.route == 1 ? launch_cgemm_rowwarp_split(g.M, g.N, g.K, X, Y, out, g.splits, s)
                            : launch_cgemm_simt_split(g.M, g.N, g.K, X, Y, out, g.splits, s);
      return g.route == 1 ? launch_cgemm_thin(g.M, g.N, g.K, X, Y, p.d_gC, s)
                          : launch_cgemm_simt(g.M, g.N, g.K, X, Y, p.d_gC, s);
    });
  }
  if (e == cudaSuccess && g.splits > 1) e = launch_splitk_reduce(p.d_gP, g.splits, g.M * g.N, p.d_gC, s);
  if (e != cudaSuccess) return e;
  // scatter C' into the target's cotangent: accumulate (FP64) for grid tensors,
  // plain write for intermediates (each is consumed by exactly one step)
  return timed(p, 1, 0, 0, double(g.M) * g.N * 16.0, s, [&] {
    if (g.target.grid) {
      double2* out = p.d_wgrid + p.gmeta[g.target.id].offset + ref_base(g.target, vals);
      return launch_permute_tiled(p.d_gC, 0, g.st, kFmtAccC128, 1, out, 0, s);
    }
    float2* out = reinterpret_cast<float2*>(p.d_warena + p.w_off[g.target.id]);
    return launch_permute_tiled(p.d_gC, 0, g.st, kFmtC64, 1, out, 0, s);
  });
}

void decode_slice(const Sub& p, int64_t s, std::vector<int64_t>& vals) {
  vals.assign(p.cuts.size(), 0);
  for (int i = int(p.cuts.size()) - 1; i >= 0; --i) {
    const int64_t r = int64_t(1) << p.K[p.cuts[i]];
    vals[i] = s % r;
    s /= r;
  }
}

// Walk the schedule of one call; `f(step index or -1 for slice sum, vals)`.
template <class F>
qflex_status walk(const Sub& p, int64_t n_bs, const int64_t* ids, int64_t n_ids, F&& f) {
  std::vector<int64_t> vals, prev;
  for (int64_t b = 0; b < n_bs; ++b) {
    if (qflex_status st = f(-2, b, vals)) return st;   // grid tensors for bitstring b
    bool first = true;
    const int64_t cnt = ids ? n_ids : p.P;
    for (int64_t k = 0; k < cnt; ++k) {
      const int64_t s = ids ? ids[k] : k;
      decode_slice(p, s, vals);
      if (p.zeros.any() && p.zeros.zero(vals)) continue;   // contributes exactly zero
      uint64_t changed = 0;
      for (size_t c = 0; c < vals.size(); ++c)
        if (first || vals[c] != prev[c]) changed |= uint64_t(1) << c;
      for (size_t i = 0; i < p.steps.size(); ++i)
        if (first || (p.steps[i].dep & changed))
          if (qflex_status st = f(int(i), b, vals)) return st;
      if (qflex_status st = f(-1, b, vals)) return st;   // slice sum
      prev = vals;
      first = false;
    }
  }
  return QFLEX_OK;
}

qflex_status check_slices(const Sub& p, const int64_t* ids, int64_t n_ids) {
  if (!ids) return QFLEX_OK;
  if (n_ids < 0) return fail(QFLEX_ERR_ARG, "n_slice_ids < 0");
  for (int64_t k = 0; k < n_ids; ++k)
    if (ids[k] < 0 || ids[k] >= p.P) return fail(QFLEX_ERR_ARG, "slice id out of range");
  return QFLEX_OK;
}

// Run `enqueue` on stream s, through a cached CUDA graph when the plan has
// graphs enabled (and is not profiling).  A call whose key (pointers, batch,
// slice list) differs from the last one runs directly; the second call with
// the same key captures its launches into a graph, and later calls with that
// key replay it.  Streams that cannot be captured (the legacy default
// stream) always run directly.
template <class F>
qflex_status with_graph(qflex_plan_s& p, const qflex_plan_s::GraphKey& key, cudaStream_t s, F&& enqueue) {
  if (!p.use_graphs || p.prof.on || s == nullptr) return enqueue();
  if (p.gexec && p.gkey == key) {
    QF_CUDA(cudaGraphLaunch(p.gexec, s));
    return QFLEX_OK;
  }
  if (!(p.gseen == key)) {
    p.gseen = key;
    return enqueue();
  }
  if (p.gexec) {
    cudaGraphExecDestroy(p.gexec);
    p.gexec = nullptr;
  }
  QF_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  qflex_status st = enqueue();
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &graph);
  if (st != QFLEX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&p.gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    p.gexec = nullptr;
    return fail(QFLEX_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  p.gkey = key;
  QF_CUDA(cudaGraphLaunch(p.gexec, s));
  return QFLEX_OK;
}

// A problem's part of one qflex_amplitudes call, enqueued on stream s:
// grid tensors per bitstring, the schedule per path (steps rerun when a cut
// they depend on changes), the FP64 slice sum into amps [n_bs][2^|tile|].
qflex_status enqueue_amplitudes(Sub& p, const double* angles, const uint8_t* bits, int64_t n_bs, const int64_t* ids,
                                int64_t n_ids, double* amps, cudaStream_t s) {
  const int64_t T = int64_t(1) << p.tile.size();
  QF_CUDA(cudaMemsetAsync(amps, 0, size_t(n_bs) * T * 2 * sizeof(double), s));
  if (p.fp16_fused) QF_CUDA(cudaMemsetAsync(p.d_bmax, 0, sizeof(unsigned) * p.bufs.size(), s));
  oc_reset(p, p.oc_b, p.oc_v);
  return walk(p, n_bs, ids, n_ids, [&](int i, int64_t b, const std::vector<int64_t>& vals) -> qflex_status {
    cudaError_t e;
    if (i == -2) {
      e = timed(p, 0, 0, 0, 8.0 * p.grid_elems, s, [&] {
        return launch_gridtensor(p.d_gmeta, p.n, p.max_bits, p.d_gops, angles, bits + b * p.n, p.d_grid, s);
      });
    } else if (i == -1) {
      const float2* src = ref_ptr(p, p.final_ref) + ref_base(p.final_ref, vals);
      e = timed(p, 4, 0, 0, 40.0 * T, s, [&] {
        return launch_slicesum(src, p.final_strides.data(), int(p.tile.size()), amps + b * T * 2, s);
      });
    } else {
      e = run_step(p, p.steps[size_t(i)], b, vals, s);
    }
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return QFLEX_OK;
  });
}

// A problem's part of one qflex_amplitudes_grad call: the forward pass on
// the dedicated buffers, then per path the reverse pass (environments of
// every intermediate and grid tensor, FP64 accumulation over paths), and
// per bitstring the angle derivatives of the grid tensors.
qflex_status enqueue_gradients(Sub& p, const double* angles, const uint8_t* bits, int64_t n_bs, const int64_t* ids,
                               int64_t n_ids, const double* g, double* amps, double* grad, cudaStream_t s) {
  const int64_t T = int64_t(1) << p.tile.size();
  const int final_buf = p.final_ref.id;
  QF_CUDA(cudaMemsetAsync(amps, 0, size_t(n_bs) * T * 2 * sizeof(double), s));
  if (p.n_params > 0) QF_CUDA(cudaMemsetAsync(grad, 0, size_t(p.n_params) * sizeof(double), s));
  oc_reset(p, p.oc_b, p.oc_v);
  qflex_status res = walk(p, n_bs, ids, n_ids, [&](int i, int64_t b, const std::vector<int64_t>& vals) -> qflex_status {
    cudaError_t e = cudaSuccess;
    if (i == -2) {
      if (b > 0 && p.n_params > 0)   // gradient of the previous bitstring
        e = launch_gridgrad(p.d_gmeta, p.n, p.max_bits, p.d_gops, angles, bits + (b - 1) * p.n, p.d_wgrid, grad, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(p.d_wgrid, 0, size_t(p.grid_elems) * 16, s);
      if (e == cudaSuccess)
        e = launch_gridtensor(p.d_gmeta, p.n, p.max_bits, p.d_gops, angles, bits + b * p.n, p.d_grid, s);
    } else if (i == -1) {
      const float2* src = ref_ptr(p, p.final_ref);
      e = launch_slicesum(src, p.final_strides.data(), int(p.tile.size()), amps + b * T * 2, s);
      // reverse pass of this slice
      if (e == cudaSuccess)
        e = launch_init_cotangent(reinterpret_cast<float2*>(p.d_warena + p.w_off[size_t(final_buf)]),
                                  p.final_strides.data(), int(p.tile.size()), g + b * T * 2, s);
      for (int k = int(p.steps.size()) - 1; k >= 0 && e == cudaSuccess; --k) {
        e = run_bwd(p, p.steps[size_t(k)], p.sg[size_t(k)].ga, vals, s);
        if (e == cudaSuccess) e = run_bwd(p, p.steps[size_t(k)], p.sg[size_t(k)].gb, vals, s);
      }
    } else {
      e = run_step(p, p.steps[size_t(i)], b, vals, s);
    }
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
    return QFLEX_OK;
  });
  if (res == QFLEX_OK && n_bs > 0 && p.n_params > 0) {
    cudaError_t e = launch_gridgrad(p.d_gmeta, p.n, p.max_bits, p.d_gops, angles, bits + (n_bs - 1) * p.n,
                                    p.d_wgrid, grad, s);
    if (e != cudaSuccess) res = fail(QFLEX_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  }
  return res;
}

// Run fn(problem, stream) for every problem of a call on stream s: one
// problem runs on s itself; several are spread round-robin over the plan's
// worker streams, forked from s by an event and joined back to it, so that
// independent problems overlap (and a capture of s records the whole
// fork-join graph).
template <class F>
qflex_status for_each_problem(qflex_plan_s& p, cudaStream_t s, F&& fn) {
  if (p.subs.size() == 1) return fn(0, s);
  QF_CUDA(cudaEventRecord(p.fork_ev[0], s));
  for (cudaStream_t w : p.workers) QF_CUDA(cudaStreamWaitEvent(w, p.fork_ev[0], 0));
  qflex_status res = QFLEX_OK;
  for (size_t i = 0; i < p.subs.size() && res == QFLEX_OK; ++i) res = fn(i, p.workers[i % p.workers.size()]);
  // join every worker even after an error, so that no stream is left forked
  for (size_t k = 0; k < p.workers.size(); ++k) {
    QF_CUDA(cudaEventRecord(p.join_ev[k], p.workers[k]));
    QF_CUDA(cudaStreamWaitEvent(s, p.join_ev[k], 0));
  }
  return res;
}

Sub* sub_of(qflex_plan p, int32_t problem) {
  if (!p || problem < 0 || size_t(problem) >= p->subs.size()) return nullptr;
  return p->subs[size_t(problem)].get();
}

}  // namespace

extern "C" {

int32_t qflex_abi_version(void) { return QFLEX_ABI_VERSION; }

const char* qflex_last_error(void) { return g_err.c_str(); }

qflex_status qflex_plan_create(const qflex_problem* problems, int32_t n_problems, qflex_precision prec,
                               size_t ws_max, int device, qflex_plan* out) {
  return guarded([&]() -> qflex_status {
    if (!problems || !out) return fail(QFLEX_ERR_ARG, "null problems or output");
    *out = nullptr;
    if (n_problems < 1 || n_problems > kMaxProblems)
      return fail(QFLEX_ERR_ARG, "n_problems must be in [1, " + std::to_string(kMaxProblems) + "]");
    if (prec < QFLEX_FP32_SIMT || prec > QFLEX_FP16X3) return fail(QFLEX_ERR_ARG, "unknown precision");
    auto plan = std::make_unique<qflex_plan_s>();
    plan->prec = prec;
    plan->device = device;
    for (int32_t i = 0; i < n_problems; ++i) {
      auto sp = std::make_unique<Sub>();
      sp->prec = prec;
      sp->device = device;
      sp->tc_kind = tc_kind_of(prec);
      sp->nsplit = nsplit_of(prec);
      sp->prof = &plan->prof;
      if (qflex_status st = build_plan(&problems[i], *sp)) {
        if (n_problems > 1) return fail(st, "problem " + std::to_string(i) + ": " + g_err);
        return st;
      }
      plan->off_qubits.push_back(plan->n_qubits_total);
      plan->off_params.push_back(plan->n_params_total);
      plan->off_amps.push_back(plan->amps_total);
      plan->n_qubits_total += sp->n;
      plan->n_params_total += sp->n_params;
      plan->amps_total += int64_t(1) << sp->tile.size();
      plan->total_bytes += align256(sp->total_bytes);
      plan->subs.push_back(std::move(sp));
    }
    if (ws_max > 0 && plan->total_bytes > ws_max)
      return fail(QFLEX_ERR_PLAN, "plan needs " + std::to_string(plan->total_bytes) + " bytes, budget " +
                                      std::to_string(ws_max));
    if (device >= 0) {
      if (prec != QFLEX_FP32_SIMT && !tc_available())
        return fail(QFLEX_ERR_UNSUPPORTED, "tensor-map encoder unavailable in this driver");
      QF_CUDA(cudaSetDevice(device));
      if (cudaMalloc(&plan->d_ws, plan->total_bytes) != cudaSuccess) {
        cudaGetLastError();
        plan->d_ws = nullptr;
        return fail(QFLEX_ERR_OOM, "workspace allocation of " + std::to_string(plan->total_bytes) + " bytes failed");
      }
      char* c = plan->d_ws;
      for (auto& sp : plan->subs) {
        if (qflex_status st = allocate(*sp, c)) return st;
        c += align256(sp->total_bytes);
      }
      if (n_problems > 1) {
        const int w = std::min<int>(kMaxWorkers, n_problems);
        plan->fork_ev.resize(1);
        QF_CUDA(cudaEventCreateWithFlags(&plan->fork_ev[0], cudaEventDisableTiming));
        for (int k = 0; k < w; ++k) {
          cudaStream_t st = nullptr;
          QF_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
          plan->workers.push_back(st);
          cudaEvent_t ev = nullptr;
          QF_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
          plan->join_ev.push_back(ev);
        }
      }
    }
    *out = plan.release();
    return QFLEX_OK;
  });
}

void qflex_plan_destroy(qflex_plan plan) {
  if (!plan) return;
  if (plan->device >= 0) cudaSetDevice(plan->device);
  delete plan;   // ~qflex_plan_s frees the workspaces, graph, streams and events
}

qflex_status qflex_plan_get_info(qflex_plan p, int32_t problem, qflex_plan_info* info) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !info) return fail(QFLEX_ERR_ARG, "null argument or problem index out of range");
    info->n_slices = sp->P;
    info->n_qubits = sp->n;
    info->n_params = sp->n_params;
    info->n_open = int(sp->tile.size());
    info->n_steps = int(sp->steps.size());
    info->max_tensor_elems = sp->max_tensor;
    info->workspace_bytes = p->total_bytes;
    info->n_tc_steps = sp->n_tc;
    info->n_persistent_buffers = sp->n_persistent;
    info->n_nonzero_slices = int64_t(sp->zeros.n_nonzero());
    info->n_problems = int32_t(p->subs.size());
    info->plane_format = sp->prec == QFLEX_FP32_SIMT ? 0 : (sp->tc_kind == 0 ? 1 : (sp->tc_kind == 1 ? 2 : 3));
    info->problem_workspace_bytes = sp->total_bytes;
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_cost(qflex_plan p, int32_t problem, int64_t n_bs, const int64_t* ids, int64_t n_ids,
                             qflex_cost* out) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !out || n_bs < 0) return fail(QFLEX_ERR_ARG, "bad argument");
    if (qflex_status st = check_slices(*sp, ids, n_ids)) return st;
    qflex_cost c{};
    const double prods = sp->nsplit == 2 ? 3.0 : 1.0;
    std::vector<int64_t> ob;
    std::vector<std::vector<int64_t>> ov;
    oc_reset(*sp, ob, ov);
    qflex_status st = walk(*sp, n_bs, ids, n_ids, [&](int i, int64_t b, const std::vector<int64_t>& vals) {
      if (i < 0) {
        ++c.launches;
        return QFLEX_OK;
      }
      const Step& s = sp->steps[i];
      const double mnk = double(s.M) * double(s.N) * double(s.K);
      c.cmacs += mnk;
      c.largest_gemm_cmacs = std::max(c.largest_gemm_cmacs, mnk);
      if (s.tc) {
        c.tc_cmacs += mnk;
        c.tc_mma_flops += mnk * 3.0 * prods * 2.0;
      }
      // operand producers that run (not in place, not a cache hit): one
      // permutation each, plus the absmax of an fp16 operand
      const bool runA = !s.A.direct && !s.A.fused &&
                        !(s.A.cache >= 0 && oc_hit(ob, ov, sp->opcache[size_t(s.A.cache)].dep, s.A.cache, b, vals));
      const bool runB = !s.B.direct && !s.B.fused &&
                        !(s.B.cache >= 0 && oc_hit(ob, ov, sp->opcache[size_t(s.B.cache)].dep, s.B.cache, b, vals));
      if (runA) c.permute_bytes += 16.0 * double(s.M) * double(s.K);
      if (runB) c.permute_bytes += 16.0 * double(s.N) * double(s.K);
      c.launches += 1 + runA + runB + (s.tc && sp->tc_kind == 2 ? int(runA) + int(runB) : 0) +
                    (!s.tc && s.fuse_out && sp->tc_kind == 2 ? 2 : 0);
      ++c.steps_executed;
      return QFLEX_OK;
    });
    if (st) return st;
    *out = c;
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_steps(qflex_plan p, int32_t problem, int64_t n_bs, const int64_t* ids, int64_t n_ids,
                              qflex_step_info* out,
                              int32_t cap, int32_t* n_steps) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !n_steps || n_bs < 0 || cap < 0 || (cap > 0 && !out)) return fail(QFLEX_ERR_ARG, "bad argument");
    if (qflex_status st = check_slices(*sp, ids, n_ids)) return st;
    std::vector<int64_t> runs(sp->steps.size(), 0), ab(sp->steps.size(), 0), bb(sp->steps.size(), 0);
    std::vector<int64_t> ob;
    std::vector<std::vector<int64_t>> ov;
    oc_reset(*sp, ob, ov);
    qflex_status st = walk(*sp, n_bs, ids, n_ids, [&](int i, int64_t b, const std::vector<int64_t>& vals) {
      if (i < 0) return QFLEX_OK;
      const Step& s = sp->steps[size_t(i)];
      ++runs[size_t(i)];
      ab[size_t(i)] += !s.A.direct && !s.A.fused &&
                       !(s.A.cache >= 0 && oc_hit(ob, ov, sp->opcache[size_t(s.A.cache)].dep, s.A.cache, b, vals));
      bb[size_t(i)] += !s.B.direct && !s.B.fused &&
                       !(s.B.cache >= 0 && oc_hit(ob, ov, sp->opcache[size_t(s.B.cache)].dep, s.B.cache, b, vals));
      return QFLEX_OK;
    });
    if (st) return st;
    *n_steps = int32_t(sp->steps.size());
    for (int i = 0; i < int(sp->steps.size()) && i < cap; ++i) {
      const Step& s = sp->steps[size_t(i)];
      qflex_step_info& o = out[i];
      o.dst = s.dst;
      o.src = s.src;
      o.M = s.M;
      o.N = s.N;
      o.K = s.K;
      if (s.tc) {
        o.kernel = 4;
      } else if (s.fp32_kernel == 1 || (s.fp32_kernel == 0 && s.N <= 32)) {
        // same rule as launch_cgemm_thin
        const int64_t cgs = (s.N + 15) / 16;
        o.kernel = (s.K >= 64 && ((s.M + 255) / 256) * cgs < 256) ? 3 : (s.N <= 16 ? 1 : 2);
      } else {
        o.kernel = 0;
      }
      o.bn = s.bn;
      o.a_direct = s.A.direct;
      o.b_direct = s.B.direct;
      o.runs = runs[size_t(i)];
      o.a_cached = s.A.cache >= 0;
      o.b_cached = s.B.cache >= 0;
      o.a_builds = ab[size_t(i)];
      o.b_builds = bb[size_t(i)];
      o.a_fused = s.A.fused;
      o.b_fused = s.B.fused;
      o.out_fused = s.fuse_out ? (s.po.n_fast ? 1 : 2) : 0;
      o.tc_wide = s.tc && tc_wide_mma(sp->nsplit, s.bn, s.K) ? 1 : 0;
    }
    return QFLEX_OK;
  });
}

qflex_status qflex_search_ordering(const qflex_circuit* c, const int32_t* tile, int32_t n_open, const int32_t* cut_edges,
                                   int32_t n_cuts, int32_t max_new_cuts, int64_t max_tensor_elems, int32_t trials,
                                   uint64_t seed, int32_t* cuts_out, int32_t* steps_out, qflex_search_result* out) {
  return guarded([&]() -> qflex_status {
    if (!c || !out || !steps_out || n_open < 0 || n_cuts < 0 || max_new_cuts < 0 || max_tensor_elems < 1 ||
        trials < 1 || trials > 4096 ||
        (n_open > 0 && !tile) || (n_cuts > 0 && !cut_edges) || (n_cuts + max_new_cuts > 0 && !cuts_out) ||
        n_cuts + max_new_cuts > 64)
      return fail(QFLEX_ERR_ARG, "bad search arguments");
    const int n = c->n_qubits, E = c->n_edges;
    if (n < 1 || E < 0 || (E > 0 && !c->edges) || c->n_gates < 0 || (c->n_gates > 0 && !c->gates))
      return fail(QFLEX_ERR_CIRCUIT, "bad circuit");
    SearchNet net;
    net.n = n;
    std::map<std::pair<int, int>, int> index;
    for (int e = 0; e < E; ++e) {
      const int a = c->edges[2 * e], b = c->edges[2 * e + 1];
      if (a < 0 || b < 0 || a >= n || b >= n || a == b) return fail(QFLEX_ERR_CIRCUIT, "bad edge");
      const auto key = std::make_pair(std::min(a, b), std::max(a, b));
      if (index.count(key)) return fail(QFLEX_ERR_CIRCUIT, "repeated edge");
      index[key] = e;
      net.edges.push_back(key);
    }
    net.bits.assign(size_t(E), 0);
    std::vector<int> gate_edge(size_t(c->n_gates), -1);
    for (int64_t i = 0; i < c->n_gates; ++i) {
      const qflex_gate& g = c->gates[i];
      if (g.kind < 0 || g.kind > QFLEX_GATE_ISWAP || g.q0 < 0 || g.q0 >= n)
        return fail(QFLEX_ERR_CIRCUIT, "bad gate kind or qubit");
      if (g.kind != QFLEX_GATE_CZ && g.kind != QFLEX_GATE_ISWAP) continue;
      auto it = index.find(std::make_pair(std::min(g.q0, g.q1), std::max(g.q0, g.q1)));
      if (it == index.end()) return fail(QFLEX_ERR_CIRCUIT, "two-qubit gate on a pair that is not a lattice edge");
      net.bits[size_t(it->second)] += g.kind == QFLEX_GATE_ISWAP ? 2 : 1;
      gate_edge[size_t(i)] = it->second;
    }
    std::vector<int64_t> order(size_t(c->n_gates));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return c->gates[x].cycle < c->gates[y].cycle; });
    net.lines = proj_lines(c, order, gate_edge, net.bits);
    net.open.assign(size_t(n), 0);
    for (int t = 0; t < n_open; ++t) {
      if (tile[t] < 0 || tile[t] >= n || net.open[size_t(tile[t])]) return fail(QFLEX_ERR_ARG, "bad tile qubit");
      net.open[size_t(tile[t])] = 1;
    }
    std::vector<int> cuts(cut_edges, cut_edges + n_cuts);
    for (int e : cuts)
      if (e < 0 || e >= E || std::count(cuts.begin(), cuts.end(), e) > 1) return fail(QFLEX_ERR_ARG, "bad cut edge");
    std::vector<int> found;
    SearchResult r;
    const bool fits = search_cuts(net, cuts, max_new_cuts, std::log2(double(max_tensor_elems)), &found, &r, trials,
                                  seed);
    if (r.steps.size() != size_t(2 * (n - 1))) return fail(QFLEX_ERR_PLAN, "search failed");
    std::copy(found.begin(), found.end(), cuts_out);
    std::copy(r.steps.begin(), r.steps.end(), steps_out);
    out->log2_max_tensor = r.log2_max;
    out->cmacs_per_bitstring = r.cmacs;
    out->n_slices = r.n_slices;
    out->n_nonzero_slices = r.n_nonzero;
    out->n_cuts = int32_t(found.size());
    out->n_steps = n - 1;
    if (!fits)
      return fail(QFLEX_ERR_PLAN, "no ordering with at most " + std::to_string(max_tensor_elems) +
                                      " entries per tensor within " + std::to_string(max_new_cuts) + " new cuts");
    return QFLEX_OK;
  });
}

namespace {

// The first n_f of a Fisher-Yates shuffle of 0..P-1 (SplitMix64 stream),
// n_f = max(1, floor(f P + 1/2)) capped at P, sorted.
qflex_status shuffle_select(int64_t P, double f, uint64_t seed, int64_t cap, std::vector<int64_t>* out) {
  if (P > (int64_t(1) << 32)) return fail(QFLEX_ERR_UNSUPPORTED, "too many slices to shuffle");
  int64_t nf = int64_t(std::floor(f * double(P) + 0.5));
  nf = std::max<int64_t>(1, std::min<int64_t>(P, nf));
  if (cap < nf) return fail(QFLEX_ERR_ARG, "slice_ids capacity too small");
  std::vector<int64_t> a(static_cast<size_t>(P));
  std::iota(a.begin(), a.end(), 0);
  uint64_t x = seed;
  auto next = [&]() {   // SplitMix64 (Steele, Lea, Flood 2014)
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int64_t i = P - 1; i > 0; --i) {
    const int64_t j = int64_t(next() % uint64_t(i + 1));
    std::swap(a[size_t(i)], a[size_t(j)]);
  }
  a.resize(size_t(nf));
  std::sort(a.begin(), a.end());
  *out = std::move(a);
  return QFLEX_OK;
}

constexpr int64_t kMaxListedSlices = int64_t(1) << 32;

}  // namespace

qflex_status qflex_select_slices(qflex_plan p, int32_t problem, double f, uint64_t seed, int64_t* ids, int64_t cap,
                                 int64_t* n_sel) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !ids || !n_sel || !(f > 0.0)) return fail(QFLEX_ERR_ARG, "bad argument");
    std::vector<int64_t> a;
    if (qflex_status st = shuffle_select(sp->P, f, seed, cap, &a)) return st;
    std::copy(a.begin(), a.end(), ids);
    *n_sel = int64_t(a.size());
    return QFLEX_OK;
  });
}

qflex_status qflex_nonzero_slices(qflex_plan p, int32_t problem, int64_t* ids, int64_t cap, int64_t* n_nonzero) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !n_nonzero || cap < 0 || (cap > 0 && !ids)) return fail(QFLEX_ERR_ARG, "bad argument");
    const double count = sp->zeros.n_nonzero();
    if (count > double(kMaxListedSlices)) return fail(QFLEX_ERR_UNSUPPORTED, "too many paths to list");
    *n_nonzero = int64_t(count);
    if (cap < *n_nonzero) return fail(QFLEX_ERR_ARG, "slice_ids capacity too small");
    std::vector<int64_t> all;
    if (!sp->zeros.list(&all, kMaxListedSlices)) return fail(QFLEX_ERR_UNSUPPORTED, "too many paths to list");
    std::copy(all.begin(), all.end(), ids);
    return QFLEX_OK;
  });
}

qflex_status qflex_select_nonzero_slices(qflex_plan p, int32_t problem, double f, uint64_t seed, int64_t* ids,
                                         int64_t cap, int64_t* n_sel) {
  return guarded([&]() -> qflex_status {
    Sub* sp = sub_of(p, problem);
    if (!sp || !ids || !n_sel || !(f > 0.0)) return fail(QFLEX_ERR_ARG, "bad argument");
    std::vector<int64_t> all;
    if (!sp->zeros.list(&all, kMaxListedSlices)) return fail(QFLEX_ERR_UNSUPPORTED, "too many paths to list");
    std::vector<int64_t> a;
    if (qflex_status st = shuffle_select(int64_t(all.size()), f, seed, cap, &a)) return st;
    for (size_t k = 0; k < a.size(); ++k) ids[k] = all[size_t(a[k])];
    *n_sel = int64_t(a.size());
    return QFLEX_OK;
  });
}

qflex_status qflex_amplitudes(qflex_plan p, const double* angles, const uint8_t* bits, int64_t n_bs,
                              const int64_t* ids, int64_t n_ids, double* amps, void* stream) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    if (n_bs < 0 || (n_bs > 0 && (!bits || !amps))) return fail(QFLEX_ERR_ARG, "bad bitstrings/output");
    if (p->n_params_total > 0 && !angles) return fail(QFLEX_ERR_ARG, "angles required");
    for (auto& sp : p->subs)
      if (qflex_status st = check_slices(*sp, ids, n_ids)) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    QF_CUDA(cudaSetDevice(p->device));
    p->last_stream = s;
    qflex_plan_s::GraphKey key;
    key.angles = angles;
    key.bits = bits;
    key.out = amps;
    key.n_bs = n_bs;
    key.kind = 0;
    key.all = ids == nullptr;
    if (ids) key.ids.assign(ids, ids + n_ids);
    return with_graph(*p, key, s, [&]() -> qflex_status {
      return for_each_problem(*p, s, [&](size_t i, cudaStream_t ws) {
        return enqueue_amplitudes(*p->subs[i], angles ? angles + p->off_params[i] : nullptr,
                                  bits + n_bs * p->off_qubits[i], n_bs, ids, n_ids,
                                  amps + 2 * n_bs * p->off_amps[i], ws);
      });
    });
  });
}

qflex_status qflex_plan_enable_gradients(qflex_plan p) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    if (p->grad_ready) return QFLEX_OK;
    QF_CUDA(cudaSetDevice(p->device));
    size_t total = 0;
    for (auto& sp : p->subs) {
      if (qflex_status st = build_grad(*sp)) return st;
      total += sp->grad_bytes;
    }
    if (cudaMalloc(&p->d_gws, total) != cudaSuccess) {
      cudaGetLastError();
      p->d_gws = nullptr;
      return fail(QFLEX_ERR_OOM, "gradient workspace allocation of " + std::to_string(total) + " bytes failed");
    }
    p->grad_bytes = total;
    char* c = p->d_gws;
    for (auto& sp : p->subs) {
      if (qflex_status st = grad_assign(*sp, c)) return st;
      c += sp->grad_bytes;
    }
    p->grad_ready = true;
    return QFLEX_OK;
  });
}

qflex_status qflex_amplitudes_grad(qflex_plan p, const double* angles, const uint8_t* bits, int64_t n_bs,
                                   const int64_t* ids, int64_t n_ids, const double* g, double* amps,
                                   double* grad, void* stream) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    if (!p->grad_ready) return fail(QFLEX_ERR_UNSUPPORTED, "call qflex_plan_enable_gradients first");
    if (n_bs < 0 || (n_bs > 0 && (!bits || !amps || !g))) return fail(QFLEX_ERR_ARG, "bad bitstrings/outputs");
    if (p->n_params_total > 0 && (!angles || !grad)) return fail(QFLEX_ERR_ARG, "angles and grad_angles required");
    for (auto& sp : p->subs) {
      if (sp->steps.empty()) return fail(QFLEX_ERR_UNSUPPORTED, "gradients need at least one contraction step");
      if (qflex_status st = check_slices(*sp, ids, n_ids)) return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    QF_CUDA(cudaSetDevice(p->device));
    p->last_stream = s;
    qflex_plan_s::GraphKey key;
    key.angles = angles;
    key.bits = bits;
    key.out = amps;
    key.grad = grad;
    key.g = g;
    key.n_bs = n_bs;
    key.kind = 1;
    key.all = ids == nullptr;
    if (ids) key.ids.assign(ids, ids + n_ids);
    for (auto& sp : p->subs) sp->grad_active = true;
    qflex_status res = with_graph(*p, key, s, [&]() -> qflex_status {
      return for_each_problem(*p, s, [&](size_t i, cudaStream_t ws) {
        const int64_t pa = p->off_params[i], pb = n_bs * p->off_qubits[i], pc = 2 * n_bs * p->off_amps[i];
        return enqueue_gradients(*p->subs[i], angles ? angles + pa : nullptr, bits + pb, n_bs, ids, n_ids, g + pc,
                                 amps + pc, grad ? grad + pa : nullptr, ws);
      });
    });
    for (auto& sp : p->subs) sp->grad_active = false;
    return res;
  });
}

qflex_status qflex_plan_autotune(qflex_plan p, int32_t reps, int32_t* n_shapes, double* gain_ms) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    if (reps < 1 || reps > 100) return fail(QFLEX_ERR_ARG, "reps must be in [1, 100]");
    QF_CUDA(cudaSetDevice(p->device));
    cudaStream_t s = nullptr;
    QF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    QF_CUDA(cudaEventCreate(&e0));
    QF_CUDA(cudaEventCreate(&e1));
    int tuned = 0;
    double gain = 0.0;
    qflex_status res = QFLEX_OK;
    for (auto& spu : p->subs) {
      Sub* sp = spu.get();
      struct Key {
        int64_t M, N, K;
        bool tc;
        bool operator<(const Key& o) const {
          return std::tie(M, N, K, tc) < std::tie(o.M, o.N, o.K, o.tc);
        }
      };
      std::map<Key, std::vector<size_t>> groups;
      for (size_t i = 0; i < sp->steps.size(); ++i) {
        const Step& st = sp->steps[i];
        groups[{st.M, st.N, st.K, st.tc}].push_back(i);
      }
      for (auto& [key, idx] : groups) {
        Step& st = sp->steps[idx.front()];
        float2* C = reinterpret_cast<float2*>(sp->d_arena + sp->bufs[st.out_buf].offset);
        std::vector<int> cands;
        bool fused_fp32 = false;   // CUDA-core producers writing planes keep their form
        for (size_t i : idx) fused_fp32 = fused_fp32 || (!sp->steps[i].tc && sp->steps[i].fuse_out);
        if (key.tc) cands = {128, 64};
        else if (key.N <= 32 && !fused_fp32) cands = {1, 2};
        else continue;
        std::vector<TcGemmMaps> maps(cands.size());
        float best = 1e30f, first = 0.f;
        int best_c = -1;
        for (size_t c = 0; c < cands.size(); ++c) {
          if (key.tc && !tc_encode_maps(sp->tc_kind, sp->nsplit, cands[c], x_buf(*sp, st.A, true, true), st.M,
                                        x_buf(*sp, st.B, false, true), st.N, st.K, &maps[c])) {
            res = fail(QFLEX_ERR_CUDA, "tensor map encoding failed");
            break;
          }
          auto launch = [&]() -> cudaError_t {
            if (key.tc)
              return launch_cgemm_tc(sp->tc_kind, sp->nsplit, cands[c], maps[c], st.M, st.N, st.K, C, sp->d_status, s,
                                     scale_word(*sp, st.A, true, true), scale_word(*sp, st.B, false, true),
                                     st.fuse_out ? &st.po : nullptr);
            // operands as the step reads them: in place when consumed directly
            // (the scratch is only sized for produced operands), else their buffer
            const float2* A = st.A.direct ? ref_ptr(*sp, st.A.ref) : static_cast<const float2*>(op_buf(*sp, st.A, true));
            const float2* B = st.B.direct ? ref_ptr(*sp, st.B.ref) : static_cast<const float2*>(op_buf(*sp, st.B, false));
            return cands[c] == 1 ? launch_cgemm_thin(st.M, st.N, st.K, A, B, C, s)
                                 : launch_cgemm_simt(st.M, st.N, st.K, A, B, C, s);
          };
          cudaError_t e = launch();   // warm-up
          for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            if (r == 0) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch();
          }
          if (e == cudaSuccess) e = cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            res = fail(QFLEX_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            break;
          }
          ms /= float(reps);
          if (c == 0) first = ms;
          if (ms < best) {
            best = ms;
            best_c = int(c);
          }
        }
        if (res != QFLEX_OK) break;
        for (size_t i : idx) {
          Step& t = sp->steps[i];
          if (key.tc) {
            // steps of one shape may read different operand buffers (caches)
            t.bn = cands[best_c];
            if (!encode_step(*sp, t)) {
              res = fail(QFLEX_ERR_CUDA, "tensor map encoding failed");
              break;
            }
          } else {
            t.fp32_kernel = cands[best_c];
          }
        }
        ++tuned;
        gain += double(first - best) * double(idx.size());
      }
      if (res != QFLEX_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (res != QFLEX_OK) return res;
    for (auto& spu : p->subs) {
      int32_t w = 0;
      QF_CUDA(cudaMemcpy(&w, spu->d_status, sizeof(w), cudaMemcpyDeviceToHost));
      if (w) return fail(QFLEX_ERR_DEVICE_TIMEOUT, "a bounded device-side wait ran out during autotuning");
    }
    if (p->gexec) {   // cached graph holds the old configuration
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
      p->gseen = qflex_plan_s::GraphKey{};
    }
    if (n_shapes) *n_shapes = tuned;
    if (gain_ms) *gain_ms = gain;
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_use_graphs(qflex_plan p, int32_t enable) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    p->use_graphs = enable != 0;
    if (!p->use_graphs && p->gexec) {
      cudaGraphExecDestroy(p->gexec);
      p->gexec = nullptr;
    }
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_profile(qflex_plan p, int32_t mode, qflex_profile* out) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    QF_CUDA(cudaSetDevice(p->device));
    Prof& pr = p->prof;
    auto drain = [&]() -> qflex_status {
      for (const auto& r : pr.recs) {   // pairs may sit on several streams
        QF_CUDA(cudaEventSynchronize(pr.pool[r.e0 + 1]));
        float ms = 0.f;
        QF_CUDA(cudaEventElapsedTime(&ms, pr.pool[r.e0], pr.pool[r.e0 + 1]));
        pr.tot.launches[r.cls] += 1;
        pr.tot.ms[r.cls] += ms;
        pr.tot.flops[r.cls] += r.flops;
        pr.tot.mma_flops[r.cls] += r.mma;
        pr.tot.bytes[r.cls] += r.bytes;
        if (r.M > 0) {
          qflex_profile_shape& q = pr.shapes[std::make_tuple(r.cls, r.M, r.N, r.K, r.planes)];
          q.cls = r.cls;
          q.out_planes = r.planes;
          q.M = r.M;
          q.N = r.N;
          q.K = r.K;
          q.launches += 1;
          q.ms += ms;
          q.mma_flops += r.mma;
        }
      }
      pr.recs.clear();
      pr.used = 0;
      return QFLEX_OK;
    };
    if (mode < 0 || mode > 31) return fail(QFLEX_ERR_ARG, "mode must be a class mask in [0, 31]");
    if (mode != 0) {
      if (qflex_status st = drain()) return st;
      pr.tot = qflex_profile{};
      pr.shapes.clear();
      pr.on = true;
      pr.mask = mode;
    } else {
      pr.on = false;
    }
    if (out) {
      if (qflex_status st = drain()) return st;
      *out = pr.tot;
    }
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_profile_shapes(qflex_plan p, qflex_profile_shape* out, int64_t cap, int64_t* n) {
  return guarded([&]() -> qflex_status {
    if (!p || !n) return fail(QFLEX_ERR_ARG, "null plan or count");
    if (cap < 0 || (cap > 0 && !out)) return fail(QFLEX_ERR_ARG, "bad output array");
    if (p->device < 0) return fail(QFLEX_ERR_UNSUPPORTED, "host-only plan");
    Prof& pr = p->prof;
    if (!pr.recs.empty()) return fail(QFLEX_ERR_ARG, "launches not yet read: call qflex_plan_profile with out first");
    *n = int64_t(pr.shapes.size());
    int64_t i = 0;
    for (const auto& kv : pr.shapes) {
      if (i >= cap) break;
      out[i++] = kv.second;
    }
    return QFLEX_OK;
  });
}

qflex_status qflex_plan_sync(qflex_plan p) {
  return guarded([&]() -> qflex_status {
    if (!p) return fail(QFLEX_ERR_ARG, "null plan");
    if (p->device < 0) return QFLEX_OK;
    QF_CUDA(cudaSetDevice(p->device));
    QF_CUDA(cudaStreamSynchronize(p->last_stream));
    int32_t w = 0;
    for (auto& sp : p->subs) {
      int32_t v = 0;
      QF_CUDA(cudaMemcpy(&v, sp->d_status, sizeof(v), cudaMemcpyDeviceToHost));
      if (v) QF_CUDA(cudaMemset(sp->d_status, 0, sizeof(int32_t)));
      w |= v;
    }
    if (w & kDevTimeout) return fail(QFLEX_ERR_DEVICE_TIMEOUT, "a bounded device-side wait ran out");
    if (w) return fail(QFLEX_ERR_PLAN, "internal: a fused epilogue destination fell outside its operand planes");
    return QFLEX_OK;
  });
}

qflex_status qflex_permute(const void* in, void* out, int32_t rank, const int64_t* dims, const int32_t* perm,
                           void* stream) {
  return guarded([&]() -> qflex_status {
    if (rank < 0 || rank > 32 || (rank > 0 && (!dims || !perm))) return fail(QFLEX_ERR_ARG, "bad permute arguments");
    std::vector<int64_t> istr(rank);
    int64_t total = 1;
    for (int a = rank - 1; a >= 0; --a) {
      if (dims[a] < 0) return fail(QFLEX_ERR_ARG, "dims must be non-negative");
      istr[a] = total;
      total *= dims[a];
    }
    std::vector<int> seen(rank, 0);
    for (int a = 0; a < rank; ++a) {
      if (perm[a] < 0 || perm[a] >= rank || seen[perm[a]]++) return fail(QFLEX_ERR_ARG, "perm is not a permutation");
    }
    if (total == 0) return QFLEX_OK;
    if (!in || !out) return fail(QFLEX_ERR_ARG, "null tensor pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool pow2 = true;
    for (int a = 0; a < rank; ++a) pow2 = pow2 && is_pow2(dims[a]);
    cudaError_t e;
    if (pow2) {
      std::vector<int64_t> w;
      for (int a = rank - 1; a >= 0; --a)
        for (int b = 0; b < ilog2(dims[perm[a]]); ++b) w.push_back(istr[perm[a]] << b);
      PermTile t;
      if (!build_perm_tile(int(w.size()), w.data(), &t)) return fail(QFLEX_ERR_UNSUPPORTED, "tensor too large");
      e = launch_permute_tiled(static_cast<const float2*>(in), 0, t, kFmtC64, 1, out, total, s);
    } else {
      GatherDesc g{};
      g.rank = rank;
      g.total = total;
      for (int a = 0; a < rank; ++a) {
        g.dims[a] = dims[perm[a]];
        g.in_strides[a] = istr[perm[a]];
      }
      e = launch_permute_gather(static_cast<const float2*>(in), 0, g, kFmtC64, 1, out, total, s);
    }
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, cudaGetErrorString(e));
    return QFLEX_OK;
  });
}

qflex_status qflex_cgemm_workspace_size(int32_t prec, int64_t M, int64_t N, int64_t K, size_t* bytes) {
  return guarded([&]() -> qflex_status {
    if (!bytes || M < 0 || N < 0 || K < 0) return fail(QFLEX_ERR_ARG, "bad argument");
    if (prec == QFLEX_FP32_SIMT) {
      *bytes = 0;
      return QFLEX_OK;
    }
    if (prec < 0 || prec > QFLEX_FP16X3) return fail(QFLEX_ERR_ARG, "unknown precision");
    const int kind = tc_kind_of(prec);
    const int nsplit = nsplit_of(prec);
    const size_t per = size_t(3) * nsplit * (kind == 0 ? 4 : 2);
    // planes of at most 2^62 bytes each, checked before multiplying out
    const uint64_t lim = uint64_t(1) << 62;
    if (K > 0 && (uint64_t(M) > lim / (per * uint64_t(K)) || uint64_t(N) > lim / (per * uint64_t(K))))
      return fail(QFLEX_ERR_ARG, "GEMM too large");
    *bytes = align256(per * size_t(M) * size_t(K)) + align256(per * size_t(N) * size_t(K)) + 256;
    return QFLEX_OK;
  });
}

qflex_status qflex_cgemm(int32_t prec, int64_t M, int64_t N, int64_t K, const void* A, const void* B, void* C,
                         void* ws, size_t ws_bytes, void* stream) {
  return guarded([&]() -> qflex_status {
    if (M < 0 || N < 0 || K < 0 || (M * N > 0 && (!A || !B || !C))) return fail(QFLEX_ERR_ARG, "bad GEMM arguments");
    if (M == 0 || N == 0) return QFLEX_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool tc = prec != QFLEX_FP32_SIMT && M >= 128 && K % 8 == 0 && K > 0 && N >= 16;
    if (!tc) {
      if (K == 0) QF_CUDA(cudaMemsetAsync(C, 0, size_t(M) * N * 8, s));
      else if (N <= 32)
        QF_CUDA(launch_cgemm_thin(M, N, K, static_cast<const float2*>(A), static_cast<const float2*>(B),
                                  static_cast<float2*>(C), s));
      else
        QF_CUDA(launch_cgemm_simt(M, N, K, static_cast<const float2*>(A), static_cast<const float2*>(B),
                                  static_cast<float2*>(C), s));
      return QFLEX_OK;
    }
    size_t need = 0;
    if (qflex_status st = qflex_cgemm_workspace_size(prec, M, N, K, &need)) return st;
    if (!ws || ws_bytes < need) return fail(QFLEX_ERR_ARG, "workspace too small");
    if (!tc_available()) return fail(QFLEX_ERR_UNSUPPORTED, "tensor-map encoder unavailable");
    const int kind = tc_kind_of(prec);
    const int nsplit = nsplit_of(prec);
    const size_t per = size_t(3) * nsplit * (kind == 0 ? 4 : 2);
    char* pa = static_cast<char*>(ws);
    char* pb = pa + align256(per * size_t(M) * size_t(K));
    unsigned* smax = reinterpret_cast<unsigned*>(pb + align256(per * size_t(N) * size_t(K)));
    const int fmt = plane_fmt(kind);
    // identity "permutation" of a [rows][K] matrix into operand planes
    auto planes = [&](const void* src, int64_t rows, void* dst, unsigned* sm) {
      std::vector<int64_t> w;
      const int64_t total = rows * K;
      if (fmt == kFmtFP16) {
        cudaError_t e = launch_absmax(static_cast<const float2*>(src), total, sm, s);
        if (e != cudaSuccess) return e;
      } else {
        sm = nullptr;
      }
      if (is_pow2(total)) {
        for (int b = 0; b < ilog2(total); ++b) w.push_back(int64_t(1) << b);
        PermTile t;
        build_perm_tile(int(w.size()), w.data(), &t);
        return launch_permute_tiled(static_cast<const float2*>(src), 0, t, fmt, nsplit, dst, total, s, sm);
      }
      GatherDesc g{};
      g.rank = 1;
      g.total = total;
      g.dims[0] = total;
      g.in_strides[0] = 1;
      return launch_permute_gather(static_cast<const float2*>(src), 0, g, fmt, nsplit, dst, total, s, sm);
    };
    QF_CUDA(planes(A, M, pa, smax));
    QF_CUDA(planes(B, N, pb, smax + 1));
    TcGemmMaps maps;
    const int bn = N >= 128 ? 128 : 64;
    if (!tc_encode_maps(kind, nsplit, bn, pa, M, pb, N, K, &maps)) return fail(QFLEX_ERR_CUDA, "tensor map encoding failed");
    int dev = 0;
    QF_CUDA(cudaGetDevice(&dev));
    QF_CUDA(launch_cgemm_tc(kind, nsplit, bn, maps, M, N, K, static_cast<float2*>(C), device_status_word(dev), s,
                            kind == 2 ? smax : nullptr, kind == 2 ? smax + 1 : nullptr));
    return QFLEX_OK;
  });
}

qflex_status qflex_norm(const double* amps, int64_t n, double* out, void* stream) {
  return guarded([&]() -> qflex_status {
    if (!amps || !out || n < 0) return fail(QFLEX_ERR_ARG, "bad argument");
    QF_CUDA(launch_norm(amps, n, out, static_cast<cudaStream_t>(stream)));
    return QFLEX_OK;
  });
}

qflex_status qflex_frugal_sample(const double* amps, int64_t n_batches, int32_t n_c, int32_t n_qubits,
                                 double M, uint64_t seed, int32_t* accepted, void* stream) {
  return guarded([&]() -> qflex_status {
    if (n_batches < 0 || n_c < 1 || n_c > 4096 || n_qubits < 0 || n_qubits > 1000 || !(M > 0.0))
      return fail(QFLEX_ERR_ARG, "bad sampling arguments");
    if (n_batches == 0) return QFLEX_OK;
    if (!amps || !accepted) return fail(QFLEX_ERR_ARG, "null pointer");
    const double scale = std::ldexp(1.0, n_qubits) / M;
    QF_CUDA(launch_frugal(amps, n_batches, n_c, scale, seed, accepted, static_cast<cudaStream_t>(stream)));
    return QFLEX_OK;
  });
}

qflex_status qflex_fidelity_samples(const uint8_t* batch_bits, const int32_t* accepted, int64_t n_batches,
                                    const int32_t* tile, int32_t n_tile, int32_t n_qubits, double fidelity,
                                    uint64_t seed, int64_t n_samples, uint8_t* samples, int32_t* source,
                                    int64_t* n_exact, void* stream) {
  return guarded([&]() -> qflex_status {
    if (!n_exact || n_batches < 0 || n_samples < 0 || n_qubits < 1 || n_qubits > 100000 || n_tile < 0 ||
        n_tile > 30 || n_tile > n_qubits || !(fidelity >= 0.0 && fidelity <= 1.0))
      return fail(QFLEX_ERR_ARG, "bad fidelity-sampling arguments");
    if (n_batches > INT32_MAX) return fail(QFLEX_ERR_ARG, "more than 2^31 - 1 batches");
    std::vector<char> seen(size_t(n_qubits), 0);
    for (int t = 0; t < n_tile; ++t) {
      if (!tile || tile[t] < 0 || tile[t] >= n_qubits || seen[tile[t]]) return fail(QFLEX_ERR_ARG, "bad tile qubit");
      seen[tile[t]] = 1;
    }
    *n_exact = 0;
    if (n_samples == 0) return QFLEX_OK;
    if (!samples || !source || (n_batches > 0 && (!batch_bits || !accepted))) return fail(QFLEX_ERR_ARG, "null pointer");
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    const size_t pool_bytes = (size_t(n_batches) * 4 + 15) / 16 * 16;
    QF_CUDA(cudaMallocAsync(&scratch, pool_bytes + 16, s));
    int32_t* pool = static_cast<int32_t*>(scratch);
    int64_t* counts = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + pool_bytes);
    int64_t host_counts[2] = {0, 0};
    cudaError_t e = launch_fidelity_mix(batch_bits, accepted, n_batches, tile, n_tile, n_qubits, fidelity, seed,
                                        n_samples, pool, source, counts, samples, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_counts, counts, sizeof(host_counts), cudaMemcpyDeviceToHost, s);
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(QFLEX_ERR_CUDA, std::string("fidelity sampling: ") + cudaGetErrorString(e));
    *n_exact = host_counts[0];
    if (host_counts[0] > host_counts[1])
      return fail(QFLEX_ERR_ARG, "fidelity sampling needs " + std::to_string(host_counts[0]) +
                                     " exact samples but only " + std::to_string(host_counts[1]) +
                                     " batches were accepted; compute more batches");
    return QFLEX_OK;
  });
}

qflex_status qflex_device_status(int device, int32_t* status) {
  return guarded([&]() -> qflex_status {
    if (!status || device < 0) return fail(QFLEX_ERR_ARG, "bad argument");
    QF_CUDA(cudaSetDevice(device));
    QF_CUDA(cudaDeviceSynchronize());
    int32_t* w = device_status_word(device);
    if (!w) return fail(QFLEX_ERR_CUDA, "status word allocation failed");
    int32_t v = 0, na = 0;
    QF_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    QF_CUDA(cudaMemset(w, 0, sizeof(v)));
    QF_CUDA(noalloc_take_status(device, &na));
    v |= na;
    // the bits as qflex_plan_sync decodes them
    *status = (v & kDevTimeout) ? QFLEX_ERR_DEVICE_TIMEOUT : (v & kDevBadIndex) ? QFLEX_ERR_PLAN : QFLEX_OK;
    return QFLEX_OK;
  });
}

qflex_status qflex_device_selftest_timeout(int device, uint64_t limit_ns, int32_t* status) {
  return guarded([&]() -> qflex_status {
    if (!status || device < 0 || limit_ns < 1000 || limit_ns > 1000000000ull)
      return fail(QFLEX_ERR_ARG, "bad argument (limit_ns must be in [1e3, 1e9])");
    QF_CUDA(cudaSetDevice(device));
    int32_t* w = device_status_word(device);
    if (!w) return fail(QFLEX_ERR_CUDA, "status word allocation failed");
    QF_CUDA(cudaDeviceSynchronize());
    QF_CUDA(cudaMemset(w, 0, sizeof(int32_t)));
    QF_CUDA(launch_wait_selftest(limit_ns, w, nullptr));
    QF_CUDA(cudaDeviceSynchronize());
    int32_t v = 0;
    QF_CUDA(cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost));
    QF_CUDA(cudaMemset(w, 0, sizeof(v)));
    // the same bounded wait on the allocation-free GEMM's private word, whose
    // bit stays set for that entry point's next call to clear and report
    QF_CUDA(noalloc_selftest(device, limit_ns));
    *status = (v & kDevTimeout) ? QFLEX_ERR_DEVICE_TIMEOUT : QFLEX_OK;
    return QFLEX_OK;
  });
}

}  // extern "C"

void qflex::set_last_error(const char* msg) { g_err = msg; }

/*
 * qflex_gb300 -- C ABI of a single-GPU (GB300, sm_103a) engine that contracts
 * the 2D-grid tensor network of a random quantum circuit into output
 * amplitudes, after Villalonga et al., "A flexible high-performance simulator
 * for verifying and benchmarking quantum circuits implemented on real
 * hardware" (arXiv:1811.09599, "qFlex").
 *
 * The calls follow the paper's problem statement: a circuit on a lattice
 * (Methods, "Revised set of RQCs" and "Overview of the simulator"), a
 * contraction ordering (Methods, "Remarks on the choice of cuts and
 * contraction ordering"), a set of cut bonds whose values define independent
 * paths (Methods, "Cutting indexes"), output bitstrings with an open tile of
 * qubits whose 2^k amplitudes come out of one contraction (Methods, "Fast
 * sampling technique"; SI A), and the fraction of paths summed for
 * fidelity-f amplitudes (Methods, "Summing a fraction of the paths").
 *
 * Conventions for every call:
 *  - Pointers documented "device" must be device memory of the plan's GPU
 *    (e.g. torch tensor data); "host" pointers are ordinary host memory.  The
 *    caller owns every input and output buffer.
 *  - A plan owns one device workspace allocated in qflex_plan_create (the
 *    paper preallocates scratch space once, Methods "Implementation of the
 *    simulator"); afterwards only qflex_plan_enable_gradients (the reverse
 *    pass's buffers, once) and qflex_fidelity_samples (stream-ordered
 *    scratch) allocate device memory.
 *  - Calls that take a stream enqueue work on it and return at once; the
 *    returned status covers argument checks and launches.  Errors detected on
 *    the device (a bounded wait that ran out; a fused store whose computed
 *    position fell outside its planes, skipped) set a status word that
 *    qflex_plan_sync / qflex_device_status report.
 *  - Nothing throws across the ABI; on failure the call returns a nonzero
 *    qflex_status and qflex_last_error() describes it (thread-local string).
 *    A failed host allocation inside a call returns QFLEX_ERR_OOM.
 *  - Complex numbers are interleaved (re, im): complex64 = 2 x float,
 *    complex128 = 2 x double.  Tensors are row-major.
 */
#ifndef QFLEX_GB300_H
#define QFLEX_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QFLEX_ABI_VERSION 4

typedef struct qflex_plan_s* qflex_plan;

typedef enum {
  QFLEX_OK = 0,
  QFLEX_ERR_ARG = 1,            /* a null pointer, size or index out of range */
  QFLEX_ERR_CIRCUIT = 2,        /* malformed circuit (gate on a non-edge, bad kind ...) */
  QFLEX_ERR_PLAN = 3,           /* invalid ordering, or the plan exceeds the memory budget */
  QFLEX_ERR_OOM = 4,            /* device allocation failed */
  QFLEX_ERR_CUDA = 5,           /* a CUDA runtime call failed */
  QFLEX_ERR_DEVICE_TIMEOUT = 6, /* a bounded device-side wait ran out (kernel returned early) */
  QFLEX_ERR_UNSUPPORTED = 7     /* valid request this build does not handle (e.g. no GPU) */
} qflex_status;

/* Arithmetic of the complex GEMMs (the cross-slice sum is always FP64). */
typedef enum {
  QFLEX_FP32_SIMT = 0,  /* plain FP32, 4 real FMAs per complex MAC on CUDA cores */
  QFLEX_TF32X3 = 1,     /* tcgen05 kind::tf32, 3-multiply complex trick, operands split
                           hi+lo, products hi*hi + hi*lo + lo*hi, FP32 accumulate */
  QFLEX_BF16X3 = 2,     /* same with bf16 hi+lo splits (kind::f16, bf16 inputs); a problem
                           whose schedule has more than 36 tensor-core steps stores its
                           operands as the scaled fp16 hi+lo of QFLEX_FP16X3 instead (16
                           significand bits per operand do not hold the amplitude within
                           1e-4 over longer chains of products); qflex_plan_info's
                           plane_format tells which */
  QFLEX_BF16_PLAIN = 3, /* one bf16 product per part (reported, not gated) */
  QFLEX_TF32_PLAIN = 4, /* one tf32 product per part (reported, not gated) */
  QFLEX_FP16X3 = 5      /* fp16 hi+lo splits (kind::f16, f16 inputs), 3 products, FP32
                           accumulate; each operand is first scaled by a power of two 2^s
                           chosen from its largest |re|, |im|, |re+im| (kept below 2^14),
                           and the product is rescaled exactly by 2^-(s_A+s_B) */
} qflex_precision;

/* Gate kinds (Methods, "Revised set of RQCs"; rotations R_P(t) = exp(-i t P/2)).
 * Two-qubit kinds act on a lattice edge and add bits to its bond: CZ 1 bit
 * (Schmidt rank 2), ISWAP = |00><00| + |11><11| + i|01><10| + i|10><01|
 * 2 bits (rank 4, Methods "Overview of the simulator"); a bond carries at
 * most 20 bits. */
enum {
  QFLEX_GATE_H = 0, QFLEX_GATE_T = 1, QFLEX_GATE_SX = 2, QFLEX_GATE_SY = 3,
  QFLEX_GATE_CZ = 4, QFLEX_GATE_RX = 5, QFLEX_GATE_RY = 6, QFLEX_GATE_RZ = 7,
  QFLEX_GATE_ISWAP = 8
};

/* One gate: cycle (time step, gates sorted by it), kind, qubits (q1 = -1 for
 * one-qubit gates), param = index into the angle vector for RX/RY/RZ, else -1. */
typedef struct {
  int32_t cycle, kind, q0, q1, param;
} qflex_gate;

typedef struct {
  int32_t n_qubits;
  const int32_t* edges;      /* host, [n_edges][2] qubit pairs (lattice bonds) */
  int32_t n_edges;
  const qflex_gate* gates;   /* host, [n_gates] */
  int64_t n_gates;
  int32_t n_params;          /* length of the angle vector */
} qflex_circuit;

/* Pairwise contraction order: steps[2i] = dst, steps[2i+1] = src; tensor q
 * starts as qubit q's grid tensor; the result of a step keeps the id dst. */
typedef struct {
  const int32_t* steps;      /* host, [n_steps][2] */
  int32_t n_steps;
} qflex_ordering;

typedef struct {
  const qflex_circuit* circuit;
  const qflex_ordering* ordering; /* NULL: qflex_search_ordering for these cuts, no cuts
                                     added, 32 trials, seed 0, limit 2^28 entries */
  const int32_t* cut_edges;       /* host, indices into circuit->edges; first = most
                                     significant digit of the slice id */
  int32_t n_cuts;
  const int32_t* open_tile;       /* host, qubit ids; amplitude index j has tile qubit t
                                     as bit (n_open-1-t) */
  int32_t n_open;
} qflex_problem;

typedef struct {
  int64_t n_slices;          /* P = prod over cuts of 2^{K_e} (Methods, "Cutting indexes") */
  int32_t n_qubits, n_params, n_open, n_steps;
  int64_t max_tensor_elems;  /* largest intermediate (complex entries) */
  size_t workspace_bytes;    /* device bytes owned by the plan */
  int32_t n_tc_steps;        /* steps whose GEMM runs on the tensor cores */
  int32_t n_persistent_buffers;
  int64_t n_nonzero_slices;  /* paths that do not vanish identically (qflex_nonzero_slices) */
  int32_t n_problems;        /* problems of the plan (qflex_plan_create) */
  int32_t plane_format;      /* operand planes of the tensor-core steps: 0 none (FP32), 1 tf32,
                                2 bf16, 3 power-of-two-scaled fp16 (see QFLEX_BF16X3) */
  size_t problem_workspace_bytes; /* this problem's part of workspace_bytes */
} qflex_plan_info;

/* Work of one qflex_amplitudes call, counted by replaying the schedule on the
 * host (reuse of slice-independent tensors included). */
typedef struct {
  double cmacs;              /* complex multiply-adds of all GEMMs (8 real flops each) */
  double tc_cmacs;           /* of which on the tensor cores */
  double tc_mma_flops;       /* real tensor-core flops executed (3M x splits) */
  double permute_bytes;      /* algorithmic bytes of operand permutations (read + write) */
  int64_t launches;          /* kernels launched */
  int64_t steps_executed;
  double largest_gemm_cmacs; /* M*N*K of the largest GEMM */
} qflex_cost;

/* One step of the plan's schedule (introspection; no counterpart in the
 * paper beyond its pairwise contraction steps, Methods "Matrix
 * multiplications"). */
typedef struct {
  int32_t dst, src;          /* tensor ids of the ordering step (result keeps dst) */
  int64_t M, N, K;           /* C[M][N] = sum_k A[M][k] B[N][k] */
  int32_t kernel;            /* 0 FP32 tiled, 1 FP32 thin (N <= 16), 2 FP32 thin (N <= 32),
                                3 FP32 block per row (few rows, long K), 4 tensor cores */
  int32_t bn;                /* tensor-core tile width (kernel 4) */
  int32_t a_direct, b_direct;/* operand read in place, without a permutation */
  int64_t runs;              /* executions in one call over n_bs bitstrings and the slices */
  int32_t a_cached, b_cached;/* operand kept in its own buffer and permuted only when its
                                source changes (it depends on fewer cuts than the step) */
  int64_t a_builds, b_builds;/* operand permutations run in that call */
  int32_t a_fused, b_fused;  /* operand planes written by the producing step's epilogue
                                (no permutation; not in gradient calls) */
  int32_t out_fused;         /* this step's epilogue writes its consumer's operand planes:
                                1 stores along its columns, 2 along its rows; 0 not fused */
  int32_t tc_wide;           /* kernel 4 with split operands: per k-step one MMA of width
                                2 bn over B hi and B lo ([hi.hi | hi.lo]) and one of width
                                bn (lo.hi) instead of three of width bn; chosen for bn = 64,
                                and for bn = 128 when K >= 256 */
} qflex_step_info;

int32_t qflex_abi_version(void);
const char* qflex_last_error(void);

/* Build a plan for n_problems independent problems (1 <= n_problems <=
 * 65536; the paper runs independent circuit instances, paths and batches as
 * separate jobs of one run, Methods "Simulation of RQCs on NASA HPC
 * clusters"; here they are one plan and one call).  Per problem: network
 * metadata (grid-tensor layouts, bond dimensions 2^{K_e}), cut/slice
 * indexing, ordering validation, per-step permutation and GEMM descriptors,
 * buffer reuse across paths (SI A: tensors independent of a cut are built
 * once and reused).  All problems share one device workspace (one
 * allocation, each problem a slice of it) and, when there are several, up to
 * 8 internal streams on which a call runs them concurrently.
 * problems: host, [n_problems] (their circuits, orderings, cuts and tiles
 * are copied; the caller may free them after the call).
 * workspace_bytes_max = 0 means no limit.  device < 0 builds a host-only plan
 * (no device memory, no CUDA calls) whose info/cost calls work and whose
 * amplitude calls return QFLEX_ERR_UNSUPPORTED; used to check plans on hosts
 * without a GPU.  Errors: QFLEX_ERR_ARG, QFLEX_ERR_CIRCUIT, QFLEX_ERR_PLAN,
 * QFLEX_ERR_OOM, QFLEX_ERR_CUDA (for a failing problem i > 0 of several the
 * message names i). */
qflex_status qflex_plan_create(const qflex_problem* problems, int32_t n_problems, qflex_precision prec,
                               size_t workspace_bytes_max, int device, qflex_plan* out);
void qflex_plan_destroy(qflex_plan plan);
/* Information on problem `problem` (0 <= problem < n_problems) of the plan;
 * workspace_bytes is the whole plan's. */
qflex_status qflex_plan_get_info(qflex_plan plan, int32_t problem, qflex_plan_info* info);

/* Cost of problem `problem`'s part of qflex_amplitudes(plan, ..., n_bs,
 * slice_ids, n_slice_ids, ...).  slice_ids: host, NULL = all slices. */
qflex_status qflex_plan_cost(qflex_plan plan, int32_t problem, int64_t n_bs, const int64_t* slice_ids,
                             int64_t n_slice_ids, qflex_cost* out);

/* The schedule's steps of problem `problem` for a call over n_bs bitstrings
 * and `slice_ids` (host, NULL = all): out[i] for i < min(cap, n_steps);
 * *n_steps = number of steps. */
qflex_status qflex_plan_steps(qflex_plan plan, int32_t problem, int64_t n_bs, const int64_t* slice_ids,
                              int64_t n_slice_ids, qflex_step_info* out, int32_t cap, int32_t* n_steps);

/* Automated cut and ordering search (the paper picks both by hand per
 * lattice: Methods "Cutting indexes", "Contraction of the 3D tensor network";
 * SI A).  Ordering: randomized greedy over the per-slice network (cut bonds
 * removed), best of `trials` passes: each step contracts the pair of live
 * tensors sharing a bond with the smallest log2(result) - alpha log2(larger
 * input) + beta log2(runs of the result) + tau * Gumbel noise, steps whose
 * result exceeds the limit last (pass 0: alpha = 1, beta = tau = 0; the
 * others draw alpha in [0, 1.5], tau in [0, 1] and, every second pass,
 * beta in [0, 2] from SplitMix64(seed)); the larger tensor keeps its id;
 * passes rank by the excess of their largest tensor over the limit, then by
 * work.  Cuts: starting from `cut_edges` (kept, in order), up to
 * `max_new_cuts` bonds are appended by a beam search (three cut sets per
 * level, same ranking) until the largest tensor has at most
 * max_tensor_elems entries; a level extends every set by one bond, or by
 * two bonds whose CZ projector halves share a diagonal stretch of one
 * qubit (tied bits: see qflex_nonzero_slices); the chosen set gets an
 * ordering search with 4 x trials.  Candidate sets are searched on the
 * host's cores (std::thread); the result does not depend on their number.  Work counts each step as often as the
 * executor runs it: once per change of the cuts it depends on, over the
 * paths that do not vanish identically (qflex_nonzero_slices).
 * circuit/open_tile/cut_edges: host, as in qflex_problem.  cuts_out: host,
 * capacity n_cuts + max_new_cuts; steps_out: host, capacity 2 (n_qubits - 1)
 * (dst, src) pairs, usable as a qflex_ordering.  Returns QFLEX_ERR_PLAN (with
 * the best result written) when the limit is not met. */
typedef struct {
  double log2_max_tensor;      /* log2 entries of the largest tensor */
  double cmacs_per_bitstring;  /* complex MACs of one bitstring over all slices, with reuse */
  double n_slices;             /* P of the cuts found */
  double n_nonzero_slices;     /* of which do not vanish identically */
  int32_t n_cuts;
  int32_t n_steps;
} qflex_search_result;
qflex_status qflex_search_ordering(const qflex_circuit* circuit, const int32_t* open_tile, int32_t n_open,
                                   const int32_t* cut_edges, int32_t n_cuts, int32_t max_new_cuts,
                                   int64_t max_tensor_elems, int32_t trials, uint64_t seed, int32_t* cuts_out,
                                   int32_t* steps_out, qflex_search_result* out);

/* Fraction-f path choice (Methods, "Summing a fraction of the paths"):
 * n_f = max(1, floor(f P + 1/2)) capped at P, the first n_f entries of a
 * Fisher-Yates shuffle of 0..P-1 driven by SplitMix64(seed), sorted.
 * slice_ids: host, capacity >= n_f. */
qflex_status qflex_select_slices(qflex_plan plan, int32_t problem, double fidelity, uint64_t seed,
                                 int64_t* slice_ids, int64_t capacity, int64_t* n_selected);

/* Paths that vanish identically.  A path fixes the cut bonds (Methods,
 * "Cutting indexes").  On one qubit, the CZ projector halves |k><k| (lower-
 * index qubit of each CZ) multiply through diagonal gates (T, R_Z, Z halves)
 * to zero unless their bits agree, and one met before the qubit's first
 * non-diagonal gate acts on |0> and needs k = 0.  A path that breaks this
 * contributes exactly zero for every bitstring and angle; qflex_amplitudes,
 * qflex_amplitudes_grad and qflex_plan_cost skip such paths, in `slice_ids`
 * lists as well.  qflex_nonzero_slices writes the other paths' ids in
 * ascending order.
 * slice_ids: host, capacity entries (may be NULL when capacity is 0).
 * *n_nonzero: their number, also set when capacity is too small
 * (QFLEX_ERR_ARG).  QFLEX_ERR_UNSUPPORTED above 2^32 paths. */
qflex_status qflex_nonzero_slices(qflex_plan plan, int32_t problem, int64_t* slice_ids, int64_t capacity,
                                  int64_t* n_nonzero);

/* Fraction-f path choice among the paths that do not vanish identically:
 * qflex_select_slices' rule over the P' entries of qflex_nonzero_slices'
 * list (n_f = max(1, floor(f P' + 1/2)) capped at P'), mapped to slice ids,
 * ascending.  slice_ids: host, capacity >= n_f. */
qflex_status qflex_select_nonzero_slices(qflex_plan plan, int32_t problem, double fidelity, uint64_t seed,
                                         int64_t* slice_ids, int64_t capacity, int64_t* n_selected);

/* Amplitudes of n_bs bitstrings of every problem, each with its open tile
 * enumerated:
 *   amps_out[b][j] = sum_{s in slice_ids} amp_s(x_b with tile bits j)
 * For a plan of several problems every array is the problems' arrays back
 * to back, problem 0 first: angles [sum_i n_params_i], bitstrings
 * [sum_i n_bs n_qubits_i], amps_out [sum_i n_bs 2^n_open_i]; slice_ids
 * apply to every problem (NULL: each problem's own P paths).
 * angles:     device, double [n_params] (may be NULL when n_params == 0)
 * bitstrings: device, uint8 [n_bs][n_qubits], one byte (0/1) per qubit; tile bits ignored
 * slice_ids:  host, int64 [n_slice_ids] distinct values in [0, P); NULL = all P slices
 * amps_out:   device, complex128 [n_bs][2^n_open], overwritten
 * Grid tensors and GEMMs run in the plan's precision; the slice sum is FP64.
 * Enqueued on `stream` (a cudaStream_t; NULL = legacy default stream); the
 * problems of a multi-problem plan run on its internal streams, forked from
 * `stream` and joined back to it before the call's work completes. */
qflex_status qflex_amplitudes(qflex_plan plan, const double* angles, const uint8_t* bitstrings,
                              int64_t n_bs, const int64_t* slice_ids, int64_t n_slice_ids,
                              double* amps_out, void* stream);

/* Allocate the workspace of qflex_amplitudes_grad (once per plan; later calls
 * return QFLEX_OK at once): dedicated buffers that keep every intermediate of
 * a slice for the reverse pass (checkpointed slice intermediates), their
 * cotangents, FP64 grid-tensor cotangents and reverse-GEMM scratch.  This is
 * the only plan call after qflex_plan_create that allocates device memory. */
qflex_status qflex_plan_enable_gradients(qflex_plan plan);

/* Amplitudes and the gradient of L = Re sum_{b,j} conj(g[b][j]) amps[b][j] with respect to
 * every angle (the paper has no gradients): environments of each grid tensor by the
 * reverse pass through the same pairwise contractions, summed over slices, then the
 * derivative of each grid tensor w.r.t. each rotation angle from prefix/suffix products of
 * its qubit's gate line.  grad_amps: device complex128 [n_bs][2^n_open] (g);
 * grad_angles: device double [n_params], overwritten; amps_out as in qflex_amplitudes.
 * Several problems: arrays back to back as in qflex_amplitudes (grad_amps as
 * amps_out, grad_angles as angles).
 * Requires qflex_plan_enable_gradients.  The reverse GEMMs run in the plan's precision;
 * grid-tensor cotangents and the angle gradients are summed in FP64. */
qflex_status qflex_amplitudes_grad(qflex_plan plan, const double* angles,
                                   const uint8_t* bitstrings, int64_t n_bs,
                                   const int64_t* slice_ids, int64_t n_slice_ids,
                                   const double* grad_amps, double* amps_out,
                                   double* grad_angles, void* stream);

/* Tile-shape autotuner: for every distinct contraction shape of the plan,
 * time the candidate kernel configurations on the plan's own workspace
 * (`reps` launches each, CUDA events, on a private stream) and keep the
 * fastest for all steps of that shape: tensor-core tile width BN in {128, 64},
 * and for narrow FP32 shapes (N <= 32) the row-per-thread thin kernel or the
 * tiled one.  Synchronous; call after qflex_plan_create and before any
 * capture.  n_shapes / gain_ms (may be NULL): shapes tuned and the estimated
 * time saved per pass over all steps against the default choice. */
qflex_status qflex_plan_autotune(qflex_plan plan, int32_t reps, int32_t* n_shapes, double* gain_ms);

/* CUDA-graph launch mode (enable != 0): a qflex_amplitudes / _grad call whose
 * arguments (pointers, n_bs, slice list) repeat those of the previous call is
 * captured into a CUDA graph on its second occurrence and replayed from then
 * on (one graph launch instead of thousands of kernel launches).  Inputs may
 * change contents between calls but not addresses.  Calls on the legacy
 * default stream (NULL) and calls while profiling run directly.  The first
 * call with new arguments runs directly, so kernel set-up happens outside
 * capture. */
qflex_status qflex_plan_use_graphs(qflex_plan plan, int32_t enable);

/* Per-kernel-class timing of a plan's launches, for roofline measurement.
 * Classes: 0 grid tensors, 1 permutation / operand producer, 2 FP32 GEMM,
 * 3 tensor-core GEMM, 4 slice sum.  mode != 0 is a bit mask of classes
 * (bit c = class c): it clears the totals and starts recording a CUDA event
 * pair around every launch of those classes in later qflex_amplitudes calls;
 * mode = 0 stops recording.  If out != NULL the call synchronizes the
 * recorded stream and returns the totals so far: launches, summed
 * event-to-event milliseconds, algorithmic flops (8 per complex MAC for the
 * GEMMs; `mma_flops` = real tensor-core flops executed) and algorithmic bytes
 * (permutation: entries read x 8 + operand bytes written). */
typedef struct {
  int64_t launches[5];
  double ms[5];
  double flops[5];
  double mma_flops[5];
  double bytes[5];
} qflex_profile;
qflex_status qflex_plan_profile(qflex_plan plan, int32_t mode, qflex_profile* out);

/* The GEMM launches of the profiled totals by product shape, for a roofline
 * per step kind (e.g. the region absorbs apart from the square products):
 * one record per (class, M, N, K, out_planes) of the class-2 and class-3
 * launches recorded since profiling was last started.  out_planes = 1 when
 * the epilogue wrote the next product's operand planes instead of complex64.
 * Call after qflex_plan_profile(plan, ., out != NULL) has read the recorded
 * events (else QFLEX_ERR_ARG).  Writes min(cap, count) records to the host
 * array out (caller-owned) in ascending (class, M, N, K) order and the count
 * to *n; cap = 0 with out = NULL queries the count.  Host-only plans:
 * QFLEX_ERR_UNSUPPORTED. */
typedef struct {
  int32_t cls;
  int32_t out_planes;
  int64_t M, N, K;
  int64_t launches;
  double ms;          /* summed event-to-event milliseconds */
  double mma_flops;   /* real tensor-core flops executed (class 3) */
} qflex_profile_shape;
qflex_status qflex_plan_profile_shapes(qflex_plan plan, qflex_profile_shape* out, int64_t cap, int64_t* n);

/* Synchronize the plan's last stream and report its device status word
 * (QFLEX_ERR_DEVICE_TIMEOUT if a bounded wait ran out; QFLEX_ERR_PLAN if a
 * fused epilogue computed a destination outside its operand planes, which
 * the kernel skipped); the word is cleared. */
qflex_status qflex_plan_sync(qflex_plan plan);

/* ---------------- standalone hot-path kernels (same kernels the plan runs) ---------------- */

/* Index permutation of a row-major complex64 tensor (Methods, "Cache-efficient index
 * permutations"): out axis i = in axis perm[i], i.e.
 *   out[j_0..j_{r-1}] = in[i] with i_{perm[a]} = j_a.
 * in, out: device, complex64, distinct non-overlapping buffers of prod(dims) entries.
 * dims, perm: host, [rank], rank <= 32.  Bit-exact (pure data movement).
 * Power-of-two dims take the shared-memory tiled kernel; others a gather kernel. */
qflex_status qflex_permute(const void* in, void* out, int32_t rank, const int64_t* dims,
                           const int32_t* perm, void* stream);

/* Complex GEMM C[m][n] = sum_k A[m][k] * B[n][k] (both operands K-contiguous),
 * A: device complex64 [M][K], B: device complex64 [N][K], C: device complex64 [M][N].
 * prec selects the arithmetic as in qflex_precision; tensor-core precisions need
 * K % 8 == 0 and M >= 128 (other shapes run on the FP32 path).  workspace: device,
 * at least qflex_cgemm_workspace_size() bytes (split operand planes). */
qflex_status qflex_cgemm_workspace_size(int32_t prec, int64_t M, int64_t N, int64_t K,
                                        size_t* bytes);
qflex_status qflex_cgemm(int32_t prec, int64_t M, int64_t N, int64_t K, const void* A,
                         const void* B, void* C, void* workspace, size_t workspace_bytes,
                         void* stream);

/* FP64 reduction sum_i |amps_i|^2 (Methods, "Summing a fraction of the paths": the
 * norm <psi~|psi~> and fidelity estimates).  amps: device complex128 [n];
 * out: device double [1], overwritten. */
qflex_status qflex_norm(const double* amps, int64_t n, double* out, void* stream);

/* Frugal rejection sampling over batches of amplitudes (Methods, "Fast sampling
 * technique"): for each batch (e.g. the 2^k open-tile amplitudes of one bitstring)
 * the entries are visited in a uniformly random order and entry j is accepted with
 * probability min(1, p_j N / M), p_j = |amp_j|^2, N = 2^n_qubits; the first
 * acceptance ends the batch (at most one per batch, which avoids correlations
 * inside a batch); the probability of a sample per batch is 1 - (1 - 1/M)^n_c.
 * Randomness: SplitMix64 stream per batch starting at seed + b * 0xD1B54A32D192ED03,
 * order by a forward Fisher-Yates walk (step k swaps entry k with entry
 * k + (x mod (n_c - k))), uniform u = (x >> 11) * 2^-53, acceptance u < p * (N / M)
 * with FP64 products rounded separately.
 * amps: device complex128 [n_batches][n_c], n_c <= 4096; accepted: device int32
 * [n_batches], the accepted index within the batch or -1. */
qflex_status qflex_frugal_sample(const double* amps, int64_t n_batches, int32_t n_c, int32_t n_qubits,
                                 double M, uint64_t seed, int32_t* accepted, void* stream);

/* Fidelity-f samples from perfect-fidelity amplitudes (Methods, "Fraction of
 * perfect fidelity amplitudes"): the output of a circuit run at fidelity f is
 * rho = f |psi><psi| + (1 - f) I / N, so each of the n_samples draws is, with
 * probability f, an exact sample of |psi> and otherwise a uniformly random
 * bitstring.  Exact samples are the batches that qflex_frugal_sample accepted,
 * used in batch order: the k-th exact draw takes the k-th accepted batch b,
 * i.e. batch_bits[b] with tile qubit t set to bit (n_tile - 1 - t) of
 * accepted[b].  Randomness: draw i runs a SplitMix64 stream from
 * seed + i * 0xD1B54A32D192ED03; its first value x gives u = (x >> 11) 2^-53
 * and the draw is exact when u < fidelity; a uniform draw takes qubit q from
 * bit 63 - (q mod 64) of value number 1 + q div 64 of the stream.
 * batch_bits: device uint8 [n_batches][n_qubits] (the bitstring each batch was
 * computed for; its tile bits are ignored); accepted: device int32 [n_batches]
 * from qflex_frugal_sample; tile: host int32 [n_tile] qubit ids (n_tile <= 30,
 * the plan's open tile order); samples: device uint8 [n_samples][n_qubits];
 * source: device int32 [n_samples], the batch of an exact draw, -1 for a
 * uniform draw, -2 for an exact draw past the accepted batches (bits zero).
 * *n_exact (host) = number of exact draws.  Uses stream-ordered scratch of
 * 4 * n_batches + 16 bytes and synchronizes the stream before returning.
 * Returns QFLEX_ERR_ARG (outputs written) when more exact draws are needed
 * than batches were accepted: compute more batches. */
qflex_status qflex_fidelity_samples(const uint8_t* batch_bits, const int32_t* accepted, int64_t n_batches,
                                    const int32_t* tile, int32_t n_tile, int32_t n_qubits, double fidelity,
                                    uint64_t seed, int64_t n_samples, uint8_t* samples, int32_t* source,
                                    int64_t* n_exact, void* stream);

/* Synchronize `device` and read (and clear) the library's device status word
 * used by the standalone kernels, together with the status and report words
 * of qflex_cgemm_noalloc on that device.  *status = QFLEX_ERR_DEVICE_TIMEOUT
 * if a bounded wait ran out, else QFLEX_ERR_PLAN if a fused store fell
 * outside its planes (the bits as qflex_plan_sync decodes them), else
 * QFLEX_OK. */
qflex_status qflex_device_status(int device, int32_t* status);

/* Self-test of failure detection (no counterpart in the paper): one CTA
 * waits, by the bounded-wait pattern of the tensor-core GEMM, on an mbarrier
 * that no one arrives at; after limit_ns (1e3 .. 1e9 ns) the wait gives up,
 * sets the timeout bit of the library's device status word and the kernel
 * returns.  Synchronizes `device`, clears the status word before and after;
 * *status = QFLEX_ERR_DEVICE_TIMEOUT when the wait ran out (the expected
 * outcome), QFLEX_OK otherwise.  The context stays usable.  The same wait
 * then runs out once more on the private status word of qflex_cgemm_noalloc
 * (set up on `device` if needed) and leaves its bit there, as a call of that
 * entry point whose wait ran out would: its next call still computes C, and
 * qflex_device_status reports QFLEX_ERR_DEVICE_TIMEOUT once for it. */
qflex_status qflex_device_selftest_timeout(int device, uint64_t limit_ns, int32_t* status);

/* ---------------- allocation-free complex GEMM ----------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory.  qflex_cgemm needs a workspace, and obtaining one
 * means cudaMalloc (or a library allocator), which may synchronize the whole
 * device and can fail under memory pressure: a serving loop that must not
 * stall other streams, or code embedded in a framework that owns every
 * device byte through its own pool, cannot do that.  This entry point
 * computes the same product as qflex_cgemm (same precisions, same kernels,
 * same results within the same tolerances) using a fixed scratch array that
 * is part of the library image instead of a caller workspace.
 *
 *  - Scratch limit: the split operand planes of A and B must fit in
 *    QFLEX_NOALLOC_SCRATCH_BYTES (64 MiB), i.e. (M + N) * K * 12 bytes for
 *    bf16 and fp16 split forms, (M + N) * K * 24 for tf32x3 (half that for the
 *    plain forms); larger tensor-core products return QFLEX_ERR_ARG.  The FP32
 *    precision needs no scratch and has no such limit.
 *  - Every GPU that loads the library's scratch holds these 64 MiB until the
 *    process exits.  The first call on a device (with that device current)
 *    looks up the scratch address and clears its status word; make that first
 *    call before any stream capture.
 *  - Every call shares the one scratch array: calls whose work overlaps on the
 *    GPU (different streams, or host threads) race and give wrong results;
 *    serialize them on one stream.  The planes are fully rewritten by each
 *    call, so leftover contents of an earlier call do not matter.
 *  - No cudaMalloc, cudaFree or allocating library routine is called.
 *  - A bounded device-side wait that runs out (a fault, not a normal
 *    condition) is recorded in a status word private to this entry point;
 *    the return value does not report it (that would need a host read and
 *    a stream synchronization per call).  Every tensor-core call starts
 *    with one stream-ordered thread that moves what earlier calls left in
 *    that word into a report word and clears it, so one timed-out call never
 *    makes later calls skip their work; qflex_device_status(device) reads
 *    and clears both words and returns QFLEX_ERR_DEVICE_TIMEOUT if any call
 *    since its last read timed out.
 *  - Sizes are checked before their products are formed: M or N above
 *    64 MiB / (plane bytes per entry x K) return QFLEX_ERR_ARG.
 * Arguments are those of qflex_cgemm without the workspace. */
#define QFLEX_NOALLOC_SCRATCH_BYTES (64ull << 20)
qflex_status qflex_cgemm_noalloc(int32_t prec, int64_t M, int64_t N, int64_t K, const void* A,
                                 const void* B, void* C, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* QFLEX_GB300_H */

/*
 * tn_gb300.h -- C ABI of the sliced sparse-state tensor-network contraction
 * (Pan, Chen, Zhang, "Solving the Sampling Problem of the Sycamore Quantum
 * Circuits", arXiv:2111.03011) on one GB300 GPU.
 *
 * What it computes.  A quantum circuit U is a tensor network (Method section):
 * |0> vectors on the initial boundary, a matrix per single-qubit gate and a
 * four-way tensor per two-qubit gate.  The final boundary is the sparse state
 * (Supplement, "The sparse-state method"): L groups, group g fixing every
 * non-open ("tail") qubit to the bits of tails[g] and leaving the h open qubits
 * free, so the result is the head tensor H[g][mu] of L x 2^h amplitudes,
 *     H[g][mu] = sum_{s in kept slices} <tails[g] (+) mu| U_s |0...0>,
 * where U_s is the network with the k sliced edges fixed to the bits of the
 * slice id s (Supplement, slicing).  Summing all 2^k slices gives the exact
 * amplitudes; summing a fraction f of them gives a state of fidelity ~ f
 * (Method, edge breaking; Supplement, slicing).  Samples are then drawn one
 * per group (Method, last paragraph).
 *
 * Conventions (the paper fixes none of these):
 *   - qubit q <-> bit q of a uint64 bitstring (LSB = qubit 0);
 *   - open index mu = sum_j bit(open_qubits[j]) << j;
 *   - group g = position of its tail in tails[]; tail bits on open qubits are ignored;
 *   - slice id s in [0, 2^k): sliced edge j (in the order given) takes (s >> j) & 1;
 *   - gate matrices: row = output, column = input; two-qubit basis |q0 q1>, q0 high bit.
 *
 * Ownership.  The library owns plans and heads.  A head may wrap a caller-owned
 * device buffer, which must outlive the head.  A plan must outlive its heads.
 * Errors.  Every call returns TN_OK (0) or a TN_ERR_* code and never aborts;
 * tn_last_error() gives a message for the calling thread's last failure.
 * Streams.  `stream` arguments are cudaStream_t values (NULL = legacy default
 * stream).  Calls that return host-visible results synchronise that stream.
 */
#ifndef TN_GB300_H
#define TN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TN_OK = 0,
  TN_ERR_INVALID = 1,       /* bad argument: qubit, edge, range, order, size */
  TN_ERR_OOM = 2,           /* size cap exceeded or device allocation failed */
  TN_ERR_NOT_IN_STATE = 3,  /* a requested bitstring's tail is not in tails[] */
  TN_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
  TN_ERR_CUDA = 5,          /* a CUDA runtime call failed */
  TN_ERR_UNSUPPORTED = 6    /* valid request this build does not implement */
};

enum { TN_EDGE_SLICE = 0, TN_EDGE_PIN = 1, TN_EDGE_COMPANION = 2 };
enum { TN_C64 = 0, TN_C128 = 1 };
/* GEMM-step engines: AUTO = TC_3XTF32.  TC_3XTF32: tcgen05, tf32 hi/lo split,
 * FP32-accurate (complex64 path, relative L2 <= 1e-5).  SIMT_FP32: CUDA-core
 * FP32 (the plain complex64 reference engine).  TC_BF16X3: tcgen05 kind::f16,
 * bf16 hi/lo split with FP32 accumulation, relative L2 <= 1e-4 (a precision
 * form with twice the tensor rate).  TC_FP16X3: tcgen05 kind::f16, fp16 hi/lo
 * split of each operand scaled by a power of two from its maximum (an extra
 * max pass per operand): fp16 and tf32 both carry 11 significant bits, so it
 * has the 3xTF32 accuracy (relative L2 <= 1e-5) at the kind::f16 rate. */
enum { TN_GEMM_AUTO = 0, TN_GEMM_TC_3XTF32 = 1, TN_GEMM_SIMT_FP32 = 2, TN_GEMM_TC_BF16X3 = 3, TN_GEMM_TC_FP16X3 = 4 };

/* One gate, in time order.  arity 1: re/im[0..3] hold the 2x2 matrix
 * (row-major, row = output); arity 2: re/im[0..15] hold the 4x4 matrix. */
typedef struct { int arity; int q0, q1; double re[16], im[16]; } tn_gate;
typedef struct { int n_qubits; int n_gates; const tn_gate* gates; } tn_circuit;

/* The sparse state: L = n_tails groups x 2^n_open members (Supplement, sparse
 * state; Results: 6 open qubits, 2^20 groups).  n_qubits <= 64, n_open <= 30. */
typedef struct {
  const int* open_qubits; int n_open;
  const uint64_t* tails; int64_t n_tails;
} tn_open_spec;

/* A cut edge: the wire entering gate `gate` on its q0 (leg 0) or q1 (leg 1).
 * SLICE: enumerated by the slice id (Supplement, slicing).
 * PIN:   fixed at `value` for every slice -- an edge broken by inserting
 *        E = (1,0)x(1,0) (value 0), each halving the fidelity estimate
 *        (Method, edge breaking); both inputs of one fSim pinned drill a hole.
 * COMPANION: slice the input leg like SLICE (it takes its slice bit) and, in the
 *        same slice, fix the partner qubit's output of the same two-qubit gate
 *        to the same value: the rank-one companion cut of Method case (ii)
 *        (pinning input a of an fSim to v keeps the partner output at v; the
 *        supplement's singular values of the sliced fSim).  It multiplies F_est
 *        by the kept norm fraction, (1 + sin^2 theta)/2 for an fSim. */
typedef struct { int gate; int leg; int kind; int value; } tn_edge;
typedef struct { int64_t begin, end; } tn_range;

typedef struct {
  double max_log2_elements;   /* cap on every intermediate, log2 complex64 elements (0: 28) */
  int    gemm;                /* TN_GEMM_*: GEMM-step engine (0: auto = tensor cores)         */
  int    host_only;           /* 1: plan on the host only (no device upload; inspect only)   */
  int    order_trials;        /* randomised greedy order restarts (0: 64)                   */
  uint64_t order_seed;        /* seed of those restarts                                      */
  int    max_host_absorb_log2;/* size cap of host-side absorption of order<=2 tensors (0: 12)*/
  int    small_max_bits;      /* contractions with <= this many contracted and new legs use the
                                 streaming small-operand kernel (0: 4; -1: none, all GEMM steps) */
  int    auto_slice;          /* 0: off.  Otherwise, when no order fits the cap, slice up to this
                                 many more wires (at most 24), chosen on the best over-cap order:
                                 each is the bond carried by the most over-cap intermediates
                                 (Supplement, slicing: sliced edges are those that cut the largest
                                 intermediates).  These internal edges take slice bits k, k+1, ...
                                 and are summed inside every user slice, so slice ids, F_est and
                                 the head are those of the k user edges, exactly. */
  int    host_fold_log2;      /* host folding: a contraction of the order whose operands are both
                                 host tensors (leaves or earlier folds) and whose result has at most
                                 2^this elements (and at most 2^6 slice variants) is done on the host
                                 in FP64 at plan time and becomes a leaf (0: 12; -1: off) */
  int    gemm_pair;           /* 0: 16-bit GEMM steps with 256-wide tiles and M >= 256 run on CTA pairs
                                 (cta_group::2, 256 x 256 tiles); -1: one-CTA 128-row tiles only.
                                 tn_plan_autotune times both and keeps the faster. */
  int    side_bprep;          /* 1: a large tensor-core B-preparation step (>= 64 MiB) whose operand
                                 is already written runs on a second stream beside the previous
                                 tensor-core GEMM if that GEMM is long (>= 2^34 complex MACs): an
                                 HBM-bound step next to a tensor-bound one; its operand and output
                                 stay allocated from that GEMM on.  0 (default): every step in order
                                 on the caller's stream; on the 30-qubit workload the side stream
                                 measured 5 % slower (the GEMM beside it slows by more than the
                                 preparation takes).  tn_profile_slices always runs in order. */
  int    tune_steps;          /* tn_plan_autotune only.  0: after choosing the order, tune every
                                 step's tile variant (tn_plan_tune_steps, 3 repetitions) when a
                                 pass (a slice, or 1/2^n_internal_sliced of it) takes at most 1 s;
                                 > 0: tune with this many repetitions whatever the time; -1: do not
                                 tune steps. */
} tn_plan_opts;

typedef struct tn_plan tn_plan_t;
typedef struct tn_head tn_head_t;

/* Per-plan figures for one slice. */
typedef struct {
  int     n_qubits, n_open;
  int64_t n_tails;            /* L */
  int64_t n_patterns;         /* distinct tails (rows of the final pattern axis) */
  int     n_sliced;           /* k */
  int     n_pinned;           /* PIN edges (each halves F_est) */
  int     n_leaves;           /* device leaves: tensors left after host simplification and folding */
  int     n_contractions;     /* pairwise contractions per slice */
  int     n_launches;         /* kernel launches per slice (steps incl. permutes/prep + accumulate) */
  double  tc_macs;            /* T_c: complex multiply-adds per slice (algorithmic) */
  double  alg_bytes;          /* algorithmic HBM bytes per slice (each operand read once, result written once) */
  double  max_log2_elements;  /* largest intermediate */
  int64_t workspace_bytes;    /* device arena of one slice */
  int     n_gemm_tc, n_gemm_simt, n_small, n_permute;  /* step counts by kernel kind */
  double  measured_slice_ms;  /* tn_plan_autotune: measured time of one slice (0 otherwise) */
  int     autotune_candidates;/* tn_plan_autotune: distinct orders timed */
  int     n_internal_sliced;  /* edges added by auto_slice; n_launches, tc_macs and alg_bytes count
                                 all 2^n_internal_sliced passes of one user slice */
  int     gemm_pair;          /* the plan's tn_plan_opts.gemm_pair (as chosen by tn_plan_autotune) */
  int     n_side_bprep;       /* B-preparation steps that run beside an earlier GEMM (side_bprep) */
  int     n_tuned_steps;      /* steps whose chosen tile variant is not the default (0: untuned) */
  double  tune_default_ms;    /* tn_plan_tune_steps: one pass of slice 0 with the variants it started from */
  double  tune_tuned_ms;      /* ... and with the variants it chose (the faster set is kept) */
} tn_plan_stats;

/* Plan the contraction (host).  `order`: n_pairs pairs (i, j) of leaf ids, the
 * result of contracting i and j stored at i (the convention of the paper's
 * contraction-order listing); NULL lets the greedy planner choose.  Leaf ids are
 * the tensors left after host simplification, see tn_plan_order().  Unless
 * opts->host_only, uploads leaves and step tables to the current device
 * (synchronous).  Errors: TN_ERR_INVALID for a bad circuit, qubit, edge or order;
 * TN_ERR_OOM if no order fits the cap. */
int tn_plan(const tn_circuit* circuit, const tn_open_spec* open_spec,
            const tn_edge* sliced_edges, int n_edges,
            const int32_t* order, int64_t n_pairs,
            const tn_plan_opts* opts, tn_plan_t** out);
void tn_plan_free(tn_plan_t* plan);
/* Autotuner: builds up to n_candidates plans whose orders come from greedy
 * searches with seeds opts->order_seed + c (each with opts->order_trials
 * restarts), times one slice of each distinct order on the current device
 * (CUDA events on `stream`, after one untimed slice), and returns the fastest
 * in *out (the others are freed).  Same arguments and errors as tn_plan. */
int tn_plan_autotune(const tn_circuit* circuit, const tn_open_spec* open_spec,
                     const tn_edge* sliced_edges, int n_edges, const tn_plan_opts* opts,
                     int n_candidates, void* stream, tn_plan_t** out);
int  tn_plan_get_stats(const tn_plan_t* plan, tn_plan_stats* out);

/* Per-step tile variants (the batched form's tuner of tile shapes and permute
 * schedules; the paper tunes nothing of this kind: its steps are PyTorch
 * calls, Results, implementation paragraph).  Every variant of a step computes
 * the same result; they differ only in how the kernel is tiled:
 *   tensor-core GEMM step: variant j picks the widest tile (real columns) and
 *     whether 256 x 256 CTA-pair tiles may be used, from (256, pairs),
 *     (256, one CTA), (128), (64), (32), keeping only choices that launch
 *     differently for this step's shape (fold of patterns side by side
 *     included); variant 0 is the default rule;
 *   permute step of >= 2^20 elements: tile schedules (input-run bits,
 *     output-run bits, tile bits) = (5, 5, 10) [default], (4, 6, 10),
 *     (6, 4, 10), (5, 5, 9), (4, 4, 8), duplicates removed, each followed
 *     by its four-outputs-per-store form where output bits 0 and 1 are bits
 *     of the tile;
 *   tensor-core B preparation of >= 2^20 elements (not beside a GEMM): the
 *     gather kernel and the permute kernel writing the real embedding, the
 *     permute first (variant 0) when the gather's loads would not coalesce;
 *   every other step: one variant.
 * tn_plan_step_variants gives step i's variant count and current choice
 * (steps as in tn_plan_step_info).  tn_plan_set_step_variant chooses one; it
 * drops the plan's captured graphs (they replay the old launches).  Errors:
 * TN_ERR_INVALID for a bad plan, step or variant. */
int  tn_plan_step_variants(const tn_plan_t* plan, int64_t i, int* n_variants, int* chosen);
int  tn_plan_set_step_variant(tn_plan_t* plan, int64_t i, int variant);
/* Tuner: times every variant of every step on the current device (one pass of
 * slice 0 per variant set, per-launch CUDA events on `stream`, in order, the
 * fastest of `reps` >= 1 repetitions after one untimed pass; variant v of
 * every step is timed in the same pass), chooses each step's fastest, then
 * times one pass of slice 0 (the whole slice unless the plan has
 * automatically sliced edges) with the starting and the chosen variants, in
 * the plan's own launch order (alternating, best of `reps`), and keeps the
 * faster set.  *default_ms / *tuned_ms (may be NULL) receive those two pass
 * times.  Synchronous; allocates a scratch
 * head; the plan's heads are not touched.  Errors: TN_ERR_INVALID for a
 * host-only plan, TN_ERR_CUDA, TN_ERR_TIMEOUT if a bounded wait gave up. */
int  tn_plan_tune_steps(tn_plan_t* plan, int reps, void* stream, double* default_ms, double* tuned_ms);
/* Copies up to `cap` pairs of the order used into pairs[2*i], pairs[2*i+1];
 * *n_pairs receives the full count. */
int  tn_plan_order(const tn_plan_t* plan, int32_t* pairs, int64_t cap, int64_t* n_pairs);
/* JSON description of leaves and steps (for tests and tooling); the string is
 * owned by the plan and valid until the next call on it. */
const char* tn_plan_describe(tn_plan_t* plan, int with_data);

/* Head tensor H[L][2^h] complex128 (row g = group).  dev_c128 = NULL: the head
 * allocates it; else it wraps the caller's device buffer of L*2^h complex128.
 * Zeroed on creation (synchronous). */
int  tn_head_create(tn_plan_t* plan, void* dev_c128, tn_head_t** out);
void tn_head_free(tn_head_t* head);
void* tn_head_data(tn_head_t* head);  /* device pointer of H */
/* Zero H (asynchronously on `stream`) and forget the accumulated slices. */
int  tn_head_reset(tn_head_t* head, void* stream);
/* F_est = 2^-n_pinned * slices_done / 2^k * prod over companion cuts of
 * their kept norm fraction (fidelity-estimate equation). */
int  tn_head_fidelity(const tn_head_t* head, double* f_est, int64_t* slices_done);
/* Override F_est for a head filled by the caller (not by contraction). */
int  tn_head_set_fidelity(tn_head_t* head, double f_est);

/* Contract slices [begin, end) and add them into the head (FP64).  Asynchronous
 * on `stream`.  A slice already accumulated into this head is rejected
 * (TN_ERR_INVALID) -- ranges are additive and may come from several calls.
 * If a launch fails part-way, the whole slices enqueued before it stay
 * recorded (a retry of the rest of the range is accepted; tn_last_error names
 * them); if the failure leaves a slice partly accumulated (between the passes
 * of an automatically sliced plan), the head becomes invalid: every later
 * call on it returns TN_ERR_INVALID until tn_head_reset.
 *
 * Bounded waits.  Every mbarrier wait of the tensor-core GEMM gives up after a
 * fixed number of polls and sets the plan's device status word instead of
 * hanging.  The calls that synchronise a stream for a head (tn_amplitudes,
 * tn_head_norm, tn_sample, tn_sample_ex) read that word after their own work;
 * a set word is cleared, the head marked invalid and TN_ERR_TIMEOUT returned.
 *
 * Fault injection (tests; host side only).  The environment variable
 * TN_FAULT_INJECT, read on every check, arms one fault: "alloc" (device
 * allocations of tn_plan and tn_head_create fail with TN_ERR_OOM before any
 * CUDA call), "slice:S" or "slice:S:T" (the contraction fails with
 * TN_ERR_CUDA before pass T, default 0, of user slice S), "status" (every
 * successful tn_contract_slices sets the plan's device status word, as a wait
 * that gave up would). */
int  tn_contract_slices(tn_plan_t* plan, tn_range slice_range, tn_head_t* head, void* stream);

/* Batched form.  tn_contract_slices_graph: the same result as
 * tn_contract_slices, but the range's launches are captured once into a CUDA
 * graph (cached per plan, range and head buffer) and replayed on `stream`.
 * tn_contract_batch: items (plans[i], ranges[i], heads[i]) as parallel
 * branches of one graph (items of the same plan share a branch, since they
 * share its workspace), so many small contractions overlap on the GPU; the
 * last batch's graph is cached per thread and replayed when the same batch is
 * submitted again.  Both asynchronous on `stream`; both reject slices already
 * accumulated into a head, and a batch rejects a head listed twice.  Items
 * with an empty range record nothing.  tn_contract_slices_graph keeps at most
 * 16 captured ranges per plan and drops the least recently replayed one. */
int  tn_contract_slices_graph(tn_plan_t* plan, tn_range slice_range, tn_head_t* head, void* stream);
int  tn_contract_batch(tn_plan_t* const* plans, const tn_range* ranges, tn_head_t* const* heads, int n,
                       void* stream);

/* out[i] = H[g(s_i)][mu(s_i)] for n bitstrings.  `bitstrings` and `out` may be
 * host or device pointers; dtype TN_C64 or TN_C128.  Synchronises `stream`.
 * TN_ERR_NOT_IN_STATE if a bitstring's tail is not a group (the first such
 * index is in tn_last_error()); `out` then holds 0 for those entries. */
int  tn_amplitudes(tn_head_t* head, const uint64_t* bitstrings, int64_t n,
                   void* out, int dtype, void* stream);

/* Draw n bitstrings: sample i from group i mod L, with probability
 * |H[g][mu]|^2 / sum_nu |H[g][nu]|^2 (exact categorical draw, the stationary law
 * of the paper's Metropolis chain), replaced with probability
 * 1 - target_fidelity / F_head by a uniform n_qubits-bit string (the noisy-state
 * mixture of the Supplement's slicing section).  target_fidelity <= 0 or
 * >= F_head: no mixing.  Random numbers: Philox-4x32-10 keyed by `seed`.
 * out_bitstrings may be host or device memory; synchronises `stream`. */
int  tn_sample(tn_head_t* head, int64_t n, double target_fidelity, uint64_t seed,
               uint64_t* out_bitstrings, void* stream);

/* Sampling methods of tn_sample_ex.
 *   EXACT: as tn_sample (exact in-group categorical draw).
 *   METROPOLIS: the paper's in-group Markov chain (Method, last paragraph;
 *     Supplement, validation): start at member 0, param proposals mu' uniform
 *     over the group (Philox counter (i, 2, t)), accept when u*w(mu) < w(mu'),
 *     w = |H|^2; param = 0 means l = 2^h proposals.
 *   FRUGAL: rejection sampling valid under Porter-Thomas (Supplement, bitstring
 *     choice): a uniform member (counter (i, 3, t)) is accepted when
 *     u*M*Z < w(mu)*l, Z the group's sum; at most 64*M rounds, the last
 *     candidate kept; param = M (0 means 10).
 * Uniform mixing for target_fidelity applies to every method as in tn_sample. */
enum { TN_SAMPLE_EXACT = 0, TN_SAMPLE_METROPOLIS = 1, TN_SAMPLE_FRUGAL = 2 };
int  tn_sample_ex(tn_head_t* head, int64_t n, double target_fidelity, uint64_t seed, int method, int64_t param,
                  uint64_t* out_bitstrings, void* stream);

/* ------------------------------------------------------------------ serving
 * A request server with continuous admission.  Circuits (a plan and its kept
 * slice range) are registered first.  Requests -- amplitude lookups or
 * samples on one circuit -- are queued by tn_server_submit and admitted by a
 * dispatcher thread into one of n_slots slots (each its own CUDA stream) as
 * soon as a slot is free and the circuit's head fits the HBM budget, so
 * requests arriving while others run overlap with them on the device.  The
 * first request on a circuit contracts its head (cached in HBM afterwards;
 * idle heads are evicted least-recently-used when a new one does not fit);
 * other requests on it wait for the head on the device.  Request buffers are
 * host memory and must stay valid until tn_server_wait returns.  Results are
 * those of tn_amplitudes / tn_sample_ex on the same head.  Plans registered
 * with a server must not be used by other calls while it runs. */
/* n_slots: 0 means 8.  hbm_budget_bytes: bytes of cached heads; 0 means the
 * device's free memory when the server is created, less 1 GiB.  Admission of
 * a new head also requires that much free device memory now (cudaMemGetInfo)
 * beyond a 1 GiB reserve; idle heads are evicted least-recently-used until
 * both hold. */
typedef struct { int n_slots; int64_t hbm_budget_bytes; } tn_server_opts;
typedef struct tn_server tn_server_t;
enum { TN_REQ_AMPLITUDES = 0, TN_REQ_SAMPLE = 1 };
typedef struct {
  int circuit;                 /* id from tn_server_add_circuit */
  int kind;                    /* TN_REQ_* */
  const uint64_t* bitstrings;  /* amplitudes: n bitstrings (host) */
  int64_t n;                   /* bitstrings, or samples */
  void* out;                   /* host: n amplitudes (dtype) or n uint64 samples */
  int dtype;                   /* amplitudes: TN_C64 / TN_C128 */
  double target_fidelity;      /* samples: as tn_sample */
  uint64_t seed;               /* samples */
  int method;                  /* samples: TN_SAMPLE_* */
  int64_t param;               /* samples: as tn_sample_ex */
} tn_request;
typedef struct { int status; double latency_us; double queue_us; } tn_request_result;
typedef struct {
  int64_t completed, failed, in_flight, queued;
  double p50_us, p99_us, mean_us;   /* submit -> result in the caller's buffer */
  int64_t heads_cached, head_bytes, evictions;
  double wall_s;
} tn_server_stats;
int  tn_server_create(const tn_server_opts* opts, tn_server_t** out);
int  tn_server_add_circuit(tn_server_t* server, tn_plan_t* plan, tn_range kept, int* circuit_id);
int  tn_server_submit(tn_server_t* server, const tn_request* request, uint64_t* ticket);
/* Blocks until the request is done; returns its status (TN_ERR_NOT_IN_STATE
 * for a bitstring outside the sparse state, with `out` holding 0 there). */
int  tn_server_wait(tn_server_t* server, uint64_t ticket, tn_request_result* result);
int  tn_server_get_stats(tn_server_t* server, tn_server_stats* out);
void tn_server_free(tn_server_t* server);   /* drains the queue first */

/* Linear and logarithmic cross-entropy benchmark of n samples against the
 * probabilities held by `ideal`, a head of exact amplitudes (all slices
 * kept): P(s) = |H(s)|^2, F_XEB = 2^n_qubits <P(s_i)> - 1 and
 * log 2^n_qubits + gamma + <log P(s_i)> (Supplement, validation: the XEB
 * formula and the logarithmic XEB; gamma = Euler's constant), with the sums
 * reduced in FP64 on the GPU.  samples: host or device uint64 bitstrings,
 * each in the sparse state (TN_ERR_NOT_IN_STATE otherwise).  Either output
 * may be NULL.  Synchronises `stream`. */
int  tn_xeb(tn_head_t* ideal, const uint64_t* samples, int64_t n, double* linear, double* log_xeb, void* stream);

/* Squared norm N = sum |H|^2 (FP64) and, if group_norms != NULL, the L
 * per-group sums (host memory).  Synchronises `stream`. */
int  tn_head_norm(tn_head_t* head, double* norm, double* group_norms, void* stream);

/* Tracing: like tn_contract_slices, but times every launch with CUDA events
 * on `stream` (synchronising once per 64 passes) and returns in step_ms[i] the
 * summed milliseconds of launch i of the per-pass launch list over the range
 * and every internal pass (i < n_launches >> n_internal_sliced of
 * tn_plan_stats; the last entry is the slice accumulation).  Accumulates
 * into the head like tn_contract_slices. */
int  tn_profile_slices(tn_plan_t* plan, tn_range slice_range, tn_head_t* head, void* stream,
                       double* step_ms, int64_t n_entries);
/* Kind (tn step kind: 0 small-operand, 1 permute, 2 B prep (tensor core),
 * 3 tensor-core GEMM, 4 B prep (SIMT), 5 SIMT GEMM, 6 operand max (FP16x3
 * scaling), -1 accumulation) and the
 * algorithmic complex multiply-adds and HBM bytes of launch i of one pass
 * (a slice runs 2^n_internal_sliced passes). */
int  tn_plan_step_info(const tn_plan_t* plan, int64_t i, int* kind, double* macs, double* bytes);

/* Largest group count tn_head_norm_noalloc accepts (its fixed scratch: 1 MiB). */
#define TN_NOALLOC_MAX_GROUPS 131072

/* tn_head_norm for callers that cannot allocate device memory -- for example
 * code running inside another framework that owns all device memory through
 * its own allocator, or a latency-critical loop where a cudaMalloc (which may
 * synchronise the device) is not allowed.  The paper has no counterpart; it is
 * an integration aid.
 *
 * Computes *norm_out = sum |H|^2 (FP64, same kernels and summation order as
 * tn_head_norm) for a complex128 head H[n_groups][2^n_open] in device memory.
 * norm_out is a device pointer; the call is asynchronous on `stream` and
 * allocates nothing (no cudaMalloc, no cudaFree, no allocating library call).
 * The per-group partial sums live in one fixed device array of
 * TN_NOALLOC_MAX_GROUPS doubles inside the library, which every GPU that loads
 * the library holds until the process exits; larger n_groups are rejected with
 * TN_ERR_INVALID.  A call looks up that array's device address with the
 * device current; outside a stream capture it does so on every call (so the
 * address stays right after cudaDeviceReset), inside a capture it uses the
 * address found by an earlier call on that device, so make the first call on
 * a device before any stream capture.  All calls share the array and it keeps the last
 * call's contents: calls whose kernels overlap on the GPU (different streams,
 * or different host threads) race on it, so serialise them. */
int  tn_head_norm_noalloc(const void* head_c128, int64_t n_groups, int n_open, double* norm_out, void* stream);

/* Standalone complex GEMM step (the contraction kernel of every GEMM step, the
 * K2 step of the contraction; Supplement complexity table, 8 flops per complex
 * multiply-add): C[p] = A[mapA(p)] B[mapB(p)] for p < PC, complex64, with
 * A [PA][M][K], B [PB][K][N] and C [PC][M][N] row-major device buffers.
 * M, N and K are powers of two (K >= 2 on the tensor-core engines; 16-bit
 * engines take K = 2 in tf32, as the planner does).  mapA / mapB are host
 * arrays of PC pattern indices, or NULL for the identity (P = PC) or pattern 0
 * (P = 1).  The operands pass through the same split permute, B preparation
 * and GEMM kernels as a plan's steps (engine TN_GEMM_*; pair as
 * tn_plan_opts.gemm_pair).  It allocates its
 * scratch (split planes, prepared B, tables) with cudaMalloc, frees it before
 * returning, and synchronises `stream`.  TN_ERR_TIMEOUT if a bounded device
 * wait gave up. */
int  tn_gemm_c64(int engine, const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K,
                 int64_t PA, int64_t PB, int64_t PC, const int32_t* mapA, const int32_t* mapB, int pair,
                 void* stream);

const char* tn_last_error(void);
const char* tn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TN_GB300_H */

// C ABI: plans, heads, slice contraction, amplitudes, sampling.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "handles.h"
#include "kernels.h"
#include "planner.h"
#include "tn_gb300.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(x)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) return fail(TN_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// NVTX range around a scope: a profiler (nsys, or ncu with --nvtx) sees each
// pass and each step's launch by name; without a tool attached the calls do
// nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

const char* step_range_name(int kind) {
  switch (kind) {
    case tn::ST_SMALL: return "tn small_operand";
    case tn::ST_PERMUTE: return "tn permute";
    case tn::ST_BPREP_TC: return "tn bprep_tc";
    case tn::ST_GEMM_TC: return "tn gemm_tc";
    case tn::ST_BPREP_C: return "tn bprep_simt";
    case tn::ST_GEMM_SIMT: return "tn gemm_simt";
    case tn::ST_ABSMAX: return "tn operand_max";
    default: return "tn step";
  }
}

}  // namespace

static const char* kVersion = "tn_gb300 0.1 (sm_103a)";

namespace tn {
// Lets other translation units of the library report through tn_last_error.
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace tn

namespace tn {
// Host-side fault injection: TN_FAULT_INJECT is read on every check, so a
// test can arm and disarm a fault between calls.
static std::string fault_env() {
  const char* e = std::getenv("TN_FAULT_INJECT");
  return e ? std::string(e) : std::string();
}
bool fault_alloc() { return fault_env() == "alloc"; }
bool fault_slice(int64_t s, int64_t t) {
  const std::string f = fault_env();
  if (f.rfind("slice:", 0) != 0) return false;
  long long S = -1, T = 0;
  if (std::sscanf(f.c_str() + 6, "%lld:%lld", &S, &T) < 1) return false;
  return s == S && t == T;
}
bool fault_status() { return fault_env() == "status"; }

// After the caller's stream is synchronised: a nonzero device status word of
// the plan means a bounded wait of a tensor-core GEMM gave up in some
// contraction of this plan since the last check.  The word is cleared, the
// head marked invalid and TN_ERR_TIMEOUT returned.
static int report_status(tn_head_t* h, unsigned int word, cudaStream_t st) {
  if (!word) return TN_OK;
  cudaMemsetAsync(h->plan->d_status, 0, sizeof(unsigned int), st);
  cudaStreamSynchronize(st);
  h->invalid = true;
  return fail(TN_ERR_TIMEOUT,
              "a bounded device wait in a contraction of this plan gave up (status " + std::to_string(word) +
                  "); the head is invalid until tn_head_reset");
}
}  // namespace tn

extern "C" const char* tn_last_error(void) { return g_err.c_str(); }
extern "C" const char* tn_version(void) { return kVersion; }

static void plan_release(tn_plan_t* p) {
  if (!p) return;
  if (p->on_device) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (p->device >= 0) cudaSetDevice(p->device);
    cudaFree(p->d_leaves);
    cudaFree(p->d_meta);
    cudaFree(p->d_arena);
    cudaFree(p->d_keys);
    cudaFree(p->d_key_groups);
    cudaFree(p->d_tails);
    cudaFree(p->d_open);
    cudaFree(p->d_status);
    cudaFree(p->d_scale);
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    for (auto& e : p->prof_events) cudaEventDestroy(e);
    for (auto& e : p->side_fork) if (e) cudaEventDestroy(e);
    for (auto& e : p->side_join) if (e) cudaEventDestroy(e);
    if (p->side_stream) cudaStreamDestroy(p->side_stream);
    if (cur >= 0) cudaSetDevice(cur);
  }
  delete p;
}

extern "C" void tn_plan_free(tn_plan_t* plan) { plan_release(plan); }

static int plan_upload(tn_plan_t* p) {
  tn::Plan& P = p->P;
  if (tn::fault_alloc()) return fail(TN_ERR_OOM, "device allocation failed (injected: TN_FAULT_INJECT=alloc)");
  CUDA_TRY(cudaGetDevice(&p->device));
  CUDA_TRY(tn::prepare_gemm_tc());
  CUDA_TRY(tn::prepare_permute());
  std::vector<float2> leaves(P.leaf_arena.size());
  for (size_t i = 0; i < leaves.size(); ++i)
    leaves[i] = make_float2((float)P.leaf_arena[i].real(), (float)P.leaf_arena[i].imag());
  p->on_device = true;
  CUDA_TRY(cudaMalloc(&p->d_leaves, std::max<size_t>(leaves.size(), 1) * sizeof(float2)));
  if (!leaves.empty())
    CUDA_TRY(cudaMemcpy(p->d_leaves, leaves.data(), leaves.size() * sizeof(float2), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(&p->d_meta, std::max<size_t>(P.meta.size(), 1) * sizeof(uint32_t)));
  if (!P.meta.empty())
    CUDA_TRY(cudaMemcpy(p->d_meta, P.meta.data(), P.meta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  if (P.workspace_bytes > 0) {
    cudaError_t e = cudaMalloc(&p->d_arena, (size_t)P.workspace_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TN_ERR_OOM, "workspace of " + std::to_string(P.workspace_bytes) + " bytes: " + cudaGetErrorString(e));
    }
  }
  // amplitude lookup table
  const size_t L = P.tails_raw.size();
  std::vector<std::pair<uint64_t, uint32_t>> kv(L);
  for (size_t g = 0; g < L; ++g) kv[g] = {P.tails_raw[g] & P.tail_mask, (uint32_t)g};
  std::sort(kv.begin(), kv.end());
  std::vector<uint64_t> keys(L);
  std::vector<uint32_t> grp(L);
  for (size_t i = 0; i < L; ++i) { keys[i] = kv[i].first; grp[i] = kv[i].second; }
  p->n_keys = (int64_t)L;
  CUDA_TRY(cudaMalloc(&p->d_keys, L * sizeof(uint64_t)));
  CUDA_TRY(cudaMalloc(&p->d_key_groups, L * sizeof(uint32_t)));
  CUDA_TRY(cudaMalloc(&p->d_tails, L * sizeof(uint64_t)));
  CUDA_TRY(cudaMemcpy(p->d_keys, keys.data(), L * sizeof(uint64_t), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(p->d_key_groups, grp.data(), L * sizeof(uint32_t), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(p->d_tails, P.tails_raw.data(), L * sizeof(uint64_t), cudaMemcpyHostToDevice));
  const size_t h = P.open_qubits.size();
  CUDA_TRY(cudaMalloc(&p->d_open, std::max<size_t>(h, 1) * sizeof(int)));
  if (h) CUDA_TRY(cudaMemcpy(p->d_open, P.open_qubits.data(), h * sizeof(int), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(&p->d_status, sizeof(unsigned int)));
  CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(unsigned int)));
  const size_t n_static = P.scale_static.size(), n_slots = n_static + (size_t)P.n_scale_slots;
  if (n_slots > 0) {
    CUDA_TRY(cudaMalloc(&p->d_scale, n_slots * sizeof(unsigned int)));
    CUDA_TRY(cudaMemset(p->d_scale, 0, n_slots * sizeof(unsigned int)));
    if (n_static)
      CUDA_TRY(cudaMemcpy(p->d_scale, P.scale_static.data(), n_static * sizeof(unsigned int), cudaMemcpyHostToDevice));
  }
  if (P.n_side_bprep > 0) {
    const size_t ns = P.steps.size();
    p->side_fork.assign(ns, nullptr);
    p->side_join.assign(ns, nullptr);
    p->forks_at.assign(ns, {});
    CUDA_TRY(cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking));
    for (size_t i = 0; i < ns; ++i) {
      const int f = P.steps[i].fork;
      if (f < 0) continue;
      if (f >= (int)i) return fail(TN_ERR_INVALID, "internal: side step forks after itself");
      p->forks_at[f].push_back((int)i);
      if (!p->side_fork[f]) CUDA_TRY(cudaEventCreateWithFlags(&p->side_fork[f], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&p->side_join[i], cudaEventDisableTiming));
    }
  }
  return TN_OK;
}

extern "C" int tn_plan(const tn_circuit* circuit, const tn_open_spec* open_spec, const tn_edge* sliced_edges,
                       int n_edges, const int32_t* order, int64_t n_pairs, const tn_plan_opts* opts,
                       tn_plan_t** out) {
  if (!out) return fail(TN_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!circuit || !open_spec) return fail(TN_ERR_INVALID, "circuit or open_spec is NULL");
  if (circuit->n_gates > 0 && !circuit->gates) return fail(TN_ERR_INVALID, "gates is NULL");
  if (open_spec->n_open < 0 || (open_spec->n_open > 0 && !open_spec->open_qubits))
    return fail(TN_ERR_INVALID, "bad open qubit list");
  if (open_spec->n_tails < 1 || !open_spec->tails) return fail(TN_ERR_INVALID, "need at least one tail");
  if (n_edges < 0 || (n_edges > 0 && !sliced_edges)) return fail(TN_ERR_INVALID, "bad edge list");
  if (order && n_pairs < 0) return fail(TN_ERR_INVALID, "n_pairs < 0");
  tn::PlanInput in;
  in.n_qubits = circuit->n_qubits;
  in.n_gates = circuit->n_gates;
  std::vector<int> ar(circuit->n_gates), q0(circuit->n_gates), q1(circuit->n_gates);
  std::vector<tn::cd> mats((size_t)circuit->n_gates * 16);
  for (int g = 0; g < circuit->n_gates; ++g) {
    const tn_gate& G = circuit->gates[g];
    ar[g] = G.arity;
    q0[g] = G.q0;
    q1[g] = G.q1;
    for (int e = 0; e < 16; ++e) mats[(size_t)g * 16 + e] = tn::cd(G.re[e], G.im[e]);
  }
  in.arity = ar.data();
  in.q0 = q0.data();
  in.q1 = q1.data();
  in.mats = mats.data();
  in.open_qubits.assign(open_spec->open_qubits, open_spec->open_qubits + open_spec->n_open);
  in.tails.assign(open_spec->tails, open_spec->tails + open_spec->n_tails);
  for (int e = 0; e < n_edges; ++e)
    in.edges.push_back({sliced_edges[e].gate, sliced_edges[e].leg, sliced_edges[e].kind, sliced_edges[e].value});
  in.order = order;
  in.n_pairs = order ? n_pairs : 0;
  bool host_only = false;
  if (opts) {
    if (opts->max_log2_elements > 0) in.cap_log2 = opts->max_log2_elements;
    in.gemm_engine = opts->gemm;
    host_only = opts->host_only != 0;
    if (opts->order_trials > 0) in.order_trials = opts->order_trials;
    if (opts->order_seed) in.order_seed = opts->order_seed;
    if (opts->max_host_absorb_log2 > 0) in.absorb_log2 = opts->max_host_absorb_log2;
    if (opts->small_max_bits != 0) in.small_max_bits = opts->small_max_bits < 0 ? -1 : std::min(4, opts->small_max_bits);
    if (opts->auto_slice < 0 || opts->auto_slice > 24) return fail(TN_ERR_INVALID, "auto_slice must be in [0, 24]");
    in.auto_slice = opts->auto_slice;
    if (opts->host_fold_log2 > 16) return fail(TN_ERR_INVALID, "host_fold_log2 must be at most 16");
    if (opts->host_fold_log2 != 0) in.fold_log2 = opts->host_fold_log2 < 0 ? -1 : opts->host_fold_log2;
    in.gemm_pair = opts->gemm_pair < 0 ? -1 : 0;
    in.side_bprep = opts->side_bprep > 0;
  }
  if (in.gemm_engine < 0 || in.gemm_engine > 4) return fail(TN_ERR_INVALID, "unknown gemm engine");
  if (in.cap_log2 > 34) return fail(TN_ERR_INVALID, "size cap above 2^34 elements");
  tn_plan_t* p = new tn_plan_t();
  std::string err;
  int rc = tn::build_plan(in, p->P, err);
  if (rc) {
    delete p;
    return fail(rc, err);
  }
  if (!host_only) {
    rc = plan_upload(p);
    if (rc) {
      plan_release(p);
      return rc;
    }
  }
  *out = p;
  return TN_OK;
}

extern "C" int tn_plan_get_stats(const tn_plan_t* plan, tn_plan_stats* s) {
  if (!plan || !s) return fail(TN_ERR_INVALID, "NULL argument");
  const tn::Plan& P = plan->P;
  std::memset(s, 0, sizeof(*s));
  s->n_qubits = P.n_qubits;
  s->n_open = (int)P.open_qubits.size();
  s->n_tails = (int64_t)P.tails_raw.size();
  s->n_patterns = P.n_patterns_final;
  s->n_sliced = P.n_sliced;
  s->n_pinned = P.n_pinned;
  s->n_leaves = (int)P.leaves.size();
  s->n_contractions = P.n_contractions;
  const double ni = std::ldexp(1.0, P.n_internal);
  s->n_launches = (int)(((int64_t)P.steps.size() + 1) << P.n_internal);
  s->tc_macs = P.tc_macs * ni;
  s->alg_bytes = P.alg_bytes * ni;
  s->n_internal_sliced = P.n_internal;
  s->gemm_pair = P.gemm_pair;
  s->n_side_bprep = P.n_side_bprep;
  s->max_log2_elements = P.max_log2;
  s->workspace_bytes = P.workspace_bytes;
  s->measured_slice_ms = plan->measured_slice_ms;
  s->autotune_candidates = plan->autotune_candidates;
  s->tune_default_ms = plan->tune_default_ms;
  s->tune_tuned_ms = plan->tune_tuned_ms;
  for (auto& st : P.steps) {
    if (st.variant != 0) ++s->n_tuned_steps;
    if (st.kind == tn::ST_GEMM_TC) ++s->n_gemm_tc;
    if (st.kind == tn::ST_GEMM_SIMT) ++s->n_gemm_simt;
    if (st.kind == tn::ST_SMALL) ++s->n_small;
    if (st.kind == tn::ST_PERMUTE) ++s->n_permute;
  }
  return TN_OK;
}

extern "C" int tn_plan_order(const tn_plan_t* plan, int32_t* pairs, int64_t cap, int64_t* n_pairs) {
  if (!plan || !n_pairs) return fail(TN_ERR_INVALID, "NULL argument");
  const auto& o = plan->P.order;
  *n_pairs = (int64_t)o.size();
  for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)o.size()); ++i) {
    pairs[2 * i] = o[i].first;
    pairs[2 * i + 1] = o[i].second;
  }
  return TN_OK;
}

extern "C" const char* tn_plan_describe(tn_plan_t* plan, int with_data) {
  if (!plan) return "";
  plan->P.describe_cache = tn::describe_plan(plan->P, with_data != 0);
  return plan->P.describe_cache.c_str();
}

// ----------------------------------------------------------------- heads

extern "C" int tn_head_create(tn_plan_t* plan, void* dev_c128, tn_head_t** out) {
  if (!plan || !out) return fail(TN_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (!plan->on_device) return fail(TN_ERR_INVALID, "plan was made host_only");
  if (tn::fault_alloc()) return fail(TN_ERR_OOM, "head allocation failed (injected: TN_FAULT_INJECT=alloc)");
  tn_head* h = new tn_head();
  h->plan = plan;
  const int64_t L = (int64_t)plan->P.tails_raw.size();
  const int64_t elems = L << plan->P.open_qubits.size();
  if (dev_c128) {
    h->H = (double2*)dev_c128;
  } else {
    cudaError_t e = cudaMalloc(&h->H, (size_t)elems * sizeof(double2));
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(TN_ERR_OOM, std::string("head allocation: ") + cudaGetErrorString(e));
    }
    h->owns = true;
  }
  cudaError_t e1 = cudaMemset(h->H, 0, (size_t)elems * sizeof(double2));
  if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(0);   // zeroed before any stream, blocking or not, uses it
  cudaError_t e2 = cudaMalloc(&h->d_Z, (size_t)std::max<int64_t>(L, 1) * sizeof(double));
  cudaError_t e3 = cudaMalloc(&h->d_N, sizeof(double));
  cudaError_t e4 = cudaMalloc(&h->d_status, sizeof(unsigned long long));
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
    cudaGetLastError();
    tn_head_free(h);
    return fail(TN_ERR_CUDA, "head set-up failed");
  }
  *out = h;
  return TN_OK;
}

extern "C" void tn_head_free(tn_head_t* h) {
  if (!h) return;
  if (h->owns) cudaFree(h->H);
  cudaFree(h->d_Z);
  cudaFree(h->d_N);
  cudaFree(h->d_status);
  cudaFree(h->d_stage);
  delete h;
}

extern "C" void* tn_head_data(tn_head_t* h) { return h ? (void*)h->H : nullptr; }

extern "C" int tn_head_reset(tn_head_t* h, void* stream) {
  if (!h) return fail(TN_ERR_INVALID, "NULL head");
  const int64_t elems = (int64_t)h->plan->P.tails_raw.size() << h->plan->P.open_qubits.size();
  CUDA_TRY(cudaMemsetAsync(h->H, 0, (size_t)elems * sizeof(double2), (cudaStream_t)stream));
  h->done.clear();
  h->slices_done = 0;
  h->f_override = false;
  h->invalid = false;
  return TN_OK;
}

extern "C" int tn_head_fidelity(const tn_head_t* h, double* f_est, int64_t* slices_done) {
  if (!h) return fail(TN_ERR_INVALID, "NULL head");
  const tn::Plan& P = h->plan->P;
  double f = h->f_override ? h->f_value
                           : std::ldexp((double)h->slices_done, -P.n_sliced) * std::ldexp(1.0, -P.n_pinned) *
                                 P.companion_factor;
  if (f_est) *f_est = f;
  if (slices_done) *slices_done = h->slices_done;
  return TN_OK;
}

extern "C" int tn_head_set_fidelity(tn_head_t* h, double f) {
  if (!h || !(f >= 0.0) || f > 1.0) return fail(TN_ERR_INVALID, "bad head or fidelity");
  h->f_override = true;
  h->f_value = f;
  return TN_OK;
}

// -------------------------------------------------------- slice execution

static inline const float2* ref_ptr(const tn_plan_t* p, const tn::Ref& r, int64_t s) {
  if (r.kind == 0) {
    const tn::LeafInfo& li = p->P.leaf_info[r.id];
    int64_t v = 0;
    for (size_t t = 0; t < li.var_slice_bits.size(); ++t) v |= ((s >> li.var_slice_bits[t]) & 1) << t;
    return p->d_leaves + li.off + v * li.size;
  }
  return (const float2*)(p->d_arena + p->P.bufs[r.id].off);
}

static inline float2* buf_ptr(const tn_plan_t* p, const tn::Ref& r) {
  return (float2*)(p->d_arena + p->P.bufs[r.id].off);
}

// FP16x3 scale slot -> device address (static slots first, then the per-pass ones)
static unsigned int* scale_ptr(const tn_plan_t* p, int slot) {
  if (slot == -1) return nullptr;
  const int64_t n_static = (int64_t)p->P.scale_static.size();
  return p->d_scale + (slot >= 0 ? n_static + slot : (int64_t)(-(slot + 2)));
}

// Launch one step of the launch list for the full slice id s on stream st
// (`side`: a B-prep beside a running GEMM, launched with one block per SM).
static cudaError_t launch_step(tn_plan_t* p, const tn::Step& x, int64_t s, cudaStream_t st, bool side) {
  const tn::Plan& P = p->P;
  NvtxRange range(step_range_name(x.kind));
  cudaError_t e = cudaSuccess;
  switch (x.kind) {
    case tn::ST_SMALL: {
      tn::SmallParams sp;
      sp.A = ref_ptr(p, x.a, s);
      sp.B = ref_ptr(p, x.b, s);
      sp.C = buf_ptr(p, x.c);
      sp.a_pstride = 1LL << x.rA;
      sp.b_pstride = 1LL << x.rB;
      sp.c_pstride = 1LL << x.rC;
      sp.M = 1LL << (x.rA - x.nk);
      sp.PC = x.PC;
      sp.rA = x.rA;
      sp.nk = x.nk;
      sp.nn = x.nn;
      for (int j = 0; j < 4; ++j) sp.kpos[j] = x.kposA[j];
      std::memcpy(sp.boffK, x.boffK, sizeof(sp.boffK));
      std::memcpy(sp.boffN, x.boffN, sizeof(sp.boffN));
      sp.mapA = p->d_meta + x.mapA_off;
      sp.mapB = p->d_meta + x.mapB_off;
      sp.mapA_mode = x.mapA_mode;
      sp.mapB_mode = x.mapB_mode;
      sp.amax = scale_ptr(p, x.max_slot);
      e = tn::launch_small(sp, st);
      break;
    }
    case tn::ST_PERMUTE: {
      tn::PermParams pp;
      pp.in = ref_ptr(p, x.a, s);
      pp.out = buf_ptr(p, x.c);
      pp.pstride = 1LL << x.rA;
      pp.P = x.PA;
      pp.t = x.t_bits;
      pp.n_rest = x.n_rest;
      std::memcpy(pp.rest_in, x.rest_in, sizeof(pp.rest_in));
      std::memcpy(pp.rest_out, x.rest_out, sizeof(pp.rest_out));
      pp.tab = p->d_meta + x.tab_off;
      pp.split = x.split;
      pp.scale = scale_ptr(p, x.slot);
      pp.vec4 = x.vec4;
      e = tn::launch_permute(pp, st);
      break;
    }
    case tn::ST_BPREP_C:
    case tn::ST_BPREP_TC: {
      if (x.kind == tn::ST_BPREP_TC && !x.alts.empty() && (x.variant == 0) == (x.bprep_embed0 != 0)) {
        // the permute kernel onto [N][K] order, writing the real embedding
        tn::PermParams pp;
        pp.in = ref_ptr(p, x.a, s);
        pp.out = buf_ptr(p, x.c);
        pp.pstride = 1LL << x.rA;
        pp.P = x.PA;
        pp.t = x.t_bits;
        pp.n_rest = x.n_rest;
        std::memcpy(pp.rest_in, x.rest_in, sizeof(pp.rest_in));
        std::memcpy(pp.rest_out, x.rest_out, sizeof(pp.rest_out));
        pp.tab = p->d_meta + x.tab_off;
        pp.split = 4 + x.h16;
        pp.scale = scale_ptr(p, x.slot);
        pp.embed_nk = x.nk;
        e = tn::launch_permute(pp, st);
        break;
      }
      tn::BPrepParams bp;
      bp.B = ref_ptr(p, x.a, s);
      bp.out = buf_ptr(p, x.c);
      bp.b_pstride = 1LL << x.rA;
      bp.PB = x.PA;
      bp.nk = x.nk;
      bp.nn = x.nn;
      bp.bk = p->d_meta + x.bk_off;
      bp.bn = p->d_meta + x.bn_off;
      bp.h16 = x.h16;
      bp.scale = scale_ptr(p, x.slot);
      e = x.kind == tn::ST_BPREP_C ? tn::launch_bprep_c(bp, st) : tn::launch_bprep_tc(bp, st, side);
      break;
    }
    case tn::ST_GEMM_SIMT:
    case tn::ST_GEMM_TC: {
      tn::GemmParams gp;
      gp.A = ref_ptr(p, x.a, s);
      gp.B = (const void*)ref_ptr(p, x.b, s);
      gp.C = buf_ptr(p, x.c);
      gp.M = 1LL << x.nm;
      gp.N = 1LL << x.nn;
      gp.K = 1LL << x.nk;
      gp.PA = x.PA;
      gp.PB = x.PB;
      gp.PC = x.PC;
      gp.mapA = p->d_meta + x.mapA_off;
      gp.mapB = p->d_meta + x.mapB_off;
      gp.mapA_mode = x.mapA_mode;
      gp.mapB_mode = x.mapB_mode;
      gp.h16 = x.h16;
      gp.scaleA = scale_ptr(p, x.slot);
      gp.scaleB = scale_ptr(p, x.slotB);
      gp.amax = scale_ptr(p, x.max_slot);
      gp.pair = P.gemm_pair < 0 ? -1 : x.pair;
      gp.tile_cap = x.tile_cap;
      e = x.kind == tn::ST_GEMM_SIMT ? tn::launch_gemm_simt(gp, st) : tn::launch_gemm_tc(gp, p->d_status, st);
      break;
    }
    case tn::ST_ABSMAX: {
      tn::AbsmaxParams ap;
      ap.in = ref_ptr(p, x.a, s);
      ap.n = x.PA << x.rA;
      ap.out = scale_ptr(p, x.slot);
      e = tn::launch_absmax(ap, st);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return e;
}

// One pass of the launch list for the full slice id s (user bits, then the
// bits of automatically sliced edges).  With per-launch timing events (ev)
// every step runs in order on st; otherwise a B-prep step with fork f is
// launched on the plan's side stream just before step f (after everything
// before f is done) and step f + ... waits for it right before the GEMM that
// consumes its output.
static int run_pass(tn_plan_t* p, int64_t s, double2* H, cudaStream_t st, cudaEvent_t* ev) {
  const tn::Plan& P = p->P;
  NvtxRange range("tn pass");
  if (P.n_scale_slots > 0) {
    cudaError_t e = cudaMemsetAsync(p->d_scale + P.scale_static.size(), 0,
                                    (size_t)P.n_scale_slots * sizeof(unsigned int), st);
    if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("scale reset: ") + cudaGetErrorString(e));
  }
  const bool use_side = !ev && p->side_stream != nullptr;
  std::vector<int> pending;      // side steps launched and not yet joined
  auto join_pending = [&]() {
    for (int j : pending) cudaStreamWaitEvent(st, p->side_join[j], 0);
    pending.clear();
  };
  int si = 0;
  for (const tn::Step& x : P.steps) {
    cudaError_t e = cudaSuccess;
    if (use_side && !p->forks_at[si].empty()) {
      e = cudaEventRecord(p->side_fork[si], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side_stream, p->side_fork[si], 0);
      for (int j : p->forks_at[si]) {
        if (e == cudaSuccess) e = launch_step(p, P.steps[j], s, p->side_stream, true);
        if (e == cudaSuccess) e = cudaEventRecord(p->side_join[j], p->side_stream);
        if (e == cudaSuccess) pending.push_back(j);
      }
      if (e != cudaSuccess) {
        join_pending();
        return fail(TN_ERR_CUDA, std::string("side launch: ") + cudaGetErrorString(e));
      }
    }
    if (ev) cudaEventRecord(ev[2 * si], st);
    if (use_side && x.fork >= 0) {
      // launched on the side stream before step x.fork: wait for it here
      e = cudaStreamWaitEvent(st, p->side_join[si], 0);
      pending.erase(std::remove(pending.begin(), pending.end(), si), pending.end());
    } else {
      e = launch_step(p, x, s, st, false);
    }
    if (e == cudaErrorInvalidValue && (x.kind < 0 || x.kind > tn::ST_ABSMAX)) {
      join_pending();
      return fail(TN_ERR_INVALID, "internal: unknown step kind");
    }
    if (e != cudaSuccess) {
      join_pending();
      return fail(TN_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    }
    if (ev) cudaEventRecord(ev[2 * si + 1], st);
    ++si;
  }
  join_pending();
  if (ev) cudaEventRecord(ev[2 * si], st);
  tn::AccumParams ap;
  ap.F = ref_ptr(p, P.fin.ref, s);
  ap.H = H;
  ap.f_pstride = 1LL << P.fin.rF;
  ap.L = (int64_t)P.tails_raw.size();
  ap.h = (int)P.open_qubits.size();
  ap.pidx = p->d_meta + P.fin.pidx_off;
  for (int j = 0; j < ap.h && j < 32; ++j) ap.open_pos[j] = P.fin.open_pos[j];
  cudaError_t e = tn::launch_accum(ap, st);
  if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("accumulate launch: ") + cudaGetErrorString(e));
  if (ev) cudaEventRecord(ev[2 * si + 1], st);
  return TN_OK;
}

// User slice s: every value t of the automatically sliced edges, slice id
// s | t << k, each pass accumulating into H.  *passes_done (if given) counts
// the passes enqueued whole: a failing pass fails before its accumulation
// launch, so exactly those passes reach H.
static int run_slice(tn_plan_t* p, int64_t s, double2* H, cudaStream_t st, int64_t* passes_done = nullptr) {
  const int64_t ni = 1LL << p->P.n_internal;
  for (int64_t t = 0; t < ni; ++t) {
    if (passes_done) *passes_done = t;
    if (tn::fault_slice(s, t))
      return fail(TN_ERR_CUDA, "injected failure before pass " + std::to_string(t) + " of slice " + std::to_string(s) +
                                   " (TN_FAULT_INJECT)");
    int rc = run_pass(p, s | (t << p->P.n_sliced), H, st, nullptr);
    if (rc) return rc;
  }
  if (passes_done) *passes_done = ni;
  return TN_OK;
}

static int check_range(tn_plan_t* plan, tn_range r, tn_head_t* head) {
  if (!plan || !head) return fail(TN_ERR_INVALID, "NULL argument");
  if (head->plan != plan) return fail(TN_ERR_INVALID, "head belongs to another plan");
  if (!plan->on_device) return fail(TN_ERR_INVALID, "plan was made host_only");
  if (head->invalid)
    return fail(TN_ERR_INVALID, "head is invalid after a failed or timed-out contraction; call tn_head_reset");
  const int64_t ns = 1LL << plan->P.n_sliced;
  if (r.begin < 0 || r.end > ns || r.begin > r.end) return fail(TN_ERR_INVALID, "slice range outside [0, 2^k)");
  auto it = head->done.upper_bound(r.begin);
  if (it != head->done.begin()) {
    auto pv = std::prev(it);
    if (pv->second > r.begin && r.begin < r.end)
      return fail(TN_ERR_INVALID, "slice range overlaps slices already accumulated");
  }
  if (it != head->done.end() && it->first < r.end)
    return fail(TN_ERR_INVALID, "slice range overlaps slices already accumulated");
  return TN_OK;
}

static void mark_done(tn_head_t* head, tn_range r) {
  if (r.begin >= r.end) return;   // an empty range records nothing (and must not replace [b, e))
  head->done[r.begin] = r.end;
  head->slices_done += r.end - r.begin;
}

extern "C" int tn_profile_slices(tn_plan_t* plan, tn_range r, tn_head_t* head, void* stream, double* step_ms,
                                 int64_t n_entries) {
  int rc = check_range(plan, r, head);
  if (rc) return rc;
  const int64_t ns = (int64_t)plan->P.steps.size() + 1;
  if (!step_ms || n_entries < ns) return fail(TN_ERR_INVALID, "step_ms needs n_launches entries");
  for (int64_t i = 0; i < ns; ++i) step_ms[i] = 0.0;
  if (r.begin == r.end) return TN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // events for up to kBatch passes, recorded back to back and read after one
  // synchronisation per batch (no host round trip between the passes of a batch)
  constexpr int64_t kBatch = 64;
  const int64_t ni = 1LL << plan->P.n_internal;
  const int64_t npass = (r.end - r.begin) * ni;
  const size_t need = (size_t)(2 * ns * std::min(npass, kBatch));
  auto& ev = plan->prof_events;
  while (ev.size() < need) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    ev.push_back(e);
  }
  int status = TN_OK;
  int64_t passes_run = 0;
  for (int64_t q0 = 0; q0 < npass && status == TN_OK; q0 += kBatch) {
    const int64_t nb = std::min(kBatch, npass - q0);
    for (int64_t j = 0; j < nb && status == TN_OK; ++j) {
      const int64_t q = r.begin * ni + q0 + j;
      const int64_t s = (q / ni) | ((q % ni) << plan->P.n_sliced);
      status = run_pass(plan, s, head->H, st, ev.data() + 2 * ns * j);
      if (status == TN_OK) ++passes_run;
    }
    if (status) break;
    cudaError_t e = cudaEventSynchronize(ev[(size_t)(2 * ns * nb - 1)]);
    if (e != cudaSuccess) { status = fail(TN_ERR_CUDA, cudaGetErrorString(e)); break; }
    for (int64_t j = 0; j < nb; ++j)
      for (int64_t i = 0; i < ns; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[(size_t)(2 * ns * j + 2 * i)], ev[(size_t)(2 * ns * j + 2 * i + 1)]);
        step_ms[i] += ms;
      }
  }
  if (status == TN_OK) mark_done(head, r);
  else if (passes_run > 0) head->invalid = true;   // H holds an unrecorded part of the range
  return status;
}

extern "C" int tn_plan_step_info(const tn_plan_t* plan, int64_t i, int* kind, double* macs, double* bytes) {
  if (!plan) return fail(TN_ERR_INVALID, "NULL plan");
  const int64_t ns = (int64_t)plan->P.steps.size();
  if (i < 0 || i > ns) return fail(TN_ERR_INVALID, "step index out of range");
  if (i == ns) {
    const tn::Plan& P = plan->P;
    const double L = (double)P.tails_raw.size(), l = std::ldexp(1.0, (int)P.open_qubits.size());
    if (kind) *kind = -1;
    if (macs) *macs = 0.0;
    if (bytes) *bytes = L * l * (8.0 + 32.0);   // read F (c64), read+write H (c128)
    return TN_OK;
  }
  const tn::Step& x = plan->P.steps[i];
  if (kind) *kind = x.kind;
  if (macs) *macs = x.macs;
  if (bytes) *bytes = x.bytes;
  return TN_OK;
}

// ------------------------------------------------ per-step tile variants

namespace {

struct GemmVariant {
  int cap, pair;
};
// widest tile (real columns) and CTA pairs allowed (0) or not (-1)
constexpr GemmVariant kGemmVariants[] = {{256, 0}, {256, -1}, {128, 0}, {64, 0}, {32, 0}};
constexpr int kNumGemmVariants = (int)(sizeof(kGemmVariants) / sizeof(kGemmVariants[0]));

// Indices into kGemmVariants of the choices that launch differently for the
// shape of tensor-core GEMM step x (independent of the plan-wide pair flag,
// so that a step's variant numbers never change).
std::vector<int> gemm_variants(const tn::Step& x) {
  std::vector<int> out;
  std::vector<tn::GemmTile> seen;
  for (int v = 0; v < kNumGemmVariants; ++v) {
    tn::GemmParams gp;
    gp.M = 1LL << x.nm;
    gp.N = 1LL << x.nn;
    gp.K = 1LL << x.nk;
    gp.PC = x.PC;
    gp.mapA_mode = x.mapA_mode;
    gp.h16 = x.h16;
    gp.pair = kGemmVariants[v].pair;
    gp.tile_cap = kGemmVariants[v].cap;
    const tn::GemmTile t = tn::gemm_tc_tile(gp);
    bool dup = false;
    for (const tn::GemmTile& q : seen) dup |= q.bn == t.bn && q.fold == t.fold && q.paired == t.paired;
    if (!dup) {
      seen.push_back(t);
      out.push_back(v);
    }
  }
  return out;
}

int step_variant_count(const tn::Step& x) {
  if (x.kind == tn::ST_GEMM_TC) return (int)gemm_variants(x).size();
  if (x.kind == tn::ST_PERMUTE) return std::max<int>(1, (int)x.alts.size());
  if (x.kind == tn::ST_BPREP_TC) return x.alts.empty() ? 1 : 2;
  return 1;
}

void apply_step_variant(tn::Step& x, int v) {
  x.variant = v;
  if (x.kind == tn::ST_GEMM_TC) {
    const GemmVariant& g = kGemmVariants[gemm_variants(x)[(size_t)v]];
    x.tile_cap = g.cap;
    x.pair = g.pair;
  } else if (x.kind == tn::ST_PERMUTE && !x.alts.empty()) {
    tn::apply_perm_schedule(x, x.alts[(size_t)v]);
  }
}

// Captured graphs replay the launches they recorded: drop them, and give the
// plan a new serial so that the batch graph cache (keyed on it) misses too.
void drop_graphs(tn_plan_t* p) {
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
  p->serial = tn::next_serial();
}

}  // namespace

extern "C" int tn_plan_step_variants(const tn_plan_t* plan, int64_t i, int* n_variants, int* chosen) {
  if (!plan) return fail(TN_ERR_INVALID, "NULL plan");
  if (i < 0 || i >= (int64_t)plan->P.steps.size()) return fail(TN_ERR_INVALID, "step index out of range");
  const tn::Step& x = plan->P.steps[(size_t)i];
  if (n_variants) *n_variants = step_variant_count(x);
  if (chosen) *chosen = x.variant;
  return TN_OK;
}

extern "C" int tn_plan_set_step_variant(tn_plan_t* plan, int64_t i, int variant) {
  if (!plan) return fail(TN_ERR_INVALID, "NULL plan");
  if (i < 0 || i >= (int64_t)plan->P.steps.size()) return fail(TN_ERR_INVALID, "step index out of range");
  tn::Step& x = plan->P.steps[(size_t)i];
  if (variant < 0 || variant >= step_variant_count(x)) return fail(TN_ERR_INVALID, "variant out of range");
  if (x.variant != variant) {
    apply_step_variant(x, variant);
    drop_graphs(plan);
  }
  return TN_OK;
}

extern "C" int tn_plan_tune_steps(tn_plan_t* plan, int reps, void* stream, double* default_ms, double* tuned_ms) {
  if (!plan) return fail(TN_ERR_INVALID, "NULL plan");
  if (!plan->on_device) return fail(TN_ERR_INVALID, "plan was made host_only");
  if (reps < 1 || reps > 64) return fail(TN_ERR_INVALID, "reps must be in [1, 64]");
  tn::Plan& P = plan->P;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ns = (int64_t)P.steps.size();
  std::vector<int> start(ns), count(ns);
  int max_v = 1;
  for (int64_t i = 0; i < ns; ++i) {
    start[i] = P.steps[i].variant;
    count[i] = step_variant_count(P.steps[i]);
    max_v = std::max(max_v, count[i]);
  }
  tn_head_t* h = nullptr;
  int rc = tn_head_create(plan, nullptr, &h);
  if (rc) return rc;
  auto& ev = plan->prof_events;
  while (ev.size() < (size_t)(2 * (ns + 1))) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      tn_head_free(h);
      return fail(TN_ERR_CUDA, "event creation failed");
    }
    ev.push_back(e);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    tn_head_free(h);
    return fail(TN_ERR_CUDA, "event creation failed");
  }
  auto set_all = [&](const std::vector<int>& v) {
    for (int64_t i = 0; i < ns; ++i)
      if (P.steps[i].variant != v[i]) apply_step_variant(P.steps[i], v[i]);
  };
  // 1. per-step times of variant v of every step (v past a step's count: its default)
  std::vector<double> best_ms(ns, 1e300);
  std::vector<int> best_v(start);
  for (int v = 0; v < max_v && rc == TN_OK; ++v) {
    std::vector<int> cur(ns);
    for (int64_t i = 0; i < ns; ++i) cur[i] = v < count[i] ? v : 0;
    set_all(cur);
    for (int r = 0; r <= reps && rc == TN_OK; ++r) {
      rc = run_pass(plan, 0, h->H, st, ev.data());
      if (rc) break;
      const cudaError_t e = cudaEventSynchronize(ev[(size_t)(2 * ns + 1)]);
      if (e != cudaSuccess) {
        rc = fail(TN_ERR_CUDA, std::string("tuning pass: ") + cudaGetErrorString(e));
        break;
      }
      if (r == 0) continue;   // untimed
      for (int64_t i = 0; i < ns; ++i) {
        if (v >= count[i]) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[(size_t)(2 * i)], ev[(size_t)(2 * i + 1)]);
        if (ms < best_ms[i]) {
          best_ms[i] = ms;
          best_v[i] = v;
        }
      }
    }
  }
  // 2. one pass of slice 0 each (a whole slice unless the plan has automatically
  // sliced edges) on the plan's own execution path, starting set against the
  // chosen one, alternating
  double t_start = 1e300, t_best = 1e300;
  for (int r = 0; r <= reps && rc == TN_OK; ++r)
    for (int which = 0; which < 2 && rc == TN_OK; ++which) {
      set_all(which == 0 ? start : best_v);
      cudaEventRecord(e0, st);
      rc = run_pass(plan, 0, h->H, st, nullptr);
      cudaEventRecord(e1, st);
      if (rc) break;
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        rc = fail(TN_ERR_CUDA, std::string("tuning slice: ") + cudaGetErrorString(e));
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 0) continue;   // untimed
      double& t = which == 0 ? t_start : t_best;
      t = std::min(t, (double)ms);
    }
  unsigned int word = 0;
  if (rc == TN_OK && cudaMemcpy(&word, plan->d_status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = fail(TN_ERR_CUDA, "status read-back failed");
  if (rc == TN_OK && word) {
    cudaMemset(plan->d_status, 0, sizeof(word));
    rc = fail(TN_ERR_TIMEOUT, "a bounded device wait gave up while tuning (status " + std::to_string(word) + ")");
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tn_head_free(h);
  const bool keep = rc == TN_OK && t_best < t_start;
  set_all(keep ? best_v : start);
  drop_graphs(plan);
  if (rc) return rc;
  plan->tune_default_ms = t_start;
  plan->tune_tuned_ms = t_best;
  if (default_ms) *default_ms = t_start;
  if (tuned_ms) *tuned_ms = t_best;
  return TN_OK;
}

extern "C" int tn_contract_slices(tn_plan_t* plan, tn_range r, tn_head_t* head, void* stream) {
  int rc = check_range(plan, r, head);
  if (rc) return rc;
  if (r.begin == r.end) return TN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t done_end = r.end;
  rc = tn::enqueue_slices(plan, r, head->H, st, &done_end);
  if (rc) {
    // the whole slices enqueued before the failure stay recorded (a retry of
    // the rest is accepted); a slice left partly accumulated invalidates H
    if (done_end < 0) {
      head->invalid = true;
      g_err += "; the head holds part of a slice and is invalid until tn_head_reset";
    } else {
      mark_done(head, {r.begin, done_end});
      g_err += "; slices [" + std::to_string(r.begin) + ", " + std::to_string(done_end) + ") were accumulated";
    }
    return rc;
  }
  mark_done(head, r);
  if (tn::fault_status())   // injected: as if a bounded wait of this contraction had given up
    CUDA_TRY(cudaMemsetAsync(plan->d_status, 1, sizeof(unsigned int), st));
  return TN_OK;
}

// ---------------------------------------------------------- CUDA graphs

// Capture the launches of `slices` of every (plan, head) item, item i on branch
// stream branch_of[i], into one graph (fork/join through events).
static int capture_items(const std::vector<tn_plan_t*>& plans, const std::vector<tn_range>& ranges,
                         const std::vector<tn_head_t*>& heads, const std::vector<int>& branch_of, int n_branches,
                         cudaGraphExec_t* exec_out) {
  static thread_local std::vector<cudaStream_t> streams;
  while ((int)streams.size() < n_branches + 1) {
    cudaStream_t st;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    streams.push_back(st);
  }
  cudaStream_t main = streams[0];
  std::vector<cudaEvent_t> ev(n_branches + 1);
  for (auto& e : ev) CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  CUDA_TRY(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
  int rc = TN_OK;
  cudaError_t ce = cudaEventRecord(ev[0], main);
  for (int b = 0; b < n_branches && ce == cudaSuccess; ++b) ce = cudaStreamWaitEvent(streams[1 + b], ev[0], 0);
  if (ce != cudaSuccess) rc = fail(TN_ERR_CUDA, std::string("graph fork: ") + cudaGetErrorString(ce));
  for (size_t i = 0; i < plans.size() && rc == TN_OK; ++i)
    for (int64_t s = ranges[i].begin; s < ranges[i].end && rc == TN_OK; ++s)
      rc = run_slice(plans[i], s, heads[i]->H, streams[1 + branch_of[i]]);
  for (int b = 0; b < n_branches && rc == TN_OK; ++b) {
    ce = cudaEventRecord(ev[1 + b], streams[1 + b]);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(main, ev[1 + b], 0);
    if (ce != cudaSuccess) rc = fail(TN_ERR_CUDA, std::string("graph join: ") + cudaGetErrorString(ce));
  }
  cudaGraph_t graph = nullptr;
  ce = cudaStreamEndCapture(main, &graph);
  if (rc == TN_OK && ce != cudaSuccess) rc = fail(TN_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(ce));
  if (rc == TN_OK) {
    ce = cudaGraphInstantiate(exec_out, graph, 0);
    if (ce != cudaSuccess) rc = fail(TN_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
  }
  if (graph) cudaGraphDestroy(graph);
  for (auto& e : ev) cudaEventDestroy(e);
  cudaGetLastError();
  return rc;
}

extern "C" int tn_contract_slices_graph(tn_plan_t* plan, tn_range r, tn_head_t* head, void* stream) {
  int rc = check_range(plan, r, head);
  if (rc) return rc;
  if (r.begin == r.end) return TN_OK;
  GraphEntry* hit = nullptr;
  for (auto& g : plan->graphs)
    if (g.begin == r.begin && g.end == r.end && g.H == (void*)head->H) hit = &g;
  if (!hit) {
    GraphEntry g;
    g.begin = r.begin;
    g.end = r.end;
    g.H = head->H;
    rc = capture_items({plan}, {r}, {head}, {0}, 1, &g.exec);
    if (rc) return rc;
    // bounded cache: the least recently replayed graph goes (an in-flight
    // executable graph is freed by CUDA once its launch completes)
    constexpr size_t kGraphCache = 16;
    if (plan->graphs.size() >= kGraphCache) {
      auto lru = std::min_element(plan->graphs.begin(), plan->graphs.end(),
                                  [](const GraphEntry& a, const GraphEntry& b) { return a.last_use < b.last_use; });
      cudaGraphExecDestroy(lru->exec);
      plan->graphs.erase(lru);
    }
    plan->graphs.push_back(g);
    hit = &plan->graphs.back();
  }
  hit->last_use = ++plan->graph_clock;
  CUDA_TRY(cudaGraphLaunch(hit->exec, (cudaStream_t)stream));
  mark_done(head, r);
  return TN_OK;
}

extern "C" int tn_contract_batch(tn_plan_t* const* plans, const tn_range* ranges, tn_head_t* const* heads, int n,
                                 void* stream) {
  if (n < 0 || (n > 0 && (!plans || !ranges || !heads))) return fail(TN_ERR_INVALID, "bad batch arrays");
  if (n == 0) return TN_OK;
  std::vector<tn_plan_t*> P(plans, plans + n);
  std::vector<tn_range> R(ranges, ranges + n);
  std::vector<tn_head_t*> Hs(heads, heads + n);
  std::vector<int> branch(n);
  std::map<tn_plan_t*, int> branch_of_plan;   // items of one plan share its arena: same branch
  std::map<tn_head_t*, int> head_seen;
  for (int i = 0; i < n; ++i) {
    int rc = check_range(P[i], R[i], Hs[i]);
    if (rc) return rc;
    if (head_seen.count(Hs[i])) return fail(TN_ERR_INVALID, "a head appears twice in one batch");
    head_seen[Hs[i]] = i;
    auto it = branch_of_plan.find(P[i]);
    if (it == branch_of_plan.end()) it = branch_of_plan.emplace(P[i], (int)branch_of_plan.size()).first;
    branch[i] = it->second;
  }
  const int n_branches = std::min<int>((int)branch_of_plan.size(), 32);
  for (int i = 0; i < n; ++i) branch[i] %= n_branches;
  // single-entry cache: the same batch again replays the same graph.  Keyed
  // on the handles' serials (never reused), not on their addresses.
  static thread_local std::vector<uint64_t> last_p;
  static thread_local std::vector<int64_t> last_r;
  static thread_local std::vector<uint64_t> last_h;
  static thread_local cudaGraphExec_t last_exec = nullptr;
  std::vector<int64_t> rr;
  for (auto& x : R) { rr.push_back(x.begin); rr.push_back(x.end); }
  std::vector<uint64_t> sp, sh;
  for (auto* x : P) sp.push_back(x->serial);
  for (auto* x : Hs) sh.push_back(x->serial);
  if (!(last_exec && last_p == sp && last_r == rr && last_h == sh)) {
    if (last_exec) cudaGraphExecDestroy(last_exec);
    last_exec = nullptr;
    int rc = capture_items(P, R, Hs, branch, n_branches, &last_exec);
    if (rc) { last_exec = nullptr; return rc; }
    last_p = sp;
    last_r = rr;
    last_h = sh;
  }
  CUDA_TRY(cudaGraphLaunch(last_exec, (cudaStream_t)stream));
  for (int i = 0; i < n; ++i) mark_done(Hs[i], R[i]);
  return TN_OK;
}

// ------------------------------------------------------ amplitudes, sampling

static int ensure_stage(tn_head* h, size_t bytes) {
  if (h->stage_bytes >= bytes) return TN_OK;
  cudaFree(h->d_stage);
  h->d_stage = nullptr;
  h->stage_bytes = 0;
  cudaError_t e = cudaMalloc(&h->d_stage, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(TN_ERR_OOM, "staging buffer allocation failed");
  }
  h->stage_bytes = bytes;
  return TN_OK;
}

extern "C" int tn_amplitudes(tn_head_t* h, const uint64_t* bitstrings, int64_t n, void* out, int dtype, void* stream) {
  if (!h || (n > 0 && (!bitstrings || !out))) return fail(TN_ERR_INVALID, "NULL argument");
  if (n < 0) return fail(TN_ERR_INVALID, "n < 0");
  if (dtype != TN_C64 && dtype != TN_C128) return fail(TN_ERR_INVALID, "dtype must be TN_C64 or TN_C128");
  if (h->invalid) return fail(TN_ERR_INVALID, "head is invalid after a failed or timed-out contraction");
  if (n == 0) return TN_OK;
  tn_plan_t* p = h->plan;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t esz = dtype == TN_C128 ? 16 : 8;
  const bool dev_in = is_device_ptr(bitstrings), dev_out = is_device_ptr(out);
  size_t need = 0;
  if (!dev_in) need += (size_t)n * 8;
  size_t out_off = (need + 255) / 256 * 256;
  if (!dev_out) need = out_off + (size_t)n * esz;
  if (need) {
    int rc = ensure_stage(h, need);
    if (rc) return rc;
  }
  const uint64_t* d_bits = bitstrings;
  if (!dev_in) {
    CUDA_TRY(cudaMemcpyAsync(h->d_stage, bitstrings, (size_t)n * 8, cudaMemcpyHostToDevice, st));
    d_bits = (const uint64_t*)h->d_stage;
  }
  void* d_out = dev_out ? out : (void*)((char*)h->d_stage + out_off);
  unsigned long long init = ~0ULL;
  CUDA_TRY(cudaMemcpyAsync(h->d_status, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  CUDA_TRY(tn::launch_amplitudes(h->H, (int)p->P.open_qubits.size(), p->d_keys, p->d_key_groups, p->n_keys,
                                 p->P.tail_mask, p->d_open, d_bits, n, d_out, dtype == TN_C128 ? 1 : 0, h->d_status,
                                 st));
  unsigned long long status = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, st));
  if (!dev_out) CUDA_TRY(cudaMemcpyAsync(out, d_out, (size_t)n * esz, cudaMemcpyDeviceToHost, st));
  unsigned int word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, p->d_status, sizeof(word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (int rc = tn::report_status(h, word, st)) return rc;
  if (status != ~0ULL)
    return fail(TN_ERR_NOT_IN_STATE, "bitstring " + std::to_string(status) + " has a tail that is not a group");
  return TN_OK;
}

extern "C" int tn_xeb(tn_head_t* h, const uint64_t* samples, int64_t n, double* linear, double* log_xeb,
                      void* stream) {
  if (!h || (n > 0 && !samples)) return fail(TN_ERR_INVALID, "NULL argument");
  if (n < 1) return fail(TN_ERR_INVALID, "n must be >= 1");
  if (h->invalid) return fail(TN_ERR_INVALID, "head is invalid after a failed or timed-out contraction");
  tn_plan_t* p = h->plan;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev_in = is_device_ptr(samples);
  // stage: [samples (host input)] [amplitudes c128] [partials] [2 sums]
  const size_t in_b = dev_in ? 0 : (size_t)n * 8;
  const size_t amp_off = (in_b + 255) / 256 * 256;
  const size_t part_off = amp_off + (size_t)n * 16;
  const size_t sums_off = part_off + (size_t)tn::xeb_partials(n) * 8;
  int rc = ensure_stage(h, sums_off + 16);
  if (rc) return rc;
  char* stg = (char*)h->d_stage;
  const uint64_t* d_bits = samples;
  if (!dev_in) {
    CUDA_TRY(cudaMemcpyAsync(stg, samples, in_b, cudaMemcpyHostToDevice, st));
    d_bits = (const uint64_t*)stg;
  }
  unsigned long long init = ~0ULL;
  CUDA_TRY(cudaMemcpyAsync(h->d_status, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  CUDA_TRY(tn::launch_amplitudes(h->H, (int)p->P.open_qubits.size(), p->d_keys, p->d_key_groups, p->n_keys,
                                 p->P.tail_mask, p->d_open, d_bits, n, stg + amp_off, 1, h->d_status, st));
  CUDA_TRY(tn::launch_xeb_sums((const double2*)(stg + amp_off), n, (double*)(stg + part_off),
                               (double*)(stg + sums_off), st));
  double sums[2] = {0.0, 0.0};
  unsigned long long status = 0;
  CUDA_TRY(cudaMemcpyAsync(sums, stg + sums_off, 16, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (status != ~0ULL)
    return fail(TN_ERR_NOT_IN_STATE, "sample " + std::to_string(status) + " has a tail that is not a group");
  const int nq = p->P.n_qubits;
  if (linear) *linear = std::ldexp(sums[0] / (double)n, nq) - 1.0;
  if (log_xeb) *log_xeb = nq * std::log(2.0) + 0.57721566490153286 + sums[1] / (double)n;
  return TN_OK;
}

extern "C" int tn_head_norm(tn_head_t* h, double* norm, double* group_norms, void* stream) {
  if (!h) return fail(TN_ERR_INVALID, "NULL head");
  if (h->invalid) return fail(TN_ERR_INVALID, "head is invalid after a failed or timed-out contraction");
  tn_plan_t* p = h->plan;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t L = (int64_t)p->P.tails_raw.size();
  CUDA_TRY(tn::launch_group_norms(h->H, L, (int)p->P.open_qubits.size(), h->d_Z, h->d_N, st));
  if (norm) CUDA_TRY(cudaMemcpyAsync(norm, h->d_N, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (group_norms) CUDA_TRY(cudaMemcpyAsync(group_norms, h->d_Z, (size_t)L * sizeof(double), cudaMemcpyDeviceToHost, st));
  unsigned int word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, p->d_status, sizeof(word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return tn::report_status(h, word, st);
}

static int sample_impl(tn_head_t* h, int64_t n, double target_fidelity, uint64_t seed, int method, int64_t param,
                       uint64_t* out, void* stream);

extern "C" int tn_sample(tn_head_t* h, int64_t n, double target_fidelity, uint64_t seed, uint64_t* out, void* stream) {
  return sample_impl(h, n, target_fidelity, seed, TN_SAMPLE_EXACT, 0, out, stream);
}

extern "C" int tn_sample_ex(tn_head_t* h, int64_t n, double target_fidelity, uint64_t seed, int method,
                            int64_t param, uint64_t* out, void* stream) {
  return sample_impl(h, n, target_fidelity, seed, method, param, out, stream);
}

static int sample_impl(tn_head_t* h, int64_t n, double target_fidelity, uint64_t seed, int method, int64_t param,
                       uint64_t* out, void* stream) {
  if (!h || (n > 0 && !out)) return fail(TN_ERR_INVALID, "NULL argument");
  if (method < TN_SAMPLE_EXACT || method > TN_SAMPLE_FRUGAL) return fail(TN_ERR_INVALID, "unknown sampling method");
  const int64_t l = 1LL << h->plan->P.open_qubits.size();
  if (method == TN_SAMPLE_METROPOLIS && param == 0) param = l;
  if (method == TN_SAMPLE_FRUGAL && param == 0) param = 10;
  if (param < 0 || (method == TN_SAMPLE_METROPOLIS && param > (1LL << 32)) ||
      (method == TN_SAMPLE_FRUGAL && param > (1LL << 20)))
    return fail(TN_ERR_INVALID, "sampling parameter out of range");
  if (n < 0) return fail(TN_ERR_INVALID, "n < 0");
  if (h->invalid) return fail(TN_ERR_INVALID, "head is invalid after a failed or timed-out contraction");
  if (n == 0) return TN_OK;
  tn_plan_t* p = h->plan;
  double f_head = 0.0;
  tn_head_fidelity(h, &f_head, nullptr);
  if (target_fidelity > f_head && target_fidelity > 0.0 && f_head > 0.0 && target_fidelity - f_head > 1e-15)
    return fail(TN_ERR_INVALID, "target fidelity above the head's estimated fidelity");
  double mix = 0.0;
  if (target_fidelity > 0.0 && f_head > 0.0 && target_fidelity < f_head) mix = 1.0 - target_fidelity / f_head;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev_out = is_device_ptr(out);
  uint64_t* d_out = out;
  if (!dev_out) {
    int rc = ensure_stage(h, (size_t)n * 8);
    if (rc) return rc;
    d_out = (uint64_t*)h->d_stage;
  }
  tn::SampleParams sp;
  sp.H = h->H;
  sp.L = (int64_t)p->P.tails_raw.size();
  sp.h = (int)p->P.open_qubits.size();
  sp.tails = p->d_tails;
  sp.open_mask = p->P.open_mask;
  sp.open_q = p->d_open;
  sp.n_qubits = p->P.n_qubits;
  sp.n = n;
  sp.mix = mix;
  sp.seed = seed;
  sp.out = d_out;
  sp.method = method;
  sp.param = param;
  CUDA_TRY(tn::launch_sample(sp, st));
  if (!dev_out) CUDA_TRY(cudaMemcpyAsync(out, d_out, (size_t)n * 8, cudaMemcpyDeviceToHost, st));
  unsigned int word = 0;
  CUDA_TRY(cudaMemcpyAsync(&word, p->d_status, sizeof(word), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return tn::report_status(h, word, st);
}

namespace tn {
int enqueue_slices(tn_plan_t* plan, tn_range r, double2* H, cudaStream_t stream, int64_t* done_end) {
  for (int64_t s = r.begin; s < r.end; ++s) {
    int64_t t = 0;
    int rc = run_slice(plan, s, H, stream, &t);
    if (rc) {
      if (done_end) *done_end = t == 0 ? s : -1;
      return rc;
    }
  }
  if (done_end) *done_end = r.end;
  return TN_OK;
}
int check_slice_range(tn_plan_t* plan, tn_range r, tn_head_t* head) { return check_range(plan, r, head); }
void mark_slices_done(tn_head_t* head, tn_range r) { mark_done(head, r); }
}  // namespace tn

// ------------------------------------------------------- standalone GEMM

extern "C" int tn_gemm_c64(int engine, const void* A, const void* B, void* C, int64_t M, int64_t N, int64_t K,
                           int64_t PA, int64_t PB, int64_t PC, const int32_t* mapA, const int32_t* mapB, int pair,
                           void* stream) {
  if (engine == TN_GEMM_AUTO) engine = TN_GEMM_TC_3XTF32;
  if (engine < TN_GEMM_TC_3XTF32 || engine > TN_GEMM_TC_FP16X3) return fail(TN_ERR_INVALID, "unknown gemm engine");
  if (!A || !B || !C) return fail(TN_ERR_INVALID, "NULL operand");
  auto pow2 = [](int64_t x) { return x >= 1 && (x & (x - 1)) == 0; };
  if (!pow2(M) || !pow2(N) || !pow2(K)) return fail(TN_ERR_INVALID, "M, N and K must be powers of two");
  if (PA < 1 || PB < 1 || PC < 1) return fail(TN_ERR_INVALID, "pattern counts must be >= 1");
  if (M * K > (1LL << 32) || K * N > (1LL << 32) || M * N > (1LL << 32))
    return fail(TN_ERR_INVALID, "operand above 2^32 elements");
  const bool simt = engine == TN_GEMM_SIMT_FP32;
  int nk = 0, nn = 0, nmk = 0;
  while ((1LL << nk) < K) ++nk;
  while ((1LL << nn) < N) ++nn;
  while ((1LL << nmk) < M * K) ++nmk;
  if (!simt && nk < 1) return fail(TN_ERR_INVALID, "tensor-core engines need K >= 2");
  // like the planner: 16-bit operands need K >= 4 (16-byte rows); K = 2 uses tf32
  const int h16 = simt ? 0 : nk >= 2 ? (engine == TN_GEMM_TC_BF16X3 ? 1 : engine == TN_GEMM_TC_FP16X3 ? 2 : 0) : 0;
  // pattern maps: a table of PC entries, or identity (P == PC) / all zero (P == 1)
  int mode[2];
  std::vector<uint32_t> maps[2];
  const int32_t* user[2] = {mapA, mapB};
  const int64_t PX[2] = {PA, PB};
  for (int x = 0; x < 2; ++x) {
    if (user[x]) {
      mode[x] = 2;
      for (int64_t p = 0; p < PC; ++p) {
        if (user[x][p] < 0 || user[x][p] >= PX[x]) return fail(TN_ERR_INVALID, "pattern map entry out of range");
        maps[x].push_back((uint32_t)user[x][p]);
      }
    } else if (PX[x] == PC) {
      mode[x] = 0;
    } else if (PX[x] == 1) {
      mode[x] = 1;
    } else {
      return fail(TN_ERR_INVALID, "a pattern count differs from PC and no map is given");
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(tn::prepare_gemm_tc());   // kernel attributes (shared-memory size), as at plan upload
  CUDA_TRY(tn::prepare_permute());
  // scratch: split A planes, prepared B, tables, scale slots
  const int64_t es = h16 ? 2 : 4;
  const int split = simt ? 0 : (h16 == 2 ? 3 : h16 == 1 ? 2 : 1);
  const int64_t a_bytes = simt ? 0 : PA * M * K * 8 * (split == 1 ? 2 : 1);
  const int64_t b_bytes = simt ? PB * K * N * 8 : 2 * PB * (2 * N) * (2 * K) * es;
  const int t = std::min(nmk, 10);
  std::vector<uint32_t> meta;
  const size_t tab_off = meta.size();
  for (int i = 0; i < (1 << t); ++i) meta.push_back((uint32_t)i);   // identity tile: in offsets
  for (int i = 0; i < (1 << t); ++i) meta.push_back((uint32_t)i);   // out offsets
  for (int i = 0; i < (1 << t); ++i) meta.push_back((uint32_t)i);   // slots
  const size_t bk_off = meta.size();
  for (int64_t k = 0; k < K; ++k) meta.push_back((uint32_t)(k * N));
  const size_t bn_off = meta.size();
  for (int64_t n = 0; n < N; ++n) meta.push_back((uint32_t)n);
  const size_t map_off[2] = {meta.size(), meta.size() + maps[0].size()};
  meta.insert(meta.end(), maps[0].begin(), maps[0].end());
  meta.insert(meta.end(), maps[1].begin(), maps[1].end());
  char* a_split = nullptr;
  char* b_prep = nullptr;
  uint32_t* d_meta = nullptr;
  unsigned int* d_scale = nullptr;   // [0] max of A, [1] max of B, [2] status
  int rc = TN_OK;
  auto cleanup = [&]() {
    cudaFree(a_split);
    cudaFree(b_prep);
    cudaFree(d_meta);
    cudaFree(d_scale);
  };
  if ((a_bytes && cudaMalloc(&a_split, (size_t)a_bytes) != cudaSuccess) ||
      cudaMalloc(&b_prep, (size_t)b_bytes) != cudaSuccess ||
      cudaMalloc(&d_meta, meta.size() * sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&d_scale, 3 * sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(TN_ERR_OOM, "tn_gemm_c64 scratch allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(d_meta, meta.data(), meta.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_scale, 0, 3 * sizeof(unsigned int), st);
  if (e == cudaSuccess && h16 == 2) {
    tn::AbsmaxParams ap{(const float2*)A, PA * M * K, d_scale};
    e = tn::launch_absmax(ap, st);
    if (e == cudaSuccess) {
      tn::AbsmaxParams bp{(const float2*)B, PB * K * N, d_scale + 1};
      e = tn::launch_absmax(bp, st);
    }
  }
  if (e == cudaSuccess && !simt) {   // A -> split planes (identity bit permutation)
    tn::PermParams pp;
    pp.in = (const float2*)A;
    pp.out = (float2*)a_split;
    pp.pstride = M * K;
    pp.P = PA;
    pp.t = t;
    pp.n_rest = nmk - t;
    for (int x = 0; x < pp.n_rest; ++x) pp.rest_in[x] = pp.rest_out[x] = (uint8_t)(t + x);
    pp.tab = d_meta + tab_off;
    pp.split = split;
    pp.scale = d_scale;
    e = tn::launch_permute(pp, st);
  }
  if (e == cudaSuccess) {   // B -> real embedding (tensor cores) or [K][N] copy (CUDA cores)
    tn::BPrepParams bp;
    bp.B = (const float2*)B;
    bp.out = b_prep;
    bp.b_pstride = K * N;
    bp.PB = PB;
    bp.nk = nk;
    bp.nn = nn;
    bp.bk = d_meta + bk_off;
    bp.bn = d_meta + bn_off;
    bp.h16 = h16;
    bp.scale = d_scale + 1;
    e = simt ? tn::launch_bprep_c(bp, st) : tn::launch_bprep_tc(bp, st);
  }
  if (e == cudaSuccess) {
    tn::GemmParams gp;
    gp.A = simt ? (const float2*)A : (const float2*)a_split;
    gp.B = b_prep;
    gp.C = (float2*)C;
    gp.M = M;
    gp.N = N;
    gp.K = K;
    gp.PA = PA;
    gp.PB = PB;
    gp.PC = PC;
    gp.mapA = d_meta + map_off[0];
    gp.mapB = d_meta + map_off[1];
    gp.mapA_mode = mode[0];
    gp.mapB_mode = mode[1];
    gp.h16 = h16;
    gp.scaleA = d_scale;
    gp.scaleB = d_scale + 1;
    gp.amax = nullptr;
    gp.pair = pair < 0 ? -1 : 0;
    e = simt ? tn::launch_gemm_simt(gp, st) : tn::launch_gemm_tc(gp, d_scale + 2, st);
  }
  unsigned int word = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&word, d_scale + 2, sizeof(word), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    rc = fail(TN_ERR_CUDA, std::string("tn_gemm_c64: ") + cudaGetErrorString(e));
  } else if (word) {
    rc = fail(TN_ERR_TIMEOUT, "tn_gemm_c64: a bounded device wait gave up");
  }
  cleanup();
  return rc;
}

extern "C" int tn_plan_autotune(const tn_circuit* circuit, const tn_open_spec* open_spec, const tn_edge* sliced_edges,
                                int n_edges, const tn_plan_opts* opts, int n_candidates, void* stream,
                                tn_plan_t** out) {
  if (!out) return fail(TN_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n_candidates < 1 || n_candidates > 64) return fail(TN_ERR_INVALID, "n_candidates must be in [1, 64]");
  tn_plan_opts o{};
  if (opts) o = *opts;
  if (o.host_only) return fail(TN_ERR_INVALID, "autotuning needs the device");
  const uint64_t seed0 = o.order_seed ? o.order_seed : 1;
  cudaStream_t st = (cudaStream_t)stream;
  tn_plan_t* best = nullptr;
  double best_ms = 1e300;
  int distinct = 0;
  std::vector<std::vector<std::pair<int, int>>> seen;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int last_rc = TN_OK;
  for (int c = 0; c < n_candidates; ++c) {
    o.order_seed = seed0 + (uint64_t)c;
    tn_plan_opts ho = o;
    ho.host_only = 1;
    tn_plan_t* hp = nullptr;
    int rc = tn_plan(circuit, open_spec, sliced_edges, n_edges, nullptr, 0, &ho, &hp);
    if (rc) { last_rc = rc; continue; }
    bool dup = false;
    for (auto& s_ : seen) dup |= s_ == hp->P.order;
    if (dup) { tn_plan_free(hp); continue; }
    seen.push_back(hp->P.order);
    // upload this candidate (its edges include any automatically sliced ones)
    tn_plan_t* p = hp;
    rc = plan_upload(p);
    if (rc) { plan_release(p); last_rc = rc; continue; }
    ++distinct;
    tn_head_t* h = nullptr;
    rc = tn_head_create(p, nullptr, &h);
    double ms = 1e300;
    if (rc == TN_OK) {
      // with 16-bit operands, time the CTA-pair and the one-CTA GEMM tiles and
      // keep the faster (unless the caller turned pairs off)
      const bool both = o.gemm_pair == 0 && (o.gemm == TN_GEMM_TC_BF16X3 || o.gemm == TN_GEMM_TC_FP16X3);
      int best_pair = p->P.gemm_pair;
      for (int v = 0; v < (both ? 2 : 1) && rc == TN_OK; ++v) {
        if (both) p->P.gemm_pair = v == 0 ? 0 : -1;
        rc = run_slice(p, 0, h->H, st);   // untimed
        if (rc != TN_OK) break;
        cudaEventRecord(e0, st);
        rc = run_slice(p, 0, h->H, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) == cudaSuccess) {
          float f = 0.f;
          cudaEventElapsedTime(&f, e0, e1);
          if (f < ms) {
            ms = f;
            best_pair = p->P.gemm_pair;
          }
        }
      }
      p->P.gemm_pair = best_pair;
      tn_head_free(h);
    }
    if (rc == TN_OK && ms < best_ms) {
      if (best) tn_plan_free(best);
      best = p;
      best_ms = ms;
    } else {
      tn_plan_free(p);
    }
    if (rc) last_rc = rc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!best) return last_rc ? last_rc : fail(TN_ERR_OOM, "no candidate plan could be built");
  best->measured_slice_ms = best_ms;
  best->autotune_candidates = distinct;
  const double passes = std::ldexp(1.0, best->P.n_internal);
  if (o.tune_steps > 0 || (o.tune_steps == 0 && best_ms / passes <= 1000.0)) {
    double t0 = 0, t1 = 0;
    const int rc = tn_plan_tune_steps(best, o.tune_steps > 0 ? o.tune_steps : 3, stream, &t0, &t1);
    if (rc) {
      tn_plan_free(best);
      return rc;
    }
    // the tuner times one pass: a slice is 2^n_internal of them
    best->measured_slice_ms = best->P.n_internal == 0 ? std::min(t0, t1) : best_ms * std::min(t0, t1) / t0;
  }
  *out = best;
  return TN_OK;
}

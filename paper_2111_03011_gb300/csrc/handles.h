// Internal handle layouts shared by the C ABI (capi.cu) and the request
// server (server.cu).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "planner.h"
#include "tn_gb300.h"

struct GraphEntry {
  int64_t begin = 0, end = 0;
  void* H = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;              // LRU stamp (the per-plan cache keeps kGraphCache entries)
};

namespace tn {
// Unique, never reused identity of a plan or head (caches must not key on
// addresses: a freed handle's address can come back for a new one).
inline uint64_t next_serial() {
  static std::atomic<uint64_t> c{1};
  return c.fetch_add(1);
}
}  // namespace tn

struct tn_plan {
  uint64_t serial = tn::next_serial();
  uint64_t graph_clock = 0;            // LRU clock of `graphs`
  tn::Plan P;
  double measured_slice_ms = 0.0;
  int autotune_candidates = 0;
  double tune_default_ms = 0.0, tune_tuned_ms = 0.0;   // tn_plan_tune_steps: slice times before / after
  std::vector<GraphEntry> graphs;     // captured slice ranges (tn_contract_slices_graph)
  std::vector<cudaEvent_t> prof_events;   // tn_profile_slices: reused timing events
  // side stream of the B-prep steps that run beside an earlier GEMM
  // (Step::fork): one fork event per fork step, one join event per side step
  cudaStream_t side_stream = nullptr;
  std::vector<cudaEvent_t> side_fork, side_join;   // indexed by step
  std::vector<std::vector<int>> forks_at;          // step -> side steps launched before it
  bool on_device = false;
  int device = -1;
  float2* d_leaves = nullptr;
  uint32_t* d_meta = nullptr;
  char* d_arena = nullptr;
  uint64_t* d_keys = nullptr;      // sorted masked tails
  uint32_t* d_key_groups = nullptr;
  uint64_t* d_tails = nullptr;     // tails in group order
  int* d_open = nullptr;
  unsigned int* d_status = nullptr;
  unsigned int* d_scale = nullptr;   // FP16x3 operand scale slots (zeroed at the start of every pass)
  int64_t n_keys = 0;
};

struct tn_head {
  uint64_t serial = tn::next_serial();
  tn_plan_t* plan = nullptr;
  double2* H = nullptr;
  bool owns = false;
  std::map<int64_t, int64_t> done;   // begin -> end of accumulated slice ranges
  int64_t slices_done = 0;
  // set when H may hold part of a slice (a call failed between the passes of
  // one slice) or a bounded device wait gave up; cleared by tn_head_reset
  bool invalid = false;
  bool f_override = false;
  double f_value = 0.0;
  // scratch
  double* d_Z = nullptr;
  double* d_N = nullptr;
  unsigned long long* d_status = nullptr;
  void* d_stage = nullptr;
  size_t stage_bytes = 0;
};


namespace tn {
void set_last_error(const std::string& msg);
// Enqueue the slices of `r` of `plan` into H on `stream` (no range checks).
// On failure *done_end (if given) is the end of the leading sub-range whose
// slices were enqueued whole, or -1 if a slice was left partly accumulated.
int enqueue_slices(tn_plan_t* plan, tn_range r, double2* H, cudaStream_t stream, int64_t* done_end = nullptr);
// Host-side fault injection (environment variable TN_FAULT_INJECT): true if
// the named fault is armed.  "alloc": device allocations of plans and heads
// fail; "slice:S[:T]": the contraction fails before pass T (default 0) of
// user slice S; "status": each plain contraction call sets the plan's device
// status word, as a bounded wait that gave up would.
bool fault_alloc();
bool fault_slice(int64_t s, int64_t t);
bool fault_status();
// Range checks and bookkeeping of tn_contract_slices.
int check_slice_range(tn_plan_t* plan, tn_range r, tn_head_t* head);
void mark_slices_done(tn_head_t* head, tn_range r);
}  // namespace tn

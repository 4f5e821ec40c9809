// Host-side planner of the sliced sparse-state contraction.
//
// Builds the tensor network of a circuit (Method section: |0> vectors, gate
// matrices and four-way tensors, the sparse-state final boundary of the
// Supplement), applies pins, absorbs order-one and order-two tensors into their
// neighbours (Results: simplification before contraction), picks a pairwise
// contraction order and lays every pairwise contraction out as device steps
// over binary-leg tensors with an optional sparse-state pattern axis.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

namespace tn {

using cd = std::complex<double>;

enum LegKind { LEG_BOND = 0, LEG_OPEN = 1, LEG_HALF = 2 };

struct Leg {
  int kind = LEG_BOND;
  int slice_bit = -1;   // LEG_HALF: slice-id bit fixing this end of a sliced edge
  int open_index = -1;  // LEG_OPEN: position j in open_qubits
};

// A tensor over binary legs (bit i of the flat index <-> legs[i]) times a
// sparse-state pattern axis: the distinct restrictions of the tails to the tail
// qubits in `tq` (Supplement, sparse-state method: only patterns present in
// the targets are kept when final-state legs merge).
struct HostTensor {
  std::vector<int> legs;
  uint64_t tq = 0;
  std::vector<uint64_t> pats{0};
  std::vector<cd> data;
  bool alive = true;
  int64_t P() const { return (int64_t)pats.size(); }
};

// Pattern lists of subsets of tail qubits.
struct PatternBook {
  std::vector<uint64_t> tails;  // masked to tail qubits
  std::unordered_map<uint64_t, std::vector<uint64_t>> cache;
  const std::vector<uint64_t>& get(uint64_t mask);
  int64_t count(uint64_t mask) { return (int64_t)get(mask).size(); }
};

enum StepKind {
  ST_SMALL = 0,      // streaming contraction with a <=16x16 operand, any A layout
  ST_PERMUTE = 1,    // bit permutation of a tensor's legs
  ST_BPREP_TC = 2,   // B -> real-embedded K-major fp32 hi/lo operand (tensor-core GEMM)
  ST_GEMM_TC = 3,    // tcgen05 complex GEMM (4M real embedding, 3xTF32)
  ST_BPREP_C = 4,    // B -> complex [K][N] row-major (SIMT GEMM)
  ST_GEMM_SIMT = 5,  // FP32 CUDA-core complex GEMM
  ST_ABSMAX = 6,     // max |re|, |im| of a GEMM operand into a scale slot (FP16x3 engine)
};

struct Ref {
  int kind = -1;   // 0 leaf, 1 workspace buffer
  int id = -1;
};

struct LeafInfo {
  int64_t off = 0;        // element offset of variant 0 in the leaf arena
  int64_t size = 0;       // elements per variant (P * 2^r)
  std::vector<int> var_slice_bits;  // variant bit t <- slice bit var_slice_bits[t]
};

struct BufInfo {
  int64_t bytes = 0;
  int64_t off = 0;
  int first = 0, last = 0;  // step lifetime (inclusive)
};

// Tile schedule of a permute step: tile bits, its tables in meta and the
// input / output positions of the remaining (tile index) bits.
struct PermSched {
  int t_bits = 0;
  int64_t tab_off = 0;
  int n_rest = 0;
  uint8_t rest_in[64] = {0}, rest_out[64] = {0};
  int vec4 = 0;            // output bits 0 and 1 are tile bits 0 and 1 (four outputs per store)
};

struct Step {
  int kind = ST_SMALL;
  Ref a, b, c;
  int vt_a = -1, vt_b = -1, vt_c = -1;   // virtual tensor ids (for describe)
  int rA = 0, rB = 0, rC = 0;
  int64_t PA = 1, PB = 1, PC = 1;
  int nk = 0, nm = 0, nn = 0;
  // pattern maps: mode 0 identity, 1 zero, 2 table in meta (int32)
  int mapA_mode = 1, mapB_mode = 1;
  int64_t mapA_off = 0, mapB_off = 0;
  // SMALL
  int kposA[4] = {0, 0, 0, 0};
  uint32_t boffK[16] = {0}, boffN[16] = {0};
  // PERMUTE: tile bits t; tables in meta: in_off[2^t], out_off[2^t], slot[2^t]
  int t_bits = 0;
  int split = 0;           // PERMUTE: 1 tf32 hi/lo planes, 2 bf16, 3 scaled fp16 (tensor-core GEMM operand)
  int h16 = 0;             // BPREP_TC / GEMM_TC: 16-bit operand planes (0 tf32, 1 bf16, 2 scaled fp16)
  // FP16x3 scale slots: -1 none, j >= 0 the j-th per-pass slot (zeroed at the
  // start of every pass), <= -2 the static slot -(slot + 2) (a leaf's maximum)
  int slot = -1;           // ABSMAX: slot written; PERMUTE (split 3), BPREP (h16 2), GEMM (h16 2): A's slot
  int slotB = -1;          // GEMM (h16 2): B's slot
  int max_slot = -1;       // GEMM_TC / SMALL: also write the output's max |re|, |im| into this slot
  int64_t tab_off = 0;
  int n_rest = 0;
  uint8_t rest_in[64] = {0}, rest_out[64] = {0};
  // PERMUTE: the schedules a plan tuner may choose from (alts[0] is the
  // default); the fields above hold the chosen one
  std::vector<PermSched> alts;
  int vec4 = 0;            // PERMUTE: of the chosen schedule
  // BPREP_TC with alts (its B operand has >= 2^20 elements): variant 0 or 1 is
  // the gather kernel, the other the permute kernel in an embedding mode with
  // the tile schedule alts[0] (fields above) onto [N][K] order; 1 here: the
  // plan's rule picked the permute (the gather's loads would not coalesce)
  int bprep_embed0 = 0;
  // GEMM_TC: widest tile (real columns, 16..256) and CTA pairs allowed (0) or
  // not (-1), as chosen by a plan tuner (default: the dispatch rule's widest)
  int tile_cap = 256;
  int pair = 0;
  int variant = 0;         // index of the chosen variant (0: default)
  // BPREP: gather tables bk[K], bn[N] in meta (uint32)
  int64_t bk_off = 0, bn_off = 0;
  // BPREP_TC run on the side stream: it may start once every step before
  // `fork` (a tensor-core GEMM) is done, and the next step waits for it
  int fork = -1;
  double macs = 0, bytes = 0;
  int contraction = -1;   // index of the pairwise contraction this step belongs to
};

struct FinalInfo {
  Ref ref;
  int vt = -1;
  int rF = 0;
  int64_t PF = 1;
  int open_pos[64] = {0};  // bit position in F of open leg j
  int64_t pidx_off = 0;    // meta offset of pidx[L] (int32)
};

struct VTensor {   // a tensor of the device network (leaf or intermediate)
  std::vector<int> legs;
  uint64_t tq = 0;
  int64_t P = 1;
  Ref ref;
  bool alive = true;
};

struct Plan {
  // inputs
  int n_qubits = 0;
  std::vector<int> open_qubits;
  std::vector<uint64_t> tails_raw;
  uint64_t open_mask = 0, tail_mask = 0;
  int n_sliced = 0, n_pinned = 0, n_companion = 0;
  int n_internal = 0;              // slice bits added by automatic slicing (summed inside every slice)
  int n_scale_slots = 0;           // FP16x3 per-pass operand scale slots
  std::vector<uint32_t> scale_static;   // FP16x3 static slots: fp32 bits of a leaf operand's max |re|, |im|
  std::vector<std::pair<int, int>> leg_edge;   // bond leg -> (gate, input leg) that consumes it
  std::vector<std::pair<int, int>> internal_edges;   // (gate, leg) of the SLICE edges automatic slicing added
  double companion_factor = 1.0;   // product of the companion cuts' kept norm fractions
  double cap_log2 = 28;
  int gemm_engine = 0;
  int gemm_pair = 0;               // GemmParams::pair of every tensor-core GEMM step
  int n_side_bprep = 0;            // B-prep steps with fork >= 0
  int small_max_bits = 4;

  std::vector<Leg> legs;
  PatternBook book;

  // device network
  std::vector<HostTensor> leaves;   // after simplification (with half legs still present)
  std::vector<LeafInfo> leaf_info;
  std::vector<cd> leaf_arena;       // variants, complex128 on host, uploaded as complex64
  std::vector<VTensor> vts;         // leaves first, then intermediates
  std::vector<std::pair<int, int>> order;
  std::vector<Step> steps;
  std::vector<BufInfo> bufs;
  std::vector<uint32_t> meta;       // int32/uint32 tables
  FinalInfo fin;
  int64_t n_patterns_final = 1;
  int64_t workspace_bytes = 0;
  double tc_macs = 0, alg_bytes = 0, max_log2 = 0;
  int n_contractions = 0;

  std::string describe_cache;
};

// Builds the whole plan; returns 0 or a TN_ERR_* code with `err` set.
struct PlanInput {
  int n_qubits;
  int n_gates;
  const int* arity;
  const int* q0;
  const int* q1;
  const cd* mats;           // n_gates * 16 (1q gates use the first 4)
  std::vector<int> open_qubits;
  std::vector<uint64_t> tails;
  struct Edge { int gate, leg, kind, value; };
  std::vector<Edge> edges;
  const int32_t* order = nullptr;
  int64_t n_pairs = 0;
  double cap_log2 = 28;
  int gemm_engine = 0;
  int order_trials = 64;
  uint64_t order_seed = 1;
  int absorb_log2 = 12;
  int small_max_bits = 4;
  int auto_slice = 0;       // at most this many extra sliced edges when no order fits the cap
  int fold_log2 = 12;       // host folding of small contractions of host tensors (-1: off)
  int gemm_pair = 0;        // 0: CTA-pair GEMM tiles where they apply; -1: one-CTA tiles only
  bool side_bprep = false;  // B-prep steps whose operand is ready run beside the previous GEMM
};

int build_plan(const PlanInput& in, Plan& plan, std::string& err);
void apply_perm_schedule(Step& s, const PermSched& ps);
std::string describe_plan(const Plan& plan, bool with_data);

}  // namespace tn

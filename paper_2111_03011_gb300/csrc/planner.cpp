// Host-side planner: network construction, simplification, order, step layout.
// See planner.h for the data model.
#include "planner.h"

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <random>
#include <set>
#include <sstream>
#include <thread>

#include "tn_gb300.h"

namespace tn {

const std::vector<uint64_t>& PatternBook::get(uint64_t mask) {
  auto it = cache.find(mask);
  if (it != cache.end()) return it->second;
  std::vector<uint64_t> v;
  v.reserve(tails.size());
  for (uint64_t t : tails) v.push_back(t & mask);
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
  return cache.emplace(mask, std::move(v)).first->second;
}

static int64_t pat_index(const std::vector<uint64_t>& pats, uint64_t v) {
  auto it = std::lower_bound(pats.begin(), pats.end(), v);
  if (it == pats.end() || *it != v) return -1;
  return (int64_t)(it - pats.begin());
}

static int find_pos(const std::vector<int>& legs, int l) {
  for (size_t i = 0; i < legs.size(); ++i)
    if (legs[i] == l) return (int)i;
  return -1;
}

// ---------------------------------------------------------------- host tensors

// Contract A and B over every leg they share; result legs = A's free legs then B's.
static HostTensor contract_host(const HostTensor& A, const HostTensor& B, PatternBook& book) {
  std::vector<int> shared;
  for (int l : A.legs)
    if (find_pos(B.legs, l) >= 0) shared.push_back(l);
  HostTensor C;
  std::vector<int> srcA, srcB;  // for C leg i: position in A (or -1), position in B (or -1)
  for (int l : A.legs)
    if (find_pos(shared, l) < 0) { C.legs.push_back(l); srcA.push_back(find_pos(A.legs, l)); srcB.push_back(-1); }
  for (int l : B.legs)
    if (find_pos(shared, l) < 0) { C.legs.push_back(l); srcA.push_back(-1); srcB.push_back(find_pos(B.legs, l)); }
  C.tq = A.tq | B.tq;
  C.pats = book.get(C.tq);
  const int rA = (int)A.legs.size(), rB = (int)B.legs.size(), rC = (int)C.legs.size();
  const int nk = (int)shared.size();
  std::vector<int64_t> ka(1LL << nk), kb(1LL << nk);
  for (int64_t k = 0; k < (1LL << nk); ++k) {
    int64_t a = 0, b = 0;
    for (int j = 0; j < nk; ++j)
      if ((k >> j) & 1) { a |= 1LL << find_pos(A.legs, shared[j]); b |= 1LL << find_pos(B.legs, shared[j]); }
    ka[k] = a; kb[k] = b;
  }
  const int64_t nC = 1LL << rC;
  C.data.assign((size_t)(C.P() * nC), cd(0, 0));
  for (int64_t p = 0; p < C.P(); ++p) {
    int64_t pa = pat_index(A.pats, C.pats[p] & A.tq);
    int64_t pb = pat_index(B.pats, C.pats[p] & B.tq);
    const cd* a0 = A.data.data() + pa * (1LL << rA);
    const cd* b0 = B.data.data() + pb * (1LL << rB);
    for (int64_t c = 0; c < nC; ++c) {
      int64_t ia = 0, ib = 0;
      for (int i = 0; i < rC; ++i)
        if ((c >> i) & 1) {
          if (srcA[i] >= 0) ia |= 1LL << srcA[i];
          else ib |= 1LL << srcB[i];
        }
      cd s(0, 0);
      for (size_t k = 0; k < ka.size(); ++k) s += a0[ia + ka[k]] * b0[ib + kb[k]];
      C.data[(size_t)(p * nC + c)] = s;
    }
  }
  return C;
}

// Fix leg at position `pos` to value v and drop it.
static void select_leg(HostTensor& T, int pos, int v) {
  const int r = (int)T.legs.size();
  const int64_t n_old = 1LL << r, n_new = 1LL << (r - 1);
  std::vector<cd> d((size_t)(T.P() * n_new));
  const int64_t lo_mask = (1LL << pos) - 1;
  for (int64_t p = 0; p < T.P(); ++p)
    for (int64_t i = 0; i < n_new; ++i) {
      int64_t src = ((i & ~lo_mask) << 1) | ((int64_t)v << pos) | (i & lo_mask);
      d[(size_t)(p * n_new + i)] = T.data[(size_t)(p * n_old + src)];
    }
  T.data.swap(d);
  T.legs.erase(T.legs.begin() + pos);
}


// --------------------------------------------------------------- network build

struct Builder {
  Plan& plan;
  std::vector<HostTensor> T;
  std::vector<int> pin_of_leg;   // -1 or pinned value
  struct Use { int leg, gate, pos; };
  std::vector<Use> consumed;     // input wires of gates

  explicit Builder(Plan& p) : plan(p) {}

  int new_leg(int kind) {
    Leg l;
    l.kind = kind;
    plan.legs.push_back(l);
    pin_of_leg.push_back(-1);
    return (int)plan.legs.size() - 1;
  }
};

static int build_network(const PlanInput& in, Plan& plan, Builder& b, std::string& err) {
  const int n = in.n_qubits;
  std::vector<int> wire(n);
  for (int q = 0; q < n; ++q) {
    int l = b.new_leg(LEG_BOND);
    HostTensor t;
    t.legs = {l};
    t.data = {cd(1, 0), cd(0, 0)};
    b.T.push_back(t);
    wire[q] = l;
  }
  // cuts by gate
  std::map<int, std::vector<std::pair<int, int>>> cuts;  // gate -> (leg, edge index)
  for (size_t e = 0; e < in.edges.size(); ++e) cuts[in.edges[e].gate].push_back({in.edges[e].leg, (int)e});
  int slice_bit = 0;
  std::vector<int> edge_slice_bit(in.edges.size(), -1);
  for (size_t e = 0; e < in.edges.size(); ++e)
    if (in.edges[e].kind == TN_EDGE_SLICE || in.edges[e].kind == TN_EDGE_COMPANION) edge_slice_bit[e] = slice_bit++;
  // companion cuts: gate -> (partner output leg position 0/1 of the outputs, slice bit)
  std::map<int, std::vector<std::pair<int, int>>> companions;
  for (size_t e = 0; e < in.edges.size(); ++e)
    if (in.edges[e].kind == TN_EDGE_COMPANION)
      companions[in.edges[e].gate].push_back({1 - in.edges[e].leg, edge_slice_bit[e]});

  for (int gi = 0; gi < in.n_gates; ++gi) {
    const int ar = in.arity[gi];
    const int q0 = in.q0[gi], q1 = in.q1[gi];
    auto it = cuts.find(gi);
    if (it != cuts.end()) {
      for (auto& c : it->second) {
        const int q = c.first == 0 ? q0 : q1;
        const auto& E = in.edges[c.second];
        int old = wire[q];
        if (plan.legs[old].kind == LEG_HALF) {
          // the wire is already fixed by a companion cut of the previous gate
          err = "edge: gate " + std::to_string(gi) + " leg " + std::to_string(c.first) +
                " cuts a wire that a companion cut already fixes";
          return TN_ERR_INVALID;
        }
        int nw = b.new_leg(LEG_HALF);
        plan.legs[old].kind = LEG_HALF;
        if (E.kind == TN_EDGE_SLICE || E.kind == TN_EDGE_COMPANION) {
          plan.legs[old].slice_bit = edge_slice_bit[c.second];
          plan.legs[nw].slice_bit = edge_slice_bit[c.second];
        } else {
          b.pin_of_leg[old] = E.value;
          b.pin_of_leg[nw] = E.value;
        }
        wire[q] = nw;
      }
    }
    const cd* U = in.mats + (size_t)gi * 16;
    // the wire this gate consumes on each input leg (for automatic slicing)
    b.consumed.push_back({wire[q0], gi, 0});
    if (ar == 2) b.consumed.push_back({wire[q1], gi, 1});
    HostTensor t;
    if (ar == 1) {
      int out = b.new_leg(LEG_BOND);
      t.legs = {wire[q0], out};
      t.data.assign(4, cd(0, 0));
      for (int o = 0; o < 2; ++o)
        for (int i = 0; i < 2; ++i) t.data[i + 2 * o] = U[o * 2 + i];
      wire[q0] = out;
    } else {
      int o0 = b.new_leg(LEG_BOND), o1 = b.new_leg(LEG_BOND);
      t.legs = {wire[q0], wire[q1], o0, o1};
      t.data.assign(16, cd(0, 0));
      for (int a0 = 0; a0 < 2; ++a0)
        for (int a1 = 0; a1 < 2; ++a1)
          for (int i0 = 0; i0 < 2; ++i0)
            for (int i1 = 0; i1 < 2; ++i1)
              t.data[i0 + 2 * i1 + 4 * a0 + 8 * a1] = U[(2 * a0 + a1) * 4 + (2 * i0 + i1)];
      wire[q0] = o0;
      wire[q1] = o1;
      // rank-one companion cut (Method case (ii)): with input leg a fixed to v
      // by the slice, the partner output is fixed to the same v, so that wire
      // becomes a pair of half legs carrying the same slice bit
      auto ic = companions.find(gi);
      if (ic != companions.end())
        for (auto& pc : ic->second) {
          const int q = pc.first == 0 ? q0 : q1;
          int old = wire[q];
          int nw = b.new_leg(LEG_HALF);
          plan.legs[old].kind = LEG_HALF;
          plan.legs[old].slice_bit = pc.second;
          plan.legs[nw].slice_bit = pc.second;
          wire[q] = nw;
        }
    }
    b.T.push_back(t);
  }
  // final boundary: open legs, tail projectors with a pattern axis
  for (int q = 0; q < n; ++q) {
    int j = find_pos(plan.open_qubits, q);
    if (j >= 0 && plan.legs[wire[q]].kind == LEG_HALF) {
      // the open qubit's last wire is fixed by a companion cut of its last
      // gate: an identity tensor carries the fixed value to a fresh open leg
      // (its variant v is the unit vector e_v on that leg)
      int ol = b.new_leg(LEG_OPEN);
      plan.legs[ol].open_index = j;
      HostTensor t;
      t.legs = {wire[q], ol};
      t.data = {cd(1, 0), cd(0, 0), cd(0, 0), cd(1, 0)};
      b.T.push_back(t);
    } else if (j >= 0) {
      plan.legs[wire[q]].kind = LEG_OPEN;
      plan.legs[wire[q]].open_index = j;
    } else {
      HostTensor t;
      t.legs = {wire[q]};
      t.tq = 1ULL << q;
      t.pats = plan.book.get(t.tq);
      t.data.assign((size_t)(2 * t.P()), cd(0, 0));
      for (int64_t p = 0; p < t.P(); ++p) t.data[(size_t)(2 * p + ((t.pats[p] >> q) & 1))] = cd(1, 0);
      b.T.push_back(t);
    }
  }
  // apply pins (both half legs of a pinned edge take its value)
  for (auto& t : b.T)
    for (int pos = (int)t.legs.size() - 1; pos >= 0; --pos) {
      int l = t.legs[pos];
      if (plan.legs[l].kind == LEG_HALF && b.pin_of_leg[l] >= 0) select_leg(t, pos, b.pin_of_leg[l]);
    }
  return TN_OK;
}

// Absorb order-one and order-two tensors into neighbours and split rank-one
// order-two tensors (the exact hole reduction of Method case (i)).
static void simplify(Plan& plan, std::vector<HostTensor>& T, int absorb_log2) {
  auto is_bond = [&](int l) { return plan.legs[l].kind == LEG_BOND; };
  bool changed = true;
  while (changed) {
    changed = false;
    // rank-one split
    const size_t n0 = T.size();
    for (size_t i = 0; i < n0; ++i) {
      HostTensor& t = T[i];
      if (!t.alive || t.legs.size() != 2 || t.tq != 0) continue;
      if (!is_bond(t.legs[0]) || !is_bond(t.legs[1])) continue;
      // data[a + 2b]
      cd m00 = t.data[0], m10 = t.data[1], m01 = t.data[2], m11 = t.data[3];
      double nrm = std::norm(m00) + std::norm(m01) + std::norm(m10) + std::norm(m11);
      if (nrm == 0.0) continue;
      if (std::abs(m00 * m11 - m01 * m10) > 1e-13 * nrm) continue;
      // pick largest entry
      int ba = 0, bb = 0;
      double best = -1;
      for (int a = 0; a < 2; ++a)
        for (int bq = 0; bq < 2; ++bq)
          if (std::abs(t.data[a + 2 * bq]) > best) { best = std::abs(t.data[a + 2 * bq]); ba = a; bb = bq; }
      HostTensor u, v;
      u.legs = {t.legs[0]};
      v.legs = {t.legs[1]};
      u.data = {t.data[0 + 2 * bb], t.data[1 + 2 * bb]};
      cd piv = t.data[ba + 2 * bb];
      v.data = {t.data[ba + 0] / piv, t.data[ba + 2] / piv};
      t.alive = false;
      T.push_back(u);
      T.push_back(v);
      changed = true;
    }
    // absorption
    std::unordered_map<int, std::vector<int>> owners;
    for (size_t i = 0; i < T.size(); ++i)
      if (T[i].alive)
        for (int l : T[i].legs)
          if (is_bond(l)) owners[l].push_back((int)i);
    for (size_t i = 0; i < T.size(); ++i) {
      HostTensor& t = T[i];
      if (!t.alive || t.legs.size() > 2) continue;
      int best_n = -1;
      double best_sz = 1e300;
      for (int l : t.legs) {
        if (!is_bond(l)) continue;
        for (int o : owners[l]) {
          if (o == (int)i || !T[o].alive) continue;
          // result size
          int shared = 0;
          for (int x : t.legs)
            if (find_pos(T[o].legs, x) >= 0) ++shared;
          double sz = std::log2((double)plan.book.count(T[o].tq | t.tq)) +
                      (double)(T[o].legs.size() + t.legs.size() - 2 * shared);
          if (sz < best_sz) { best_sz = sz; best_n = o; }
        }
      }
      if (best_n < 0 || best_sz > absorb_log2) continue;
      HostTensor merged = contract_host(T[best_n], t, plan.book);
      T[best_n] = std::move(merged);
      T[i].alive = false;
      changed = true;
      // refresh owners (cheap enough at circuit sizes)
      owners.clear();
      for (size_t k = 0; k < T.size(); ++k)
        if (T[k].alive)
          for (int l : T[k].legs)
            if (is_bond(l)) owners[l].push_back((int)k);
    }
  }
}

// ------------------------------------------------------------------- ordering

struct GNode {
  std::vector<int> legs;  // device legs (bond + open)
  uint64_t tq = 0;
  double lsz = 0;         // log2 elements
  bool alive = true;
};

static std::vector<int> sym_diff_bond(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> out;
  for (int l : a)
    if (find_pos(b, l) < 0) out.push_back(l);
  for (int l : b)
    if (find_pos(a, l) < 0) out.push_back(l);
  return out;
}

static int shared_count(const std::vector<int>& a, const std::vector<int>& b) {
  int s = 0;
  for (int l : a)
    if (find_pos(b, l) >= 0) ++s;
  return s;
}

// Execution-time model of a pairwise contraction (seconds), calibrated on the
// GB300 kernels (streaming steps ~5 TB/s; tensor-core GEMM ~200 TFLOP/s
// algorithmic; split permute 24 B/element at ~4 TB/s; B prep 40 B/element;
// ~4 us per launch).  Used only to pick among greedy restarts.
static double step_time_model(double lA, double lB, double lC, int nk, int nn_small, bool tc) {
  double A = std::exp2(lA), B = std::exp2(lB), C = std::exp2(lC);
  const double big = std::max(A, B), sml = std::min(A, B);
  const double macs = C * std::exp2(nk);
  const bool small = nk <= 4 && nn_small <= 4;
  if (small) return 8.0 * (A + B + C) / 5.0e12 + 4e-6;
  const double peak = tc ? 200e12 : 40e12;
  double t = std::max(8.0 * macs / peak, (16.0 * big + 8.0 * C) / 5.5e12);   // GEMM
  t += 24.0 * big / 4.0e12;                                                     // permute (split)
  t += 40.0 * sml / 3.0e12;                                                     // B prep
  return t + 12e-6;
}

struct TrialResult {
  bool fits = false;
  double cost = 1e300, mx = 1e300;
  std::vector<std::pair<int, int>> order;
  std::vector<int> legs;   // legs automatic slicing cuts on this order
  std::string why;
};

// One randomised greedy trial; trial 0 is the plain greedy (alpha 1, no noise).
static TrialResult greedy_trial(const Plan& plan, PatternBook& book, const std::vector<GNode>& init, double cap,
                                uint64_t seed, int trial) {
  std::mt19937_64 rng(seed * 0x9E3779B97F4A7C15ULL + (uint64_t)trial * 0xD1B54A32D192ED03ULL + 1);
  std::uniform_real_distribution<double> ud(1e-12, 1.0);
  const double alpha = trial == 0 ? 1.0 : 0.3 + 1.2 * ud(rng);
  const double tau = trial == 0 ? 0.0 : 0.05 + 0.6 * ud(rng);
  std::vector<GNode> g = init;
  TrialResult res;
  double cost = 0, mx = 0;
  int alive = 0;
  for (auto& x : g) {
    alive += x.alive;
    mx = std::max(mx, x.lsz);
  }
  std::unordered_map<int, std::vector<int>> owners;
  for (size_t i = 0; i < g.size(); ++i)
    if (g[i].alive)
      for (int l : g[i].legs)
        if (plan.legs[l].kind == LEG_BOND) owners[l].push_back((int)i);
  while (alive > 1) {
    std::set<std::pair<int, int>> cand;
    for (auto& kv : owners)
      if (kv.second.size() == 2) {
        int a = std::min(kv.second[0], kv.second[1]), b = std::max(kv.second[0], kv.second[1]);
        cand.insert({a, b});
      }
    int bi = -1, bj = -1;
    double bs = 1e300;
    for (auto& pr : cand) {
      const GNode &A = g[pr.first], &B = g[pr.second];
      std::vector<int> cl = sym_diff_bond(A.legs, B.legs);
      double lc = std::log2((double)book.count(A.tq | B.tq)) + (double)cl.size();
      double score = std::exp2(lc) - alpha * (std::exp2(A.lsz) + std::exp2(B.lsz));
      // log-domain key keeps the noise scale-free; pairs over the cap go last
      double key = (score >= 0 ? std::log2(1.0 + score) : -std::log2(1.0 - score));
      if (tau > 0) key -= tau * std::log(-std::log(ud(rng)));
      if (lc > cap + 1e-9) key += 1e6 + lc;
      if (key < bs) { bs = key; bi = pr.first; bj = pr.second; }
    }
    if (bi < 0) {
      // disconnected: outer product of the two smallest
      std::vector<int> al;
      for (size_t i = 0; i < g.size(); ++i)
        if (g[i].alive) al.push_back((int)i);
      std::sort(al.begin(), al.end(), [&](int a, int b) { return g[a].lsz < g[b].lsz; });
      bi = std::min(al[0], al[1]);
      bj = std::max(al[0], al[1]);
    }
    GNode &A = g[bi], &B = g[bj];
    int nk = shared_count(A.legs, B.legs);
    std::vector<int> cl = sym_diff_bond(A.legs, B.legs);
    GNode C;
    C.legs = cl;
    C.tq = A.tq | B.tq;
    C.lsz = std::log2((double)book.count(C.tq)) + (double)cl.size();
    mx = std::max(mx, C.lsz);
    int nn_small = (int)((A.lsz <= B.lsz ? A.legs.size() : B.legs.size())) - nk;
    cost += step_time_model(A.lsz, B.lsz, C.lsz, nk, nn_small, plan.gemm_engine != TN_GEMM_SIMT_FP32);
    for (int l : A.legs)
      if (plan.legs[l].kind == LEG_BOND) {
        auto& v = owners[l];
        v.erase(std::remove(v.begin(), v.end(), bi), v.end());
        if (v.empty()) owners.erase(l);
      }
    for (int l : B.legs)
      if (plan.legs[l].kind == LEG_BOND) {
        auto& v = owners[l];
        v.erase(std::remove(v.begin(), v.end(), bj), v.end());
        if (v.empty()) owners.erase(l);
      }
    for (int l : C.legs)
      if (plan.legs[l].kind == LEG_BOND) owners[l].push_back(bi);
    res.order.push_back({bi, bj});
    g[bi] = C;
    g[bj].alive = false;
    --alive;
  }
  res.fits = mx <= cap + 1e-9;
  res.cost = cost;
  res.mx = mx;
  return res;
}

static bool better(const TrialResult& a, const TrialResult& b) {   // is a better than b
  if (a.fits != b.fits) return a.fits;
  if (a.fits) return a.cost < b.cost;
  return a.mx < b.mx || (a.mx == b.mx && a.cost < b.cost);
}

// Automatic slicing.  Slicing a bond leg that survives host simplification
// turns it into a variant axis of the two leaves holding it: the leaf set, and
// with it any order over the leaves, stays as it is.  For a fixed order the
// slicer replays the contractions once, then adds legs one at a time: the
// candidates are the bond legs of the largest intermediate that are wires of
// the circuit, and the pick is the one with the smallest modelled time of all
// 2^|S| passes.  It stops when every intermediate fits the cap.
struct StepLegs {
  std::vector<int> a, b, c, k;   // legs of A, B, C and the contracted ones
  double pa = 0, pb = 0, pc = 0; // log2 pattern counts
};

struct SliceResult {
  bool ok = false;
  double cost = 1e300, mx = 1e300;   // modelled time of all passes; largest intermediate
  std::vector<int> legs;             // sliced legs, in the order they were picked
  std::string why;
};

static std::vector<StepLegs> replay_steps(PatternBook& book, const std::vector<GNode>& init,
                                          const std::vector<std::pair<int, int>>& order) {
  std::vector<GNode> g = init;
  std::vector<StepLegs> out;
  out.reserve(order.size());
  for (auto& pr : order) {
    StepLegs st;
    const GNode &A = g[pr.first], &B = g[pr.second];
    st.a = A.legs;
    st.b = B.legs;
    for (int l : A.legs)
      if (find_pos(B.legs, l) >= 0) st.k.push_back(l);
    st.c = sym_diff_bond(A.legs, B.legs);
    st.pa = std::log2((double)book.count(A.tq));
    st.pb = std::log2((double)book.count(B.tq));
    const uint64_t tq = A.tq | B.tq;
    st.pc = std::log2((double)book.count(tq));
    GNode C;
    C.legs = st.c;
    C.tq = tq;
    C.lsz = st.pc + (double)st.c.size();
    g[pr.first] = C;
    g[pr.second].alive = false;
    out.push_back(std::move(st));
  }
  return out;
}

static inline int count_sliced(const std::vector<int>& legs, const std::vector<char>& sl) {
  int n = 0;
  for (int l : legs) n += sl[l];
  return n;
}

static double sliced_step_time(const StepLegs& st, const std::vector<char>& sl, bool tc, double* lc) {
  const double lA = st.pa + (double)st.a.size() - count_sliced(st.a, sl);
  const double lB = st.pb + (double)st.b.size() - count_sliced(st.b, sl);
  const double lC = st.pc + (double)st.c.size() - count_sliced(st.c, sl);
  const int nk = (int)st.k.size() - count_sliced(st.k, sl);
  const int ra = (int)st.a.size() - count_sliced(st.a, sl), rb = (int)st.b.size() - count_sliced(st.b, sl);
  const int nn_small = (lA <= lB ? ra : rb) - nk;
  if (lc) *lc = lC;
  return step_time_model(lA, lB, lC, nk, nn_small, tc);
}

static SliceResult slice_order(const Plan& plan, PatternBook& book, const std::vector<GNode>& init,
                               const std::vector<std::pair<int, int>>& order, double cap, int budget) {
  SliceResult r;
  const bool tc = plan.gemm_engine != TN_GEMM_SIMT_FP32;
  std::vector<StepLegs> steps = replay_steps(book, init, order);
  const int nl = (int)plan.legs.size();
  std::vector<char> sl(nl, 0);
  std::vector<std::vector<int>> touch(nl);   // leg -> steps whose operands or result carry it
  for (size_t i = 0; i < steps.size(); ++i) {
    std::set<int> u(steps[i].a.begin(), steps[i].a.end());
    u.insert(steps[i].b.begin(), steps[i].b.end());
    for (int l : u) touch[l].push_back((int)i);
  }
  double leaf_mx = 0;
  for (auto& x : init) leaf_mx = std::max(leaf_mx, x.lsz);
  std::vector<double> t(steps.size()), lcs(steps.size());
  double sum = 0;
  for (size_t i = 0; i < steps.size(); ++i) sum += t[i] = sliced_step_time(steps[i], sl, tc, &lcs[i]);
  while (true) {
    int im = -1;
    double mx = leaf_mx;
    for (size_t i = 0; i < steps.size(); ++i)
      if (lcs[i] > mx) { mx = lcs[i]; im = (int)i; }
    r.mx = mx;
    if (mx <= cap + 1e-9) break;
    if (im < 0) { r.why = "a leaf exceeds the cap"; return r; }
    if ((int)r.legs.size() >= budget) {
      r.why = "more than " + std::to_string(budget) + " extra edges needed";
      return r;
    }
    int best = -1;
    double best_sum = 1e300;
    for (int l : steps[im].c) {
      if (sl[l] || plan.legs[l].kind != LEG_BOND) continue;
      if (l >= (int)plan.leg_edge.size() || plan.leg_edge[l].first < 0) continue;
      sl[l] = 1;
      double s2 = sum;
      for (int i : touch[l]) s2 += sliced_step_time(steps[i], sl, tc, nullptr) - t[i];
      sl[l] = 0;
      if (s2 < best_sum) { best_sum = s2; best = l; }
    }
    if (best < 0) { r.why = "open legs and tail patterns alone exceed the cap"; return r; }
    sl[best] = 1;
    r.legs.push_back(best);
    for (int i : touch[best]) {
      const double tn_ = sliced_step_time(steps[i], sl, tc, &lcs[i]);
      sum += tn_ - t[i];
      t[i] = tn_;
    }
  }
  r.ok = true;
  r.cost = std::ldexp(sum, (int)r.legs.size());
  return r;
}

// One partition trial.  Recursive bisection of the leaf graph (nodes = leaves,
// edge weight = the bond legs two leaves share, i.e. log2 of the dimension cut)
// gives a contraction tree whose largest intermediates sit at the smallest
// cuts: each part is contracted on its own and the two results are contracted
// last.  A part is split by a region grown breadth-first from a random node to
// a random share of 40-60 % of the nodes, then refined by Fiduccia-Mattheyses
// passes (move the unlocked node of largest cut reduction that keeps the
// balance, keep the best prefix of moves).  The tree becomes a pairwise order
// (each result stored at its first operand's slot) and is scored like a greedy
// trial: modelled time of its steps and largest intermediate.
static TrialResult partition_trial(const Plan& plan, PatternBook& book, const std::vector<GNode>& init, double cap,
                                   uint64_t seed, int trial) {
  std::mt19937_64 rng(seed * 0xA24BAED4963EE407ULL + (uint64_t)trial * 0x9FB21C651E98DF25ULL + 7);
  std::uniform_real_distribution<double> ud(0.0, 1.0);
  const int n = (int)init.size();
  // weighted adjacency over bond legs held by exactly two leaves
  std::unordered_map<int, std::vector<int>> owners;
  for (int i = 0; i < n; ++i)
    for (int l : init[i].legs)
      if (plan.legs[l].kind == LEG_BOND) owners[l].push_back(i);
  std::vector<std::unordered_map<int, int>> adj(n);
  for (auto& kv : owners)
    if (kv.second.size() == 2) {
      ++adj[kv.second[0]][kv.second[1]];
      ++adj[kv.second[1]][kv.second[0]];
    }
  const double share = 0.4 + 0.2 * ud(rng);
  std::vector<std::pair<int, int>> order;
  std::vector<int> side(n, -1);
  // returns the slot holding the part's result
  std::function<int(std::vector<int>&)> build = [&](std::vector<int>& part) -> int {
    const int m = (int)part.size();
    if (m == 1) return part[0];
    if (m == 2) {
      order.push_back({part[0], part[1]});
      return part[0];
    }
    for (int v : part) side[v] = 0;
    // initial cut: a region grown breadth-first from a random node
    const int target = std::max(1, std::min(m - 1, (int)std::lround(share * m)));
    std::vector<int> q{part[(size_t)(ud(rng) * m) % m]};
    side[q[0]] = 1;
    int grown = 1;
    for (size_t h = 0; h < q.size() && grown < target; ++h)
      for (auto& nb : adj[q[h]])
        if (side[nb.first] == 0 && grown < target) {
          side[nb.first] = 1;
          q.push_back(nb.first);
          ++grown;
        }
    for (size_t i = 0; grown < target && i < part.size(); ++i)   // disconnected remainder
      if (side[part[i]] == 0) { side[part[i]] = 1; ++grown; }
    // Fiduccia-Mattheyses refinement within balance [lo, hi] for side 1
    const int lo = std::max(1, (int)std::floor(0.35 * m)), hi = std::min(m - 1, (int)std::ceil(0.65 * m));
    for (int pass = 0; pass < 6; ++pass) {
      std::vector<char> locked(n, 0);
      std::vector<int> moves;
      int cur = 0, best = 0, best_len = 0, size1 = grown;
      for (int step = 0; step < m; ++step) {
        int bv = -1, bg = INT32_MIN;
        for (int v : part) {
          if (locked[v]) continue;
          const int to = 1 - side[v];
          const int ns = size1 + (to == 1 ? 1 : -1);
          if (ns < lo || ns > hi) continue;
          int g = 0;
          for (auto& nb : adj[v])
            if (side[nb.first] >= 0) g += side[nb.first] == side[v] ? -nb.second : nb.second;
          if (g > bg || (g == bg && ud(rng) < 0.5)) { bg = g; bv = v; }
        }
        if (bv < 0) break;
        size1 += side[bv] == 0 ? 1 : -1;
        side[bv] = 1 - side[bv];
        locked[bv] = 1;
        moves.push_back(bv);
        cur += bg;
        if (cur > best) { best = cur; best_len = (int)moves.size(); }
      }
      for (int i = (int)moves.size() - 1; i >= best_len; --i) side[moves[i]] = 1 - side[moves[i]];
      grown = 0;
      for (int v : part) grown += side[v] == 1;
      if (best <= 0) break;
    }
    std::vector<int> a, b;
    for (int v : part) (side[v] == 1 ? a : b).push_back(v);
    for (int v : part) side[v] = -1;
    if (a.empty() || b.empty()) {   // degenerate split: halve by position
      a.assign(part.begin(), part.begin() + m / 2);
      b.assign(part.begin() + m / 2, part.end());
    }
    const int sa = build(a);
    const int sb = build(b);
    order.push_back({sa, sb});
    return sa;
  };
  std::vector<int> all(n);
  for (int i = 0; i < n; ++i) all[i] = i;
  if (n > 1) build(all);
  TrialResult res;
  std::vector<StepLegs> steps = replay_steps(book, init, order);
  const std::vector<char> none(plan.legs.size(), 0);
  double mx = 0, cost = 0;
  for (auto& x : init) mx = std::max(mx, x.lsz);
  for (auto& st : steps) {
    double lc = 0;
    cost += sliced_step_time(st, none, plan.gemm_engine != TN_GEMM_SIMT_FP32, &lc);
    mx = std::max(mx, lc);
  }
  res.order = std::move(order);
  res.fits = mx <= cap + 1e-9;
  res.cost = cost;
  res.mx = mx;
  return res;
}

// Order search (restarts).  Even trials are randomised greedy; odd trials are
// recursive bisections (partition_trial).  A greedy trial repeatedly contracts the
// connected pair minimising size(C) - alpha * (size(A) + size(B)), with alpha
// drawn per trial and Gumbel noise of temperature tau on log-scores after the
// first trial.  A trial never stops at the cap: it records its largest
// intermediate, and the best trial is the one under the cap with the lowest
// modelled time (or, if none fits, the one with the smallest maximum).  Trials
// are seeded independently and spread over the host's cores; the result does
// not depend on the number of threads (ties go to the lower trial index).
//
// With a slicing budget, a third of the trials run under the cap as above, a
// third with no cap and a third with the cap raised by 2..7; every trial's
// order is then sliced to the cap (slice_order) and trials compete on the
// modelled time of all their passes.
static int greedy_order(Plan& plan, const std::vector<GNode>& init, double cap, int trials, uint64_t seed,
                        int budget, std::vector<std::pair<int, int>>& best_order, std::vector<int>& best_legs,
                        std::string& err) {
  trials = std::max(1, trials);
  const int nthreads = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), std::min(trials, 32)));
  // pattern counts of every tail-qubit subset a trial may meet, warmed serially
  // per thread (PatternBook is not thread-safe): each thread gets its own copy
  std::vector<TrialResult> best(nthreads);
  std::vector<int> best_idx(nthreads, -1);
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&, t] {
      PatternBook book;
      book.tails = plan.book.tails;
      for (int trial = t; trial < trials; trial += nthreads) {
        double tcap = cap;
        if (budget > 0 && trial % 3 == 1) tcap = 1e9;
        if (budget > 0 && trial % 3 == 2) tcap = cap + 2 + (trial / 3) % 6;
        // odd trials (from the second on) build the order by recursive bisection
        TrialResult r = (trial % 2 == 1 && init.size() >= 8) ? partition_trial(plan, book, init, tcap, seed, trial)
                                                             : greedy_trial(plan, book, init, tcap, seed, trial);
        if (budget > 0) {
          SliceResult sr = slice_order(plan, book, init, r.order, cap, budget);
          r.fits = sr.ok;
          if (sr.ok) {
            r.cost = sr.cost;
            r.mx = sr.mx;
          }
          r.legs = std::move(sr.legs);
          r.why = std::move(sr.why);
        }
        if (best_idx[t] < 0 || better(r, best[t])) {
          best[t] = std::move(r);
          best_idx[t] = trial;
        }
      }
    });
  for (auto& th : pool) th.join();
  int bt = -1;
  for (int t = 0; t < nthreads; ++t) {
    if (best_idx[t] < 0) continue;
    if (bt < 0 || better(best[t], best[bt]) ||
        (!better(best[bt], best[t]) && best_idx[t] < best_idx[bt]))
      bt = t;
  }
  if (bt < 0 || !best[bt].fits) {
    err = "no contraction order found keeps every intermediate under the size cap (best 2^" +
          std::to_string(bt < 0 ? 0.0 : best[bt].mx) + " elements); slice more edges or raise the cap";
    if (budget > 0 && bt >= 0) err += " (automatic slicing: " + best[bt].why + ")";
    return TN_ERR_OOM;
  }
  best_order = best[bt].order;
  best_legs = best[bt].legs;
  return TN_OK;
}

// ---------------------------------------------------------------- step layout

static int64_t meta_push(Plan& plan, const std::vector<uint32_t>& v) {
  while (plan.meta.size() % 4) plan.meta.push_back(0);
  int64_t off = (int64_t)plan.meta.size();
  plan.meta.insert(plan.meta.end(), v.begin(), v.end());
  return off;
}

static int new_buf(Plan& plan, int64_t bytes, int step) {
  BufInfo b;
  b.bytes = (bytes + 255) / 256 * 256;
  b.first = step;
  b.last = step;
  plan.bufs.push_back(b);
  return (int)plan.bufs.size() - 1;
}

static void touch(Plan& plan, const Ref& r, int step) {
  if (r.kind == 1) plan.bufs[r.id].last = std::max(plan.bufs[r.id].last, step);
}

static int64_t vt_elems(const VTensor& v) { return v.P * (1LL << v.legs.size()); }

// Pattern maps of C's pattern axis onto an operand's.
static void set_map(Plan& plan, const VTensor& X, const VTensor& C, int& mode, int64_t& off) {
  if (X.tq == 0) { mode = 1; off = 0; return; }
  if (X.tq == C.tq) { mode = 0; off = 0; return; }
  const auto& pc = plan.book.get(C.tq);
  const auto& px = plan.book.get(X.tq);
  std::vector<uint32_t> m(pc.size());
  for (size_t p = 0; p < pc.size(); ++p) m[p] = (uint32_t)pat_index(px, pc[p] & X.tq);
  mode = 2;
  off = meta_push(plan, m);
}

// max |re|, |im| of X into scale slot `slot` (FP16x3 operand scaling)
static void add_absmax(Plan& plan, const VTensor& X, int slot, int ci) {
  Step s;
  s.kind = ST_ABSMAX;
  s.a = X.ref;
  s.rA = (int)X.legs.size();
  s.PA = X.P;
  s.slot = slot;
  s.contraction = ci;
  s.bytes = 8.0 * (double)vt_elems(X);
  touch(plan, X.ref, (int)plan.steps.size());
  plan.steps.push_back(s);
}

// One tile schedule of a permute: the tile's input bits are the `a` lowest
// input positions and the input positions of the `bq` lowest output
// positions, grown with further low input bits up to `tmax` bits (longer
// contiguous runs, fewer tiles); the remaining bits index the tiles.
static PermSched perm_schedule(Plan& plan, const std::vector<int>& in_pos, const std::vector<int>& inv, int a,
                               int bq, int tmax) {
  const int r = (int)in_pos.size();
  a = std::min(r, a);
  bq = std::min(r, bq);
  std::vector<int> Tin;
  for (int x = 0; x < a; ++x) Tin.push_back(x);
  for (int o = 0; o < bq; ++o)
    if (std::find(Tin.begin(), Tin.end(), in_pos[o]) == Tin.end()) Tin.push_back(in_pos[o]);
  for (int x = 0; x < r && (int)Tin.size() < tmax; ++x)
    if (std::find(Tin.begin(), Tin.end(), x) == Tin.end()) Tin.push_back(x);
  std::sort(Tin.begin(), Tin.end());
  const int t = (int)Tin.size();
  std::vector<int> Tout;
  for (int x : Tin) Tout.push_back(inv[x]);
  std::sort(Tout.begin(), Tout.end());
  const int nt = 1 << t;
  std::vector<uint32_t> tab(3 * (size_t)nt);
  for (int i = 0; i < nt; ++i) {
    uint32_t io = 0, oo = 0, sl = 0;
    for (int u = 0; u < t; ++u)
      if ((i >> u) & 1) {
        io |= 1u << Tin[u];
        oo |= 1u << Tout[u];
        int ip = in_pos[Tout[u]];
        int slot_bit = (int)(std::find(Tin.begin(), Tin.end(), ip) - Tin.begin());
        sl |= 1u << slot_bit;
      }
    tab[i] = io;
    tab[nt + i] = oo;
    tab[2 * nt + i] = sl;
  }
  PermSched ps;
  ps.t_bits = t;
  ps.vec4 = 0;
  ps.tab_off = meta_push(plan, tab);
  ps.n_rest = 0;
  for (int x = 0; x < r; ++x)
    if (std::find(Tin.begin(), Tin.end(), x) == Tin.end()) {
      ps.rest_in[ps.n_rest] = (uint8_t)x;
      ps.rest_out[ps.n_rest] = (uint8_t)inv[x];
      ++ps.n_rest;
    }
  return ps;
}

void apply_perm_schedule(Step& s, const PermSched& ps) {
  s.t_bits = ps.t_bits;
  s.tab_off = ps.tab_off;
  s.n_rest = ps.n_rest;
  s.vec4 = ps.vec4;
  std::memcpy(s.rest_in, ps.rest_in, sizeof(s.rest_in));
  std::memcpy(s.rest_out, ps.rest_out, sizeof(s.rest_out));
}

static void add_permute(Plan& plan, const VTensor& X, const std::vector<int>& target, Ref out, int ci,
                        int split) {
  Step s;
  s.kind = ST_PERMUTE;
  s.split = split;
  s.a = X.ref;
  s.c = out;
  s.contraction = ci;
  const int r = (int)X.legs.size();
  s.rA = s.rC = r;
  s.PA = s.PC = X.P;
  std::vector<int> in_pos(r), inv(r);  // in_pos[o] = input position of output position o
  for (int o = 0; o < r; ++o) in_pos[o] = find_pos(X.legs, target[o]);
  for (int o = 0; o < r; ++o) inv[in_pos[o]] = o;
  // schedule 0 (the default): 32-element runs on both sides, 2^10-element
  // tiles.  Permutes of at least 2^20 elements also get the alternatives
  // that a plan tuner may time: wider input or output runs, smaller tiles
  // (more resident blocks per SM).
  // Each schedule whose output bits 0 and 1 are tile bits 0 and 1 also
  // comes in the four-outputs-per-store form (same tables).
  static const int kSched[][3] = {{5, 5, 10}, {4, 6, 10}, {6, 4, 10}, {5, 5, 9}, {4, 4, 8}};
  const int n_sched = (int64_t)X.P << r >= (1LL << 20) ? 5 : 1;
  for (int v = 0; v < n_sched; ++v) {
    PermSched ps = perm_schedule(plan, in_pos, inv, kSched[v][0], kSched[v][1], kSched[v][2]);
    bool dup = false;
    for (const PermSched& q : s.alts)
      dup |= q.t_bits == ps.t_bits && q.n_rest == ps.n_rest &&
             std::memcmp(q.rest_in, ps.rest_in, sizeof(ps.rest_in)) == 0;
    if (dup) {
      plan.meta.resize((size_t)ps.tab_off);   // the table just pushed is not needed
      continue;
    }
    s.alts.push_back(ps);
    const uint32_t* out_off = plan.meta.data() + ps.tab_off + ((size_t)1 << ps.t_bits);
    if (n_sched > 1 && ps.t_bits >= 2 && out_off[1] == 1 && out_off[2] == 2) {
      ps.vec4 = 1;
      s.alts.push_back(ps);
    }
  }
  apply_perm_schedule(s, s.alts[0]);
  s.bytes = (split == 1 ? 24.0 : 16.0) * (double)vt_elems(X);
  plan.steps.push_back(s);
}

static int layout_steps(Plan& plan, std::string& err) {
  plan.steps.clear();
  plan.bufs.clear();
  plan.n_scale_slots = 0;
  plan.scale_static.clear();
  std::map<int, int> producer;   // workspace buffer id -> index of the step that writes it
  int ci = 0;
  // FP16x3 scale slot of a GEMM operand X: a leaf's maximum is known on the
  // host (static slot, over all its slice variants); an intermediate written
  // by a tensor-core GEMM or a small-operand step has its maximum recorded by
  // that step's epilogue; anything else gets an ABSMAX pass.
  auto operand_slot = [&](const VTensor& X) -> int {
    if (X.ref.kind == 0) {
      const LeafInfo& li = plan.leaf_info[X.ref.id];
      const int64_t n = li.size << li.var_slice_bits.size();
      float m = 0.0f;
      for (int64_t e = 0; e < n; ++e) {
        const cd& v = plan.leaf_arena[(size_t)(li.off + e)];
        m = std::max(m, std::max(std::fabs((float)v.real()), std::fabs((float)v.imag())));
      }
      uint32_t bits;
      std::memcpy(&bits, &m, sizeof(bits));
      plan.scale_static.push_back(bits);
      return -(int)plan.scale_static.size() - 1;
    }
    const int slot = plan.n_scale_slots++;
    auto it = producer.find(X.ref.id);
    if (it != producer.end() && (plan.steps[it->second].kind == ST_GEMM_TC || plan.steps[it->second].kind == ST_SMALL))
      plan.steps[it->second].max_slot = slot;
    else
      add_absmax(plan, X, slot, ci);
    return slot;
  };
  for (auto& pr : plan.order) {
    const int i = pr.first, j = pr.second;
    VTensor A = plan.vts[i], B = plan.vts[j];
    std::vector<int> shared;
    for (int l : A.legs)
      if (find_pos(B.legs, l) >= 0) shared.push_back(l);
    // roles: big operand streams (rows), small operand is the "gate"
    const VTensor& big = vt_elems(A) >= vt_elems(B) ? A : B;
    const VTensor& sml = vt_elems(A) >= vt_elems(B) ? B : A;
    std::vector<int> K, M, N;
    for (int l : big.legs)
      if (find_pos(shared, l) >= 0) K.push_back(l); else M.push_back(l);
    for (int l : sml.legs)
      if (find_pos(shared, l) < 0) N.push_back(l);
    const int nk = (int)K.size(), nm = (int)M.size(), nn = (int)N.size();
    VTensor C;
    C.tq = A.tq | B.tq;
    C.P = plan.book.count(C.tq);
    int mapA_mode, mapB_mode;
    int64_t mapA_off, mapB_off;
    C.legs.clear();
    std::vector<int> cl;
    const bool use_small = nk <= plan.small_max_bits && nn <= plan.small_max_bits;
    if (use_small) {
      for (int l : M) cl.push_back(l);
      for (int l : N) cl.push_back(l);
    } else {
      for (int l : N) cl.push_back(l);
      for (int l : M) cl.push_back(l);
    }
    C.legs = cl;
    const double lc = std::log2((double)C.P) + (double)cl.size();
    if (lc > plan.cap_log2 + 1e-9) {
      err = "contraction " + std::to_string(ci) + " exceeds the size cap (2^" + std::to_string(lc) + " elements)";
      return TN_ERR_OOM;
    }
    plan.max_log2 = std::max(plan.max_log2, lc);
    set_map(plan, big, C, mapA_mode, mapA_off);
    set_map(plan, sml, C, mapB_mode, mapB_off);
    const int64_t eC = vt_elems(C);
    const double macs = (double)C.P * std::exp2((double)(nm + nn + nk));
    plan.tc_macs += macs;
    plan.alg_bytes += 8.0 * (double)(vt_elems(big) + vt_elems(sml) + eC);

    std::vector<uint32_t> bk(1u << nk), bn(1u << nn);
    for (uint32_t k = 0; k < bk.size(); ++k) {
      uint32_t o = 0;
      for (int q = 0; q < nk; ++q)
        if ((k >> q) & 1) o |= 1u << find_pos(sml.legs, K[q]);
      bk[k] = o;
    }
    for (uint32_t n = 0; n < bn.size(); ++n) {
      uint32_t o = 0;
      for (int q = 0; q < nn; ++q)
        if ((n >> q) & 1) o |= 1u << find_pos(sml.legs, N[q]);
      bn[n] = o;
    }

    if (use_small) {
      Step s;
      s.kind = ST_SMALL;
      s.contraction = ci;
      s.a = big.ref;
      s.b = sml.ref;
      s.rA = (int)big.legs.size();
      s.rB = (int)sml.legs.size();
      s.rC = (int)cl.size();
      s.PA = big.P; s.PB = sml.P; s.PC = C.P;
      s.nk = nk; s.nm = nm; s.nn = nn;
      s.mapA_mode = mapA_mode; s.mapA_off = mapA_off;
      s.mapB_mode = mapB_mode; s.mapB_off = mapB_off;
      for (int q = 0; q < nk; ++q) s.kposA[q] = find_pos(big.legs, K[q]);
      for (size_t k = 0; k < bk.size(); ++k) s.boffK[k] = bk[k];
      for (size_t n = 0; n < bn.size(); ++n) s.boffN[n] = bn[n];
      s.macs = macs;
      s.bytes = 8.0 * (double)(vt_elems(big) + vt_elems(sml) + eC);
      const int st = (int)plan.steps.size();
      touch(plan, s.a, st);
      touch(plan, s.b, st);
      s.c = Ref{1, new_buf(plan, eC * 8, st)};
      C.ref = s.c;
      plan.steps.push_back(s);
      producer[s.c.id] = (int)plan.steps.size() - 1;
    } else {
      // A' = big permuted to [K][M] (K legs low) unless already so
      std::vector<int> target;
      for (int l : K) target.push_back(l);
      for (int l : M) target.push_back(l);
      Ref aref = big.ref;
      // 16-bit operands need K >= 4 (16-byte rows); K = 2 steps use the tf32 kernel
      const int h16 = nk >= 2 ? (plan.gemm_engine == TN_GEMM_TC_BF16X3 ? 1 : plan.gemm_engine == TN_GEMM_TC_FP16X3 ? 2 : 0) : 0;
      const bool bf16 = h16 != 0;
      const bool tc = plan.gemm_engine != TN_GEMM_SIMT_FP32 && nk >= 1;
      int slot_a = -1, slot_b = -1;
      if (tc || target != big.legs) {
        // the tensor-core GEMM reads A as hi/lo planes: always a (possibly
        // identity) permute in split mode
        if (h16 == 2) slot_a = operand_slot(big);
        const int st = (int)plan.steps.size();
        touch(plan, big.ref, st);
        Ref out{1, new_buf(plan, vt_elems(big) * 8 * (tc && !bf16 ? 2 : 1), st)};
        add_permute(plan, big, target, out, ci, tc ? (h16 == 2 ? 3 : h16 == 1 ? 2 : 1) : 0);
        plan.steps.back().slot = slot_a;
        aref = out;
      }
      // B' prep
      Step p;
      p.kind = tc ? ST_BPREP_TC : ST_BPREP_C;
      p.h16 = h16;
      if (h16 == 2) slot_b = operand_slot(sml);
      p.slot = slot_b;
      p.contraction = ci;
      p.a = sml.ref;
      p.rA = (int)sml.legs.size();
      p.PA = sml.P;
      p.nk = nk; p.nn = nn;
      p.bk_off = meta_push(plan, bk);
      p.bn_off = meta_push(plan, bn);
      if (tc && (int)sml.legs.size() == nk + nn && vt_elems(sml) >= (1LL << 20)) {
        // the permute alternative: B's legs to [N][K] order (K legs low),
        // written as the real embedding; the plan's rule takes it when the
        // gather's consecutive k are not consecutive in memory
        std::vector<int> target;
        for (int l : K) target.push_back(l);
        for (int l : N) target.push_back(l);
        const int r = (int)target.size();
        std::vector<int> in_pos(r), inv(r);
        for (int o = 0; o < r; ++o) in_pos[o] = find_pos(sml.legs, target[o]);
        for (int o = 0; o < r; ++o) inv[in_pos[o]] = o;
        PermSched ps = perm_schedule(plan, in_pos, inv, 5, 5, 10);
        p.alts.push_back(ps);
        apply_perm_schedule(p, ps);
        p.bprep_embed0 = nk >= 1 && bk[1] != 1u;
      }
      const int64_t bprep_bytes =
          tc ? 2LL * sml.P * (2LL << nn) * (2LL << nk) * (bf16 ? 2 : 4) : sml.P * (1LL << (nk + nn)) * 8;
      {
        const int st = (int)plan.steps.size();
        touch(plan, sml.ref, st);
        p.c = Ref{1, new_buf(plan, bprep_bytes, st)};
        p.bytes = 8.0 * (double)vt_elems(sml) + (double)bprep_bytes;
        plan.steps.push_back(p);
      }
      Step g;
      g.kind = tc ? ST_GEMM_TC : ST_GEMM_SIMT;
      g.h16 = h16;
      g.slot = slot_a;
      g.slotB = slot_b;
      g.contraction = ci;
      g.a = aref;
      g.b = p.c;
      g.rA = (int)big.legs.size();
      g.rB = (int)sml.legs.size();
      g.rC = (int)cl.size();
      g.PA = big.P; g.PB = sml.P; g.PC = C.P;
      g.nk = nk; g.nm = nm; g.nn = nn;
      g.mapA_mode = mapA_mode; g.mapA_off = mapA_off;
      g.mapB_mode = mapB_mode; g.mapB_off = mapB_off;
      g.macs = macs;
      g.bytes = 8.0 * (double)(vt_elems(big) + eC) + (double)bprep_bytes;
      const int st = (int)plan.steps.size();
      touch(plan, g.a, st);
      touch(plan, g.b, st);
      g.c = Ref{1, new_buf(plan, eC * 8, st)};
      C.ref = g.c;
      plan.steps.push_back(g);
      producer[g.c.id] = (int)plan.steps.size() - 1;
    }
    for (auto& s : plan.steps)
      if (s.contraction == ci) { s.vt_a = i; s.vt_b = j; s.vt_c = (int)plan.vts.size(); }
    plan.vts.push_back(C);
    plan.vts[i].alive = false;
    plan.vts[j].alive = false;
    // the result lives at slot i: keep a pointer from i to the new tensor
    // (the order refers to slots, see build_plan)
    ++ci;
  }
  plan.n_contractions = ci;
  return TN_OK;
}

// Tensor-core B-preparation steps that may run beside an earlier GEMM.  The
// B operand of a stem contraction is usually a branch finished long before
// (only the A side comes from the step just before), so its preparation, an
// HBM-bound pass, can run on a second stream during the previous tensor-core
// GEMM, which leaves HBM mostly idle.  A step qualifies when its operand was
// written before that GEMM and its FP16 scale (if any) is a leaf's static
// slot or the operand producer's epilogue maximum (not an ABSMAX step of its
// own), and it is large (at least 64 MiB) beside a long GEMM (at least 2^34
// complex MACs).  Its output buffer then starts at the fork, so nothing running
// between the fork and the consuming GEMM shares its memory; its operand is
// live from its producer to the B-prep already.
constexpr double kSideMinBytes = 64.0 * (1 << 20);   // B-prep algorithmic bytes
constexpr double kSideMinMacs = 0x1p34;              // complex MACs of the GEMM it runs beside

static void schedule_side_bprep(Plan& plan) {
  std::map<int, int> producer;   // workspace buffer id -> step that writes it
  const int n = (int)plan.steps.size();
  plan.n_side_bprep = 0;
  for (int i = 0; i < n; ++i) {
    Step& x = plan.steps[i];
    if (x.kind == ST_BPREP_TC && i + 1 < n && plan.steps[i + 1].kind == ST_GEMM_TC &&
        plan.steps[i + 1].b.kind == 1 && plan.steps[i + 1].b.id == x.c.id) {
      int prod = -1;
      bool ok = true;
      if (x.a.kind == 1) {
        auto it = producer.find(x.a.id);
        ok = it != producer.end();
        if (ok) prod = it->second;
      }
      if (ok && x.slot >= 0) ok = prod >= 0 && plan.steps[prod].max_slot == x.slot;
      int q = -1;
      for (int j = i - 1; ok && j > prod; --j)
        if (plan.steps[j].kind == ST_GEMM_TC) { q = j; break; }
      // only a large preparation beside a long GEMM gains: each fork and join
      // costs a dependency edge, and a short GEMM leaves nothing to hide under
      if (q >= 0 && (x.bytes < kSideMinBytes || plan.steps[q].macs < kSideMinMacs)) q = -1;
      if (ok && q >= 0) {
        x.fork = q;
        plan.bufs[x.c.id].first = std::min(plan.bufs[x.c.id].first, q);
        ++plan.n_side_bprep;
        // beside a GEMM only the gather kernel fits (one small block per SM)
        x.alts.clear();
        x.bprep_embed0 = 0;
      }
    }
    if (x.c.kind == 1) producer[x.c.id] = i;
  }
}

static void plan_arena(Plan& plan) {
  std::vector<int> idx(plan.bufs.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (plan.bufs[a].bytes != plan.bufs[b].bytes) return plan.bufs[a].bytes > plan.bufs[b].bytes;
    return a < b;
  });
  std::vector<int> placed;
  int64_t peak = 0;
  for (int b : idx) {
    BufInfo& B = plan.bufs[b];
    std::vector<std::pair<int64_t, int64_t>> busy;
    for (int o : placed) {
      const BufInfo& O = plan.bufs[o];
      if (O.last < B.first || B.last < O.first) continue;
      busy.push_back({O.off, O.off + O.bytes});
    }
    std::sort(busy.begin(), busy.end());
    int64_t off = 0;
    for (auto& iv : busy) {
      if (off + B.bytes <= iv.first) break;
      off = std::max(off, iv.second);
    }
    B.off = off;
    peak = std::max(peak, off + B.bytes);
    placed.push_back(b);
  }
  plan.workspace_bytes = peak;
}

// --------------------------------------------------------------------- driver

// Leaves: the tensors left after simplification, each stored once per value
// of its sliced (half) legs, and their virtual tensors (device legs only).
static void build_leaves(Plan& plan, const std::vector<HostTensor>& T) {
  plan.leaves.clear();
  for (auto& t : T)
    if (t.alive) plan.leaves.push_back(t);
  plan.leaf_info.clear();
  plan.leaf_arena.clear();
  plan.vts.clear();
  for (auto& t : plan.leaves) {
    LeafInfo li;
    std::vector<int> half_pos;
    std::vector<int> dev_legs;
    for (size_t p = 0; p < t.legs.size(); ++p) {
      if (plan.legs[t.legs[p]].kind == LEG_HALF) {
        half_pos.push_back((int)p);
        li.var_slice_bits.push_back(plan.legs[t.legs[p]].slice_bit);
      } else dev_legs.push_back(t.legs[p]);
    }
    li.size = t.P() * (1LL << dev_legs.size());
    // align each leaf to 16 complex elements (128 bytes)
    while (plan.leaf_arena.size() % 16) plan.leaf_arena.push_back(cd(0, 0));
    li.off = (int64_t)plan.leaf_arena.size();
    const int nh = (int)half_pos.size();
    for (int v = 0; v < (1 << nh); ++v) {
      HostTensor x = t;
      for (int hh = nh - 1; hh >= 0; --hh) select_leg(x, half_pos[hh], (v >> hh) & 1);
      plan.leaf_arena.insert(plan.leaf_arena.end(), x.data.begin(), x.data.end());
    }
    plan.leaf_info.push_back(li);
    VTensor vt;
    vt.legs = dev_legs;
    vt.tq = t.tq;
    vt.P = t.P();
    vt.ref = Ref{0, (int)plan.leaf_info.size() - 1};
    plan.vts.push_back(vt);
  }
}

// Two half legs of one tensor that carry the same slice bit (the two ends of
// a cut edge, brought together by a host contraction) always take the same
// value: keep the entries where they agree and drop the second leg.
static void merge_half_legs(const Plan& plan, HostTensor& T) {
  for (bool again = true; again;) {
    again = false;
    for (size_t a = 0; a < T.legs.size() && !again; ++a)
      for (size_t b = a + 1; b < T.legs.size() && !again; ++b) {
        const Leg& La = plan.legs[T.legs[a]];
        const Leg& Lb = plan.legs[T.legs[b]];
        if (La.kind != LEG_HALF || Lb.kind != LEG_HALF || La.slice_bit != Lb.slice_bit) continue;
        const int r = (int)T.legs.size();
        const int64_t n_old = 1LL << r, n_new = 1LL << (r - 1);
        std::vector<cd> d((size_t)(T.P() * n_new));
        const int64_t lo_mask = (1LL << b) - 1;
        for (int64_t p = 0; p < T.P(); ++p)
          for (int64_t i = 0; i < n_new; ++i) {
            const int64_t v = (i >> a) & 1;    // leg b takes leg a's value
            const int64_t src = ((i & ~lo_mask) << 1) | (v << b) | (i & lo_mask);
            d[(size_t)(p * n_new + i)] = T.data[(size_t)(p * n_old + src)];
          }
        T.data.swap(d);
        T.legs.erase(T.legs.begin() + b);
        again = true;
      }
  }
}

// Host folding.  A contraction of the order whose two operands are host
// tensors (leaves, or results folded before) and whose result is small
// (pattern axis times device legs at most 2^fold_log2 elements, at most 2^6
// slice variants) is carried out here, once, in FP64, and its result becomes a
// leaf: the device then runs only the contractions that involve an
// intermediate.  A pair sharing an automatically sliced leg (one leg id on
// both operands, summed by the passes of a slice) is left to the device.
// On return `device_order` holds the remaining pairs over the new leaves and
// plan.leaves / leaf_info / vts describe those leaves.
static void fold_small(Plan& plan, const std::vector<std::pair<int, int>>& slot_order, int fold_log2,
                       std::vector<std::pair<int, int>>& device_order) {
  const int nleaf = (int)plan.leaves.size();
  std::vector<HostTensor> T = plan.leaves;
  std::vector<char> host(nleaf, 1), is_leaf(nleaf, 0);
  std::vector<int> newslot(nleaf, -1);
  std::vector<std::pair<int, int>> dev;
  auto use_on_device = [&](int s) {   // the tensor in slot s (leaf or fold) is a device leaf
    if (host[s]) {
      host[s] = 0;
      is_leaf[s] = 1;
    }
  };
  int last = -1;
  for (auto pr : slot_order) {
    const int i = pr.first, j = pr.second;
    last = i;
    if (fold_log2 >= 0 && host[i] && host[j]) {
      bool shared_half = false;
      int dev_legs = 0, half_bits = 0;
      std::vector<int> bits;
      for (int l : T[i].legs) {
        const bool in_b = find_pos(T[j].legs, l) >= 0;
        if (plan.legs[l].kind == LEG_HALF && in_b) shared_half = true;
        if (in_b) continue;
        if (plan.legs[l].kind == LEG_HALF) bits.push_back(plan.legs[l].slice_bit); else ++dev_legs;
      }
      for (int l : T[j].legs) {
        if (find_pos(T[i].legs, l) >= 0) continue;
        if (plan.legs[l].kind == LEG_HALF) bits.push_back(plan.legs[l].slice_bit); else ++dev_legs;
      }
      std::sort(bits.begin(), bits.end());
      half_bits = (int)(std::unique(bits.begin(), bits.end()) - bits.begin());
      const double lsz = std::log2((double)plan.book.count(T[i].tq | T[j].tq)) + dev_legs;
      if (!shared_half && lsz <= fold_log2 + 1e-9 && half_bits <= 6) {
        T[i] = contract_host(T[i], T[j], plan.book);
        merge_half_legs(plan, T[i]);
        host[j] = 0;
        continue;
      }
    }
    use_on_device(i);
    use_on_device(j);
    dev.push_back(pr);
  }
  if (dev.empty()) is_leaf[last >= 0 ? last : 0] = 1;   // everything folded: the result is the only leaf
  // device leaves keep the order of their slots (with nothing folded, the
  // leaves and their ids are those of the simplified network)
  std::vector<HostTensor> leaves;
  for (int s = 0; s < nleaf; ++s)
    if (is_leaf[s]) {
      newslot[s] = (int)leaves.size();
      leaves.push_back(T[s]);
    }
  device_order.clear();
  for (auto& pr : dev) device_order.push_back({newslot[pr.first], newslot[pr.second]});
  build_leaves(plan, leaves);
}

// Slice `legs` (bond legs between leaves) as internal edges: each becomes a
// half leg with slice bit k, k+1, ... on both leaves that hold it.
static void apply_internal_slices(Plan& plan, const std::vector<HostTensor>& T, const std::vector<int>& legs) {
  plan.n_internal = (int)legs.size();
  plan.internal_edges.clear();
  for (size_t i = 0; i < legs.size(); ++i) {
    plan.legs[legs[i]].kind = LEG_HALF;
    plan.legs[legs[i]].slice_bit = plan.n_sliced + (int)i;
    plan.internal_edges.push_back(plan.leg_edge[legs[i]]);
  }
  build_leaves(plan, T);
}

int build_plan(const PlanInput& in, Plan& plan, std::string& err) {
  const int n = in.n_qubits;
  if (n < 1 || n > 64) { err = "n_qubits must be in [1, 64]"; return TN_ERR_INVALID; }
  if (in.n_gates < 0) { err = "n_gates < 0"; return TN_ERR_INVALID; }
  for (int g = 0; g < in.n_gates; ++g) {
    const int ar = in.arity[g];
    if (ar != 1 && ar != 2) { err = "gate " + std::to_string(g) + ": arity must be 1 or 2"; return TN_ERR_INVALID; }
    if (in.q0[g] < 0 || in.q0[g] >= n || (ar == 2 && (in.q1[g] < 0 || in.q1[g] >= n || in.q1[g] == in.q0[g]))) {
      err = "gate " + std::to_string(g) + ": bad qubit";
      return TN_ERR_INVALID;
    }
  }
  plan.n_qubits = n;
  plan.open_qubits = in.open_qubits;
  if ((int)in.open_qubits.size() > 30) { err = "at most 30 open qubits"; return TN_ERR_INVALID; }
  plan.open_mask = 0;
  for (int q : in.open_qubits) {
    if (q < 0 || q >= n) { err = "open qubit out of range"; return TN_ERR_INVALID; }
    if ((plan.open_mask >> q) & 1) { err = "duplicate open qubit"; return TN_ERR_INVALID; }
    plan.open_mask |= 1ULL << q;
  }
  const uint64_t full = n == 64 ? ~0ULL : ((1ULL << n) - 1);
  plan.tail_mask = full & ~plan.open_mask;
  if (in.tails.empty()) { err = "n_tails must be >= 1"; return TN_ERR_INVALID; }
  plan.tails_raw = in.tails;
  plan.book.tails.clear();
  for (uint64_t t : in.tails) plan.book.tails.push_back(t & plan.tail_mask);
  plan.cap_log2 = in.cap_log2;
  plan.gemm_engine = in.gemm_engine;
  plan.gemm_pair = in.gemm_pair;
  plan.small_max_bits = in.small_max_bits;

  // edges
  std::set<std::pair<int, int>> seen;
  int k = 0, pins = 0, companions = 0;
  double comp_factor = 1.0;
  for (auto& e : in.edges) {
    if (e.gate < 0 || e.gate >= in.n_gates) { err = "edge: gate out of range"; return TN_ERR_INVALID; }
    if (e.leg < 0 || e.leg >= in.arity[e.gate]) { err = "edge: leg out of range"; return TN_ERR_INVALID; }
    if (!seen.insert({e.gate, e.leg}).second) { err = "edge listed twice"; return TN_ERR_INVALID; }
    if (e.kind == TN_EDGE_SLICE) ++k;
    else if (e.kind == TN_EDGE_PIN) {
      if (e.value != 0 && e.value != 1) { err = "pin value must be 0 or 1"; return TN_ERR_INVALID; }
      ++pins;
    } else if (e.kind == TN_EDGE_COMPANION) {
      if (in.arity[e.gate] != 2) { err = "companion edge on a single-qubit gate"; return TN_ERR_INVALID; }
      ++k;
      ++companions;
      // kept norm fraction of the rank-one cut, averaged over the two values of
      // the pinned input: |F[partner out = v]|^2 / |F|^2 with F = gate[:, in_a = v]
      const cd* U = in.mats + (size_t)e.gate * 16;
      double frac = 0.0;
      for (int v = 0; v < 2; ++v) {
        double kept = 0.0, tot = 0.0;
        for (int o0 = 0; o0 < 2; ++o0)
          for (int o1 = 0; o1 < 2; ++o1)
            for (int other = 0; other < 2; ++other) {
              const int i0 = e.leg == 0 ? v : other, i1 = e.leg == 0 ? other : v;
              const double w = std::norm(U[(2 * o0 + o1) * 4 + (2 * i0 + i1)]);
              tot += w;
              const int partner_out = e.leg == 0 ? o1 : o0;
              if (partner_out == v) kept += w;
            }
        frac += 0.5 * (tot > 0 ? kept / tot : 1.0);
      }
      comp_factor *= frac;
    } else { err = "edge: unknown kind"; return TN_ERR_INVALID; }
  }
  if (k > 40) { err = "at most 40 sliced edges"; return TN_ERR_INVALID; }
  if (k + in.auto_slice > 62) { err = "sliced edges plus auto_slice above 62"; return TN_ERR_INVALID; }
  plan.n_sliced = k;
  plan.n_internal = 0;
  plan.internal_edges.clear();
  plan.n_pinned = pins;
  plan.n_companion = companions;
  plan.companion_factor = comp_factor;

  Builder b(plan);
  int rc = build_network(in, plan, b, err);
  if (rc) return rc;
  plan.leg_edge.assign(plan.legs.size(), {-1, -1});
  for (auto& u : b.consumed)
    if (plan.legs[u.leg].kind == LEG_BOND) plan.leg_edge[u.leg] = {u.gate, u.pos};
  simplify(plan, b.T, in.absorb_log2);

  build_leaves(plan, b.T);
  const int nleaf = (int)plan.leaves.size();

  // order over slots 0..nleaf-1 (result of (i, j) stored at slot i)
  std::vector<std::pair<int, int>> slot_order;
  std::vector<GNode> init(nleaf);
  for (int i = 0; i < nleaf; ++i) {
    init[i].legs = plan.vts[i].legs;
    init[i].tq = plan.vts[i].tq;
    init[i].lsz = std::log2((double)plan.vts[i].P) + (double)plan.vts[i].legs.size();
  }
  if (in.order) {
    std::vector<char> alive(nleaf, 1);
    for (int64_t p = 0; p < in.n_pairs; ++p) {
      int i = in.order[2 * p], j = in.order[2 * p + 1];
      if (i < 0 || j < 0 || i >= nleaf || j >= nleaf || i == j || !alive[i] || !alive[j]) {
        err = "order: pair " + std::to_string(p) + " names a bad or consumed tensor";
        return TN_ERR_INVALID;
      }
      alive[j] = 0;
      slot_order.push_back({i, j});
    }
    // finish with outer products if tensors remain
    std::vector<int> rest;
    for (int i = 0; i < nleaf; ++i)
      if (alive[i]) rest.push_back(i);
    for (size_t r = 1; r < rest.size(); ++r) slot_order.push_back({rest[0], rest[r]});
    if (in.auto_slice > 0) {
      // the caller's order, sliced to the cap
      SliceResult sr = slice_order(plan, plan.book, init, slot_order, plan.cap_log2, in.auto_slice);
      if (!sr.ok) {
        err = "the given order exceeds the size cap (automatic slicing: " + sr.why + ")";
        return TN_ERR_OOM;
      }
      if (!sr.legs.empty()) apply_internal_slices(plan, b.T, sr.legs);
    }
  } else {
    std::vector<int> cut;
    rc = greedy_order(plan, init, plan.cap_log2, in.order_trials, in.order_seed, in.auto_slice, slot_order, cut, err);
    if (rc) return rc;
    if (!cut.empty()) apply_internal_slices(plan, b.T, cut);
  }
  // keep the user-visible order in slot form (over the simplified leaves)
  std::vector<std::pair<int, int>> saved_slots = slot_order;
  // small contractions of host tensors become leaves; the device runs the rest
  std::vector<std::pair<int, int>> device_order;
  fold_small(plan, slot_order, in.fold_log2, device_order);
  const int ndev = (int)plan.leaves.size();
  // translate slot pairs to virtual-tensor pairs
  std::vector<int> slot_vt(ndev);
  for (int i = 0; i < ndev; ++i) slot_vt[i] = i;
  plan.order.clear();
  std::vector<std::pair<int, int>> vt_pairs;
  for (auto& pr : device_order) {
    vt_pairs.push_back({slot_vt[pr.first], slot_vt[pr.second]});
    slot_vt[pr.first] = ndev + (int)vt_pairs.size() - 1;
  }
  plan.order = vt_pairs;
  plan.max_log2 = 0;
  for (auto& v : plan.vts) plan.max_log2 = std::max(plan.max_log2, std::log2((double)v.P) + (double)v.legs.size());
  plan.tc_macs = 0;
  plan.alg_bytes = 0;
  rc = layout_steps(plan, err);
  if (rc) return rc;
  plan.order = saved_slots;

  // final tensor
  int fvt = ndev == 1 && device_order.empty() ? 0 : (int)plan.vts.size() - 1;
  if (nleaf == 0) { err = "empty network"; return TN_ERR_INVALID; }
  const VTensor& F = plan.vts[fvt];
  // the final tensor must carry exactly the open legs and every tail projector
  for (int l : F.legs)
    if (plan.legs[l].kind != LEG_OPEN) { err = "internal: final tensor has a non-open leg"; return TN_ERR_INVALID; }
  if ((int)F.legs.size() != (int)plan.open_qubits.size()) { err = "internal: open legs missing"; return TN_ERR_INVALID; }
  if (F.tq != plan.tail_mask) { err = "internal: tail projectors missing"; return TN_ERR_INVALID; }
  plan.fin.ref = F.ref;
  plan.fin.vt = fvt;
  plan.fin.rF = (int)F.legs.size();
  plan.fin.PF = F.P;
  for (size_t p = 0; p < F.legs.size(); ++p) plan.fin.open_pos[plan.legs[F.legs[p]].open_index] = (int)p;
  const auto& fp = plan.book.get(plan.tail_mask);
  plan.n_patterns_final = (int64_t)fp.size();
  std::vector<uint32_t> pidx(plan.book.tails.size());
  for (size_t g = 0; g < pidx.size(); ++g) pidx[g] = (uint32_t)pat_index(fp, plan.book.tails[g]);
  plan.fin.pidx_off = meta_push(plan, pidx);
  touch(plan, F.ref, (int)plan.steps.size());
  if (in.side_bprep) schedule_side_bprep(plan);
  plan_arena(plan);
  return TN_OK;
}

// ------------------------------------------------------------------- describe

std::string describe_plan(const Plan& plan, bool with_data) {
  std::ostringstream o;
  o.precision(17);
  o << "{\"n_qubits\":" << plan.n_qubits << ",\"n_sliced\":" << plan.n_sliced << ",\"n_pinned\":" << plan.n_pinned;
  o << ",\"n_internal\":" << plan.n_internal << ",\"internal_edges\":[";
  for (size_t e = 0; e < plan.internal_edges.size(); ++e)
    o << (e ? "," : "") << "[" << plan.internal_edges[e].first << "," << plan.internal_edges[e].second << "]";
  o << "]";
  o << ",\"tail_mask\":" << plan.tail_mask << ",\"open_mask\":" << plan.open_mask;
  o << ",\"legs\":[";
  for (size_t l = 0; l < plan.legs.size(); ++l) {
    if (l) o << ",";
    o << "[" << plan.legs[l].kind << "," << plan.legs[l].slice_bit << "," << plan.legs[l].open_index << "]";
  }
  o << "],\"leaves\":[";
  for (size_t i = 0; i < plan.leaves.size(); ++i) {
    const auto& t = plan.leaves[i];
    const auto& li = plan.leaf_info[i];
    if (i) o << ",";
    o << "{\"legs\":[";
    for (size_t p = 0; p < t.legs.size(); ++p) o << (p ? "," : "") << t.legs[p];
    o << "],\"dev_legs\":[";
    bool first = true;
    for (int l : plan.vts[i].legs) { o << (first ? "" : ",") << l; first = false; }
    o << "],\"tq\":" << t.tq << ",\"P\":" << t.P() << ",\"var_slice_bits\":[";
    for (size_t p = 0; p < li.var_slice_bits.size(); ++p) o << (p ? "," : "") << li.var_slice_bits[p];
    o << "],\"size\":" << li.size;
    if (with_data) {
      o << ",\"re\":[";
      const int64_t nv = li.size << li.var_slice_bits.size();
      for (int64_t e = 0; e < nv; ++e) o << (e ? "," : "") << plan.leaf_arena[(size_t)(li.off + e)].real();
      o << "],\"im\":[";
      for (int64_t e = 0; e < nv; ++e) o << (e ? "," : "") << plan.leaf_arena[(size_t)(li.off + e)].imag();
      o << "]";
    }
    o << "}";
  }
  o << "],\"vts\":[";
  for (size_t v = 0; v < plan.vts.size(); ++v) {
    if (v) o << ",";
    o << "{\"legs\":[";
    for (size_t p = 0; p < plan.vts[v].legs.size(); ++p) o << (p ? "," : "") << plan.vts[v].legs[p];
    o << "],\"tq\":" << plan.vts[v].tq << ",\"P\":" << plan.vts[v].P << "}";
  }
  o << "],\"order\":[";
  for (size_t p = 0; p < plan.order.size(); ++p) o << (p ? "," : "") << "[" << plan.order[p].first << "," << plan.order[p].second << "]";
  o << "],\"steps\":[";
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    const Step& st = plan.steps[s];
    if (s) o << ",";
    o << "{\"kind\":" << st.kind << ",\"contraction\":" << st.contraction << ",\"vt_a\":" << st.vt_a << ",\"vt_b\":"
      << st.vt_b << ",\"vt_c\":" << st.vt_c << ",\"nk\":" << st.nk << ",\"nm\":" << st.nm << ",\"nn\":" << st.nn
      << ",\"PA\":" << st.PA << ",\"PB\":" << st.PB << ",\"PC\":" << st.PC << ",\"macs\":" << st.macs
      << ",\"bytes\":" << st.bytes << ",\"rA\":" << st.rA << ",\"rB\":" << st.rB << ",\"rC\":" << st.rC
      << ",\"a\":[" << st.a.kind << "," << st.a.id << "],\"b\":[" << st.b.kind << "," << st.b.id << "],\"c\":["
      << st.c.kind << "," << st.c.id << "],\"t_bits\":" << st.t_bits << ",\"split\":" << st.split << ",\"h16\":" << st.h16 << ",\"slot\":" << st.slot << ",\"slotB\":" << st.slotB << ",\"max_slot\":" << st.max_slot << ",\"fork\":" << st.fork
      << ",\"tab_off\":" << st.tab_off << ",\"vec4\":" << st.vec4 << ",\"n_rest\":" << st.n_rest << ",\"rest_in\":[";
    for (int v = 0; v < st.n_rest; ++v) o << (v ? "," : "") << (int)st.rest_in[v];
    o << "],\"rest_out\":[";
    for (int v = 0; v < st.n_rest; ++v) o << (v ? "," : "") << (int)st.rest_out[v];
    o << "],\"kposA\":[" << st.kposA[0] << "," << st.kposA[1] << "," << st.kposA[2] << "," << st.kposA[3]
      << "],\"boffK\":[";
    for (int v = 0; v < 16; ++v) o << (v ? "," : "") << st.boffK[v];
    o << "],\"boffN\":[";
    for (int v = 0; v < 16; ++v) o << (v ? "," : "") << st.boffN[v];
    o << "],\"mapA\":[" << st.mapA_mode << "," << st.mapA_off << "],\"mapB\":[" << st.mapB_mode << ","
      << st.mapB_off << "],\"bk_off\":" << st.bk_off << ",\"bn_off\":" << st.bn_off << ",\"bprep_embed0\":" << st.bprep_embed0 << ",\"variant\":" << st.variant
      << ",\"tile_cap\":" << st.tile_cap << ",\"pair\":" << st.pair << ",\"alts\":[";
    for (size_t a = 0; a < st.alts.size(); ++a) {
      const PermSched& ps = st.alts[a];
      o << (a ? "," : "") << "{\"t_bits\":" << ps.t_bits << ",\"vec4\":" << ps.vec4 << ",\"tab_off\":" << ps.tab_off << ",\"n_rest\":" << ps.n_rest
        << ",\"rest_in\":[";
      for (int v = 0; v < ps.n_rest; ++v) o << (v ? "," : "") << (int)ps.rest_in[v];
      o << "],\"rest_out\":[";
      for (int v = 0; v < ps.n_rest; ++v) o << (v ? "," : "") << (int)ps.rest_out[v];
      o << "]}";
    }
    o << "]}";
  }
  o << "],\"final\":{\"vt\":" << plan.fin.vt << ",\"open_pos\":[";
  for (size_t j = 0; j < plan.open_qubits.size(); ++j) o << (j ? "," : "") << plan.fin.open_pos[j];
  o << "],\"rF\":" << plan.fin.rF << ",\"PF\":" << plan.fin.PF << ",\"ref\":[" << plan.fin.ref.kind << ","
    << plan.fin.ref.id << "],\"pidx_off\":" << plan.fin.pidx_off << "}";
  o << ",\"bufs\":[";
  for (size_t b = 0; b < plan.bufs.size(); ++b)
    o << (b ? "," : "") << "[" << plan.bufs[b].off << "," << plan.bufs[b].bytes << "," << plan.bufs[b].first << ","
      << plan.bufs[b].last << "]";
  o << "],\"leaf_arena_elems\":" << plan.leaf_arena.size();
  if (with_data) {
    o << ",\"meta\":[";
    for (size_t m = 0; m < plan.meta.size(); ++m) o << (m ? "," : "") << plan.meta[m];
    o << "],\"leaf_info\":[";
    for (size_t l = 0; l < plan.leaf_info.size(); ++l) o << (l ? "," : "") << "[" << plan.leaf_info[l].off << "," << plan.leaf_info[l].size << "," << plan.leaf_info[l].var_slice_bits.size() << "]";
    o << "]";
  }
  o << ",\"tc_macs\":" << plan.tc_macs << ",\"alg_bytes\":" << plan.alg_bytes << ",\"max_log2\":" << plan.max_log2
    << ",\"workspace_bytes\":" << plan.workspace_bytes << "}";
  return o.str();
}

}  // namespace tn

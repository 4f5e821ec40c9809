// Request server: continuous admission of amplitude and sampling requests on
// several circuits, with head tensors cached in HBM.
//
// A dispatcher thread owns `n_slots` slots, each a CUDA stream with pinned and
// device staging buffers.  Queued requests are admitted into free slots as
// soon as a slot and the HBM budget allow; admitted requests run concurrently
// on their slots' streams, so work that arrives while other requests are on
// the GPU overlaps with it.  The first request on a circuit contracts its kept
// slices into a new head (the circuit is BUILDING); later requests on that
// circuit wait on the head's ready event on the device, not on the host.
// Heads are freed least-recently-used first when a new head does not fit the
// budget.  Completion is detected by polling per-slot events; latency is
// measured from submit to the moment the result is in the caller's buffer.
// Amplitude requests on the same ready circuit (and output type) that wait in
// the queue when a slot frees up are merged into that slot: one staging copy,
// one lookup launch and one copy back serve up to kMaxMerge of them, each
// with its own status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "handles.h"
#include "kernels.h"
#include "tn_gb300.h"

namespace {

using Clock = std::chrono::steady_clock;

int fail(int code, const std::string& msg) {
  tn::set_last_error(msg);
  return code;
}

struct Request {
  uint64_t ticket = 0;
  tn_request r{};
  Clock::time_point t_submit, t_start, t_done;
  int status = TN_OK;
  std::string err;
  bool done = false;
  bool merged = false;   // taken into another request's slot
};

enum { C_EMPTY = 0, C_BUILDING = 1, C_READY = 2 };

struct Circuit {
  tn_plan_t* plan = nullptr;
  tn_range kept{0, 0};
  tn_head_t* head = nullptr;
  int state = C_EMPTY;
  cudaEvent_t ready = nullptr;
  int builder_slot = -1;
  int users = 0;           // admitted requests not yet retired
  uint64_t last_use = 0;
  int64_t bytes = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Request* req = nullptr;
  std::vector<Request*> extra;   // amplitude requests merged into this slot's launch
  int circuit = -1;
  bool building = false;
  void* d_buf = nullptr;     // device: bitstrings then results
  size_t d_cap = 0;
  void* h_buf = nullptr;     // pinned host staging
  size_t h_cap = 0;
  unsigned long long* d_status = nullptr;
  unsigned long long* h_status = nullptr;
};

}  // namespace

struct tn_server {
  tn_server_opts opts{};
  std::vector<Circuit> circuits;
  std::vector<Slot> slots;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> reqs;
  std::vector<double> latencies_us;
  int64_t failed = 0, evictions = 0, head_bytes = 0;
  uint64_t next_ticket = 1, tick = 0;
  Clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
};

namespace {

int ensure_slot_buffers(Slot& s, size_t dev_bytes, size_t host_bytes) {
  if (s.d_cap < dev_bytes) {
    cudaFree(s.d_buf);
    s.d_buf = nullptr;
    s.d_cap = 0;
    if (cudaMalloc(&s.d_buf, dev_bytes) != cudaSuccess) {
      cudaGetLastError();
      return TN_ERR_OOM;
    }
    s.d_cap = dev_bytes;
  }
  if (s.h_cap < host_bytes) {
    cudaFreeHost(s.h_buf);
    s.h_buf = nullptr;
    s.h_cap = 0;
    if (cudaMallocHost(&s.h_buf, host_bytes) != cudaSuccess) {
      cudaGetLastError();
      return TN_ERR_OOM;
    }
    s.h_cap = host_bytes;
  }
  return TN_OK;
}

int64_t head_bytes_of(tn_plan_t* p) {
  return (int64_t)p->P.tails_raw.size() * ((int64_t)16 << p->P.open_qubits.size());
}

constexpr int kMaxMerge = 16;                       // amplitude requests per slot
constexpr int64_t kMaxMergeKeys = (int64_t)1 << 22;  // bitstrings per merged launch

// Staging of an amplitude batch: [bitstrings][results][status per request][segment ends]
struct AmpLayout {
  size_t out = 0, status = 0, seg = 0, total = 0;
  int64_t n = 0;
};

AmpLayout amp_layout(const Slot& s) {
  AmpLayout L;
  L.n = s.req->r.n;
  for (auto* q : s.extra) L.n += q->r.n;
  const size_t m = 1 + s.extra.size();
  const size_t esz = s.req->r.dtype == TN_C128 ? 16 : 8;
  L.out = ((size_t)L.n * 8 + 255) / 256 * 256;
  L.status = (L.out + (size_t)L.n * esz + 255) / 256 * 256;
  L.seg = L.status + m * 8;
  L.total = L.seg + m * 8;
  return L;
}

// Enqueue a slot's amplitude batch (s.req and s.extra, one circuit and dtype).
int enqueue_amplitudes(Slot& s, Circuit& c) {
  tn_plan_t* p = c.plan;
  const AmpLayout L = amp_layout(s);
  if (ensure_slot_buffers(s, std::max<size_t>(L.total, 256), std::max<size_t>(L.total, 256)))
    return fail(TN_ERR_OOM, "server: slot staging allocation failed");
  cudaStream_t st = s.stream;
  if (c.state == C_BUILDING && !s.building) cudaStreamWaitEvent(st, c.ready, 0);
  char* d = (char*)s.d_buf;
  char* hs = (char*)s.h_buf;
  size_t o = 0;
  unsigned long long* status = (unsigned long long*)(hs + L.status);
  int64_t* seg = (int64_t*)(hs + L.seg);
  int64_t end = 0;
  for (size_t j = 0; j <= s.extra.size(); ++j) {
    const tn_request& r = (j == 0 ? s.req : s.extra[j - 1])->r;
    std::memcpy(hs + o, r.bitstrings, (size_t)r.n * 8);
    o += (size_t)r.n * 8;
    end += r.n;
    status[j] = ~0ULL;
    seg[j] = end;
  }
  const size_t m = 1 + s.extra.size();
  if (cudaMemcpyAsync(d, hs, (size_t)L.n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d + L.status, hs + L.status, 2 * m * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return fail(TN_ERR_CUDA, "server: H2D copy");
  cudaError_t e = tn::launch_amplitudes(c.head->H, (int)p->P.open_qubits.size(), p->d_keys, p->d_key_groups,
                                        p->n_keys, p->P.tail_mask, p->d_open, (const uint64_t*)d, L.n, d + L.out,
                                        s.req->r.dtype == TN_C128 ? 1 : 0, (unsigned long long*)(d + L.status), st,
                                        (const int64_t*)(d + L.seg), (int)m);
  if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("server: amplitudes: ") + cudaGetErrorString(e));
  if (cudaMemcpyAsync(hs + L.out, d + L.out, L.seg - L.out, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(TN_ERR_CUDA, "server: D2H copy");
  return TN_OK;
}

// Enqueue one request's device work on its slot (the head is, or will be,
// ready): an amplitude batch, or one sampling request.
int enqueue_op(Slot& s, Request* q, Circuit& c) {
  if (q->r.kind == TN_REQ_AMPLITUDES) return enqueue_amplitudes(s, c);
  const tn_request& r = q->r;
  tn_plan_t* p = c.plan;
  const int h = (int)p->P.open_qubits.size();
  const size_t n = (size_t)r.n;
  if (ensure_slot_buffers(s, std::max<size_t>(n * 8, 256), std::max<size_t>(n * 8, 256)))
    return fail(TN_ERR_OOM, "server: slot staging allocation failed");
  cudaStream_t st = s.stream;
  if (c.state == C_BUILDING && !s.building) cudaStreamWaitEvent(st, c.ready, 0);
  char* d = (char*)s.d_buf;
  double f_head = 0.0;
  tn_head_fidelity(c.head, &f_head, nullptr);
  double mix = 0.0;
  if (r.target_fidelity > 0.0 && f_head > 0.0 && r.target_fidelity < f_head) mix = 1.0 - r.target_fidelity / f_head;
  tn::SampleParams sp;
  sp.H = c.head->H;
  sp.L = (int64_t)p->P.tails_raw.size();
  sp.h = h;
  sp.tails = p->d_tails;
  sp.open_mask = p->P.open_mask;
  sp.open_q = p->d_open;
  sp.n_qubits = p->P.n_qubits;
  sp.n = (int64_t)n;
  sp.mix = mix;
  sp.seed = r.seed;
  sp.out = (uint64_t*)d;
  sp.method = r.method;
  sp.param = r.param != 0 ? r.param
                          : (r.method == TN_SAMPLE_METROPOLIS ? ((int64_t)1 << h) : (r.method == TN_SAMPLE_FRUGAL ? 10 : 0));
  cudaError_t e = tn::launch_sample(sp, st);
  if (e != cudaSuccess) return fail(TN_ERR_CUDA, std::string("server: sample: ") + cudaGetErrorString(e));
  if (cudaMemcpyAsync(s.h_buf, d, n * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return fail(TN_ERR_CUDA, "server: D2H copy");
  return TN_OK;
}

void finish(tn_server* sv, Request* q, Circuit& c) {
  q->t_done = Clock::now();
  q->done = true;
  if (q->status == TN_OK)
    sv->latencies_us.push_back(std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count());
  else
    ++sv->failed;
  --c.users;
}

void retire(tn_server* sv, int si) {
  Slot& s = sv->slots[si];
  Request* q = s.req;
  Circuit& c = sv->circuits[s.circuit];
  if (s.building) {
    c.state = C_READY;
    c.builder_slot = -1;
    s.building = false;
  }
  if (q->r.kind == TN_REQ_AMPLITUDES) {
    const AmpLayout L = amp_layout(s);
    const size_t esz = q->r.dtype == TN_C128 ? 16 : 8;
    const unsigned long long* status = (const unsigned long long*)((char*)s.h_buf + L.status);
    size_t off = 0;
    for (size_t j = 0; j <= s.extra.size(); ++j) {
      Request* x = j == 0 ? q : s.extra[j - 1];
      if (x->status == TN_OK) {
        std::memcpy(x->r.out, (char*)s.h_buf + L.out + off * esz, (size_t)x->r.n * esz);
        if (status[j] != ~0ULL) {
          x->status = TN_ERR_NOT_IN_STATE;
          x->err = "bitstring " + std::to_string(status[j]) + " has a tail that is not a group";
        }
      }
      off += (size_t)x->r.n;
      finish(sv, x, c);
    }
  } else {
    const tn_request& r = q->r;
    if (q->status == TN_OK) std::memcpy(r.out, (char*)s.h_buf, (size_t)r.n * 8);
    finish(sv, q, c);
  }
  s.req = nullptr;
  s.extra.clear();
  s.circuit = -1;
}

// Device memory kept free beside the heads (request staging, workspaces).
constexpr int64_t kHbmReserve = (int64_t)1 << 30;

// Admission by memory: a new head must fit both the byte budget and the
// device's free memory as the driver reports it now (cudaMemGetInfo), less a
// reserve.  Least-recently-used idle heads are freed until it does.
bool make_room(tn_server* sv, int64_t need) {
  while (true) {
    size_t fr = 0, tot = 0;
    const bool dev_ok = cudaMemGetInfo(&fr, &tot) != cudaSuccess || (int64_t)fr >= need + kHbmReserve;
    if (sv->head_bytes + need <= sv->opts.hbm_budget_bytes && dev_ok) return true;
    int victim = -1;
    for (size_t i = 0; i < sv->circuits.size(); ++i) {
      Circuit& c = sv->circuits[i];
      if (c.state == C_READY && c.users == 0 && (victim < 0 || c.last_use < sv->circuits[victim].last_use))
        victim = (int)i;
    }
    if (victim < 0) return false;
    Circuit& c = sv->circuits[victim];
    tn_head_free(c.head);
    c.head = nullptr;
    c.state = C_EMPTY;
    sv->head_bytes -= c.bytes;
    ++sv->evictions;
  }
  return true;
}

bool plan_building(tn_server* sv, tn_plan_t* p) {
  for (auto& c : sv->circuits)
    if (c.plan == p && c.state == C_BUILDING) return true;
  return false;
}

void dispatcher(tn_server* sv) {
  cudaSetDevice(sv->circuits.empty() ? 0 : sv->circuits[0].plan->device);
  std::unique_lock<std::mutex> lock(sv->mu);
  while (true) {
    // retire finished slots
    bool progressed = false;
    for (size_t si = 0; si < sv->slots.size(); ++si) {
      Slot& s = sv->slots[si];
      if (!s.req) continue;
      cudaError_t e = cudaEventQuery(s.done);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) {
        s.req->status = TN_ERR_CUDA;
        s.req->err = std::string("server: ") + cudaGetErrorString(e);
        for (auto* x : s.extra) {
          x->status = TN_ERR_CUDA;
          x->err = s.req->err;
        }
      }
      retire(sv, (int)si);
      progressed = true;
    }
    if (progressed) sv->cv_done.notify_all();
    if (sv->stop && sv->queue.empty()) {
      bool busy = false;
      for (auto& s : sv->slots) busy |= s.req != nullptr;
      if (!busy) break;
    }
    // admit queued requests into free slots (requests that need no new
    // memory may pass one that waits for room)
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      int free_slot = -1;
      for (size_t si = 0; si < sv->slots.size(); ++si)
        if (!sv->slots[si].req) { free_slot = (int)si; break; }
      if (free_slot < 0) break;
      Request* q = *it;
      Circuit& c = sv->circuits[q->r.circuit];
      Slot& s = sv->slots[free_slot];
      bool build = false;
      if (c.state == C_EMPTY) {
        if (plan_building(sv, c.plan)) { ++it; continue; }   // the plan's workspace is in use
        if (!make_room(sv, c.bytes)) { ++it; continue; }
        tn_head_t* hd = nullptr;
        if (tn_head_create(c.plan, nullptr, &hd) != TN_OK) {
          q->status = TN_ERR_OOM;
          q->err = "server: head allocation failed";
          q->done = true;
          ++sv->failed;
          it = sv->queue.erase(it);
          sv->cv_done.notify_all();
          continue;
        }
        c.head = hd;
        sv->head_bytes += c.bytes;
        c.state = C_BUILDING;
        c.builder_slot = free_slot;
        build = true;
      }
      q->t_start = Clock::now();
      s.req = q;
      s.extra.clear();
      s.circuit = q->r.circuit;
      s.building = build;
      ++c.users;
      c.last_use = ++sv->tick;
      // continuous batching: waiting amplitude requests on the same ready
      // circuit and output type join this slot's launch
      if (q->r.kind == TN_REQ_AMPLITUDES && c.state == C_READY) {
        int64_t total = q->r.n;
        for (auto jt = std::next(it); jt != sv->queue.end() && (int)s.extra.size() < kMaxMerge - 1; ++jt) {
          Request* o = *jt;
          if (o->merged || o->r.kind != TN_REQ_AMPLITUDES || o->r.circuit != q->r.circuit ||
              o->r.dtype != q->r.dtype || total + o->r.n > kMaxMergeKeys)
            continue;
          total += o->r.n;
          o->merged = true;
          o->t_start = q->t_start;
          s.extra.push_back(o);
          ++c.users;
        }
      }
      int rc = TN_OK;
      if (build) {
        rc = tn::enqueue_slices(c.plan, c.kept, c.head->H, s.stream);
        if (rc == TN_OK) {
          tn::mark_slices_done(c.head, c.kept);
          cudaEventRecord(c.ready, s.stream);
        }
      }
      if (rc == TN_OK) rc = enqueue_op(s, q, c);
      if (rc != TN_OK) {
        q->status = rc;
        q->err = "server: enqueue failed";
        for (auto* x : s.extra) {
          x->status = rc;
          x->err = q->err;
        }
        if (build) {   // leave the circuit unbuilt: the next request starts over
          cudaStreamSynchronize(s.stream);
          tn_head_free(c.head);
          c.head = nullptr;
          sv->head_bytes -= c.bytes;
          c.state = C_EMPTY;
          c.builder_slot = -1;
          s.building = false;
        }
      }
      cudaEventRecord(s.done, s.stream);
      it = sv->queue.erase(it);
      if (!s.extra.empty()) {   // drop the merged requests from the queue; rescan from the front
        sv->queue.erase(std::remove_if(sv->queue.begin(), sv->queue.end(), [](Request* x) { return x->merged; }),
                        sv->queue.end());
        it = sv->queue.begin();
      }
    }
    // wait for new work or poll the device again shortly
    sv->cv_work.wait_for(lock, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" int tn_server_create(const tn_server_opts* opts, tn_server_t** out) {
  if (!out) return fail(TN_ERR_INVALID, "out is NULL");
  *out = nullptr;
  tn_server* sv = new tn_server();
  sv->opts.n_slots = opts && opts->n_slots > 0 ? opts->n_slots : 8;
  if (opts && opts->hbm_budget_bytes > 0) {
    sv->opts.hbm_budget_bytes = opts->hbm_budget_bytes;
  } else {   // the device's free memory now, less the reserve
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = (size_t)64 << 30;
    }
    sv->opts.hbm_budget_bytes = std::max<int64_t>((int64_t)fr - kHbmReserve, (int64_t)1 << 26);
  }
  if (sv->opts.n_slots > 64) {
    delete sv;
    return fail(TN_ERR_INVALID, "at most 64 slots");
  }
  sv->slots.resize(sv->opts.n_slots);
  for (auto& s : sv->slots) {
    if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&s.d_status, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&s.h_status, sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      tn_server_free(sv);
      return fail(TN_ERR_CUDA, "server: slot set-up failed");
    }
  }
  sv->t0 = Clock::now();
  *out = sv;
  return TN_OK;
}

extern "C" int tn_server_add_circuit(tn_server_t* sv, tn_plan_t* plan, tn_range kept, int* circuit_id) {
  if (!sv || !plan || !circuit_id) return fail(TN_ERR_INVALID, "NULL argument");
  if (!plan->on_device) return fail(TN_ERR_INVALID, "plan was made host_only");
  const int64_t ns = 1LL << plan->P.n_sliced;
  if (kept.begin < 0 || kept.end > ns || kept.begin >= kept.end) return fail(TN_ERR_INVALID, "bad kept slice range");
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->worker.joinable()) return fail(TN_ERR_INVALID, "add circuits before the first submit");
  Circuit c;
  c.plan = plan;
  c.kept = kept;
  c.bytes = head_bytes_of(plan);
  if (cudaEventCreateWithFlags(&c.ready, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(TN_ERR_CUDA, "server: event");
  }
  sv->circuits.push_back(c);
  *circuit_id = (int)sv->circuits.size() - 1;
  return TN_OK;
}

extern "C" int tn_server_submit(tn_server_t* sv, const tn_request* r, uint64_t* ticket) {
  if (!sv || !r || !ticket) return fail(TN_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return fail(TN_ERR_INVALID, "server is stopping");
  if (r->circuit < 0 || r->circuit >= (int)sv->circuits.size()) return fail(TN_ERR_INVALID, "unknown circuit");
  if (r->kind != TN_REQ_AMPLITUDES && r->kind != TN_REQ_SAMPLE) return fail(TN_ERR_INVALID, "unknown request kind");
  if (r->n < 1 || !r->out || (r->kind == TN_REQ_AMPLITUDES && !r->bitstrings))
    return fail(TN_ERR_INVALID, "request needs n >= 1 and its buffers");
  if (r->kind == TN_REQ_AMPLITUDES && r->dtype != TN_C64 && r->dtype != TN_C128)
    return fail(TN_ERR_INVALID, "dtype must be TN_C64 or TN_C128");
  if (r->kind == TN_REQ_SAMPLE && (r->method < TN_SAMPLE_EXACT || r->method > TN_SAMPLE_FRUGAL))
    return fail(TN_ERR_INVALID, "unknown sampling method");
  if (sv->circuits[r->circuit].bytes > sv->opts.hbm_budget_bytes)
    return fail(TN_ERR_OOM, "the circuit's head is larger than the server's HBM budget");
  Request* q = new Request();
  q->ticket = sv->next_ticket++;
  q->r = *r;
  q->t_submit = Clock::now();
  sv->reqs[q->ticket] = q;
  sv->queue.push_back(q);
  if (!sv->worker.joinable()) sv->worker = std::thread(dispatcher, sv);
  *ticket = q->ticket;
  sv->cv_work.notify_one();
  return TN_OK;
}

extern "C" int tn_server_wait(tn_server_t* sv, uint64_t ticket, tn_request_result* res) {
  if (!sv) return fail(TN_ERR_INVALID, "NULL server");
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(TN_ERR_INVALID, "unknown ticket");
  Request* q = it->second;
  sv->cv_done.wait(lock, [&] { return q->done; });
  if (res) {
    res->status = q->status;
    res->latency_us = std::chrono::duration<double, std::micro>(q->t_done - q->t_submit).count();
    res->queue_us = q->t_start.time_since_epoch().count() == 0
                        ? 0.0
                        : std::chrono::duration<double, std::micro>(q->t_start - q->t_submit).count();
  }
  const int st = q->status;
  const std::string err = q->err;
  sv->reqs.erase(it);
  delete q;
  if (st != TN_OK) return fail(st, err);
  return TN_OK;
}

extern "C" int tn_server_get_stats(tn_server_t* sv, tn_server_stats* out) {
  if (!sv || !out) return fail(TN_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lock(sv->mu);
  std::memset(out, 0, sizeof(*out));
  std::vector<double> v = sv->latencies_us;
  std::sort(v.begin(), v.end());
  out->completed = (int64_t)v.size();
  out->failed = sv->failed;
  out->queued = (int64_t)sv->queue.size();
  for (auto& s : sv->slots) out->in_flight += s.req != nullptr;
  if (!v.empty()) {
    out->p50_us = v[(v.size() - 1) / 2];
    out->p99_us = v[std::min(v.size() - 1, (size_t)((v.size() - 1) * 0.99 + 0.5))];
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_us = sum / (double)v.size();
  }
  for (auto& c : sv->circuits) out->heads_cached += c.state != C_EMPTY;
  out->head_bytes = sv->head_bytes;
  out->evictions = sv->evictions;
  out->wall_s = std::chrono::duration<double>(Clock::now() - sv->t0).count();
  return TN_OK;
}

extern "C" void tn_server_free(tn_server_t* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& s : sv->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    cudaStreamDestroy(s.stream);
    cudaEventDestroy(s.done);
    cudaFree(s.d_buf);
    cudaFreeHost(s.h_buf);
    cudaFree(s.d_status);
    cudaFreeHost(s.h_status);
  }
  for (auto& c : sv->circuits) {
    if (c.head) tn_head_free(c.head);
    if (c.ready) cudaEventDestroy(c.ready);
  }
  for (auto& kv : sv->reqs) delete kv.second;
  delete sv;
}

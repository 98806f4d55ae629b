// Serving loop with continuous batching (C ABI, declared in include/mea.h).
//
// One worker thread drives n_slots CUDA streams.  Requests are split into
// chunks of about the same device cost (kChunkFlop FLOPs by the process's
// operation count, at most chunk_events events), so that no chunk holds a
// slot for long.  Whenever a slot is free the worker dispatches the next
// chunk of the admitted request with the least remaining work, counted in
// estimated device seconds, minus kAging times the seconds it has waited
// since submission: short requests overtake long ones (shortest remaining
// work first), and a long request gains priority as it ages, so none
// starves.  Work of different requests overlaps on the device.
//
// Memory: every slot keeps one scratch set per process it has run (sized
// once, never regrown between chunks), so the scratch a process can hold is
// at most (its slots) x (its chunk's estimate), whatever the number of its
// requests.  Admission commits that per process against mem_budget_bytes: a
// request whose process is committed is admitted at once (no head-of-line
// blocking behind requests of other processes); a process's chunks run only
// on as many distinct slots as are committed for it; when the budget is
// short, the scratch of processes with no request left is released.
// Completion is observed with cudaEventQuery (never a blocking device call in
// the loop); every host-side wait has a bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "process.h"

namespace {

using Clock = std::chrono::steady_clock;

// Dispatch and chunking constants (see the comment at the top).
constexpr double kChunkFlop = 1e11;    // target device work of one chunk
constexpr int64_t kChunkQuantum = 128; // chunk sizes are multiples of this (or the whole request)
constexpr double kAging = 0.25;        // priority gained per second waited, in seconds of work
constexpr double kFp64Cost = 24.0;     // FP64 path cost per FLOP relative to the mixed path (measured 19-28)
constexpr double kInitialRate = 1e13;  // FLOP/s assumed until the server has measured its own

struct SrvReq {
  uint64_t id = 0;
  mea_process_t proc = nullptr;
  const double* mom = nullptr;
  int64_t n = 0;
  mea_prec_mode prec = MEA_PREC_MIXED;
  double* me2 = nullptr;
  uint8_t* flags = nullptr;
  int64_t next = 0;     // first event not yet dispatched
  int64_t done = 0;     // events whose chunk completed
  int in_flight = 0;
  int64_t chunk = 1;    // events per chunk
  double flop_per_event = 0;
  size_t slot_bytes = 0;  // scratch estimate of one chunk (one slot's scratch set)
  mea_status status = MEA_OK;
  std::string error;  // message of the failure (the worker thread's mea_last_error), if any
  bool complete = false;
  Clock::time_point t_submit, t_done;
};

struct SrvSlot {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  // one scratch set per process the slot has run: sized once, so that chunks
  // of different processes never regrow (and free) buffers between them
  std::map<mea_process_t, std::unique_ptr<mea::EvalScratch>> scratch;
  SrvReq* req = nullptr;
  int64_t cn = 0;
  double flop = 0;  // estimated work of the chunk in flight
  bool busy = false;
};

// Per process: the scratch committed against the budget and its use.
struct ProcState {
  size_t slot_bytes = 0;  // committed per slot (largest chunk estimate seen)
  int allowed = 0;        // slots committed: distinct slots that may hold its scratch
  int holding = 0;        // slots that hold a scratch set of it
  int requests = 0;       // admitted requests not yet complete
};

}  // namespace

struct mea_server_s {
  size_t budget = 0, reserved = 0;  // reserved: sum of the processes' commitments
  int64_t chunk = 1 << 14;          // largest chunk (events)
  std::vector<SrvSlot> slots;
  std::deque<SrvReq*> waiting;  // submitted, not admitted (memory)
  std::vector<SrvReq*> active;  // admitted, events left to dispatch
  std::unordered_map<uint64_t, std::unique_ptr<SrvReq>> reqs;
  std::unordered_map<mea_process_t, ProcState> procs;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t n_submitted = 0, n_completed = 0, n_rejected = 0, ev_completed = 0;
  std::vector<double> lat_ms;
  int device = 0;
  double busy_s = 0;
  double flop_done = 0;  // estimated work of the completed chunks (for the rate)
  Clock::time_point busy_since;
  int chunks_in_flight = 0;

  void run();
  double rate() const { return busy_s > 0.05 && flop_done > 0 ? flop_done / busy_s : kInitialRate; }
  bool admit(SrvReq* r);
  void release_idle(mea_process_t keep);
};

namespace {

void complete_req(mea_server_s* S, SrvReq* r, mea_status st) {
  if (r->complete) return;
  if (st != MEA_OK && r->status == MEA_OK) r->status = st;
  r->complete = true;
  r->t_done = Clock::now();
  S->procs[r->proc].requests--;
  S->n_completed++;
  S->ev_completed += (uint64_t)r->done;
  S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  S->active.erase(std::remove(S->active.begin(), S->active.end(), r), S->active.end());
  S->cv_done.notify_all();
}

}  // namespace

// Release the scratch of every process other than `keep` that has no
// admitted request left and no chunk in flight, and its commitment.
void mea_server_s::release_idle(mea_process_t keep) {
  for (auto& kv : procs) {
    ProcState& ps = kv.second;
    if (kv.first == keep || ps.requests > 0 || ps.allowed == 0) continue;
    bool in_flight = false;
    for (auto& sl : slots)
      if (sl.busy && sl.req && sl.req->proc == kv.first) in_flight = true;
    if (in_flight) continue;
    for (auto& sl : slots) {
      auto it = sl.scratch.find(kv.first);
      if (it == sl.scratch.end()) continue;
      it->second->release();
      sl.scratch.erase(it);
    }
    reserved -= std::min(reserved, ps.slot_bytes * (size_t)ps.allowed);
    ps.allowed = 0;
    ps.holding = 0;
    ps.slot_bytes = 0;
  }
}

// Commit scratch for r's process (at least one slot, up to one per chunk of
// r, at most every slot) and admit r; false if not even one slot fits.
bool mea_server_s::admit(SrvReq* r) {
  ProcState& ps = procs[r->proc];
  if (r->slot_bytes > ps.slot_bytes) {
    // a larger chunk estimate (another precision): recommit what is held at the new size
    const size_t extra = (r->slot_bytes - ps.slot_bytes) * (size_t)ps.allowed;
    if (reserved + extra > budget) release_idle(r->proc);
    if (reserved + extra > budget) return false;
    reserved += extra;
    ps.slot_bytes = r->slot_bytes;
  }
  const int64_t chunks = (r->n + r->chunk - 1) / r->chunk;
  const int want = (int)std::min<int64_t>((int64_t)slots.size(), std::max<int64_t>(1, chunks));
  while (ps.allowed < want) {
    if (reserved + ps.slot_bytes > budget) release_idle(r->proc);
    if (reserved + ps.slot_bytes > budget) break;
    reserved += ps.slot_bytes;
    ps.allowed++;
  }
  if (ps.allowed == 0) return false;
  ps.requests++;
  active.push_back(r);
  return true;
}

void mea_server_s::run() {
  cudaSetDevice(device);  // the worker drives the device the server was created on
  std::unique_lock<std::mutex> lk(mu);
  Clock::time_point stop_deadline;
  bool stopping = false;
  for (;;) {
    bool progress = false;
    // 1. completions
    for (auto& sl : slots) {
      if (!sl.busy) continue;
      cudaError_t q = cudaEventQuery(sl.ev);
      if (q == cudaErrorNotReady) continue;
      SrvReq* r = sl.req;
      sl.busy = false;
      sl.req = nullptr;
      --chunks_in_flight;
      if (chunks_in_flight == 0) busy_s += std::chrono::duration<double>(Clock::now() - busy_since).count();
      r->in_flight--;
      progress = true;
      if (q != cudaSuccess) {
        if (r->error.empty()) r->error = std::string("chunk failed on the device: ") + cudaGetErrorString(q);
        cudaGetLastError();
        r->next = r->n;
        active.erase(std::remove(active.begin(), active.end(), r), active.end());
        if (r->in_flight == 0) complete_req(this, r, MEA_E_CUDA);
        else r->status = MEA_E_CUDA;
        continue;
      }
      flop_done += sl.flop;
      r->done += sl.cn;
      if (r->done == r->n || (r->next == r->n && r->in_flight == 0)) complete_req(this, r, MEA_OK);
    }
    // 2. admission by memory, in arrival order, skipping requests that do not fit yet
    if (!stop) {
      for (auto it = waiting.begin(); it != waiting.end();) {
        if (admit(*it)) {
          it = waiting.erase(it);
          progress = true;
        } else {
          ++it;
        }
      }
    }
    // 3. dispatch: each free slot takes a chunk of the eligible request with the
    //    least remaining work (device seconds) less kAging x its age
    const Clock::time_point now = Clock::now();
    const double R = rate();
    for (auto& sl : slots) {
      if (sl.busy || active.empty() || stop) continue;
      SrvReq* r = nullptr;
      double best = 0;
      for (SrvReq* c : active) {
        const ProcState& ps = procs[c->proc];
        if (!sl.scratch.count(c->proc) && ps.holding >= ps.allowed) continue;  // no committed slot left for it
        const double age = std::chrono::duration<double>(now - c->t_submit).count();
        const double key = (double)(c->n - c->next) * c->flop_per_event / R - kAging * age;
        if (!r || key < best) {
          r = c;
          best = key;
        }
      }
      if (!r) continue;
      const int64_t c0 = r->next, cn = std::min(r->chunk, r->n - r->next);
      auto& sc = sl.scratch[r->proc];
      if (!sc) {
        sc.reset(new mea::EvalScratch());
        procs[r->proc].holding++;
      }
      const int n_ext = r->proc->prog.n_ext;
      mea_status st = mea::evaluate_with(r->proc, *sc, r->mom + (size_t)c0 * n_ext * 4, cn, MEA_HEL_SUM_NONZERO,
                                         nullptr, r->prec, r->me2 + c0, r->flags ? r->flags + c0 : nullptr, sl.s);
      r->next += cn;
      progress = true;
      if (st != MEA_OK) {
        if (r->error.empty()) r->error = mea_last_error();
        r->status = st;
        r->next = r->n;
        active.erase(std::remove(active.begin(), active.end(), r), active.end());
        if (r->in_flight == 0) complete_req(this, r, st);
        continue;
      }
      cudaEventRecord(sl.ev, sl.s);
      sl.busy = true;
      sl.req = r;
      sl.cn = cn;
      sl.flop = (double)cn * r->flop_per_event;
      if (chunks_in_flight == 0) busy_since = Clock::now();
      ++chunks_in_flight;
      r->in_flight++;
      if (r->next >= r->n) active.erase(std::remove(active.begin(), active.end(), r), active.end());
    }
    if (stop) {
      if (!stopping) { stopping = true; stop_deadline = Clock::now() + std::chrono::seconds(60); }
      if (chunks_in_flight == 0 || Clock::now() > stop_deadline) break;
    }
    if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
}

extern "C" {

mea_status mea_server_create(size_t budget, int n_slots, int64_t chunk, mea_server_t* out) {
  if (!out || n_slots <= 0 || n_slots > 64 || budget == 0) return mea::set_error(MEA_E_ARG, "mea_server_create: bad arguments");
  *out = nullptr;
  mea_server_s* S = new mea_server_s();
  S->budget = budget;
  S->chunk = chunk > 0 ? chunk : (1 << 14);
  S->slots.resize(n_slots);
  cudaGetDevice(&S->device);
  for (auto& sl : S->slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (auto& x : S->slots) {
        if (x.s) cudaStreamDestroy(x.s);
        if (x.ev) cudaEventDestroy(x.ev);
      }
      delete S;
      return mea::set_error(MEA_E_CUDA, std::string("mea_server_create: ") + cudaGetErrorString(e));
    }
  }
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return MEA_OK;
}

mea_status mea_server_submit(mea_server_t S, mea_process_t P, const double* mom, int64_t n, mea_prec_mode prec,
                             double* me2, uint8_t* flags, uint64_t* req_id) {
  if (!S || !P || !req_id || n < 0 || (n > 0 && (!mom || !me2)))
    return mea::set_error(MEA_E_ARG, "mea_server_submit: bad arguments");
  if (P->host_only) return mea::set_error(MEA_E_UNSUPPORTED, "mea_server_submit: host-only process handle");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return mea::set_error(MEA_E_ARG, "mea_server_submit: bad precision");
  std::unique_ptr<SrvReq> r(new SrvReq());
  r->proc = P;
  r->mom = mom;
  r->n = n;
  r->prec = prec;
  r->me2 = me2;
  r->flags = flags;
  // cost model: the process's operation count per event (helicity sum), the
  // FP64 path weighted by its measured slowdown; chunks of about kChunkFlop
  r->flop_per_event = std::max(1.0, P->prog.flops_per_hel * (double)std::max(1, P->prog.n_hel) *
                                        (prec == MEA_PREC_FP64 ? kFp64Cost : 1.0));
  int64_t cn = (int64_t)(kChunkFlop / r->flop_per_event) / kChunkQuantum * kChunkQuantum;
  cn = std::min(S->chunk, std::max(kChunkQuantum, cn));
  r->chunk = std::min<int64_t>(std::max<int64_t>(n, 1), cn);
  r->slot_bytes = mea::scratch_estimate(P, r->chunk, prec);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return mea::set_error(MEA_E_REJECTED, "mea_server_submit: server is stopping");
  S->n_submitted++;
  if (r->slot_bytes > S->budget) {
    S->n_rejected++;
    return mea::set_error(MEA_E_REJECTED, "mea_server_submit: one chunk of the request needs " +
                                              std::to_string(r->slot_bytes) + " bytes of scratch, budget is " +
                                              std::to_string(S->budget));
  }
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  *req_id = r->id;
  SrvReq* raw = r.get();
  S->reqs.emplace(r->id, std::move(r));
  if (n == 0) {
    raw->complete = true;
    raw->t_done = raw->t_submit;
    S->n_completed++;
    S->lat_ms.push_back(0.0);
  } else {
    S->waiting.push_back(raw);
  }
  S->cv_work.notify_all();
  return MEA_OK;
}

mea_status mea_server_wait(mea_server_t S, uint64_t id, int timeout_ms, double* latency_ms) {
  if (!S) return mea::set_error(MEA_E_ARG, "mea_server_wait: null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return mea::set_error(MEA_E_ARG, "mea_server_wait: unknown request id");
  SrvReq* r = it->second.get();
  const int ms = timeout_ms < 0 ? 600000 : timeout_ms;
  if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(ms), [r] { return r->complete; }))
    return mea::set_error(MEA_E_TIMEOUT, "mea_server_wait: request " + std::to_string(id) + " not complete");
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  mea_status st = r->status;
  const std::string why = r->error;
  S->reqs.erase(it);
  if (st != MEA_OK) return mea::set_error(st, "mea_server_wait: request failed: " + why);
  return MEA_OK;
}

mea_status mea_server_stats(mea_server_t S, mea_server_stats_t* out) {
  if (!S || !out) return mea::set_error(MEA_E_ARG, "mea_server_stats: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->submitted = S->n_submitted;
  out->completed = S->n_completed;
  out->rejected = S->n_rejected;
  out->events_completed = S->ev_completed;
  std::vector<double> l = S->lat_ms;
  std::sort(l.begin(), l.end());
  auto q = [&](double f) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(f * (double)(l.size() - 1) + 0.5))]; };
  out->p50_ms = q(0.50);
  out->p99_ms = q(0.99);
  out->max_ms = l.empty() ? 0.0 : l.back();
  double b = S->busy_s;
  if (S->chunks_in_flight > 0) b += std::chrono::duration<double>(Clock::now() - S->busy_since).count();
  out->busy_seconds = b;
  out->reserved_bytes = S->reserved;
  return MEA_OK;
}

mea_status mea_server_destroy(mea_server_t S) {
  if (!S) return mea::set_error(MEA_E_ARG, "mea_server_destroy: null server");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (SrvReq* r : S->waiting) {
      S->procs[r->proc].requests++;  // never admitted: balance the count complete_req takes back
      complete_req(S, r, MEA_E_REJECTED);
    }
    S->waiting.clear();
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& sl : S->slots) {
    if (sl.busy) cudaStreamSynchronize(sl.s);
    for (auto& kv : sl.scratch) kv.second->release();
    cudaStreamDestroy(sl.s);
    cudaEventDestroy(sl.ev);
  }
  delete S;
  return MEA_OK;
}

}  // extern "C"

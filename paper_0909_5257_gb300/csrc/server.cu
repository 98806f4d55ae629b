// Serving loop with continuous batching (C ABI, declared in include/mea.h).
//
// One worker thread drives n_slots CUDA streams.  Requests are split into
// chunks; whenever a slot is free the worker dispatches the next chunk of the
// admitted request that has waited longest since its last chunk (round robin
// over requests), so new requests start as soon as any slot frees up and work
// of different requests overlaps on the GPU.  Admission is by memory:
// each request reserves its scratch estimate from the budget until it is
// complete.  Completion is observed with cudaEventQuery (never a blocking
// device call in the loop); every host-side wait has a bound.
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
  size_t reserve = 0;
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
  bool busy = false;
};

}  // namespace

struct mea_server_s {
  size_t budget = 0, reserved = 0;
  int64_t chunk = 1 << 14;
  std::vector<SrvSlot> slots;
  std::deque<SrvReq*> waiting;  // submitted, not admitted (memory)
  std::deque<SrvReq*> active;   // admitted, events left to dispatch
  std::unordered_map<uint64_t, std::unique_ptr<SrvReq>> reqs;
  std::mutex mu;
  std::condition_variable cv_done, cv_work;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  uint64_t n_submitted = 0, n_completed = 0, n_rejected = 0, ev_completed = 0;
  std::vector<double> lat_ms;
  int device = 0;
  double busy_s = 0;
  Clock::time_point busy_since;
  int chunks_in_flight = 0;

  void run();
};

namespace {

void complete_req(mea_server_s* S, SrvReq* r, mea_status st) {
  if (r->complete) return;
  if (st != MEA_OK && r->status == MEA_OK) r->status = st;
  r->complete = true;
  r->t_done = Clock::now();
  S->reserved -= std::min(S->reserved, r->reserve);
  S->n_completed++;
  S->ev_completed += (uint64_t)r->done;
  S->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
  S->active.erase(std::remove(S->active.begin(), S->active.end(), r), S->active.end());
  S->cv_done.notify_all();
}

}  // namespace

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
        if (r->in_flight == 0) complete_req(this, r, MEA_E_CUDA);
        else r->status = MEA_E_CUDA;
        continue;
      }
      r->done += sl.cn;
      if (r->done == r->n || (r->next == r->n && r->in_flight == 0)) complete_req(this, r, MEA_OK);
    }
    // 2. admission by memory
    while (!stop && !waiting.empty() && reserved + waiting.front()->reserve <= budget) {
      SrvReq* r = waiting.front();
      waiting.pop_front();
      reserved += r->reserve;
      active.push_back(r);
      progress = true;
    }
    // 3. dispatch chunks to free slots, round robin over admitted requests
    for (auto& sl : slots) {
      if (sl.busy || active.empty() || stop) continue;
      SrvReq* r = active.front();
      active.pop_front();
      const int64_t c0 = r->next, cn = std::min(chunk, r->n - r->next);
      auto& sc = sl.scratch[r->proc];
      if (!sc) sc.reset(new mea::EvalScratch());
      const int n_ext = r->proc->prog.n_ext;
      mea_status st = mea::evaluate_with(r->proc, *sc, r->mom + (size_t)c0 * n_ext * 4, cn, MEA_HEL_SUM_NONZERO,
                                         nullptr, r->prec, r->me2 + c0, r->flags ? r->flags + c0 : nullptr, sl.s);
      r->next += cn;
      progress = true;
      if (st != MEA_OK) {
        if (r->error.empty()) r->error = mea_last_error();
        r->status = st;
        r->next = r->n;
        if (r->in_flight == 0) complete_req(this, r, st);
        continue;
      }
      cudaEventRecord(sl.ev, sl.s);
      sl.busy = true;
      sl.req = r;
      sl.cn = cn;
      if (chunks_in_flight == 0) busy_since = Clock::now();
      ++chunks_in_flight;
      r->in_flight++;
      if (r->next < r->n) active.push_back(r);  // back of the line: interleave requests
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
  const int64_t cn = std::min<int64_t>(std::max<int64_t>(n, 1), S->chunk);
  const int64_t n_chunks = (n + S->chunk - 1) / S->chunk;
  r->reserve = mea::scratch_estimate(P, cn, prec) * (size_t)std::max<int64_t>(1, std::min<int64_t>(n_chunks, (int64_t)S->slots.size()));
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return mea::set_error(MEA_E_REJECTED, "mea_server_submit: server is stopping");
  S->n_submitted++;
  if (r->reserve > S->budget) {
    S->n_rejected++;
    return mea::set_error(MEA_E_REJECTED, "mea_server_submit: request needs " + std::to_string(r->reserve) +
                                              " bytes of scratch, budget is " + std::to_string(S->budget));
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
      r->reserve = 0;  // never admitted: nothing reserved
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

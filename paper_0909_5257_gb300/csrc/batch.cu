// Autotuner and batched launch (C ABI, declared in include/mea.h).
//
// mea_autotune times every candidate tile shape / shared-memory placement of
// a process's amplitude kernel on a sample and keeps the fastest.
// mea_batch_* evaluate several subprocesses of very uneven cost with one
// CUDA-graph launch: the graph holds one evaluation per item, each on its own
// branch so that independent subprocesses fill the GPU together; it is
// captured once and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kernels.h"
#include "process.h"

#define MEA_CK(call)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return mea::set_error(MEA_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct mea_batch_s {
  std::vector<mea_batch_item> items;
  mea_prec_mode prec = MEA_PREC_MIXED;
  std::vector<mea::EvalScratch> scratch;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaStream_t origin = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernel_nodes = 0;
};

namespace {

void destroy_batch(mea_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->origin) cudaStreamDestroy(b->origin);
  for (auto& s : b->scratch) s.release();
  delete b;
}

}  // namespace

extern "C" {

mea_status mea_autotune(mea_process_t P, const double* mom, int64_t n, mea_prec_mode prec, double* me2,
                        mea_tune_result* out) {
  if (!P || !mom || !me2 || n <= 0) return mea::set_error(MEA_E_ARG, "mea_autotune: bad arguments");
  if (P->host_only) return mea::set_error(MEA_E_UNSUPPORTED, "mea_autotune: host-only process handle");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return mea::set_error(MEA_E_ARG, "mea_autotune: bad precision");
  std::lock_guard<std::mutex> lk(P->mu);
  return mea::autotune_locked(P, mom, n, prec, me2, out);
}

}  // extern "C"

namespace mea {

mea_status autotune_locked(mea_process_s* P, const double* mom, int64_t n, mea_prec_mode prec, double* me2,
                           mea_tune_result* out) {
  P->auto_tuned[prec == MEA_PREC_FP64 ? 1 : 0] = true;
  const bool fp64 = prec == MEA_PREC_FP64;
  const int ti = fp64 ? 1 : 0;
  const int H = P->prog.n_hel;
  mea::DevProgram dp = P->dev;
  const bool tc = mea::uses_tensor_path(P, prec, MEA_HEL_SUM_NONZERO);
  mea::DevBuf abuf, rowmax, pairk, evf;
  int64_t lda = 0;
  if (tc) {
    // the tensor-core path runs the amplitude-output interpreter: time that
    dp.gen = nullptr;
    dp.n_colour = 0;
    // the sample is one chunk of the size an evaluation of n events launches
    // (its grid fill and its slot traffic in L2 decide between tiles)
    n = mea::tensor_chunk_events(P, H, n);
    lda = ((2 * n * H + 127) / 128) * 128;
    if (abuf.ensure(sizeof(float) * (size_t)P->jmap.kd * (size_t)lda) != cudaSuccess ||
        rowmax.ensure(sizeof(float) * 2 * (size_t)H * n) != cudaSuccess ||
        pairk.ensure(sizeof(float) * (size_t)H * n) != cudaSuccess || evf.ensure((size_t)n) != cudaSuccess) {
      abuf.release(); rowmax.release(); pairk.release(); evf.release();
      return mea::set_error(MEA_E_NOMEM, "mea_autotune: no room for the amplitude sample");
    }
  }
  std::vector<mea::AmpConfig> cands =
      mea::candidate_configs(dp, fp64, H, n, P->num_sms, P->smem_optin, P->smem_per_sm);
  mea::AmpConfig def = mea::plan_amp(dp, fp64, H, n, P->num_sms, P->smem_optin, P->smem_per_sm);
  cands.insert(cands.begin(), def);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  {
    cudaError_t ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {  // release what this call holds before reporting
      if (e0) cudaEventDestroy(e0);
      if (s) cudaStreamDestroy(s);
      abuf.release(); rowmax.release(); pairk.release(); evf.release();
      return mea::set_error(MEA_E_CUDA, std::string("mea_autotune: ") + cudaGetErrorString(ce));
    }
  }
  // Every timed launch starts with a cold L2 (a buffer of twice the L2 is
  // written before it), as in an evaluation that follows other work: a
  // kernel timed back to back on its own input finds that input and its own
  // spill lines in L2 and can rank candidates differently.  Skipped when the
  // buffer cannot be had.
  mea::DevBuf flush;
  size_t flush_bytes = 0;
  {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) == cudaSuccess &&
        l2 > 0 && flush.ensure(2 * (size_t)l2) == cudaSuccess)
      flush_bytes = 2 * (size_t)l2;
    cudaGetLastError();
  }
  mea::EvalScratch S;
  double best = 1e30, def_ms = 0;
  int best_i = 0;
  mea_status st = MEA_OK;
  // time candidate i: best of `reps` launches on the sample (1e30 if it cannot run)
  auto time_cand = [&](size_t i, int reps) -> double {
    const mea::AmpConfig& c = cands[i];
    mea::AmpLaunch a;
    a.mom = mom;
    a.n_events = n;
    a.me2 = me2;
    a.flag_threshold = (float)P->opts.flag_threshold;
    if (tc) {
      a.amp_out = reinterpret_cast<float*>(abuf.p);
      a.lda = lda;
      a.amp_rowmax = reinterpret_cast<float*>(rowmax.p);
      a.pair_kappa = reinterpret_cast<float*>(pairk.p);
      a.ev_flags = reinterpret_cast<uint8_t*>(evf.p);
    }
    size_t jb = (mea::jamp_scratch_bytes_needed(dp, fp64, c) + 255) & ~size_t(255);
    size_t sb = mea::slot_scratch_bytes_needed(dp, fp64, c);
    mea::DevBuf& buf = fp64 ? S.s64 : S.s32;
    if (buf.ensure(jb + sb + 256) != cudaSuccess) return 1e30;  // too large: skip the candidate
    a.jamp_scratch = reinterpret_cast<float*>(buf.p);
    a.slot_scratch = reinterpret_cast<float*>(reinterpret_cast<char*>(buf.p) + jb);
    double t_best = 1e30;
    for (int rep = 0; rep < reps; ++rep) {
      if (flush_bytes) cudaMemsetAsync(flush.p, rep, flush_bytes, s);
      cudaEventRecord(e0, s);
      cudaError_t le = mea::launch_amp(dp, fp64, c, a, s);
      cudaEventRecord(e1, s);
      if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); return 1e30; }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t_best = std::min<double>(t_best, ms);
    }
    return t_best;
  };
  std::vector<double> round1(cands.size(), 1e30);
  for (size_t i = 0; i < cands.size(); ++i) {
    round1[i] = time_cand(i, 3);
    if (i == 0) def_ms = round1[i];
    if (round1[i] < best) { best = round1[i]; best_i = (int)i; }
  }
  // second round: the three fastest candidates again, five repetitions each,
  // so that timing noise on the sample does not decide between near-equal tiles
  // (the heuristic default is always among them, so that best_ms and
  // default_ms come from the same round)
  if (st == MEA_OK && cands.size() > 1) {
    std::vector<std::pair<double, int>> order;
    for (size_t i = 0; i < round1.size(); ++i) order.push_back({round1[i], (int)i});
    std::sort(order.begin(), order.end());
    std::vector<int> again{0};
    for (size_t r = 0; r < order.size() && again.size() < 4; ++r)
      if (order[r].second != 0 && order[r].first < 1e30) again.push_back(order[r].second);
    // the fastest tile without register forwarding is also timed again: a
    // forwarding tile must beat it clearly (the sample is one evaluation chunk;
    // the serving loop's chunks are smaller and run side by side, where a
    // forwarding tile faster by under 1 % on the sample measured slower)
    for (size_t r = 0; r < order.size(); ++r)
      if (order[r].first < 1e30 && !cands[order[r].second].fwd) {
        if (std::find(again.begin(), again.end(), order[r].second) == again.end()) again.push_back(order[r].second);
        break;
      }
    best = 1e30;
    double best_plain = 1e30;
    int plain_i = -1;
    for (int i : again) {
      const double t = time_cand((size_t)i, 5);
      if (i == 0) def_ms = t;
      if (t < best) { best = t; best_i = i; }
      if (!cands[i].fwd && t < best_plain) { best_plain = t; plain_i = i; }
    }
    if (cands[best_i].fwd && plain_i >= 0 && best_plain <= best * 1.03) {
      best = best_plain;
      best_i = plain_i;
    }
  }
  S.release();
  flush.release();
  abuf.release();
  rowmax.release();
  pairk.release();
  evf.release();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (best >= 1e30) return mea::set_error(MEA_E_CUDA, "mea_autotune: no candidate ran");
  mea::AmpConfig c = cands[best_i];
  // keep the per-SM residency; the grid is re-capped per call
  c.grid = std::max(c.grid, P->num_sms);
  if (best_i != 0) {
    // store the full-size grid of this shape
    std::vector<mea::AmpConfig> full =
        mea::candidate_configs(dp, fp64, H, (int64_t)1 << 40, P->num_sms, P->smem_optin, P->smem_per_sm);
    for (auto& f : full)
      if (f.E_cta == c.E_cta && f.threads == c.threads && f.jamp_in_smem == c.jamp_in_smem &&
          f.slots_in_smem == c.slots_in_smem && f.regvar == c.regvar && f.per_sm == c.per_sm &&
          f.helshare == c.helshare && f.hsplit == c.hsplit && f.fwd == c.fwd)
        c.grid = f.grid;
    P->tuned[ti] = c;
    P->tuned_H[ti] = H;
  } else {
    P->tuned[ti] = mea::AmpConfig();  // the heuristic default won: keep using it
    P->tuned_H[ti] = 0;
  }
  if (out) {
    out->threads = c.threads;
    out->events_per_cta = c.E_cta;
    out->grid = c.grid;
    out->colour_amps_in_shared = c.jamp_in_smem ? 1 : 0;
    out->slots_in_shared = c.slots_in_smem ? 1 : 0;
    out->candidates = (int)cands.size();
    out->best_ms = best;
    out->default_ms = def_ms;
    out->register_cap = dp.gen ? (fp64 ? 128 : mea::kGenCapRegisters[c.regvar / 2]) : ((c.helshare && c.regvar == 0) ? 64 : 0);
    out->vertex_partials = (dp.gen && !fp64 && (c.regvar & 1)) ? 0 : 1;
    out->helicity_shared = c.helshare ? 1 : (c.hsplit ? 2 : 0);
    out->forwarding = c.fwd ? 1 : 0;
  }
  return MEA_OK;
}

}  // namespace mea

extern "C" {

mea_status mea_batch_create(const mea_batch_item* items, int n_items, mea_prec_mode prec, mea_batch_t* out) {
  if (!items || n_items <= 0 || !out) return mea::set_error(MEA_E_ARG, "mea_batch_create: bad arguments");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return mea::set_error(MEA_E_ARG, "mea_batch_create: bad precision");
  for (int i = 0; i < n_items; ++i) {
    const mea_batch_item& it = items[i];
    if (!it.proc || it.proc->host_only || it.n_events < 0 || (it.n_events > 0 && (!it.momenta_dev || !it.me2_dev)))
      return mea::set_error(MEA_E_ARG, "mea_batch_create: bad item " + std::to_string(i));
  }
  *out = nullptr;
  mea_batch_s* b = new mea_batch_s();
  b->items.assign(items, items + n_items);
  b->prec = prec;
  b->scratch.resize(n_items);
  auto bail = [&](mea_status st) {
    destroy_batch(b);
    return st;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < n_items && e == cudaSuccess; ++i) {
    cudaStream_t s;
    cudaEvent_t j;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) { b->streams.push_back(s); e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming); }
    if (e == cudaSuccess) b->joins.push_back(j);
  }
  if (e != cudaSuccess) return bail(mea::set_error(MEA_E_CUDA, std::string("mea_batch_create: ") + cudaGetErrorString(e)));
  // eager pass: sizes every scratch set and loads every kernel
  for (int i = 0; i < n_items; ++i) {
    const mea_batch_item& it = b->items[i];
    if (it.n_events == 0) continue;
    std::lock_guard<std::mutex> lk(it.proc->mu);
    mea_status st = mea::evaluate_with(it.proc, b->scratch[i], it.momenta_dev, it.n_events, MEA_HEL_SUM_NONZERO,
                                       nullptr, prec, it.me2_dev, it.flags_dev, b->streams[i]);
    if (st != MEA_OK) return bail(st);
  }
  for (auto s : b->streams)
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
      return bail(mea::set_error(MEA_E_CUDA, std::string("mea_batch_create: ") + cudaGetErrorString(e)));
  // capture: fork from the origin stream, one branch per item, join back
  uint64_t k0 = mea::launch_counter();
  e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return bail(mea::set_error(MEA_E_CUDA, std::string("mea_batch_create: ") + cudaGetErrorString(e)));
  mea_status cst = MEA_OK;
  cudaEventRecord(b->fork, b->origin);
  for (int i = 0; i < n_items && cst == MEA_OK; ++i) {
    const mea_batch_item& it = b->items[i];
    cudaStreamWaitEvent(b->streams[i], b->fork, 0);
    if (it.n_events > 0) {
      std::lock_guard<std::mutex> lk(it.proc->mu);
      cst = mea::evaluate_with(it.proc, b->scratch[i], it.momenta_dev, it.n_events, MEA_HEL_SUM_NONZERO, nullptr,
                               prec, it.me2_dev, it.flags_dev, b->streams[i]);
    }
    cudaEventRecord(b->joins[i], b->streams[i]);
    cudaStreamWaitEvent(b->origin, b->joins[i], 0);
  }
  e = cudaStreamEndCapture(b->origin, &b->graph);
  if (cst != MEA_OK) return bail(cst);
  if (e != cudaSuccess) return bail(mea::set_error(MEA_E_CUDA, std::string("mea_batch_create: capture: ") + cudaGetErrorString(e)));
  b->kernel_nodes = (int)(mea::launch_counter() - k0);
  mea::launch_counter() = k0;  // captured launches run only when the graph is launched
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return bail(mea::set_error(MEA_E_CUDA, std::string("mea_batch_create: instantiate: ") + cudaGetErrorString(e)));
  *out = b;
  return MEA_OK;
}

mea_status mea_batch_launch(mea_batch_t b, void* stream) {
  if (!b || !b->exec) return mea::set_error(MEA_E_ARG, "mea_batch_launch: null batch");
  MEA_CK(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)));
  mea::launch_counter() += (uint64_t)b->kernel_nodes;
  return MEA_OK;
}

mea_status mea_batch_info(mea_batch_t b, int* n_kernel_nodes) {
  if (!b || !n_kernel_nodes) return mea::set_error(MEA_E_ARG, "mea_batch_info: null argument");
  *n_kernel_nodes = b->kernel_nodes;
  return MEA_OK;
}

mea_status mea_batch_destroy(mea_batch_t b) {
  if (!b) return mea::set_error(MEA_E_ARG, "mea_batch_destroy: null batch");
  cudaStreamSynchronize(b->origin);
  destroy_batch(b);
  return MEA_OK;
}

}  // extern "C"

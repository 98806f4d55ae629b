// C ABI of libmea.so (declared in include/mea.h): process handles, device
// residency of the process tables, scratch management and the evaluation
// entry points.  No compute happens here; every step of the path runs in the
// CUDA kernels of amp_kernel.cu and ps_kernel.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../phasespace/phasespace.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mea.h"
#include "colour_gemm.h"
#include "jamp_gemm.h"
#include "generator.h"
#include "kernels.h"
#include "process.h"

namespace {

thread_local std::string g_err;

mea_status fail(mea_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define MEA_CUDA(call)                                                            \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(MEA_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace


namespace {

template <typename T>
cudaError_t upload(mea_process_s* P, const std::vector<T>& v, const T** out) {
  void* d = nullptr;
  size_t b = std::max<size_t>(v.size() * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&d, b);
  if (e != cudaSuccess) return e;
  P->owned.push_back(d);
  if (!v.empty()) e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  *out = reinterpret_cast<const T*>(d);
  return e;
}

void destroy(mea_process_s* P) {
  if (!P) return;
  for (cudaEvent_t e : P->st_events) cudaEventDestroy(e);
  for (void* d : P->owned) cudaFree(d);
  for (auto& x : P->scr) x.release();
  for (int i = 0; i < 2; ++i) {
    if (P->pin_in[i]) cudaFreeHost(P->pin_in[i]);
    if (P->pin_out[i]) cudaFreeHost(P->pin_out[i]);
    if (P->pin_flags[i]) cudaFreeHost(P->pin_flags[i]);
    P->d_in[i].release();
    P->d_out[i].release();
    P->d_flags[i].release();
    if (P->st[i]) cudaStreamDestroy(P->st[i]);
    if (P->done[i]) cudaEventDestroy(P->done[i]);
  }
  delete P;
}

cudaError_t place_scratch(mea::DevBuf& buf, const mea::DevProgram& d, bool fp64, const mea::AmpConfig& c,
                          mea::AmpLaunch& a) {
  size_t jb = (mea::jamp_scratch_bytes_needed(d, fp64, c) + 255) & ~size_t(255);
  size_t sb = mea::slot_scratch_bytes_needed(d, fp64, c);
  cudaError_t e = buf.ensure(jb + sb + 256);
  if (e != cudaSuccess) return e;
  a.jamp_scratch = reinterpret_cast<float*>(buf.p);
  a.slot_scratch = reinterpret_cast<float*>(reinterpret_cast<char*>(buf.p) + jb);
  return cudaSuccess;
}

// Stage timing: CUDA events on the launching stream around one stage's
// launches, when the process has stage timing enabled (off by default; the
// pool of events only grows).
class StageTimer {
 public:
  StageTimer(mea_process_s* P, cudaStream_t s, int stage) : P_(P), s_(s) {
    if (!P->stage_timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> lk(P->st_mu);
    const size_t k = P->st_used;
    while (P->st_events.size() < 2 * (k + 1)) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      P->st_events.push_back(e);
    }
    if (P->st_stage.size() < k + 1) P->st_stage.resize(k + 1);
    P->st_stage[k] = stage;
    if (cudaEventRecord(P->st_events[2 * k], s) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    pair_ = (long)k;
    P->st_used = k + 1;
  }
  ~StageTimer() {
    if (pair_ < 0) return;
    std::lock_guard<std::mutex> lk(P_->st_mu);
    if (cudaEventRecord(P_->st_events[2 * pair_ + 1], s_) != cudaSuccess) cudaGetLastError();
  }
  StageTimer(const StageTimer&) = delete;
  StageTimer& operator=(const StageTimer&) = delete;

 private:
  mea_process_s* P_;
  cudaStream_t s_;
  long pair_ = -1;
};

// Mixed path with both colour stages on the tensor cores: the interpreter
// writes every diagram amplitude (no colour accumulators), the colour
// amplitudes are formed as an exact integer contraction (jamp_gemm.cu), the
// colour sum as a split-precision contraction (colour_gemm.cu).  Used for
// processes without a straight-line kernel, or on request (colour_mode 2).
bool use_tensor_colour(const mea_process_s* P, mea_prec_mode prec, mea_hel_mode hm) {
  if (prec != MEA_PREC_MIXED || hm == MEA_HEL_GIVEN || P->opts.colour_mode == 1) return false;
  if (!P->jmap.ok) return false;
  if (P->opts.colour_mode == 2) return true;
  return P->dev.gen == nullptr;
}

// Events per chunk of the tensor-core path.  A chunk should hold enough
// (event, helicity) lanes to fill every SM with the amplitude kernel
// (kLanesPerSm), with its diagram amplitudes (8 bytes per diagram and pair)
// between kAmpMin and kAmpMax bytes.
constexpr size_t kAmpMin = size_t(1) << 30;
constexpr size_t kAmpMax = size_t(24) << 30;
constexpr int64_t kLanesPerSm = 2048;

int64_t tc_chunk_events(const mea_process_s* P, int H, int64_t n) {
  if (P->opts.chunk_events > 0) return std::max<int64_t>(1, std::min<int64_t>(n, P->opts.chunk_events));
  const size_t per_pair = 2 * (size_t)P->jmap.kd * sizeof(float);
  size_t bytes = (size_t)P->num_sms * kLanesPerSm * per_pair;
  bytes = std::min(kAmpMax, std::max(kAmpMin, bytes));
  const size_t per_event = (size_t)H * per_pair;
  return std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(bytes / std::max<size_t>(per_event, 1))));
}

// Launch configuration of the amplitude-output interpreter for H lanes per event.
mea::AmpConfig tc_amp_config(const mea_process_s* P, const mea::DevProgram& dp, int H, int64_t cn) {
  mea::AmpConfig c = mea::cached_plan(const_cast<mea_process_s*>(P), dp, false, true, H, cn);
  if (P->tuned[0].grid > 0 && P->tuned_H[0] == H) {  // configuration chosen by mea_autotune
    c = P->tuned[0];
    int64_t tiles = (cn + c.E_cta - 1) / c.E_cta;
    if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
  }
  return c;
}

mea_status do_evaluate_tc(mea_process_s* P, mea::EvalScratch& S, const double* mom, int64_t n, mea_hel_mode hm,
                          double* me2, uint8_t* flags, cudaStream_t s) {
  const mea::Program& G = P->prog;
  const mea::JampMap& JM = P->jmap;
  const int n_ext = G.n_ext;
  const int H = (hm == MEA_HEL_SUM_NONZERO) ? G.n_hel : (1 << n_ext);
  const int m = G.n_jamp;
  const int ldj = ((m + 15) / 16) * 16;
  const int64_t chunk = tc_chunk_events(P, H, n);
  const int64_t lda = ((2 * chunk * H + 127) / 128) * 128;
  MEA_CUDA(S.abuf.ensure(sizeof(float) * (size_t)JM.kd * (size_t)lda));
  MEA_CUDA(S.rowmax.ensure(sizeof(float) * 2 * (size_t)H * chunk));
  MEA_CUDA(S.jabs.ensure(sizeof(float) * (size_t)JM.n_splits * (size_t)H * chunk));
  MEA_CUDA(S.jbuf.ensure(sizeof(float) * 2 * (size_t)ldj * (size_t)H * chunk));
  MEA_CUDA(S.pairval.ensure(sizeof(double) * (size_t)H * chunk));
  MEA_CUDA(S.pairk.ensure(sizeof(float) * (size_t)H * chunk));
  MEA_CUDA(S.flag_list.ensure(sizeof(int32_t) * (size_t)chunk));
  MEA_CUDA(S.flag_count.ensure(sizeof(int32_t)));
  MEA_CUDA(S.evf.ensure((size_t)chunk));
  mea::DevProgram dp = P->dev;
  dp.gen = nullptr;   // the interpreter writes the diagram amplitudes
  dp.n_colour = 0;    // and holds no colour accumulators
  mea::JampGemmArgs jg;
  jg.A = reinterpret_cast<const float*>(S.abuf.p);
  jg.lda = lda;
  jg.rowmax = reinterpret_cast<const float*>(S.rowmax.p);
  jg.kd = JM.kd;
  jg.kpad = JM.kpad;
  jg.m = m;
  jg.nc = JM.nc;
  jg.n_splits = JM.n_splits;
  jg.q = JM.q;
  jg.cfac = JM.cfac;
  jg.tiles = P->jmap_tiles;
  jg.J = reinterpret_cast<float*>(S.jbuf.p);
  jg.ldj = ldj;
  jg.jabs = reinterpret_cast<float*>(S.jabs.p);
  jg.status = P->status;
  mea::ColourGemmArgs cg;
  cg.m = m;
  cg.ldj = ldj;
  cg.nc = P->cf_nc;
  cg.np = P->cf_np;
  cg.kp = P->cf_kp;
  cg.b_hi = P->cf_hi;
  cg.b_lo = P->cf_lo;
  cg.inv_den = P->dev.cf_inv_den;
  cg.status = P->status;
  cg.J = reinterpret_cast<const float*>(S.jbuf.p);
  cg.pairval = reinterpret_cast<double*>(S.pairval.p);
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t cn = std::min(chunk, n - c0);
    mea::AmpConfig c = tc_amp_config(P, dp, H, cn);
    mea::AmpLaunch a;
    a.mom = mom + (size_t)c0 * n_ext * 4;
    a.n_events = cn;
    a.hel_mode = (int)hm;
    a.me2 = me2 + c0;
    a.flags = flags ? flags + c0 : nullptr;
    a.flag_threshold = (float)P->opts.flag_threshold;
    a.amp_out = reinterpret_cast<float*>(S.abuf.p);
    a.lda = lda;
    a.amp_rowmax = reinterpret_cast<float*>(S.rowmax.p);
    a.pair_kappa = reinterpret_cast<float*>(S.pairk.p);
    a.ev_flags = reinterpret_cast<uint8_t*>(S.evf.p);
    MEA_CUDA(place_scratch(S.s32, dp, false, c, a));
    {
      StageTimer tm(P, s, MEA_STAGE_AMPLITUDES);
      MEA_CUDA(mea::launch_amp(dp, false, c, a, s));
    }
    jg.n_pairs = cn * H;
    {
      StageTimer tm(P, s, MEA_STAGE_COLOUR_AMPLITUDES);
      MEA_CUDA(mea::launch_jamp_gemm(jg, P->num_sms, s));
    }
    cg.n_pairs = cn * H;
    {
      StageTimer tm(P, s, MEA_STAGE_COLOUR_SUM);
      MEA_CUDA(mea::launch_colour_gemm(cg, P->num_sms, s));
    }
    mea::AmpLaunch f = a;
    f.amp_out = nullptr;
    bool reeval = P->opts.reeval_fp64 != 0;
    if (reeval) {
      MEA_CUDA(cudaMemsetAsync(S.flag_count.p, 0, sizeof(int32_t), s));
      f.flag_list = reinterpret_cast<int32_t*>(S.flag_list.p);
      f.flag_count = reinterpret_cast<int32_t*>(S.flag_count.p);
    }
    {
      StageTimer tm(P, s, MEA_STAGE_FINISH);
      MEA_CUDA(mea::launch_finish(f, H, reinterpret_cast<const double*>(S.pairval.p),
                                  reinterpret_cast<const float*>(S.pairk.p), s,
                                  reinterpret_cast<const float*>(S.jabs.p), JM.n_splits));
    }
    if (reeval) {
      mea::AmpConfig c2 = mea::cached_plan(P, P->dev, true, false, H, cn);
      mea::AmpLaunch b = f;
      b.event_list = f.flag_list;
      b.list_count = f.flag_count;
      b.flag_list = nullptr;
      b.flag_count = nullptr;
      b.write_flags_mode = 1;
      MEA_CUDA(place_scratch(S.s64, P->dev, true, c2, b));
      StageTimer tm(P, s, MEA_STAGE_REEVALUATION);
      MEA_CUDA(mea::launch_amp(P->dev, true, c2, b, s));
    }
  }
  return MEA_OK;
}

// Tuning on first use: the first evaluation of at least kAutoTuneMin events
// with the non-zero helicity sum (outside stream capture) waits for its
// stream, times the candidate tiles on its first events with me2 as scratch
// (mea_autotune), and then evaluates with the chosen tile.  The sample is
// kAutoTuneMin events, or up to kAutoTuneGen for the straight-line kernels,
// whose choice between bodies depends on how their spills share L2 with the
// streamed inputs at full size.  Tile shape and register cap never change a
// result bit; the body (vertex partials or not) changes the FP32 rounding
// order only (kernel_variant pins it).
constexpr int64_t kAutoTuneMin = 1 << 16;
constexpr int64_t kAutoTuneGen = 1 << 20;

void maybe_autotune(mea_process_s* P, const double* mom, int64_t n, mea_hel_mode hm, mea_prec_mode prec,
                    double* me2, cudaStream_t s) {
  const int ti = prec == MEA_PREC_FP64 ? 1 : 0;
  if (!P->opts.auto_tune || P->auto_tuned[ti] || n < kAutoTuneMin || hm != MEA_HEL_SUM_NONZERO) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  P->auto_tuned[ti] = true;
  if (cudaStreamSynchronize(s) != cudaSuccess) return;  // the error resurfaces at the evaluation's own launches
  const std::string keep = g_err;
  mea_tune_result r;
  const int64_t sample = (P->dev.gen && prec != MEA_PREC_FP64) ? std::min(n, kAutoTuneGen) : kAutoTuneMin;
  if (mea::autotune_locked(P, mom, sample, prec, me2, &r) != MEA_OK) g_err = keep;  // keep the heuristic
}

mea_status do_evaluate(mea_process_s* P, mea::EvalScratch& S, const double* mom, int64_t n, mea_hel_mode hm,
                       const int8_t* hel, mea_prec_mode prec, double* me2, uint8_t* flags,
                       cudaStream_t s) {
  maybe_autotune(P, mom, n, hm, prec, me2, s);
  if (use_tensor_colour(P, prec, hm)) return do_evaluate_tc(P, S, mom, n, hm, me2, flags, s);
  const mea::Program& G = P->prog;
  int H = (hm == MEA_HEL_SUM_NONZERO) ? G.n_hel : (hm == MEA_HEL_SUM_ALL ? (1 << G.n_ext) : 1);
  bool fp64 = prec == MEA_PREC_FP64;
  mea::AmpConfig c = mea::cached_plan(P, P->dev, fp64, false, H, n);
  const int ti = fp64 ? 1 : 0;
  if (P->tuned[ti].grid > 0 && P->tuned_H[ti] == H) {  // configuration chosen by mea_autotune
    c = P->tuned[ti];
    int64_t tiles = (n + c.E_cta - 1) / c.E_cta;
    if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
  }
  mea::AmpLaunch a;
  a.mom = mom;
  a.n_events = n;
  a.hel_given = hel;
  a.hel_mode = (int)hm;
  a.me2 = me2;
  a.flags = flags;
  a.flag_threshold = (float)P->opts.flag_threshold;
  MEA_CUDA(place_scratch(fp64 ? S.s64 : S.s32, P->dev, fp64, c, a));
  bool reeval = !fp64 && P->opts.reeval_fp64 && hm != MEA_HEL_GIVEN;
  if (reeval) {
    MEA_CUDA(S.flag_list.ensure(sizeof(int32_t) * (size_t)n));
    MEA_CUDA(S.flag_count.ensure(sizeof(int32_t)));
    MEA_CUDA(cudaMemsetAsync(S.flag_count.p, 0, sizeof(int32_t), s));
    a.flag_list = reinterpret_cast<int32_t*>(S.flag_list.p);
    a.flag_count = reinterpret_cast<int32_t*>(S.flag_count.p);
  }
  {
    StageTimer tm(P, s, MEA_STAGE_AMPLITUDES);
    MEA_CUDA(mea::launch_amp(P->dev, fp64, c, a, s));
  }
  if (reeval) {
    // FP64 re-evaluation of the flagged events; their count is read on the device
    mea::AmpConfig c2 = mea::cached_plan(P, P->dev, true, false, H, n);
    mea::AmpLaunch b = a;
    b.event_list = a.flag_list;
    b.list_count = a.flag_count;
    b.flag_list = nullptr;
    b.flag_count = nullptr;
    b.write_flags_mode = 1;
    MEA_CUDA(place_scratch(S.s64, P->dev, true, c2, b));
    StageTimer tm(P, s, MEA_STAGE_REEVALUATION);
    MEA_CUDA(mea::launch_amp(P->dev, true, c2, b, s));
  }
  return MEA_OK;
}

}  // namespace

namespace mea {
mea_status set_error(mea_status s, const std::string& msg) { return fail(s, msg); }

AmpConfig cached_plan(mea_process_s* P, const DevProgram& dp, bool fp64, bool tc, int H, int64_t n) {
  AmpConfig c;
  {
    std::lock_guard<std::mutex> lk(P->plan_mu);
    auto key = std::make_tuple(fp64, tc, H);
    auto it = P->plan_cache.find(key);
    if (it == P->plan_cache.end())
      it = P->plan_cache.emplace(key, plan_amp(dp, fp64, H, (int64_t)1 << 40, P->num_sms, P->smem_optin,
                                               P->smem_per_sm)).first;
    c = it->second;
  }
  const int64_t tiles = (n + c.E_cta - 1) / c.E_cta;
  if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
  return c;
}
bool uses_tensor_path(const mea_process_s* P, mea_prec_mode prec, mea_hel_mode hm) {
  return use_tensor_colour(P, prec, hm);
}
int64_t tensor_chunk_events(const mea_process_s* P, int H, int64_t n) { return tc_chunk_events(P, H, n); }
mea_status evaluate_with(mea_process_s* P, EvalScratch& S, const double* mom, int64_t n, mea_hel_mode hm,
                         const int8_t* hel, mea_prec_mode prec, double* me2, uint8_t* flags, cudaStream_t s) {
  return do_evaluate(P, S, mom, n, hm, hel, prec, me2, flags, s);
}

size_t scratch_estimate(mea_process_s* P, int64_t n, mea_prec_mode prec) {
  const Program& G = P->prog;
  const int H = G.n_hel;
  const bool fp64 = prec == MEA_PREC_FP64;
  auto work = [&](const DevProgram& d, bool f64, int64_t ne) {
    AmpConfig c = plan_amp(d, f64, H, ne, P->num_sms, P->smem_optin, P->smem_per_sm);
    return jamp_scratch_bytes_needed(d, f64, c) + slot_scratch_bytes_needed(d, f64, c) + 512;
  };
  if (use_tensor_colour(P, prec, MEA_HEL_SUM_NONZERO)) {
    const int ldj = ((G.n_jamp + 15) / 16) * 16;
    const int64_t chunk = tc_chunk_events(P, H, n);
    const int64_t lda = ((2 * chunk * H + 127) / 128) * 128;
    DevProgram dp = P->dev;
    dp.gen = nullptr;
    dp.n_colour = 0;
    return sizeof(float) * (size_t)P->jmap.kd * (size_t)lda + sizeof(float) * (size_t)H * chunk * (3 + P->jmap.n_splits) +
           sizeof(float) * 2 * (size_t)ldj * (size_t)H * chunk + sizeof(double) * (size_t)H * chunk +
           (size_t)chunk * 5 + 4096 + work(dp, false, chunk) + work(P->dev, true, chunk);
  }
  size_t b = work(P->dev, fp64, n);
  if (!fp64 && P->opts.reeval_fp64) b += (size_t)n * 4 + 256 + work(P->dev, true, n);
  return b;
}
}  // namespace mea

extern "C" {

const char* mea_last_error(void) { return g_err.c_str(); }

uint64_t mea_kernel_launch_count(void) { return mea::launch_counter(); }

mea_status mea_create_process(const int* pdg, int n_ext, const mea_options* opts, mea_process_t* out) {
  if (!pdg || !out || n_ext < 4 || n_ext > 7) return fail(MEA_E_ARG, "mea_create_process: bad arguments");
  *out = nullptr;
  mea_process_s* P = new (std::nothrow) mea_process_s();
  if (!P) return fail(MEA_E_NOMEM, "mea_create_process: out of host memory");
  P->opts.alpha_s = 0.118;
  P->opts.flag_threshold = 1e-5;
  P->opts.reeval_fp64 = 1;
  P->opts.colour_mode = 0;
  P->opts.chunk_events = 0;
  P->opts.auto_tune = 1;
  P->opts.kernel_variant = 0;
  if (opts && (opts->kernel_variant < 0 || opts->kernel_variant > mea::kGenRegVariants)) {
    destroy(P);
    return fail(MEA_E_ARG, "mea_create_process: kernel_variant out of range");
  }
  if (opts && (opts->helicity_sharing < 0 || opts->helicity_sharing > 4)) {
    destroy(P);
    return fail(MEA_E_ARG, "mea_create_process: helicity_sharing out of range");
  }
  P->opts.helicity_sharing = 0;
  if (opts) {
    P->opts.kernel_variant = opts->kernel_variant;
    if (opts->alpha_s > 0) P->opts.alpha_s = opts->alpha_s;
    if (opts->flag_threshold > 0) P->opts.flag_threshold = opts->flag_threshold;
    P->opts.reeval_fp64 = opts->reeval_fp64;
    P->opts.colour_mode = opts->colour_mode;
    P->opts.chunk_events = opts->chunk_events;
    P->opts.auto_tune = opts->auto_tune;
    P->opts.helicity_sharing = opts->helicity_sharing;
  }
  try {
    P->prog = mea::build_program(std::vector<int>(pdg, pdg + n_ext));
  } catch (std::exception& e) {
    destroy(P);
    return fail(MEA_E_UNSUPPORTED, std::string("mea_create_process: ") + e.what());
  }
  try {
    P->hs = mea::build_helicity_shared(P->prog, P->prog.n_hel);
    P->hs_ok = true;
  } catch (std::exception&) {
    P->hs_ok = false;  // the per-lane interpreter covers the process alone
  }
  try {
    P->hsp = mea::build_split_shared(P->prog, P->prog.n_hel);
    P->hsp_ok = P->hsp.levels <= 8 && !P->hsp.main_ops.empty();
  } catch (std::exception&) {
    P->hsp_ok = false;
  }
  const mea::Program& G = P->prog;
  cudaError_t e = cudaGetDevice(&P->device);
  if (e != cudaSuccess) { destroy(P); return fail(MEA_E_CUDA, cudaGetErrorString(e)); }
  int v = 0;
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  P->smem_optin = (size_t)v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, P->device);
  P->smem_per_sm = (size_t)v;

  std::vector<int8_t> leg(4 * (size_t)n_ext, 0);
  for (int l = 0; l < n_ext; ++l) {
    int type = G.leg_type[l];
    int kind = 0;
    if (type == 1) kind = G.incoming[l] ? 0 : 1;       // u (incoming quark) or v (outgoing antiquark)
    if (type == 2) kind = G.incoming[l] ? 3 : 2;       // vbar (incoming antiquark) or ubar (outgoing quark)
    leg[4 * l] = (int8_t)type;
    leg[4 * l + 1] = (int8_t)kind;
    leg[4 * l + 2] = (int8_t)G.incoming[l];
  }
  std::vector<float> cff(G.cf_jamp.size());
  std::vector<double> cfd(G.cf_jamp.size());
  for (size_t i = 0; i < G.cf_jamp.size(); ++i) {
    cff[i] = (float)G.cf_jamp[i];
    cfd[i] = (double)G.cf_jamp[i];
  }
  mea::DevProgram& D = P->dev;
  const mea::Op* dops;
  const mea::ColEntry* dcol;
  const uint32_t* dmask;
  const int8_t *dleg, *dhel, *dhall;
  const float* dcff;
  const double* dcfd;
  if ((e = upload(P, G.ops, &dops)) != cudaSuccess || (e = upload(P, G.col, &dcol)) != cudaSuccess ||
      (e = upload(P, G.masks, &dmask)) != cudaSuccess || (e = upload(P, leg, &dleg)) != cudaSuccess ||
      (e = upload(P, G.hel, &dhel)) != cudaSuccess || (e = upload(P, G.hel_all, &dhall)) != cudaSuccess ||
      (e = upload(P, cff, &dcff)) != cudaSuccess || (e = upload(P, cfd, &dcfd)) != cudaSuccess) {
    destroy(P);
    return fail(e == cudaErrorMemoryAllocation ? MEA_E_NOMEM : MEA_E_CUDA,
                std::string("mea_create_process: ") + cudaGetErrorString(e));
  }
  D.ops = dops;
  D.n_ops = (int)G.ops.size();
  D.col = dcol;
  D.masks = dmask;
  D.n_masks = (int)G.masks.size();
  D.leg_info = dleg;
  D.n_ext = n_ext;
  D.n_slots = G.n_slots;
  D.n_colour = G.n_jamp;  // colour amplitudes accumulated (folded for gluons)
  D.cf_f = dcff;
  D.cf_d = dcfd;
  D.cf_inv_den = 1.0 / (double)G.cf_den;
  D.hel = dhel;
  D.n_hel = G.n_hel;
  D.hel_all = dhall;
  D.g = std::sqrt(4.0 * M_PI * P->opts.alpha_s);
  D.gen = (P->opts.colour_mode == 2) ? nullptr : mea::find_generated(pdg, n_ext);
  D.gen_forced = (D.gen && P->opts.kernel_variant > 0) ? P->opts.kernel_variant - 1 : -1;
  {
    // colour matrix as tensor-core operand tiles, and the status word
    mea::ColourTiles T = mea::build_colour_tiles(G.cf_jamp, G.n_jamp);
    const __half* dh = nullptr;
    const __half* dl = nullptr;
    std::vector<int> st(1, 0);
    const int* dst = nullptr;
    if ((e = upload(P, T.hi, &dh)) != cudaSuccess || (!T.exact && (e = upload(P, T.lo, &dl)) != cudaSuccess) ||
        (e = upload(P, st, &dst)) != cudaSuccess) {
      destroy(P);
      return fail(MEA_E_CUDA, std::string("mea_create_process: ") + cudaGetErrorString(e));
    }
    P->cf_hi = dh;
    P->cf_lo = T.exact ? nullptr : dl;
    P->cf_nc = T.nc;
    P->cf_np = T.np;
    P->cf_kp = T.kp;
    P->status = const_cast<int*>(dst);
  }
  {
    // diagram -> colour-amplitude coefficients for the tensor-core stage
    P->jmap = mea::build_jamp_map(G);
    if (P->jmap.ok) {
      const __half* dt = nullptr;
      const float* dw = nullptr;
      if ((e = upload(P, P->jmap.tiles, &dt)) != cudaSuccess || (e = upload(P, P->jmap.weight, &dw)) != cudaSuccess) {
        destroy(P);
        return fail(MEA_E_CUDA, std::string("mea_create_process: ") + cudaGetErrorString(e));
      }
      P->jmap_tiles = dt;
      D.amp_w = dw;
      std::vector<__half>().swap(P->jmap.tiles);
    }
  }
  if (P->jmap.ok && P->opts.helicity_sharing != 2 && P->opts.helicity_sharing != 3) {
    D.fwd_only = P->opts.helicity_sharing == 4;
    // register forwarding for the amplitude-output interpreter (helshare.h)
    const std::vector<uint8_t> fw = mea::build_forwarding_flags(G);
    const uint8_t* dfw = nullptr;
    if ((e = upload(P, fw, &dfw)) != cudaSuccess) {
      destroy(P);
      return fail(MEA_E_CUDA, std::string("mea_create_process: ") + cudaGetErrorString(e));
    }
    D.fwd = dfw;
  }
  if (P->hsp_ok && P->jmap.ok && (P->opts.helicity_sharing == 0 || P->opts.helicity_sharing == 3)) {
    // split layout for the tensor-core path's amplitude stage
    const uint32_t* dt = nullptr;
    const mea::HsOp *dr = nullptr, *dmr = nullptr;
    const mea::Op* dmo = nullptr;
    if ((e = upload(P, P->hsp.tasks, &dt)) != cudaSuccess || (e = upload(P, P->hsp.rec, &dr)) != cudaSuccess ||
        (e = upload(P, P->hsp.main_ops, &dmo)) != cudaSuccess || (e = upload(P, P->hsp.main_rec, &dmr)) != cudaSuccess) {
      destroy(P);
      return fail(MEA_E_CUDA, std::string("mea_create_process: ") + cudaGetErrorString(e));
    }
    D.hsp_tasks = dt;
    D.hsp_rec = dr;
    D.hsp_main_ops = dmo;
    D.hsp_main_rec = dmr;
    D.hsp_n_main = (int)P->hsp.main_ops.size();
    D.hsp_levels = P->hsp.levels;
    for (int l = 0; l < P->hsp.levels; ++l) D.hsp_level_end[l] = P->hsp.level_end[l];
    D.hsp_area = P->hsp.area;
    D.hsp_only = P->opts.helicity_sharing == 3;
  }
  if (P->hs_ok && P->jmap.ok && (P->opts.helicity_sharing == 0 || P->opts.helicity_sharing == 2)) {
    // helicity-shared layout for the tensor-core path's amplitude stage
    const mea::HsOp* dhs = nullptr;
    if ((e = upload(P, P->hs.ops, &dhs)) != cudaSuccess) {
      destroy(P);
      return fail(MEA_E_CUDA, std::string("mea_create_process: ") + cudaGetErrorString(e));
    }
    D.hs = dhs;
    D.hs_arena = P->hs.arena;
    D.hs_only = P->opts.helicity_sharing == 2;
  }
  *out = P;
  return MEA_OK;
}

mea_status mea_create_process_host_only(const int* pdg, int n_ext, const mea_options* opts, mea_process_t* out) {
  if (!pdg || !out || n_ext < 4 || n_ext > 7) return fail(MEA_E_ARG, "mea_create_process_host_only: bad arguments");
  *out = nullptr;
  mea_process_s* P = new (std::nothrow) mea_process_s();
  if (!P) return fail(MEA_E_NOMEM, "mea_create_process_host_only: out of host memory");
  P->host_only = true;
  P->opts.alpha_s = (opts && opts->alpha_s > 0) ? opts->alpha_s : 0.118;
  try {
    P->prog = mea::build_program(std::vector<int>(pdg, pdg + n_ext));
  } catch (std::exception& e) {
    destroy(P);
    return fail(MEA_E_UNSUPPORTED, std::string("mea_create_process_host_only: ") + e.what());
  }
  try {
    P->hs = mea::build_helicity_shared(P->prog, P->prog.n_hel);
    P->hs_ok = true;
  } catch (std::exception&) {
    P->hs_ok = false;
  }
  try {
    P->hsp = mea::build_split_shared(P->prog, P->prog.n_hel);
    P->hsp_ok = P->hsp.levels <= 8 && !P->hsp.main_ops.empty();
  } catch (std::exception&) {
    P->hsp_ok = false;
  }
  *out = P;
  return MEA_OK;
}

mea_status mea_process_info(mea_process_t P, mea_process_info_t* info) {
  if (!P || !info) return fail(MEA_E_ARG, "mea_process_info: null argument");
  const mea::Program& G = P->prog;
  std::memset(info, 0, sizeof(*info));
  info->n_ext = G.n_ext;
  info->n_diagrams = G.n_diagrams;
  info->n_colour = G.n_colour;
  info->n_hel_nonzero = G.n_hel;
  info->n_currents = G.n_currents;
  info->n_ops = (int)G.ops.size();
  info->n_slots = G.n_slots;
  info->cf_denominator = G.cf_den;
  info->cf_max_abs_numerator = G.cf_max_abs;
  info->n_colour_amplitudes = G.n_jamp;
  info->flops_per_hel = G.flops_per_hel;
  info->colour_flops_per_hel = 4.0 * (double)G.n_jamp * (double)G.n_jamp;
  info->flops_per_hel_plain = G.flops_per_hel_plain;
  int64_t nnz = 0;
  for (const mea::Op& op : G.ops)
    if (mea::is_amp_op(op.type)) nnz += op.col_count;
  info->n_colour_entries = nnz;
  if (P->hs_ok) {
    info->hs_variants = P->hs.variants;
    info->hs_arena_variants = P->hs.arena;
    info->hs_flops_per_event = P->hs.flops_event;
  }
  if (P->hsp_ok) {
    info->hsp_area_variants = P->hsp.area;
    info->hsp_flops_per_event = P->hsp.flops_event;
  }
  return MEA_OK;
}

mea_status mea_colour_matrix(mea_process_t P, int64_t* num, int64_t* den) {
  if (!P || !num || !den) return fail(MEA_E_ARG, "mea_colour_matrix: null argument");
  std::copy(P->prog.cf_num.begin(), P->prog.cf_num.end(), num);
  *den = P->prog.cf_den;
  return MEA_OK;
}

mea_status mea_helicities(mea_process_t P, int8_t* hel, int cap, int* n_hel) {
  if (!P || !n_hel) return fail(MEA_E_ARG, "mea_helicities: null argument");
  *n_hel = P->prog.n_hel;
  if (hel) {
    if (cap < P->prog.n_hel) return fail(MEA_E_ARG, "mea_helicities: buffer too small");
    std::copy(P->prog.hel.begin(), P->prog.hel.end(), hel);
  }
  return MEA_OK;
}

mea_status mea_check_status(mea_process_t P, void* stream) {
  if (!P) return fail(MEA_E_ARG, "mea_check_status: null process");
  if (P->host_only) return MEA_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MEA_CUDA(cudaStreamSynchronize(s));
  int v = 0;
  MEA_CUDA(cudaMemcpy(&v, P->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) {
    int z = 0;
    MEA_CUDA(cudaMemcpy(P->status, &z, sizeof(int), cudaMemcpyHostToDevice));
    return fail(MEA_E_TIMEOUT, "mea_check_status: a bounded wait in a tensor-core kernel expired");
  }
  return MEA_OK;
}

mea_status mea_probe_bounded_wait(mea_process_t P, uint32_t spin_limit, void* stream) {
  if (!P) return fail(MEA_E_ARG, "mea_probe_bounded_wait: null process");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_probe_bounded_wait: host-only process handle");
  if (spin_limit < 1 || spin_limit > (1u << 20)) return fail(MEA_E_ARG, "mea_probe_bounded_wait: limit out of range");
  MEA_CUDA(mea::launch_wait_probe(P->status, spin_limit, reinterpret_cast<cudaStream_t>(stream)));
  return MEA_OK;
}

mea_status mea_set_stage_timing(mea_process_t P, int enable) {
  if (!P) return fail(MEA_E_ARG, "mea_set_stage_timing: null process");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_set_stage_timing: host-only process handle");
  std::lock_guard<std::mutex> lk(P->st_mu);
  P->stage_timing = enable != 0;
  P->st_used = 0;
  return MEA_OK;
}

mea_status mea_get_stage_times(mea_process_t P, mea_stage_times* out) {
  if (!P || !out) return fail(MEA_E_ARG, "mea_get_stage_times: null argument");
  std::memset(out, 0, sizeof(*out));
  if (P->host_only) return MEA_OK;
  std::lock_guard<std::mutex> lk(P->st_mu);
  for (size_t k = 0; k < P->st_used; ++k) {
    MEA_CUDA(cudaEventSynchronize(P->st_events[2 * k + 1]));
    float ms = 0.f;
    MEA_CUDA(cudaEventElapsedTime(&ms, P->st_events[2 * k], P->st_events[2 * k + 1]));
    const int st = P->st_stage[k];
    if (st >= 0 && st < MEA_N_STAGES) {
      out->ms[st] += ms;
      out->launches[st] += 1;
    }
  }
  P->st_used = 0;
  return MEA_OK;
}

mea_status mea_destroy_process(mea_process_t P) {
  if (!P) return fail(MEA_E_ARG, "mea_destroy_process: null handle");
  if (!P->host_only) cudaDeviceSynchronize();
  destroy(P);
  return MEA_OK;
}

mea_status mea_evaluate(mea_process_t P, const double* mom, int64_t n, mea_hel_mode hm, const int8_t* hel,
                        mea_prec_mode prec, double* me2, uint8_t* flags, void* stream) {
  if (!P) return fail(MEA_E_ARG, "mea_evaluate: null process");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_evaluate: host-only process handle");
  if (n < 0 || n > (int64_t)0x7fffffff) return fail(MEA_E_ARG, "mea_evaluate: n_events out of range");
  if (n == 0) return MEA_OK;
  if (!mom || !me2) return fail(MEA_E_ARG, "mea_evaluate: null momenta or me2");
  if (hm != MEA_HEL_SUM_NONZERO && hm != MEA_HEL_SUM_ALL && hm != MEA_HEL_GIVEN)
    return fail(MEA_E_ARG, "mea_evaluate: bad helicity mode");
  if (hm == MEA_HEL_GIVEN && !hel) return fail(MEA_E_ARG, "mea_evaluate: MEA_HEL_GIVEN needs hel_dev");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return fail(MEA_E_ARG, "mea_evaluate: bad precision");
  std::lock_guard<std::mutex> lk(P->mu);
  return do_evaluate(P, P->scr[0], mom, n, hm, hel, prec, me2, flags, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {
// Releases device buffers local to one call when the call returns, on every
// path (mea::DevBuf itself is a plain record that longer-lived holders copy,
// so it has no destructor).
class ScopedBufs {
 public:
  ScopedBufs(std::initializer_list<mea::DevBuf*> bufs) : bufs_(bufs) {}
  ScopedBufs(const ScopedBufs&) = delete;
  ScopedBufs& operator=(const ScopedBufs&) = delete;
  ~ScopedBufs() {
    for (mea::DevBuf* b : bufs_) b->release();
  }

 private:
  std::vector<mea::DevBuf*> bufs_;
};

// Host copy into / out of the pinned staging buffers, split over host threads
// for large blocks (one core's memcpy bandwidth would bound the pipeline).
void host_copy(void* dst, const void* src, size_t bytes) {
  constexpr size_t kPerThread = size_t(4) << 20;
  const int nt = (int)std::min<size_t>(16, bytes / kPerThread);
  if (nt <= 1) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t part = ((bytes + nt - 1) / nt + 63) & ~size_t(63);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int i = 0; i < nt; ++i) {
    const size_t b0 = (size_t)i * part;
    if (b0 < bytes)
      std::memcpy(static_cast<char*>(dst) + b0, static_cast<const char*>(src) + b0, std::min(part, bytes - b0));
  }
}
// True when [p, p + bytes) starts and ends in page-locked host memory, so the
// DMA engines can read or write it without a staging copy.
bool page_locked(const void* p, size_t bytes) {
  if (!p || bytes == 0) return false;
  const void* ends[2] = {p, static_cast<const char*>(p) + bytes - 1};
  for (const void* q : ends) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (at.type != cudaMemoryTypeHost) return false;
  }
  return true;
}
}  // namespace

extern "C" {

mea_status mea_evaluate_host(mea_process_t P, const double* mom_h, int64_t n, mea_prec_mode prec,
                             double* me2_h, uint8_t* flags_h) {
  if (!P) return fail(MEA_E_ARG, "mea_evaluate_host: null process");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_evaluate_host: host-only process handle");
  if (n < 0) return fail(MEA_E_ARG, "mea_evaluate_host: negative n_events");
  if (n == 0) return MEA_OK;
  if (!mom_h || !me2_h) return fail(MEA_E_ARG, "mea_evaluate_host: null buffer");
  std::lock_guard<std::mutex> lk(P->mu);
  const int n_ext = P->prog.n_ext;
  const int64_t chunk = std::min<int64_t>(n, 1 << 18);
  if (P->pipe_chunk < chunk) {
    for (int i = 0; i < 2; ++i) {
      if (P->pin_in[i]) cudaFreeHost(P->pin_in[i]);
      if (P->pin_out[i]) cudaFreeHost(P->pin_out[i]);
      if (P->pin_flags[i]) cudaFreeHost(P->pin_flags[i]);
      P->pin_in[i] = P->pin_out[i] = P->pin_flags[i] = nullptr;
      MEA_CUDA(cudaHostAlloc(&P->pin_in[i], sizeof(double) * 4 * n_ext * chunk, cudaHostAllocDefault));
      MEA_CUDA(cudaHostAlloc(&P->pin_out[i], sizeof(double) * chunk, cudaHostAllocDefault));
      MEA_CUDA(cudaHostAlloc(&P->pin_flags[i], chunk, cudaHostAllocDefault));
      MEA_CUDA(P->d_in[i].ensure(sizeof(double) * 4 * n_ext * chunk));
      MEA_CUDA(P->d_out[i].ensure(sizeof(double) * chunk));
      MEA_CUDA(P->d_flags[i].ensure(chunk));
      if (!P->st[i]) MEA_CUDA(cudaStreamCreateWithFlags(&P->st[i], cudaStreamNonBlocking));
      if (!P->done[i]) MEA_CUDA(cudaEventCreateWithFlags(&P->done[i], cudaEventDisableTiming));
    }
    P->pipe_chunk = chunk;
  }
  const int64_t n_chunks = (n + chunk - 1) / chunk;
  // page-locked caller buffers are read and written by the copy engines directly
  const bool in_direct = page_locked(mom_h, sizeof(double) * 4 * n_ext * (size_t)n);
  const bool out_direct = page_locked(me2_h, sizeof(double) * (size_t)n);
  const bool fl_direct = flags_h && page_locked(flags_h, (size_t)n);
  int64_t pending[2] = {-1, -1};
  auto drain = [&](int b) -> mea_status {
    if (pending[b] < 0) return MEA_OK;
    MEA_CUDA(cudaEventSynchronize(P->done[b]));
    int64_t c0 = pending[b] * chunk;
    int64_t cn = std::min(chunk, n - c0);
    if (!out_direct) host_copy(me2_h + c0, P->pin_out[b], sizeof(double) * cn);
    if (flags_h && !fl_direct) host_copy(flags_h + c0, P->pin_flags[b], cn);
    pending[b] = -1;
    return MEA_OK;
  };
  for (int64_t k = 0; k < n_chunks; ++k) {
    int b = (int)(k & 1);
    mea_status s = drain(b);
    if (s != MEA_OK) return s;
    int64_t c0 = k * chunk, cn = std::min(chunk, n - c0);
    const double* src = mom_h + (size_t)c0 * n_ext * 4;
    if (!in_direct) {
      host_copy(P->pin_in[b], src, sizeof(double) * 4 * n_ext * cn);
      src = static_cast<const double*>(P->pin_in[b]);
    }
    MEA_CUDA(cudaMemcpyAsync(P->d_in[b].p, src, sizeof(double) * 4 * n_ext * cn, cudaMemcpyHostToDevice, P->st[b]));
    s = do_evaluate(P, P->scr[1 + b], reinterpret_cast<const double*>(P->d_in[b].p), cn, MEA_HEL_SUM_NONZERO, nullptr, prec,
                    reinterpret_cast<double*>(P->d_out[b].p), reinterpret_cast<uint8_t*>(P->d_flags[b].p), P->st[b]);
    if (s != MEA_OK) return s;
    MEA_CUDA(cudaMemcpyAsync(out_direct ? me2_h + c0 : P->pin_out[b], P->d_out[b].p, sizeof(double) * cn,
                             cudaMemcpyDeviceToHost, P->st[b]));
    if (flags_h)
      MEA_CUDA(cudaMemcpyAsync(fl_direct ? flags_h + c0 : P->pin_flags[b], P->d_flags[b].p, cn, cudaMemcpyDeviceToHost,
                               P->st[b]));
    MEA_CUDA(cudaEventRecord(P->done[b], P->st[b]));
    pending[b] = k;
  }
  for (int b = 0; b < 2; ++b) {
    mea_status s = drain(b);
    if (s != MEA_OK) return s;
  }
  return MEA_OK;
}

// ---- evaluation without allocation ------------------------------------------
// Scratch for mea_evaluate_noalloc: one fixed array in the device image.  Host
// code must not use its name as a device address: the address is looked up
// with cudaGetSymbolAddress, with the device current, once per device and CUDA
// context (a context created after cudaDeviceReset reloads the module, so the
// lookup is repeated when the context's unique id changes).
static __device__ __align__(256) unsigned char g_noalloc_scratch[MEA_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
struct NoallocSlot {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
NoallocSlot g_noalloc[64];

// Unique id of the calling thread's current CUDA context (driver entry points
// resolved through the runtime, so the library does not link libcuda).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    resolved = true;
  }
  void* ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}
}  // namespace

mea_status mea_evaluate_noalloc(mea_process_t P, const double* mom, int64_t n, mea_prec_mode prec, double* me2,
                                uint8_t* flags, void* stream) {
  if (!P) return fail(MEA_E_ARG, "mea_evaluate_noalloc: null process");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_evaluate_noalloc: host-only process handle");
  if (n < 0 || n > (int64_t)0x7fffffff) return fail(MEA_E_ARG, "mea_evaluate_noalloc: n_events out of range");
  if (n == 0) return MEA_OK;
  if (!mom || !me2) return fail(MEA_E_ARG, "mea_evaluate_noalloc: null momenta or me2");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return fail(MEA_E_ARG, "mea_evaluate_noalloc: bad precision");
  int dev = 0;
  MEA_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MEA_E_ARG, "mea_evaluate_noalloc: device index out of range");
  if (dev != P->device) return fail(MEA_E_ARG, "mea_evaluate_noalloc: process belongs to another device");
  void* base = nullptr;
  {
    // set-up: the array's device address for this device and context
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx);
    NoallocSlot& slot = g_noalloc[dev];
    if (!slot.ptr || !have_ctx || slot.ctx_id != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(MEA_E_CUDA, std::string("mea_evaluate_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      slot.ptr = p;
      slot.ctx_id = have_ctx ? ctx : 0;
    }
    base = slot.ptr;
  }
  const mea::Program& G = P->prog;
  const int H = G.n_hel;
  const bool fp64 = prec == MEA_PREC_FP64;
  const bool reeval = !fp64 && P->opts.reeval_fp64;
  const int ti = fp64 ? 1 : 0;
  std::lock_guard<std::mutex> lk(P->mu);
  // the launch configuration mea_evaluate uses: the tuned one when mea_autotune
  // (explicit or on first use) has chosen one for this helicity count
  mea::AmpConfig c = mea::cached_plan(P, P->dev, fp64, false, H, n);
  if (P->tuned[ti].grid > 0 && P->tuned_H[ti] == H && !mea::uses_tensor_path(P, prec, MEA_HEL_SUM_NONZERO)) {
    c = P->tuned[ti];
    const int64_t tiles = (n + c.E_cta - 1) / c.E_cta;
    if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
  }
  mea::AmpConfig c2 = mea::cached_plan(P, P->dev, true, false, H, n);
  auto work_bytes = [&](bool f64, const mea::AmpConfig& cc) {
    size_t jb = (mea::jamp_scratch_bytes_needed(P->dev, f64, cc) + 255) & ~size_t(255);
    return jb + ((mea::slot_scratch_bytes_needed(P->dev, f64, cc) + 255) & ~size_t(255));
  };
  // layout: [count word | flagged-event list | work space shared by both launches]
  const size_t list_off = 256;
  const size_t list_bytes = reeval ? (((size_t)n * sizeof(int32_t) + 255) & ~size_t(255)) : 0;
  const size_t work_off = list_off + list_bytes;
  size_t work = work_bytes(fp64, c);
  if (reeval) work = std::max(work, work_bytes(true, c2));
  const size_t need = work_off + work;
  if (need > (size_t)MEA_NOALLOC_SCRATCH_BYTES)
    return fail(MEA_E_ARG, "mea_evaluate_noalloc: request needs " + std::to_string(need) +
                               " bytes of scratch, the fixed array holds " +
                               std::to_string((size_t)MEA_NOALLOC_SCRATCH_BYTES));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* b = reinterpret_cast<char*>(base);
  auto place = [&](bool f64, const mea::AmpConfig& cc, mea::AmpLaunch& a) {
    size_t jb = (mea::jamp_scratch_bytes_needed(P->dev, f64, cc) + 255) & ~size_t(255);
    a.jamp_scratch = reinterpret_cast<float*>(b + work_off);
    a.slot_scratch = reinterpret_cast<float*>(b + work_off + jb);
  };
  mea::AmpLaunch a;
  a.mom = mom;
  a.n_events = n;
  a.hel_mode = 0;
  a.me2 = me2;
  a.flags = flags;
  a.flag_threshold = (float)P->opts.flag_threshold;
  place(fp64, c, a);
  if (reeval) {
    MEA_CUDA(cudaMemsetAsync(b, 0, sizeof(int32_t), s));  // the count must start at zero every call
    a.flag_count = reinterpret_cast<int32_t*>(b);
    a.flag_list = reinterpret_cast<int32_t*>(b + list_off);
  }
  MEA_CUDA(mea::launch_amp(P->dev, fp64, c, a, s));
  if (reeval) {
    mea::AmpLaunch r = a;
    r.event_list = a.flag_list;
    r.list_count = a.flag_count;
    r.flag_list = nullptr;
    r.flag_count = nullptr;
    r.write_flags_mode = 1;
    place(true, c2, r);
    MEA_CUDA(mea::launch_amp(P->dev, true, c2, r, s));
  }
  return MEA_OK;
}

mea_status mea_generate_phase_space(const mea_ps_config* cfg, uint64_t first_event, int64_t n, double* mom,
                                    int32_t* attempts, void* stream) {
  if (!cfg || n < 0) return fail(MEA_E_ARG, "mea_generate_phase_space: bad arguments");
  if (cfg->n_final < 2 || cfg->n_final > 8 || !(cfg->rs_lo > 0) || !(cfg->rs_hi >= cfg->rs_lo))
    return fail(MEA_E_ARG, "mea_generate_phase_space: bad configuration");
  if (n == 0) return MEA_OK;
  if (!mom) return fail(MEA_E_ARG, "mea_generate_phase_space: null momenta");
  mea::PsConfigDev c{cfg->seed, cfg->n_final, cfg->rs_lo, cfg->rs_hi, cfg->pt_min, cfg->eta_max, cfg->dr_min,
                     cfg->ptij_min};
  MEA_CUDA(mea::launch_phase_space(c, first_event, n, mom, attempts, reinterpret_cast<cudaStream_t>(stream)));
  return MEA_OK;
}

mea_status mea_partonic_cross_section(mea_process_t P, double sqrt_s, const mea_ps_config* cuts,
                                      uint64_t first_event, int64_t n, mea_prec_mode prec, mea_xsec_result* out) {
  if (!P || !cuts || !out || n <= 0 || !(sqrt_s > 0) || !std::isfinite(sqrt_s))
    return fail(MEA_E_ARG, "mea_partonic_cross_section: bad arguments");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_partonic_cross_section: host-only process handle");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED) return fail(MEA_E_ARG, "mea_partonic_cross_section: bad precision");
  const mea::Program& G = P->prog;
  const int n_ext = G.n_ext, nf = n_ext - 2;
  if (cuts->n_final != nf) return fail(MEA_E_ARG, "mea_partonic_cross_section: cuts->n_final != n_ext - 2");
  // Phi_n(s) = (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!), symmetry 1/prod k!
  const double s_hat = sqrt_s * sqrt_s;
  double fact_n1 = 1.0, fact_n2 = 1.0;
  for (int k = 2; k <= nf - 1; ++k) fact_n1 *= k;
  for (int k = 2; k <= nf - 2; ++k) fact_n2 *= k;
  const double phi = std::pow(2.0 * M_PI, 4.0 - 3.0 * nf) * std::pow(M_PI / 2.0, nf - 1) * std::pow(s_hat, nf - 2) /
                     (fact_n1 * fact_n2);
  std::map<int, int> count;
  for (int l = 2; l < n_ext; ++l) count[G.pdg[l]]++;
  double sym = 1.0;
  for (auto& kv : count)
    for (int k = 2; k <= kv.second; ++k) sym /= k;
  const int64_t chunk = std::min<int64_t>(n, 1 << 20);
  constexpr int kBlocks = 256;
  mea::DevBuf mom, me2, att, pf, pf2, pa;
  const ScopedBufs held{&mom, &me2, &att, &pf, &pf2, &pa};
  MEA_CUDA(mom.ensure(sizeof(double) * 4 * n_ext * chunk));
  MEA_CUDA(me2.ensure(sizeof(double) * chunk));
  MEA_CUDA(att.ensure(sizeof(int32_t) * chunk));
  MEA_CUDA(pf.ensure(sizeof(double) * kBlocks));
  MEA_CUDA(pf2.ensure(sizeof(double) * kBlocks));
  MEA_CUDA(pa.ensure(sizeof(long long) * 2 * kBlocks));
  cudaStream_t s;
  MEA_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  mea::PsConfigDev c{cuts->seed, nf, sqrt_s, sqrt_s, cuts->pt_min, cuts->eta_max, cuts->dr_min, cuts->ptij_min};
  double sum_f = 0.0, sum_f2 = 0.0;
  long long drawn = 0, accepted = 0;
  std::vector<double> hf(kBlocks), hf2(kBlocks);
  std::vector<long long> ha(2 * kBlocks);
  mea_status st = MEA_OK;
  {
    std::lock_guard<std::mutex> lk(P->mu);
    for (int64_t c0 = 0; c0 < n && st == MEA_OK; c0 += chunk) {
      const int64_t cn = std::min(chunk, n - c0);
      cudaError_t e = mea::launch_phase_space(c, first_event + (uint64_t)c0, cn, reinterpret_cast<double*>(mom.p),
                                              reinterpret_cast<int32_t*>(att.p), s);
      if (e != cudaSuccess) { st = fail(MEA_E_CUDA, cudaGetErrorString(e)); break; }
      st = do_evaluate(P, P->scr[0], reinterpret_cast<const double*>(mom.p), cn, MEA_HEL_SUM_NONZERO, nullptr, prec,
                       reinterpret_cast<double*>(me2.p), nullptr, s);
      if (st != MEA_OK) break;
      e = mea::launch_xsec_sums(reinterpret_cast<const double*>(me2.p), reinterpret_cast<const int32_t*>(att.p), cn,
                                reinterpret_cast<double*>(pf.p), reinterpret_cast<double*>(pf2.p),
                                reinterpret_cast<long long*>(pa.p), kBlocks, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hf.data(), pf.p, sizeof(double) * kBlocks, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hf2.data(), pf2.p, sizeof(double) * kBlocks, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), pa.p, sizeof(long long) * 2 * kBlocks, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { st = fail(MEA_E_CUDA, cudaGetErrorString(e)); break; }
      for (int b = 0; b < kBlocks; ++b) {
        sum_f += hf[b];
        sum_f2 += hf2[b];
        drawn += ha[2 * b];
        accepted += ha[2 * b + 1];
      }
    }
  }
  cudaStreamDestroy(s);
  if (st != MEA_OK) return st;
  const double pre = sym * phi / (2.0 * s_hat) * 0.3893794e9;
  const double mean = sum_f / (double)drawn;
  const double var = std::max(0.0, sum_f2 / (double)drawn - mean * mean);
  out->sigma_pb = pre * mean;
  out->error_pb = pre * std::sqrt(var / (double)drawn);
  out->n_accepted = accepted;
  out->n_drawn = drawn;
  out->phase_space = phi;
  out->symmetry = sym;
  return MEA_OK;
}

}  // extern "C"

namespace {
// One VEGAS grid refinement of one dimension (Lepage 1978): d[i] is the sum
// of (weight f)^2 over the iteration's points in interval i; the sums are
// smoothed over neighbours, compressed to r_i = ((1 - x_i) / ln(1 / x_i))^alpha
// with x_i the smoothed share, and the new edges give every interval an equal
// share of sum r, each old interval's r spread uniformly over its width.
void vegas_refine(std::vector<double>& e, const std::vector<double>& d, double alpha) {
  const int nb = (int)d.size();
  if (nb < 2) return;
  std::vector<double> ds(nb);
  ds[0] = 0.5 * (d[0] + d[1]);
  ds[nb - 1] = 0.5 * (d[nb - 2] + d[nb - 1]);
  for (int i = 1; i < nb - 1; ++i) ds[i] = (d[i - 1] + d[i] + d[i + 1]) / 3.0;
  double D = 0.0;
  for (double v : ds) D += v;
  if (!(D > 0.0)) return;
  std::vector<double> r(nb);
  double R = 0.0;
  for (int i = 0; i < nb; ++i) {
    const double x = ds[i] / D;
    r[i] = (x > 0.0) ? (x < 1.0 ? std::pow((1.0 - x) / -std::log(x), alpha) : 1.0) : 0.0;
    R += r[i];
  }
  if (!(R > 0.0)) return;
  std::vector<double> ne(nb + 1);
  ne[0] = 0.0;
  ne[nb] = 1.0;
  double acc = 0.0;
  int i = 0;
  for (int j = 1; j < nb; ++j) {
    const double need = R * (double)j / (double)nb;
    while (i < nb - 1 && acc + r[i] < need) acc += r[i++];
    const double frac = r[i] > 0.0 ? std::min(1.0, std::max(0.0, (need - acc) / r[i])) : 0.0;
    ne[j] = e[i] + frac * (e[i + 1] - e[i]);
  }
  e = ne;
}
}  // namespace

extern "C" {

mea_status mea_partonic_cross_section_vegas(mea_process_t P, double sqrt_s, const mea_ps_config* cuts,
                                            uint64_t first_event, const mea_vegas_config* vc, mea_prec_mode prec,
                                            mea_vegas_result* out) {
  if (!P || !cuts || !vc || !out || !(sqrt_s > 0) || !std::isfinite(sqrt_s))
    return fail(MEA_E_ARG, "mea_partonic_cross_section_vegas: bad arguments");
  if (vc->iterations < 1 || vc->points_per_iteration < 2 || vc->bins < 1 || vc->bins > PS_VEGAS_MAX_BINS ||
      !(vc->alpha >= 0.0))
    return fail(MEA_E_ARG, "mea_partonic_cross_section_vegas: bad VEGAS configuration");
  if (P->host_only) return fail(MEA_E_UNSUPPORTED, "mea_partonic_cross_section_vegas: host-only process handle");
  if (prec != MEA_PREC_FP64 && prec != MEA_PREC_MIXED)
    return fail(MEA_E_ARG, "mea_partonic_cross_section_vegas: bad precision");
  const mea::Program& G = P->prog;
  const int n_ext = G.n_ext, nf = n_ext - 2;
  if (cuts->n_final != nf) return fail(MEA_E_ARG, "mea_partonic_cross_section_vegas: cuts->n_final != n_ext - 2");
  const double s_hat = sqrt_s * sqrt_s;
  double fact_n1 = 1.0, fact_n2 = 1.0;
  for (int k = 2; k <= nf - 1; ++k) fact_n1 *= k;
  for (int k = 2; k <= nf - 2; ++k) fact_n2 *= k;
  const double phi = std::pow(2.0 * M_PI, 4.0 - 3.0 * nf) * std::pow(M_PI / 2.0, nf - 1) * std::pow(s_hat, nf - 2) /
                     (fact_n1 * fact_n2);
  std::map<int, int> count;
  for (int l = 2; l < n_ext; ++l) count[G.pdg[l]]++;
  double sym = 1.0;
  for (auto& kv : count)
    for (int k = 2; k <= kv.second; ++k) sym /= k;
  const double pre = sym * phi / (2.0 * s_hat) * 0.3893794e9;
  const int nb = vc->bins, dims = ps_rambo_dims(nf);
  const int64_t N = vc->points_per_iteration;
  const int64_t chunk = std::min<int64_t>(N, 1 << 20);
  mea::DevBuf mom, me2, wgt, bins, edges_d;
  const ScopedBufs held{&mom, &me2, &wgt, &bins, &edges_d};
  MEA_CUDA(mom.ensure(sizeof(double) * 4 * n_ext * chunk));
  MEA_CUDA(me2.ensure(sizeof(double) * chunk));
  MEA_CUDA(wgt.ensure(sizeof(double) * chunk));
  MEA_CUDA(bins.ensure((size_t)dims * chunk));
  MEA_CUDA(edges_d.ensure(sizeof(double) * dims * (nb + 1)));
  std::vector<double> edges((size_t)dims * (nb + 1));
  for (int d = 0; d < dims; ++d)
    for (int b = 0; b <= nb; ++b) edges[(size_t)d * (nb + 1) + b] = (double)b / nb;
  std::vector<double> hw(chunk), hm(chunk);
  std::vector<unsigned char> hb((size_t)dims * chunk);
  mea::PsConfigDev c{cuts->seed, nf, sqrt_s, sqrt_s, cuts->pt_min, cuts->eta_max, cuts->dr_min, cuts->ptij_min};
  cudaStream_t s;
  MEA_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double sum_w = 0.0, sum_wi = 0.0, sum_chi = 0.0;
  std::vector<double> Ik, Vk;
  int64_t accepted = 0;
  mea_status st = MEA_OK;
  {
    std::lock_guard<std::mutex> lk(P->mu);
    for (int k = 0; k < vc->iterations && st == MEA_OK; ++k) {
      std::vector<double> dsum((size_t)dims * nb, 0.0);
      double f1 = 0.0, f2 = 0.0;
      cudaError_t e = cudaMemcpyAsync(edges_d.p, edges.data(), sizeof(double) * edges.size(), cudaMemcpyHostToDevice, s);
      for (int64_t c0 = 0; c0 < N && st == MEA_OK; c0 += chunk) {
        const int64_t cn = std::min(chunk, N - c0);
        const uint64_t ev0 = first_event + (uint64_t)k * (uint64_t)N + (uint64_t)c0;
        if (e == cudaSuccess)
          e = mea::launch_vegas_points(c, reinterpret_cast<const double*>(edges_d.p), nb, ev0, cn,
                                       reinterpret_cast<double*>(mom.p), reinterpret_cast<double*>(wgt.p),
                                       reinterpret_cast<unsigned char*>(bins.p), s);
        if (e != cudaSuccess) { st = fail(MEA_E_CUDA, cudaGetErrorString(e)); break; }
        st = do_evaluate(P, P->scr[0], reinterpret_cast<const double*>(mom.p), cn, MEA_HEL_SUM_NONZERO, nullptr, prec,
                         reinterpret_cast<double*>(me2.p), nullptr, s);
        if (st != MEA_OK) break;
        e = cudaMemcpyAsync(hw.data(), wgt.p, sizeof(double) * cn, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), me2.p, sizeof(double) * cn, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), bins.p, (size_t)dims * cn, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = fail(MEA_E_CUDA, cudaGetErrorString(e)); break; }
        // host sums in event order (reproducible)
        for (int64_t i = 0; i < cn; ++i) {
          const double f = hw[i] > 0.0 ? hw[i] * hm[i] : 0.0;
          if (hw[i] > 0.0) ++accepted;
          f1 += f;
          f2 += f * f;
          for (int d = 0; d < dims; ++d) dsum[(size_t)d * nb + hb[(size_t)i * dims + d]] += f * f;
        }
      }
      if (st != MEA_OK) break;
      const double mean = f1 / (double)N;
      const double var = std::max(0.0, (f2 / (double)N - mean * mean) / (double)(N - 1));
      Ik.push_back(pre * mean);
      Vk.push_back(pre * pre * var);
      if (k + 1 < vc->iterations)
        for (int d = 0; d < dims; ++d) {
          std::vector<double> ed(edges.begin() + (size_t)d * (nb + 1), edges.begin() + (size_t)(d + 1) * (nb + 1));
          std::vector<double> dd(dsum.begin() + (size_t)d * nb, dsum.begin() + (size_t)(d + 1) * nb);
          vegas_refine(ed, dd, vc->alpha);
          std::copy(ed.begin(), ed.end(), edges.begin() + (size_t)d * (nb + 1));
        }
    }
  }
  cudaStreamDestroy(s);
  if (st != MEA_OK) return st;
  for (size_t k = 0; k < Ik.size(); ++k) {
    const double wk = Vk[k] > 0.0 ? 1.0 / Vk[k] : 0.0;
    sum_w += wk;
    sum_wi += wk * Ik[k];
  }
  const double I = sum_w > 0.0 ? sum_wi / sum_w : Ik.back();
  for (size_t k = 0; k < Ik.size(); ++k)
    if (Vk[k] > 0.0) sum_chi += (Ik[k] - I) * (Ik[k] - I) / Vk[k];
  out->sigma_pb = I;
  out->error_pb = sum_w > 0.0 ? 1.0 / std::sqrt(sum_w) : 0.0;
  out->chi2_per_dof = Ik.size() > 1 ? sum_chi / (double)(Ik.size() - 1) : 0.0;
  out->last_sigma_pb = Ik.back();
  out->last_error_pb = std::sqrt(Vk.back());
  out->n_points = (int64_t)vc->iterations * N;
  out->n_accepted = accepted;
  return MEA_OK;
}

}  // extern "C"


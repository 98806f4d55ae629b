// Internal definitions shared by the C ABI translation units (api.cu,
// batch.cu, server.cu): the process handle and the evaluation driver.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mea.h"
#include "generator.h"
#include "helshare.h"
#include "jamp_gemm.h"
#include "kernels.h"

namespace mea {

// Growable device buffer (cudaMalloc on growth only).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  cudaError_t ensure(size_t b) {
    if (b <= bytes) return cudaSuccess;
    release();
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    return e;
  }
};


// Scratch of one in-flight evaluation.  Evaluations that may overlap on the
// GPU (different streams, graph branches, server slots) use distinct sets.
struct EvalScratch {
  DevBuf s32, s64, flag_list, flag_count, jbuf, pairval, pairk, abuf, rowmax, jabs, evf;
  void release() {
    s32.release(); s64.release(); flag_list.release(); flag_count.release();
    jbuf.release(); pairval.release(); pairk.release(); abuf.release(); rowmax.release(); jabs.release();
    evf.release();
  }
};

mea_status set_error(mea_status s, const std::string& msg);

}  // namespace mea

struct mea_process_s {
  mea::Program prog;
  mea::HsProgram hs;  // helicity-shared layout of prog (valid when hs_ok)
  bool hs_ok = false;
  mea::HsSplitProgram hsp;  // split layout of prog (valid when hsp_ok)
  bool hsp_ok = false;
  mea::DevProgram dev;
  mea_options opts;
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0, smem_per_sm = 0;
  std::vector<void*> owned;
  std::mutex mu;
  // scratch sets: 0 for mea_evaluate, 1 and 2 for the two host-pipeline streams
  mea::EvalScratch scr[3];
  // configurations chosen by mea_autotune, per precision (0 mixed, 1 FP64), or grid 0
  mea::AmpConfig tuned[2];
  int tuned_H[2] = {0, 0};
  bool auto_tuned[2] = {false, false};  // tuned once already (explicitly or on first large evaluation)
  // heuristic launch plans, computed once per (FP64?, tensor path?, H) with an
  // unbounded event count; each call only caps the grid by its tiles
  std::map<std::tuple<bool, bool, int>, mea::AmpConfig> plan_cache;
  std::mutex plan_mu;
  // status word of the bounded device waits
  const __half* cf_hi = nullptr;   // colour matrix operand tiles (colour_gemm.h ColourTiles)
  const __half* cf_lo = nullptr;
  int cf_nc = 0, cf_np = 0, cf_kp = 0;
  int* status = nullptr;
  // diagram -> colour-amplitude map for the tensor-core colour-amplitude stage
  mea::JampMap jmap;                  // host description (tiles released after upload)
  const __half* jmap_tiles = nullptr;  // device copy of the coefficient tiles
  // host-buffer pipeline
  void* pin_in[2] = {nullptr, nullptr};
  void* pin_out[2] = {nullptr, nullptr};
  void* pin_flags[2] = {nullptr, nullptr};
  mea::DevBuf d_in[2], d_out[2], d_flags[2];
  cudaStream_t st[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  int64_t pipe_chunk = 0;
  bool host_only = false;
  // stage timing (mea_set_stage_timing): a pair of CUDA events recorded on the
  // evaluation's stream around every kernel launch, resolved by mea_get_stage_times
  bool stage_timing = false;
  std::mutex st_mu;
  std::vector<cudaEvent_t> st_events;  // pool: 2 per recorded launch
  std::vector<int> st_stage;           // stage of each recorded pair
  size_t st_used = 0;                  // pairs recorded since the last query
};

namespace mea {
// Enqueue one evaluation on stream s using scratch set S (see api.cu).
mea_status evaluate_with(mea_process_s* P, EvalScratch& S, const double* mom, int64_t n, mea_hel_mode hm,
                         const int8_t* hel, mea_prec_mode prec, double* me2, uint8_t* flags, cudaStream_t s);
// True when evaluations of this precision / helicity mode run the tensor-core
// path (amplitude-output interpreter + colour-amplitude and colour GEMMs).
bool uses_tensor_path(const mea_process_s* P, mea_prec_mode prec, mea_hel_mode hm);
// Events per chunk the tensor-core path launches for an evaluation of n events.
int64_t tensor_chunk_events(const mea_process_s* P, int H, int64_t n);
// mea_autotune with the process lock already held.
mea_status autotune_locked(mea_process_s* P, const double* mom, int64_t n, mea_prec_mode prec, double* me2,
                           mea_tune_result* out);
// Heuristic launch plan of this process for n events (cached per precision,
// path and helicity count); dp is P->dev or its tensor-path copy.
AmpConfig cached_plan(mea_process_s* P, const DevProgram& dp, bool fp64, bool tc, int H, int64_t n);
// Device scratch bytes an evaluation of n events would hold (admission control).
size_t scratch_estimate(mea_process_s* P, int64_t n, mea_prec_mode prec);
}  // namespace mea

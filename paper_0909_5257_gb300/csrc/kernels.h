// Host-side declarations of the CUDA kernels' launch helpers.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "generator.h"

namespace mea {

struct DevProgram;
struct AmpConfig;
struct AmpLaunch;
struct HsOp;

// A straight-line per-process kernel emitted by codegen.cpp at build time.
struct GenEntry {
  const char* key;  // PDG codes joined by commas
  // regvar: variant of the FP32 kernel, 2 * cap + body -- cap 0 / 1 / 2 =
  // 128 / 85 / 168 registers per thread, body 0 with vertex partials, 1 with
  // one vertex call per diagram; the FP64 kernel has one variant (partials, 128)
  void (*launch)(bool fp64, int regvar, const DevProgram&, const AmpConfig&, const AmpLaunch&, cudaStream_t);
  const void* (*kernel)(bool fp64, int regvar);
};
constexpr int kGenCaps = 3;
constexpr int kGenRegVariants = 2 * kGenCaps;
constexpr int kGenCapRegisters[kGenCaps] = {128, 85, 168};
const GenEntry* generated_table(int* n);
const GenEntry* find_generated(const int* pdg, int n_ext);

// Device copy of a process program (all pointers are device memory).
struct DevProgram {
  const Op* ops = nullptr;
  int n_ops = 0;
  const ColEntry* col = nullptr;
  const uint32_t* masks = nullptr;
  int n_masks = 0;
  const int8_t* leg_info = nullptr;   // [n_ext][4]: type, spinor kind, incoming, pad
  int n_ext = 0;
  int n_slots = 0;
  int n_colour = 0;
  const float* cf_f = nullptr;        // K as float [m*m]
  const double* cf_d = nullptr;       // K as double [m*m]
  double cf_inv_den = 0;              // 1 / D
  const int8_t* hel = nullptr;        // [n_hel][n_ext] helicities summed in MEA_HEL_SUM_NONZERO
  int n_hel = 0;
  const int8_t* hel_all = nullptr;    // [2^n_ext][n_ext]
  double g = 0;                       // g_s
  const GenEntry* gen = nullptr;      // straight-line kernel of this process, if emitted
  int gen_forced = -1;                // FP32 variant pinned by mea_options.kernel_variant (-1: free)
  const float* amp_w = nullptr;       // [n_diagrams] sum_alpha |c_alpha d| (amplitude-output mode)
  const HsOp* hs = nullptr;           // helicity-shared layout of the program (helshare.h), or null
  int hs_arena = 0;                   // its variants per event
  bool hs_only = false;               // amplitude-output mode: plan and tune the helicity-shared kernel only
  // split evaluation (helshare.h build_split_shared), or null
  const uint32_t* hsp_tasks = nullptr;  // prologue tasks, level by level
  int hsp_level_end[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int hsp_levels = 0;
  const HsOp* hsp_rec = nullptr;        // [n_ops] records of the whole program
  const Op* hsp_main_ops = nullptr;     // the per-lane ops
  const HsOp* hsp_main_rec = nullptr;
  int hsp_n_main = 0;
  int hsp_area = 0;                     // prologue variants per event
  bool hsp_only = false;                // amplitude-output mode: plan and tune the split kernel only
  // per op: bits 0..3 input k is the previous op's output, bit 4 the op's
  // output is read only by the next op (amplitude-output interpreter with
  // register forwarding), or null
  const uint8_t* fwd = nullptr;
  bool fwd_only = false;                // amplitude-output interpreter: plan and tune with forwarding only
};

struct AmpLaunch {
  const double* mom = nullptr;        // [n_events][n_ext][4]
  int64_t n_events = 0;
  const int32_t* event_list = nullptr;  // optional: evaluate mom[event_list[i]] for i < *list_count
  const int32_t* list_count = nullptr;  // device count for event_list mode
  const int8_t* hel_given = nullptr;  // [n_events][n_ext] for one given helicity per event
  int hel_mode = 0;                   // 0 nonzero set, 1 all 2^n, 2 given
  double* me2 = nullptr;
  uint8_t* flags = nullptr;
  float flag_threshold = 1e-5f;
  int write_flags_mode = 0;           // 0: write flags; 1: OR in MEA_FLAG_REEVALUATED (re-evaluation)
  int32_t* flag_list = nullptr;       // mixed path: indices of flagged events are appended here
  int32_t* flag_count = nullptr;
  float* pair_kappa = nullptr;        // per-pair indicator (see amp_out)
  uint8_t* ev_flags = nullptr;        // amplitude-output mode: per-event input-check bits out;
                                      //   finish_kernel ORs them into the flags
  float* amp_out = nullptr;           // amplitude-output mode: A[d][lda], (Re, Im) of pair p at 2p, 2p+1;
  int64_t lda = 0;                    //   pair_kappa then receives sum_d w_d |A_d| and
  float* amp_rowmax = nullptr;        //   amp_rowmax[2p], [2p+1] the row maxima of |Re A|, |Im A|
  float* jamp_scratch = nullptr;      // global colour-amplitude accumulators when not in SMEM
  float* slot_scratch = nullptr;      // global wavefunction slots when not in SMEM
};

struct AmpConfig {
  int H = 1;           // helicity lanes per event
  int E_cta = 1;       // events per tile
  int threads = 32;
  int grid = 1;
  size_t smem = 0;
  bool jamp_in_smem = true;
  bool slots_in_smem = true;
  int regvar = 0;  // straight-line kernels: variant, 2 * cap + body (see GenEntry)
  int per_sm = 1;  // CTAs meant to be resident per SM (sets the shared-memory carveout)
  bool fwd = false;       // amplitude-output interpreter: the previous op's output forwarded in registers
  bool hsplit = false;    // amplitude-output mode: the split kernel (amp_hsp_kernel, amp_hs_kernel.cu):
                          // E_cta events x H lanes; slots_in_smem = its prologue area in shared memory
  bool helshare = false;  // amplitude-output mode: the helicity-shared kernel (amp_hs_kernel.cu):
                          // one warp per event, E_cta = warps per CTA, regvar its register
                          // variant (0: 64 registers, 1: uncapped)
};

// Shared-memory carveout (percent of the SM's unified L1/shared storage) that
// holds per_sm CTAs of smem bytes each and leaves the rest as L1: the
// straight-line kernels spill and the interpreter keeps wavefunction slots in
// global memory, both of which live in L1.
int carveout_percent(const AmpConfig& c);

// Choose tile shape and grid for a program, precision and helicity mode.
AmpConfig plan_amp(const DevProgram& p, bool fp64, int H, int64_t n_events, int num_sms,
                   size_t max_smem_per_block, size_t smem_per_sm, int events_per_tile_hint = 0);

// Every distinct tile shape / placement worth timing (autotuner).
std::vector<AmpConfig> candidate_configs(const DevProgram& p, bool fp64, int H, int64_t n_events, int num_sms,
                                         size_t max_smem, size_t smem_per_sm);

size_t jamp_scratch_bytes_needed(const DevProgram& p, bool fp64, const AmpConfig& c);
size_t slot_scratch_bytes_needed(const DevProgram& p, bool fp64, const AmpConfig& c);

cudaError_t launch_amp(const DevProgram& p, bool fp64, const AmpConfig& c, const AmpLaunch& a,
                       cudaStream_t s);

// Helicity-shared amplitude kernel (amp_hs_kernel.cu): amplitude-output mode,
// FP32, helicity sums of up to 128 combinations, processes of up to 7 legs.
bool hs_supported(const DevProgram& p, bool fp64, int H);
size_t hs_smem_bytes(const DevProgram& p, int warps);  // dynamic shared memory of a CTA
size_t hs_arena_bytes(const DevProgram& p, const AmpConfig& c);  // global variant arena of a launch
std::vector<AmpConfig> hs_candidates(const DevProgram& p, int H, int num_sms, size_t max_smem, size_t smem_per_sm);
AmpConfig hs_plan(const DevProgram& p, int H, int num_sms, size_t max_smem, size_t smem_per_sm);  // grid 0: none
cudaError_t launch_amp_hs(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s);
// Split kernel: prologue of shared short wavefunctions, the rest per lane.
bool hsp_supported(const DevProgram& p, bool fp64, int H);
size_t hsp_smem_bytes(const DevProgram& p, int events, bool area_in_smem);
size_t hsp_area_bytes(const DevProgram& p, const AmpConfig& c);
std::vector<AmpConfig> hsp_candidates(const DevProgram& p, int H, int num_sms, size_t max_smem, size_t smem_per_sm);
cudaError_t launch_amp_hsp(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s);

// Helicity sum + flags for the split colour stage: me2 = 1/4 sum_h pairval.
// With jabs ([n_splits][n_events*H] sums of |J|), pair_kappa holds sum |c A|
// and the per-pair indicator is pair_kappa / sum_splits jabs.
cudaError_t launch_finish(const AmpLaunch& a, int H, const double* pairval, const float* pair_kappa,
                          cudaStream_t s, const float* jabs = nullptr, int n_splits = 0);

// Phase-space generator kernel (input generator).
struct PsConfigDev {
  uint64_t seed;
  int n_final;
  double rs_lo, rs_hi, pt_min, eta_max, dr_min, ptij_min;
};
cudaError_t launch_phase_space(const PsConfigDev& cfg, uint64_t first_event, int64_t n,
                               double* mom, int32_t* attempts, cudaStream_t s);
// VEGAS points at fixed sqrt(s_hat) = cfg.rs_lo (edges: device [dims][nb + 1]).
cudaError_t launch_vegas_points(const PsConfigDev& cfg, const double* edges, int nb, uint64_t first_event,
                                int64_t n, double* mom, double* weight, unsigned char* bins, cudaStream_t s);
// Per-block sums for the partonic cross section (blocks x 256 threads);
// part_a[2b], part_a[2b+1] = points drawn, points accepted.
cudaError_t launch_xsec_sums(const double* me2, const int32_t* att, int64_t n, double* part_f, double* part_f2,
                             long long* part_a, int blocks, cudaStream_t s);

uint64_t& launch_counter();

// Raise the largest dynamic shared memory a kernel may be launched with to at
// least `bytes` (never lowers it).  Serialised across host threads: a launch
// on one thread must not see another thread's smaller setting between its own
// setting and its launch.
cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes);

}  // namespace mea

/*
 * mea.h -- C ABI of the GB300 tree-level QCD matrix-element library
 * (libmea.so).  "mea" = matrix-element amplitudes.
 *
 * What the library computes (arXiv:0909.5257, Sec. 2.1):
 *   for every event, the helicity-summed, colour-summed tree-level squared
 *   matrix element averaged over the initial helicities and colours,
 *     me2 = 1/4 sum_lambda sum_{alpha,beta} J_alpha N_{alpha beta} J_beta^*,
 *   with J_alpha the colour amplitudes of Eq. (color-amplitude), built from the
 *   Feynman-diagram sum of Eq. (matrix-element) with HELAS-style wavefunction,
 *   vertex and off-shell-current functions (Sec. 4), and N the colour matrix of
 *   Eq. (color-matrix) (which already holds 1/(n_a n_b)).  No identical-
 *   particle factor and no flux factor are applied (they belong on the phase
 *   space, Sec. 2.1).
 *
 * Supported processes: massless QCD with gluons (PDG 21) and light quarks
 * (PDG 1..5, antiquarks negative), at most two quark lines, 4 <= n_ext <= 7,
 * e.g. g g -> n g, u u~ -> n g, u u -> u u + n g.
 *
 * Conventions.
 *   - Momenta: double[n_events][n_ext][4] = (E, px, py, pz) in GeV, legs ordered
 *     (incoming a, incoming b, outgoing 1..n).  Partons are massless.
 *   - Helicities are physical helicities +-1 of each parton.
 *   - Every entry point is host-callable and thread-safe for distinct handles.
 *     Device pointers are CUDA device memory of the current device; "stream"
 *     is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Work on device buffers is stream-ordered and asynchronous: a call returns
 *     after enqueueing; results are valid once the stream reaches that point.
 *   - Ownership: the caller owns every buffer it passes; the library owns the
 *     process tables, colour matrices and its scratch memory (per process
 *     handle) and frees them in mea_destroy_process.
 *   - Errors: every call returns a mea_status; nothing is thrown across the ABI.
 *     On failure mea_last_error() gives a thread-local message.  A CUDA launch or
 *     runtime failure maps to MEA_E_CUDA.  Invalid arguments are detected on the
 *     host before anything is enqueued (MEA_E_ARG).
 */
#ifndef MEA_H
#define MEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mea_process_s *mea_process_t;

typedef enum {
  MEA_OK = 0,
  MEA_E_ARG = -1,          /* invalid argument */
  MEA_E_UNSUPPORTED = -2,  /* process or mode outside what the library covers */
  MEA_E_NOMEM = -3,        /* host or device allocation failed */
  MEA_E_CUDA = -4,         /* CUDA runtime error */
  MEA_E_TIMEOUT = -5,      /* a bounded wait expired */
  MEA_E_REJECTED = -6      /* admission control refused the request */
} mea_status;

/* Which helicity combinations are summed. */
typedef enum {
  MEA_HEL_SUM_NONZERO = 0, /* only those allowed by the massless helicity
                              selection rules (the others vanish identically) */
  MEA_HEL_SUM_ALL = 1,     /* all 2^n_ext combinations */
  MEA_HEL_GIVEN = 2        /* one combination per event, given in hel_dev
                              (int8 [n_events][n_ext], entries +1/-1); the
                              result is that combination's colour-summed,
                              colour-averaged |M|^2 times 1/4 (the paper's
                              sampled-helicity mode, Sec. 3.2 step 2) */
} mea_hel_mode;

/* Arithmetic of the amplitude and colour stages. */
typedef enum {
  MEA_PREC_FP64 = 0,   /* everything in FP64 */
  MEA_PREC_MIXED = 1   /* FP32 amplitudes with compensated (two-sum) colour-
                          amplitude accumulation; colour sum on the tensor
                          cores (FP16 hi/lo split of J against the exact
                          integer colour matrix, FP32 accumulate) or on FP32
                          CUDA cores for small colour bases; events whose
                          error indicator exceeds flag_threshold are
                          re-evaluated in FP64 when reeval_fp64 != 0 */
} mea_prec_mode;

typedef struct {
  double alpha_s;        /* strong coupling, g = sqrt(4 pi alpha_s); <= 0 -> 0.118 */
  double flag_threshold; /* relative error indicator above which an event is
                            flagged in MEA_PREC_MIXED; <= 0 -> 1e-5.  The
                            indicator is u (32 + kappa), u = 2^-24 the FP32
                            roundoff and kappa the cancellation sum |c A| /
                            sum |J| of the colour-amplitude sum averaged over
                            the helicities with their |M_h|^2; it bounds the
                            measured relative error of the mixed result for
                            >= 99 % of the events */
  int reeval_fp64;       /* 1: re-evaluate flagged events in FP64 (default) */
  int colour_mode;       /* 0 auto, 1 CUDA-core colour sum, 2 tensor-core GEMM */
  int64_t chunk_events;  /* tensor-core path: events per chunk (bounds its device
                            scratch, ~8 bytes per diagram per helicity per event);
                            <= 0 -> automatic (enough lanes to fill the GPU) */
  int auto_tune;         /* 1 (default): the first mea_evaluate of >= 65536 events per
                            precision with MEA_HEL_SUM_NONZERO, outside stream capture,
                            synchronises its stream and runs mea_autotune on its first
                            65536 events (up to 2^20 for the straight-line FP32 kernels
                            of processes with up to five partons; me2 as scratch)
                            before evaluating; 0: off */
  int kernel_variant;    /* straight-line kernels (processes with up to five partons),
                            MEA_PREC_MIXED: 0 (default) the tuned or heuristic variant;
                            1..6 pin one (planning and tuning then use only it):
                            1 / 2 at 128 registers per thread, 3 / 4 at 85, 5 / 6 at
                            168, the odd ones the body with shared vertex partials, the
                            even ones the body with one vertex call per diagram (pins
                            the rounding order for reproducible results); other
                            values -> MEA_E_ARG */
  int helicity_sharing;  /* amplitude stage of the tensor-core path (MEA_PREC_MIXED,
                            helicity sums): 0 (default) the autotuner chooses
                            (untuned: the per-lane interpreter) among the per-lane
                            interpreter (one
                            lane per event and helicity combination), the
                            helicity-shared kernel (one warp per event; every
                            off-shell current evaluated once per helicity pattern
                            of its own legs instead of once per combination) and
                            the split kernel (the currents of up to n_ext - 3
                            legs shared that way in a prologue, the rest per
                            lane); all three apply the same operations to the
                            same inputs (bit-identical results); the per-lane
                            interpreter is tuned with and without forwarding each
                            op's output to the next op in registers; 1 per-lane
                            interpreter only; 2 helicity-shared kernel only; 3
                            split kernel only; 4 per-lane interpreter with
                            forwarding only; other values -> MEA_E_ARG */
} mea_options;

/* Per-event flag bits written to flags_dev.  An event re-evaluated in FP64
 * keeps the bits that sent it there (MEA_FLAG_CANCEL, MEA_FLAG_QGUARD) and
 * gains MEA_FLAG_REEVALUATED; MEA_FLAG_NONFINITE then describes the FP64
 * result. */
#define MEA_FLAG_REEVALUATED 0x01u  /* result comes from the FP64 re-evaluation */
#define MEA_FLAG_NONFINITE   0x02u  /* a non-finite value was met */
#define MEA_FLAG_CANCEL      0x04u  /* error indicator of the mixed path above flag_threshold */
#define MEA_FLAG_QGUARD      0x08u  /* a propagator invariant |q^2| is below 1e-10 of the
                                       squared energy flowing through it (near-singular
                                       kinematics; re-evaluated in FP64 on the mixed path) */
#define MEA_FLAG_MOMENTUM    0x10u  /* momentum conservation violated by more than
                                       1e-9 sqrt(s) in some component (input check) */

typedef struct {
  int n_ext;              /* external partons */
  int n_diagrams;         /* Feynman diagrams (a gggg vertex counts three times,
                             once per colour structure, as in Table 1) */
  int n_colour;           /* colour basis vectors (Table 1) */
  int n_hel_nonzero;      /* helicity combinations kept by the selection rules */
  int n_currents;         /* off-shell currents in the shared current graph */
  int n_ops;              /* operations in the per-(event,helicity) program */
  int n_slots;            /* wavefunction slots the program needs at once */
  int n_colour_amplitudes;  /* colour amplitudes the kernels accumulate: n_colour,
                              or n_colour/2 for pure-gluon processes (reflection
                              identity J_rev(a) = (-1)^n J_a, folded colour matrix) */
  int64_t cf_denominator; /* N = K / cf_denominator with K integer */
  int64_t cf_max_abs_numerator; /* max |K| */
  double flops_per_hel;   /* algorithmic FLOPs of the amplitude stage per
                             (event, helicity): wavefunctions, vertices (with
                             the shared vertex partials), currents and
                             colour-amplitude accumulation */
  double colour_flops_per_hel; /* 4 n_colour_amplitudes^2: FLOPs of the colour quadratic form */
  double flops_per_hel_plain;  /* flops_per_hel when every diagram amplitude is its own
                                  vertex call (no shared vertex partials) */
  int64_t n_colour_entries;    /* non-zero diagram -> colour-amplitude coefficients c_{alpha d}
                                  of Eq. (color-amplitude) over the accumulated colour
                                  amplitudes; flops_per_hel holds 4 FLOPs for each */
  int64_t hs_variants;         /* helicity-shared evaluation, per event: wavefunction
                                  variants evaluated (each produced wavefunction once per
                                  helicity pattern of its legs); 0 when not available */
  int hs_arena_variants;       /* its work space per event, in 32-byte FP32 wavefunctions */
  double hs_flops_per_event;   /* its FLOPs per event for the non-zero helicity sum:
                                  variants and n_hel_nonzero x diagram amplitudes, each at
                                  its operation's cost (no colour entries) */
  int hsp_area_variants;       /* split evaluation: prologue variants per event (the
                                  wavefunctions of up to n_ext - 3 legs); 0 when not available */
  double hsp_flops_per_event;  /* its FLOPs per event: the prologue variants and
                                  n_hel_nonzero x the per-lane ops, each at its cost */
} mea_process_info_t;

/* ---- process handles ---------------------------------------------------- */

/* Build the process g(pdg[0]) g(pdg[1]) -> pdg[2..n_ext-1]: enumerate its tree
 * diagrams (Sec. 2.1, Table 1), build the shared off-shell-current program,
 * the colour decomposition onto the Table 1 basis and the exact colour matrix
 * of Eq. (color-matrix); upload everything to the current device.
 * opts may be NULL (defaults).  *out receives the handle. */
mea_status mea_create_process(const int *pdg, int n_ext, const mea_options *opts,
                              mea_process_t *out);

/* Same as mea_create_process but builds the host-side tables only and touches
 * no GPU: the handle answers mea_process_info, mea_colour_matrix and
 * mea_helicities (for planning and inspection); mea_evaluate on it returns
 * MEA_E_UNSUPPORTED. */
mea_status mea_create_process_host_only(const int *pdg, int n_ext, const mea_options *opts,
                                        mea_process_t *out);

mea_status mea_process_info(mea_process_t proc, mea_process_info_t *info);

/* Exact colour matrix: num[m*m] integers K with N = K / *den.  Host buffers. */
mea_status mea_colour_matrix(mea_process_t proc, int64_t *num, int64_t *den);

/* Helicity combinations kept by MEA_HEL_SUM_NONZERO: hel[n_hel][n_ext] (+1/-1),
 * host buffer of capacity cap rows; *n_hel receives the count. */
mea_status mea_helicities(mea_process_t proc, int8_t *hel, int cap, int *n_hel);

mea_status mea_destroy_process(mea_process_t proc);

/* Synchronise `stream` and report whether any bounded device wait of this
 * process's kernels expired since the last check (MEA_E_TIMEOUT; the affected
 * results are invalid).  Resets the indicator. */
mea_status mea_check_status(mea_process_t proc, void *stream);

/* Diagnostics, no counterpart in the paper: enqueue on `stream` a one-warp
 * kernel that waits on an mbarrier nothing arrives on, with the bounded wait
 * the tensor-core kernels use, limited to spin_limit polls (1..2^20), and
 * records the expiry in the process's status word as those kernels do -- so
 * that the next mea_check_status returns MEA_E_TIMEOUT.  Lets a caller (and
 * the tests) exercise the timeout path without a hung or faulted GPU; the
 * context stays usable.  MEA_E_ARG for a limit out of range. */
mea_status mea_probe_bounded_wait(mea_process_t proc, uint32_t spin_limit, void *stream);

/* Diagnostics, no counterpart in the paper: per-stage device time of this
 * process's evaluations.  With timing enabled, every evaluation records a
 * pair of CUDA events on its stream around the kernel launches of each stage
 * (amplitudes; colour amplitudes and colour sum of the tensor-core path; the
 * helicity sum of that path; the FP64 re-evaluation of flagged events).
 * mea_get_stage_times synchronises with the recorded events, returns the
 * summed milliseconds and launch counts per stage since the previous query
 * (or since timing was enabled) and starts a new count.  Stages that ran
 * concurrently on several streams are each counted in full; launches made
 * during stream capture are not timed.  Timing costs two event records per
 * stage launch; off by default.  The straight-line kernels
 * of small processes fuse amplitudes, colour amplitudes, colour sum and
 * helicity sum into one launch, counted as MEA_STAGE_AMPLITUDES. */
enum {
  MEA_STAGE_AMPLITUDES = 0,        /* amplitude kernel (fused kernel for small processes) */
  MEA_STAGE_COLOUR_AMPLITUDES = 1, /* tensor-core colour amplitudes J = C A */
  MEA_STAGE_COLOUR_SUM = 2,        /* tensor-core colour sum J^+ K J */
  MEA_STAGE_FINISH = 3,            /* helicity sum and flags after the tensor-core stages */
  MEA_STAGE_REEVALUATION = 4,      /* FP64 re-evaluation of flagged events */
  MEA_N_STAGES = 5
};
typedef struct {
  double ms[MEA_N_STAGES];
  int64_t launches[MEA_N_STAGES];
} mea_stage_times;

mea_status mea_set_stage_timing(mea_process_t proc, int enable);
mea_status mea_get_stage_times(mea_process_t proc, mea_stage_times *out);

/* ---- evaluation ----------------------------------------------------------- */

/* me2_dev[n_events] (double, device) <- |M|^2 of every event.
 * momenta_dev: device, layout above.  hel_dev: device, only for MEA_HEL_GIVEN
 * (else NULL).  flags_dev: device uint8[n_events] or NULL.
 * n_events may be 0 (nothing is enqueued). */
mea_status mea_evaluate(mea_process_t proc, const double *momenta_dev, int64_t n_events,
                        mea_hel_mode hel_mode, const int8_t *hel_dev, mea_prec_mode prec,
                        double *me2_dev, uint8_t *flags_dev, void *stream);

/* Same result through host buffers: momenta_host[n_events][n_ext][4] and
 * me2_host[n_events] (flags_host nullable) are host memory.  The library
 * works in chunks, overlapping copies with compute on two streams, and
 * returns when me2_host is filled (synchronous).  A buffer that is
 * page-locked over its whole extent (cudaHostAlloc, cudaHostRegister, a
 * pinned PyTorch tensor) is copied to or from the device directly; pageable
 * memory goes through the library's own pinned staging buffers. */
mea_status mea_evaluate_host(mea_process_t proc, const double *momenta_host, int64_t n_events,
                             mea_prec_mode prec, double *me2_host, uint8_t *flags_host);

/* ---- autotuning ------------------------------------------------------------
 * Times the candidate tile shapes and data placements of the amplitude kernel
 * for this process on n_sample events of momenta_dev (device) with the given
 * precision, keeps the fastest for later mea_evaluate calls of that precision
 * (helicity sum over the non-vanishing combinations), and reports it.  The
 * paper scanned register caps and block sizes by hand (Sec. 5.2); this is the
 * automated counterpart.  Synchronous; overwrites nothing the caller owns
 * except scratch_me2_dev (double[n_sample], device). */
typedef struct {
  int threads;           /* threads per CTA */
  int events_per_cta;    /* events per tile */
  int grid;              /* CTAs launched */
  int colour_amps_in_shared;  /* 1: colour amplitudes in shared memory */
  int slots_in_shared;   /* 1: wavefunction slots in shared memory */
  int candidates;        /* configurations timed */
  double best_ms;        /* time of the chosen configuration on the sample */
  double default_ms;     /* time of the heuristic default on the sample */
  int register_cap;      /* straight-line kernels: registers per thread of the
                            chosen variant (128, 85 or 168); helicity-shared kernel:
                            64 for its capped variant, 0 for the uncapped one; 0
                            for the interpreter */
  int vertex_partials;   /* 1: diagrams sharing a vertex partial use it (always
                            for the interpreter and FP64); 0: the straight-line
                            body with one vertex call per diagram was faster */
  int helicity_shared;   /* 1: the helicity-shared amplitude kernel was chosen
                            (threads = 32 x events_per_cta, one warp per event);
                            2: the split kernel */
  int forwarding;        /* 1: the per-lane interpreter with each op's output
                            forwarded to the next op in registers (and not stored
                            when nothing else reads it) was chosen */
} mea_tune_result;

mea_status mea_autotune(mea_process_t proc, const double *momenta_dev, int64_t n_sample,
                        mea_prec_mode prec, double *scratch_me2_dev, mea_tune_result *out);

/* ---- batched launch ---------------------------------------------------------
 * Several subprocesses of uneven size evaluated by one CUDA-graph launch.
 * mea_batch_create evaluates every item once (eagerly, to size scratch and
 * load kernels), then captures one evaluation of every item -- each on its own
 * branch of the graph, so that independent subprocesses run concurrently --
 * and instantiates the graph.  mea_batch_launch replays it on `stream`: it
 * re-reads the items' momenta buffers and rewrites their me2/flags buffers
 * (same pointers and event counts as at creation).  Items must not alias each
 * other's outputs.  The batch owns its scratch (one set per item). */
typedef struct {
  mea_process_t proc;
  const double *momenta_dev;
  int64_t n_events;
  double *me2_dev;
  uint8_t *flags_dev;   /* nullable */
} mea_batch_item;

typedef struct mea_batch_s *mea_batch_t;

mea_status mea_batch_create(const mea_batch_item *items, int n_items, mea_prec_mode prec,
                            mea_batch_t *out);
mea_status mea_batch_launch(mea_batch_t batch, void *stream);
/* Kernel nodes in the batch's graph (kernels launched per mea_batch_launch). */
mea_status mea_batch_info(mea_batch_t batch, int *n_kernel_nodes);
mea_status mea_batch_destroy(mea_batch_t batch);

/* ---- serving loop -----------------------------------------------------------
 * Continuous batching of evaluation requests on one GPU.  A worker thread owns
 * n_slots CUDA streams; each request (a process, device momenta and output
 * buffers) is split into chunks of about 1e11 FLOPs by the process's operation
 * count (the FP64 path weighted 24x), a multiple of 128 events and at most
 * chunk_events events.  Whenever a slot is free the worker dispatches a chunk
 * of the admitted request with the least remaining estimated device time
 * minus a quarter of the time it has waited since submission (shortest
 * remaining work first, with aging so that long requests are not starved);
 * requests arriving while others run start as soon as a slot frees up, and
 * work of different requests overlaps on the device.  Admission is by memory:
 * every slot keeps one scratch set per process it has run, so the scratch of
 * a process is committed per process (slots x one chunk's estimate, up to its
 * requests' chunk counts) against mem_budget_bytes and a process's chunks run
 * on at most that many distinct slots; a request whose process is committed
 * is admitted at once, the scratch of processes without requests is released
 * when the budget is short, a request waits while not even one slot fits, and
 * a request whose single chunk exceeds the budget is rejected at submission
 * (MEA_E_REJECTED).  Per-event results do not depend on chunking or on the
 * other requests in flight (bitwise), because every event is evaluated by the
 * same arithmetic in any tile.
 * Thread-safe.  The caller keeps the buffers alive until the request is
 * complete.  No call blocks without a bound: mea_server_wait returns
 * MEA_E_TIMEOUT when timeout_ms expires. */
typedef struct mea_server_s *mea_server_t;

typedef struct {
  uint64_t submitted, completed, rejected;
  uint64_t events_completed;
  double p50_ms, p99_ms, max_ms;  /* latency submit -> completion observed */
  double busy_seconds;            /* wall time with at least one chunk in flight */
  size_t reserved_bytes;          /* scratch currently committed to processes */
} mea_server_stats_t;

mea_status mea_server_create(size_t mem_budget_bytes, int n_slots, int64_t chunk_events, mea_server_t *out);
mea_status mea_server_submit(mea_server_t srv, mea_process_t proc, const double *momenta_dev, int64_t n_events,
                             mea_prec_mode prec, double *me2_dev, uint8_t *flags_dev, uint64_t *req_id);
/* Wait up to timeout_ms (< 0: 10 minutes) for the request; returns its status
 * (MEA_OK, MEA_E_TIMEOUT, or the error it failed with).  *latency_ms (nullable)
 * receives submit-to-completion time. */
mea_status mea_server_wait(mea_server_t srv, uint64_t req_id, int timeout_ms, double *latency_ms);
mea_status mea_server_stats(mea_server_t srv, mea_server_stats_t *out);
/* Stops accepting work, waits (bounded) for in-flight chunks, frees everything. */
mea_status mea_server_destroy(mea_server_t srv);

/* ---- evaluation without allocation ----------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot let the library allocate device memory: applications whose device
 * memory is owned entirely by a pool allocator of their own (a cudaMalloc
 * behind the pool's back can fail or fragment it), and latency-critical loops
 * that cannot afford the implicit device-wide synchronisation of cudaMalloc /
 * cudaFree.  mea_evaluate may grow per-process scratch with cudaMalloc; this
 * variant never calls cudaMalloc, cudaFree or any allocating routine.
 *
 * Same result as mea_evaluate(proc, momenta_dev, n_events, MEA_HEL_SUM_NONZERO,
 * NULL, prec, me2_dev, flags_dev, stream), bit for bit -- with the same launch
 * configuration, the one mea_autotune chose if it has run -- except that the
 * colour sum always runs on CUDA cores: where mea_evaluate would use the
 * tensor-core colour stages (MEA_PREC_MIXED for processes of six or more
 * partons, or colour_mode 2) the two agree within the mixed-path tolerance
 * (median 1e-6, max 1e-4 relative) instead of bitwise.  Events flagged on the
 * mixed path are re-evaluated in FP64 as in mea_evaluate.  Its scratch (the
 * flagged-event list and, for processes without a straight-line kernel,
 * wavefunction and colour-amplitude work space) is a fixed array of
 * MEA_NOALLOC_SCRATCH_BYTES in the library's device image, which every GPU
 * that loads the library holds until the process exits.
 *   - A request whose scratch would exceed that size is rejected with
 *     MEA_E_ARG before anything is enqueued (mea_last_error() gives the bytes
 *     needed); for gg -> ggg the flagged-event list limits n_events to about
 *     8.38 million per call, for gg -> gggg the work space to a few hundred
 *     events.
 *   - The first call on each device (and the first after its CUDA context was
 *     recreated, e.g. by cudaDeviceReset) looks up the array's device address
 *     with that device current; make that first call before any stream
 *     capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (the event-count word is cleared on the stream at the start of every
 *     call).  Calls whose GPU work overlaps -- on different streams, or from
 *     different host threads -- race on the array and give wrong results;
 *     order them on one stream or with events.
 *   - The process handle must have been created on the current device. */
#define MEA_NOALLOC_SCRATCH_BYTES (32u << 20)
mea_status mea_evaluate_noalloc(mea_process_t proc, const double *momenta_dev, int64_t n_events,
                                mea_prec_mode prec, double *me2_dev, uint8_t *flags_dev,
                                void *stream);

/* ---- synthetic phase space (input generator) ------------------------------ */

typedef struct {
  uint64_t seed;
  int n_final;          /* 2..8 */
  double rs_lo, rs_hi;  /* sqrt(s_hat) log-uniform range, GeV */
  double pt_min, eta_max, dr_min;
  double ptij_min;      /* GeV: min(pT_i, pT_j) Delta R_ij > ptij_min for every pair
                           (Eq. (cuts-ptjj)); <= 0 off */
} mea_ps_config;

/* momenta_dev[n][2 + n_final][4] <- events first_event .. first_event+n-1 of
 * the seeded generator (Philox4x32-10, RAMBO, cuts; identical to the host
 * generator).  attempts_dev (int32[n], nullable) receives the accepted attempt
 * index or -1.  Stream-ordered. */
mea_status mea_generate_phase_space(const mea_ps_config *cfg, uint64_t first_event, int64_t n,
                                    double *momenta_dev, int32_t *attempts_dev, void *stream);

/* ---- partonic cross section ------------------------------------------------ *
 * The subprocess cross section of Sec. 2.1 (the leading-order d sigma_hat with
 * the invariant phase space of Eq. (phase-space) and the statistical factor on
 * it):
 * sigma_hat(s_hat) = 1/(2 s_hat) * S * integral over the cut region of
 * dPhi_n |M|^2, with |M|^2 as mea_evaluate returns it (initial helicities and
 * colours averaged), S = 1 / prod k! over identical final-state partons, and
 * the Lorentz-invariant n-body phase space of massless partons,
 * Phi_n(s) = (2 pi)^(4-3n) (pi/2)^(n-1) s^(n-2) / ((n-1)! (n-2)!).
 * Estimated at fixed sqrt(s_hat) by the seeded generator (flat RAMBO points,
 * cut points redrawn): sigma = 1/(2 s) S Phi_n sum_accepted |M|^2 / (points
 * drawn), error from the variance over all drawn points (rejected ones count
 * 0).  Events first_event .. first_event + n_events - 1 of the generator with
 * rs_lo = rs_hi = sqrt_s; device work in chunks on an internal stream;
 * synchronous.  Result in pb (1 GeV^-2 = 0.3893794e9 pb).  MEA_E_ARG for bad
 * arguments; the generator's config must have n_final = n_ext - 2. */
typedef struct {
  double sigma_pb;       /* estimate */
  double error_pb;       /* one standard deviation, statistical */
  int64_t n_accepted;    /* events evaluated */
  int64_t n_drawn;       /* phase-space points drawn (accepted + rejected) */
  double phase_space;    /* Phi_n(s_hat), GeV^(2n-4) */
  double symmetry;       /* S */
} mea_xsec_result;

mea_status mea_partonic_cross_section(mea_process_t proc, double sqrt_s, const mea_ps_config *cuts,
                                      uint64_t first_event, int64_t n_events, mea_prec_mode prec,
                                      mea_xsec_result *out);

/* The same sigma_hat by adaptive importance sampling (VEGAS, G. P. Lepage,
 * J. Comput. Phys. 27 (1978) 192) over RAMBO's uniforms: a grid of `bins`
 * intervals per dimension maps each uniform, points that fail the cuts weigh
 * 0, and after every iteration each dimension's grid is refined from the sums
 * of (weight |M|^2)^2 per interval (smoothed over neighbours, compressed with
 * exponent alpha).  Iteration k uses generator events first_event + k *
 * points_per_iteration onwards (the VEGAS counter range, distinct from the
 * flat generator's); the iterations are combined with inverse-variance
 * weights.  Points are made and |M|^2 evaluated on the device; the grid lives
 * on the host.  Synchronous.  bins in [1, 64] (1: flat sampling without
 * redraws), iterations >= 1, points_per_iteration >= 2, alpha >= 0;
 * otherwise MEA_E_ARG. */
typedef struct {
  int iterations;
  int64_t points_per_iteration;
  int bins;
  double alpha;          /* grid compression exponent; 1.5 is customary */
} mea_vegas_config;

typedef struct {
  double sigma_pb;       /* inverse-variance weighted over the iterations */
  double error_pb;
  double chi2_per_dof;   /* consistency of the iterations (0 for one) */
  double last_sigma_pb;  /* the last iteration alone */
  double last_error_pb;
  int64_t n_points;      /* all iterations */
  int64_t n_accepted;    /* points that passed the cuts */
} mea_vegas_result;

mea_status mea_partonic_cross_section_vegas(mea_process_t proc, double sqrt_s, const mea_ps_config *cuts,
                                            uint64_t first_event, const mea_vegas_config *vc,
                                            mea_prec_mode prec, mea_vegas_result *out);

/* ---- diagnostics ------------------------------------------------------------ */

const char *mea_last_error(void);

/* Measured arithmetic peak of the FP32 (fp64 = 0) or FP64 (fp64 = 1) pipe of
 * the current device, the denominator of the amplitude kernels' rooflines (no
 * counterpart in the paper): a kernel of independent fused multiply-add
 * chains, every SM several CTAs deep, timed with CUDA events after a warm-up
 * launch, the timed launch sized for about `seconds` (0 < seconds <= 10).
 * *tflops receives 2 FLOP per FMA over the launch's duration, *ms that
 * duration.  Changes no clock or power setting: the result holds at whatever
 * SM clock the GPU ran (sample it alongside to normalise).  Synchronous. */
mea_status mea_measure_alu_peak(int fp64, double seconds, double *tflops, double *ms);

/* Number of kernels this library has launched in this process (all devices). */
uint64_t mea_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* MEA_H */

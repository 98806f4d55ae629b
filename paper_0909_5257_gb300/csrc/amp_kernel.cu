// Amplitude stage, table-driven: one lane per (event, helicity combination).
//
// A CTA owns a tile of E events x H helicity lanes.  Per tile:
//   phase 0  preparation, shared by the helicity lanes of an event
//            (amp_common.cuh): transverse polarisation bases and helicity
//            spinor blocks of every leg, and for every momentum sum ("mask")
//            used by the program its flowing-out momentum and 1/P^2, the
//            invariant formed in FP64 (FP64 path) or compensated FP32 (FP32
//            path) before the cast to the lane precision; input checks;
//   phase 1  every lane runs the process program (op table): external
//            wavefunctions, shared off-shell currents, one amplitude per
//            Feynman diagram.  Default mode: each amplitude is added into the
//            colour amplitudes J_alpha of its colour entries
//            (Eq. (color-amplitude); two-sum compensated in FP32), then the
//            colour quadratic form of Eq. (color-averaged-amplitude) with the
//            integer colour matrix.  Amplitude-output mode (AOUT, FP32): the
//            diagram amplitudes go to global memory for the tensor-core colour
//            stages (jamp_gemm.cu, colour_gemm.cu), with per-row maxima and
//            the cancellation mass;
//   phase 2  the helicity sum of each event in fixed order, x 1/4, written to
//            me2 together with the event flags (default mode; in AOUT mode
//            finish_kernel does it after the colour stages).
// Wavefunction slots live in shared or global memory as [slot][lane][8 reals];
// colour amplitudes as [alpha][component][lane], so consecutive lanes touch
// consecutive words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <mutex>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/mea.h"
#include "amp_common.cuh"
#include "heget.cuh"
#include "kernels.h"

namespace mea {

uint64_t& launch_counter() {
  static uint64_t c = 0;
  return c;
}

cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> set;
  std::lock_guard<std::mutex> lk(mu);
  auto it = set.find(kernel);
  if (it != set.end() && it->second >= bytes) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) set[kernel] = bytes;
  return e;
}

namespace {

constexpr int kMaxThreads = 512;

union OpWords {
  int4 v[2];
  Op op;
};

// Wavefunction slots are stored [slot][lane][8 reals]: one lane's wavefunction
// is 32 (FP32) or 64 (FP64) contiguous bytes, moved with 16-byte vector
// accesses -- a quarter warp then covers 128 contiguous bytes, conflict-free in
// shared memory and whole sectors in global memory.
template <typename R>
__device__ __forceinline__ W4<R> ld_slot(const R* slots, int s, int L, int t) {
  const R* b = slots + ((size_t)s * L + t) * 8;
  W4<R> w;
  if constexpr (std::is_same<R, float>::value) {
    const float4 u = *reinterpret_cast<const float4*>(b);
    const float4 v = *reinterpret_cast<const float4*>(b + 4);
    w.c[0] = {u.x, u.y}; w.c[1] = {u.z, u.w}; w.c[2] = {v.x, v.y}; w.c[3] = {v.z, v.w};
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 u = *reinterpret_cast<const double2*>(b + 2 * k);
      w.c[k] = {u.x, u.y};
    }
  }
  return w;
}
template <typename R>
__device__ __forceinline__ void st_slot(R* slots, int s, int L, int t, const W4<R>& w) {
  R* b = slots + ((size_t)s * L + t) * 8;
  if constexpr (std::is_same<R, float>::value) {
    *reinterpret_cast<float4*>(b) = make_float4(w.c[0].r, w.c[0].i, w.c[1].r, w.c[1].i);
    *reinterpret_cast<float4*>(b + 4) = make_float4(w.c[2].r, w.c[2].i, w.c[3].r, w.c[3].i);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) *reinterpret_cast<double2*>(b + 2 * k) = make_double2(w.c[k].r, w.c[k].i);
  }
}

// One op of the process program for the (pair) lane t of a slot array with
// stride L: external wavefunction or current into its slot (returns false), or
// a diagram amplitude into amp (returns true).
//
// FWD (amplitude-output FP32 path): the previous op's output is also held in
// `last`; fwd bit k (0..3) marks an input that is that output (read from the
// register instead of the slot), bit 4 an output read by nothing but the next
// op (kept in the register only, never stored).
template <typename R, bool FWD = false>
__device__ __forceinline__ bool eval_op(const Op& op, const DevProgram& P, R* slots, int L, int t, const R* et,
                                        const R* mt, uint32_t lam_bits, R g, R gg, cx<R>& amp,
                                        uint32_t fwd = 0u, W4<R>* last = nullptr) {
  auto in_ = [&](int k) -> W4<R> {
    if constexpr (FWD) {
      if (fwd >> k & 1u) return *last;
    }
    return ld_slot(slots, op.in[k], L, t);
  };
  auto out_ = [&](const W4<R>& x) {
    if constexpr (FWD) {
      *last = x;
      if (fwd & 16u) return;
    }
    st_slot(slots, op.out, L, t, x);
  };
  switch (op.type) {
    case OP_EXT: {
      int l = op.leg;
      int type = P.leg_info[4 * l], kind = P.leg_info[4 * l + 1];
      bool in = P.leg_info[4 * l + 2] != 0;
      const R* o = et + 8 * l;
      W4<R> x;
      int lam = (lam_bits >> l & 1u) ? 1 : -1;
      if (type == 0) x = ext_gluon<R>(o, o + 3, lam, !in);
      else x = ext_spinor<R>(o[0], o[1], mk<R>(o[2], o[3]), lam, kind);
      out_(x);
      return false;
    }
    case OP_JVV: {
      W4<R> a = in_(0);
      W4<R> b = in_(1);
      const R* pa = mt + 5 * op.min[0];
      const R* pb = mt + 5 * op.min[1];
      W4<R> j = jvv<R>(a, b, pa, pb, mt[5 * op.mout + 4], g);
      out_(j);
      return false;
    }
    case OP_JGGG: {
      W4<R> a = in_(0);
      W4<R> b = in_(1);
      W4<R> c = in_(2);
      W4<R> j = jggg<R>(a, b, c, mt[5 * op.mout + 4], gg);
      out_(j);
      return false;
    }
    case OP_FVI: {
      W4<R> f = in_(0);
      W4<R> v = in_(1);
      const R* pq = mt + 5 * op.mout;
      W4<R> j = fvi<R>(f, v, pq, pq[4], g);
      out_(j);
      return false;
    }
    case OP_FVO: {
      W4<R> f = in_(0);
      W4<R> v = in_(1);
      const R* pq = mt + 5 * op.mout;
      W4<R> j = fvo<R>(f, v, pq, pq[4], g);
      out_(j);
      return false;
    }
    case OP_JIO: {
      W4<R> f = in_(0);
      W4<R> o = in_(1);
      W4<R> j = jio<R>(f, o, mt[5 * op.mout + 4], g);
      out_(j);
      return false;
    }
    case OP_AVVV: {
      W4<R> a = in_(0);
      W4<R> b = in_(1);
      W4<R> c = in_(2);
      amp = vvv_amp<R>(a, b, c, mt + 5 * op.min[0], mt + 5 * op.min[1], mt + 5 * op.min[2], g);
      return true;
    }
    case OP_AGGGG: {
      W4<R> a = in_(0);
      W4<R> b = in_(1);
      W4<R> c = in_(2);
      W4<R> d = in_(3);
      amp = gggg_amp<R>(a, b, c, d, gg);
      return true;
    }
    case OP_AIOV: {
      W4<R> f = in_(0);
      W4<R> o = in_(1);
      W4<R> v = in_(2);
      amp = iov_amp<R>(f, o, v, g);
      return true;
    }
    case OP_ADOT: {  // diagram amplitude from its free wavefunction and the group's partial
      W4<R> w = in_(0);
      W4<R> p = in_(1);
      amp = part_contract<R>(w, p, (op.leg & 1u) != 0, (op.leg & 2u) != 0);
      return true;
    }
    case OP_PVVV: {
      W4<R> b = in_(0);
      W4<R> c = in_(1);
      W4<R> u = vvv_part<R>(b, c, mt + 5 * op.min[0], mt + 5 * op.min[1], mt + 5 * op.min[2], g);
      out_(u);
      return false;
    }
    case OP_PGGGG: {
      W4<R> x = in_(0);
      W4<R> y = in_(1);
      W4<R> z = in_(2);
      W4<R> u = gggg_part<R>(x, y, z, gg);
      out_(u);
      return false;
    }
    case OP_PIOV: {  // free fi: (fo, V); free fo: (fi, V); free V: (fi, fo)
      W4<R> a = in_(0);
      W4<R> b = in_(1);
      W4<R> u = op.leg == 0 ? iov_part_i<R>(a, b, g) : (op.leg == 1 ? iov_part_o<R>(a, b, g) : iov_part_v<R>(a, b, g));
      out_(u);
      return false;
    }
    default:
      return false;
  }
  return false;
}

template <typename R, bool JSMEM, bool SSMEM, bool AOUT, bool FWD = false>
__global__ void __launch_bounds__(kMaxThreads) amp_kernel(const DevProgram P, const AmpLaunch A,
                                                   const AmpConfig C) {
  static_assert(!AOUT || std::is_same<R, float>::value, "amplitude output is an FP32 path");
  static_assert(!FWD || AOUT, "register forwarding is built for the amplitude-output path");
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool F32 = std::is_same<R, float>::value;
  constexpr int JW = F32 ? 4 : 2;  // FP32: hi re, hi im, lo re, lo im
  const int L = blockDim.x;
  const int t = threadIdx.x;
  const int n_ext = P.n_ext, m = P.n_colour, H = C.H, E = C.E_cta;
  const int tab_stride = event_table_stride(n_ext, P.n_masks);

  size_t off = 0;
  R* slots;
  if (SSMEM) {
    slots = reinterpret_cast<R*>(smem);
    off += (size_t)P.n_slots * 8 * L * sizeof(R);
  } else {
    slots = reinterpret_cast<R*>(A.slot_scratch) + (size_t)blockIdx.x * P.n_slots * 8 * L;
  }
  R* jam;
  if (JSMEM) {
    jam = reinterpret_cast<R*>(smem + off);
    off += (size_t)m * JW * L * sizeof(R);
  } else {
    jam = reinterpret_cast<R*>(A.jamp_scratch) + (size_t)blockIdx.x * m * JW * L;
  }
  R* tab = reinterpret_cast<R*>(smem + off);
  off += (size_t)E * tab_stride * sizeof(R);
  off = (off + 7) & ~size_t(7);
  double* res = reinterpret_cast<double*>(smem + off);
  off += (size_t)L * sizeof(double);
  float* kap = reinterpret_cast<float*>(smem + off);
  unsigned int* evflag = reinterpret_cast<unsigned int*>(kap + L);  // [E] input-check bits
  for (int i = t; i < E; i += L) evflag[i] = 0u;

  const bool listed = A.event_list != nullptr;
  const int64_t n = listed ? (int64_t)(*A.list_count) : A.n_events;
  const int64_t n_tiles = (n + E - 1) / E;
  const R g = (R)P.g;
  const R gg = (R)(P.g * P.g);
  const OpWords* ops = reinterpret_cast<const OpWords*>(P.ops);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t ev0 = tile * E;
    // ---- phase 0: FP64 preparation
    __syncthreads();  // evflag cleared (first tile) / released by the previous finish
    tile_prep<R>(P, A, tab, tab_stride, ev0, n, E, t, L, evflag);
    __syncthreads();

    // ---- phase 1: one (event, helicity) per lane
    const int e = t / H, h = t - (t / H) * H;
    const int64_t ev = ev0 + e;
    const bool active = (t < E * H) && (ev < n);
    double val = 0.0;
    float kappa = 0.f;
    int bad = 0;
    if (active) {
      const int64_t gev = listed ? (int64_t)A.event_list[ev] : ev;
      uint32_t lam_bits = 0;  // bit l set: leg l has helicity +1
      for (int l = 0; l < n_ext; ++l) {
        int8_t v;
        if (A.hel_mode == 0) v = P.hel[h * n_ext + l];
        else if (A.hel_mode == 1) v = P.hel_all[h * n_ext + l];
        else v = A.hel_given[gev * n_ext + l];
        if (v > 0) lam_bits |= 1u << l;
      }
      const R* et = tab + (size_t)e * tab_stride;
      const R* mt = et + 8 * n_ext;
      if (!AOUT)
        for (int a = 0; a < m * JW; ++a) jam[(size_t)a * L + t] = (R)0;
      float abs_mass = 0.f;  // sum of |c A| over all colour entries (FP32 indicator)
      // amplitude output: diagram ordinal, row maxima of |Re A|, |Im A|, finiteness
      const int64_t pair = ev * H + h;
      int d_amp = 0;
      float mx_re = 0.f, mx_im = 0.f;
      bool finite_amps = true;

      // one diagram amplitude: to the tensor-core stage (AOUT) or into the
      // colour amplitudes through its colour entries
      auto take_amp = [&](uint32_t col_begin, uint32_t col_count, const cx<R>& amp) {
        if (AOUT) {
          float2* dst = reinterpret_cast<float2*>(A.amp_out + (size_t)d_amp * A.lda + 2 * pair);
          *dst = make_float2((float)amp.r, (float)amp.i);
          const float ar = fabsf((float)amp.r), ai = fabsf((float)amp.i);
          finite_amps = finite_amps && isfinite(ar) && isfinite(ai);
          mx_re = fmaxf(mx_re, ar);
          mx_im = fmaxf(mx_im, ai);
          abs_mass += __ldg(P.amp_w + d_amp) * (ar + ai);
          ++d_amp;
        } else {
          const ColEntry* ce = P.col + col_begin;
          for (uint32_t k = 0; k < col_count; ++k) {
            ColEntry c = ce[k];
            R cr = (R)c.re, ci = (R)c.im;
            R xr = cr * amp.r - ci * amp.i;
            R xi = cr * amp.i + ci * amp.r;
            R* jr = jam + (size_t)c.alpha * JW * L + t;
            if constexpr (F32) {
              float s, er;
              two_sum(jr[0], xr, s, er);
              jr[0] = s;
              jr[2 * L] += er;
              two_sum(jr[L], xi, s, er);
              jr[L] = s;
              jr[3 * L] += er;
              abs_mass += fabsf(xr) + fabsf(xi);
            } else {
              jr[0] += xr;
              jr[L] += xi;
            }
          }
        }
      };
      W4<R> last;  // the previous op's output (FWD)
      for (int i = 0; i < P.n_ops; ++i) {
        OpWords w;
        w.v[0] = __ldg(&ops[i].v[0]);
        w.v[1] = __ldg(&ops[i].v[1]);
        cx<R> amp;
        bool is_amp;
        if constexpr (FWD) {
          is_amp = eval_op<R, true>(w.op, P, slots, L, t, et, mt, lam_bits, g, gg, amp, __ldg(P.fwd + i), &last);
        } else {
          is_amp = eval_op<R>(w.op, P, slots, L, t, et, mt, lam_bits, g, gg, amp);
        }
        if (is_amp) take_amp(w.op.col_begin, w.op.col_count, amp);
      }
      if (AOUT) {
        const float nan = __int_as_float(0x7fc00000);
        A.amp_rowmax[2 * pair] = finite_amps ? mx_re : nan;
        A.amp_rowmax[2 * pair + 1] = finite_amps ? mx_im : nan;
        A.pair_kappa[pair] = abs_mass;  // divided by sum |J| after the colour-amplitude stage

      } else {
      // ---- colour sum: sum_ab J_a K_ab J_b^* / D
      R tot = (R)0;
      float jabs = 0.f;
      for (int a = 0; a < m; ++a) {
        const R* ja = jam + (size_t)a * JW * L + t;
        R ar = ja[0], ai = ja[L];
        if constexpr (F32) { ar += ja[2 * L]; ai += ja[3 * L]; jabs += fabsf(ar) + fabsf(ai); }
        R zr = (R)0, zi = (R)0;
        for (int b = 0; b < m; ++b) {
          R k;
          if constexpr (F32) k = __ldg(P.cf_f + (size_t)a * m + b);
          else k = __ldg(P.cf_d + (size_t)a * m + b);
          if (k == (R)0) continue;
          const R* jb = jam + (size_t)b * JW * L + t;
          R br = jb[0], bi = jb[L];
          if constexpr (F32) { br += jb[2 * L]; bi += jb[3 * L]; }
          zr += k * br;
          zi += k * bi;
        }
        tot += ar * zr + ai * zi;
      }
      val = (double)tot * P.cf_inv_den;
      if (F32) kappa = (jabs > 0.f) ? abs_mass / jabs : 0.f;
      bad = isfinite(val) ? 0 : 1;
      }
    }
    res[t] = bad ? __longlong_as_double(0x7ff8000000000000ll) : val;
    kap[t] = kappa;
    __syncthreads();

    // ---- phase 2: helicity sum per event, fixed order
    if (!AOUT) {
      tile_finish<F32>(A, t, E, H, ev0, n, listed, res, kap, evflag);
    } else if (t < E) {
      // the helicity sum runs after the colour stages: hand over the input checks
      if (ev0 + t < n) A.ev_flags[ev0 + t] = (uint8_t)evflag[t];
      evflag[t] = 0u;
    }
    __syncthreads();
  }
}

template <typename R>
size_t smem_bytes(const DevProgram& p, int threads, int E, bool jsmem, bool ssmem) {
  const int JW = std::is_same<R, float>::value ? 4 : 2;
  size_t b = ssmem ? (size_t)p.n_slots * 8 * threads * sizeof(R) : 0;
  if (jsmem) b += (size_t)p.n_colour * JW * threads * sizeof(R);
  b += (size_t)E * event_table_stride(p.n_ext, p.n_masks) * sizeof(R);
  b = (b + 7) & ~size_t(7);
  b += (size_t)threads * (sizeof(double) + sizeof(float) + sizeof(unsigned int)) + 16;
  return b;
}

// pk: per-pair indicator; with jabs (sum |J| of each column split, [n_splits][n_pairs])
// pk holds sum |c A| and the indicator is pk / sum_splits jabs.
__global__ void finish_kernel(const AmpLaunch A, int H, const double* pairval, const float* pk,
                              const float* jabs, int n_splits) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= A.n_events) return;
  const int64_t n_pairs = A.n_events * H;
  double s = 0.0, wk = 0.0;
  for (int h = 0; h < H; ++h) {
    const int64_t p = e * H + h;
    double v = pairval[p];
    float k = pk[p];
    if (jabs) {
      float ja = 0.f;
      for (int q = 0; q < n_splits; ++q) ja += jabs[(size_t)q * n_pairs + p];
      k = (ja > 0.f) ? k / ja : 0.f;
    }
    s += v;
    wk += v * (double)k;
  }
  double me = 0.25 * s;
  A.me2[e] = me;
  uint8_t fl = A.ev_flags ? A.ev_flags[e] : (uint8_t)0;
  if (!isfinite(me)) fl |= MEA_FLAG_NONFINITE;
  const double ind = error_indicator(wk, s);
  if (!(ind <= (double)A.flag_threshold)) fl |= MEA_FLAG_CANCEL;
  if (A.flags) A.flags[e] = fl;
  if (A.flag_list && (fl & (MEA_FLAG_CANCEL | MEA_FLAG_NONFINITE | MEA_FLAG_QGUARD))) {
    int slot = atomicAdd(A.flag_count, 1);
    A.flag_list[slot] = (int32_t)e;
  }
}

}  // namespace

cudaError_t launch_finish(const AmpLaunch& a, int H, const double* pairval, const float* pair_kappa,
                          cudaStream_t s, const float* jabs, int n_splits) {
  if (a.n_events <= 0) return cudaSuccess;
  int threads = 256;
  int64_t blocks = (a.n_events + threads - 1) / threads;
  finish_kernel<<<(unsigned)blocks, threads, 0, s>>>(a, H, pairval, pair_kappa, jabs, n_splits);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

const GenEntry* find_generated(const int* pdg, int n_ext) {
  int n = 0;
  const GenEntry* t = generated_table(&n);
  std::string key;
  for (int i = 0; i < n_ext; ++i) key += (i ? "," : "") + std::to_string(pdg[i]);
  for (int i = 0; i < n; ++i)
    if (key == t[i].key) return &t[i];
  return nullptr;
}

// Straight-line kernels keep the lane state in registers: pick the tile so
// that threads <= kGenMaxThreads with few idle lanes, then fill the SMs by
// occupancy.
//
// Body of the FP32 straight-line kernel at a register cap (0: 128, 1: 85):
// the one with shared vertex partials (fewer FLOPs) unless it needs more
// local memory (spills) than the body with one vertex call per diagram.
// Spilled lines compete with the streamed inputs for L2 and reach DRAM at
// full size, which costs more than the FLOPs save (gg>ggg at 2^20 events:
// 82.7 M events/s with partials, 92.2 M without; the partials body spills
// 1104 bytes per thread at 128 registers, the other 936).  The rule depends
// only on the compiled kernels, so the choice -- and the FP32 rounding order
// -- is the same on every run.
static int gen_body_variant(const DevProgram& p, int cap) {
  cudaFuncAttributes with, without;
  if (cudaFuncGetAttributes(&with, p.gen->kernel(false, 2 * cap)) != cudaSuccess ||
      cudaFuncGetAttributes(&without, p.gen->kernel(false, 2 * cap + 1)) != cudaSuccess)
    return 2 * cap;
  return without.localSizeBytes < with.localSizeBytes ? 2 * cap + 1 : 2 * cap;
}

static AmpConfig plan_generated(const DevProgram& p, bool fp64, int H, int64_t n_events, int num_sms) {
  AmpConfig best;
  best.H = H;
  best.jamp_in_smem = true;
  best.slots_in_smem = true;
  const int tab_stride = event_table_stride(p.n_ext, p.n_masks);
  double best_score = -1;
  // default: the 128-register variant (mea_autotune also tries 85 and 168 registers)
  const int regvar = fp64 ? 0 : (p.gen_forced >= 0 ? p.gen_forced : gen_body_variant(p, 0));
  const void* k = p.gen->kernel(fp64, regvar);
  cudaFuncAttributes fa;
  int max_threads = 256;
  if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) max_threads = std::min(max_threads, fa.maxThreadsPerBlock);
  for (int E = 1; E * H <= max_threads; ++E) {
    int threads = ((E * H + 31) / 32) * 32;
    if (threads > max_threads) break;
    size_t sm = (((size_t)E * tab_stride * (fp64 ? 8 : 4) + 7) & ~size_t(7)) + (size_t)threads * 16 + 16;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, sm) != cudaSuccess) per_sm = 0;
    if (per_sm < 1) continue;  // this tile cannot be resident: skip it
    double util = (double)(E * H) / threads;
    double score = std::min<double>((double)per_sm * threads, 1024.0) * util;
    // within 2 % of the best score prefer the larger tile: fewer per-tile
    // preparation rounds and barriers (measured: gg>ggg 160 threads x 3 CTAs
    // 11.6 ms vs 64 x 8 13.8 ms for 2^20 events, same resident lanes)
    const bool better = score > best_score * 1.02 || (score >= best_score * 0.98 && threads > best.threads);
    if (best_score < 0 || better) {
      best_score = std::max(best_score, score);
      best.E_cta = E; best.threads = threads; best.smem = sm; best.grid = per_sm * num_sms; best.regvar = regvar;
      best.per_sm = per_sm;
    }
  }
  if (best_score < 0) {  // nothing resident at all: one warp per tile
    best.E_cta = std::max(1, 32 / std::max(H, 1));
    best.threads = ((best.E_cta * H + 31) / 32) * 32;
    best.smem = (((size_t)best.E_cta * tab_stride * (fp64 ? 8 : 4) + 7) & ~size_t(7)) + (size_t)best.threads * 16 + 16;
    best.grid = num_sms;
    best.regvar = regvar;
  }
  int64_t tiles = (n_events + best.E_cta - 1) / best.E_cta;
  if (tiles < best.grid) best.grid = (int)std::max<int64_t>(tiles, 1);
  return best;
}

// CTAs of the interpreter kernel of this placement that registers and
// threads allow on one SM (shared memory is limited by the caller): the
// kernel is persistent (a grid-stride loop over tiles), so a grid beyond what
// is resident at once would leave the CTAs that start late to finish their
// share of the tiles alone.  Computed from the kernel's register count
// (cudaFuncGetAttributes, read only): planning may run on any host thread
// while another launches these kernels, so it changes no function attribute.
static int interp_resident(bool fp64, bool jsm, bool ssm, bool aout, int threads, bool fwd = false) {
  const void* k;
  if (aout && fwd)
    k = ssm ? (const void*)amp_kernel<float, true, true, true, true> : (const void*)amp_kernel<float, true, false, true, true>;
  else if (aout) k = ssm ? (const void*)amp_kernel<float, true, true, true> : (const void*)amp_kernel<float, true, false, true>;
  else if (fp64)
    k = jsm ? (ssm ? (const void*)amp_kernel<double, true, true, false> : (const void*)amp_kernel<double, true, false, false>)
            : (ssm ? (const void*)amp_kernel<double, false, true, false> : (const void*)amp_kernel<double, false, false, false>);
  else
    k = jsm ? (ssm ? (const void*)amp_kernel<float, true, true, false> : (const void*)amp_kernel<float, true, false, false>)
            : (ssm ? (const void*)amp_kernel<float, false, true, false> : (const void*)amp_kernel<float, false, false, false>);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((std::max(fa.numRegs, 1) + 7) / 8) * 8 * 32;  // allocated per warp in units of 8 per thread
  const int by_regs = 65536 / std::max(regs_warp * warps, 1);
  return std::max(0, std::min({by_regs, 2048 / (warps * 32), 32}));
}

AmpConfig plan_amp(const DevProgram& p, bool fp64, int H, int64_t n_events, int num_sms,
                   size_t max_smem, size_t smem_per_sm, int hint) {
  if (p.gen && hint == 0) return plan_generated(p, fp64, H, n_events, num_sms);
  if (hint == 0 && p.hsp_only && hsp_supported(p, fp64, H)) {
    // split evaluation only: the candidate with the most resident lanes
    std::vector<AmpConfig> cs = hsp_candidates(p, H, num_sms, max_smem, smem_per_sm);
    if (!cs.empty()) {
      AmpConfig c = cs.front();
      for (const AmpConfig& x : cs)
        if ((int64_t)x.per_sm * x.E_cta > (int64_t)c.per_sm * c.E_cta) c = x;
      const int64_t tiles = (n_events + c.E_cta - 1) / c.E_cta;
      if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
      return c;
    }
  }
  if (hint == 0 && p.hs_only && hs_supported(p, fp64, H)) {
    // helicity-shared kernel only (without the option, the per-lane heuristic
    // below is the untuned default: measured at least as fast untuned on every
    // process; the tuner picks the shared kernels where they are faster)
    AmpConfig c = hs_plan(p, H, num_sms, max_smem, smem_per_sm);
    if (c.grid > 0) {
      const int64_t tiles = (n_events + c.E_cta - 1) / c.E_cta;
      if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
      return c;
    }
  }
  AmpConfig best;
  best.H = H;
  double best_score = -1;
  // Every placement is scored by the lanes it keeps resident per SM (latency
  // hiding) times the fraction of busy lanes: everything in shared memory
  // counts up to 512 lanes per SM, placements that go through L1/L2 up to 256.
  // A shared-memory placement that leaves only a few lanes per SM loses to a
  // global one with many (measured: gg>gggg 2.6x, uu~>gggg 2.5x faster).
  const int placements[4][2] = {{1, 1}, {1, 0}, {0, 1}, {0, 0}};
  for (int pl = 0; pl < 4; ++pl) {
    bool jsm = placements[pl][0] != 0, ssm = placements[pl][1] != 0;
    if (p.n_colour == 0 && !jsm) continue;  // no colour accumulators: one placement axis
    for (int E = 1; E * H <= kMaxThreads; ++E) {
      if (hint > 0 && E != hint) continue;
      int threads = ((E * H + 31) / 32) * 32;
      size_t sm = fp64 ? smem_bytes<double>(p, threads, E, jsm, ssm)
                       : smem_bytes<float>(p, threads, E, jsm, ssm);
      if (sm > max_smem) break;
      int per_sm = (int)std::min<size_t>(smem_per_sm / std::max<size_t>(sm, 1), 2048 / threads);
      per_sm = std::min(per_sm, 32);
      if (per_sm < 1) continue;
      const int res = interp_resident(fp64, jsm, ssm, p.n_colour == 0 && !fp64, threads);
      if (res >= 1) per_sm = std::min(per_sm, res);
      double util = (double)(E * H) / threads;
      double lanes_sm = (double)per_sm * E * H;
      // enough lanes per SM to hide latency, then as few idle lanes as possible
      double score = std::min(lanes_sm, 512.0) * util;
      if (!jsm || !ssm) score = std::min(lanes_sm, 256.0) * util;
      if (score > best_score + 1e-9) {
        best_score = score;
        best.E_cta = E; best.threads = threads; best.smem = sm;
        best.jamp_in_smem = jsm; best.slots_in_smem = ssm;
        best.grid = per_sm * num_sms;
        best.per_sm = per_sm;
      }
    }
  }
  if (best_score < 0) {
    best.E_cta = 1;
    best.threads = ((H + 31) / 32) * 32;
    best.jamp_in_smem = false;
    best.slots_in_smem = false;
    best.smem = fp64 ? smem_bytes<double>(p, best.threads, 1, false, false)
                     : smem_bytes<float>(p, best.threads, 1, false, false);
    best.grid = num_sms;
  }
  if (p.fwd_only && p.fwd && p.n_colour == 0 && !fp64) {
    // forwarding only: the same tile, within the forwarding kernel's residency
    best.fwd = true;
    const int rf = interp_resident(false, true, best.slots_in_smem, true, best.threads, true);
    if (rf >= 1 && rf < best.per_sm) {
      best.per_sm = rf;
      best.grid = rf * num_sms;
    }
  }
  int64_t tiles = (n_events + best.E_cta - 1) / best.E_cta;
  if (tiles < best.grid) best.grid = (int)std::max<int64_t>(tiles, 1);
  return best;
}

std::vector<AmpConfig> candidate_configs(const DevProgram& p, bool fp64, int H, int64_t n_events, int num_sms,
                                         size_t max_smem, size_t smem_per_sm) {
  std::vector<AmpConfig> out;
  auto cap = [&](AmpConfig c) {
    int64_t tiles = (n_events + c.E_cta - 1) / c.E_cta;
    if (tiles < c.grid) c.grid = (int)std::max<int64_t>(tiles, 1);
    return c;
  };
  if (p.gen) {
    // FP64: one variant; FP32: every register cap, each with its body (see
    // gen_body_variant)
    const int n_caps = (fp64 || p.gen_forced >= 0) ? 1 : kGenCaps;
    for (int cap_i = 0; cap_i < n_caps; ++cap_i) {
    const int rv = fp64 ? 0 : (p.gen_forced >= 0 ? p.gen_forced : gen_body_variant(p, cap_i));
    const void* k = p.gen->kernel(fp64, rv);
    cudaFuncAttributes fa;
    int max_threads = 256;
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) max_threads = std::min(max_threads, fa.maxThreadsPerBlock);
    const int tab_stride = event_table_stride(p.n_ext, p.n_masks);
    int last_threads = -1;
    for (int E = 1; E * H <= max_threads; ++E) {
      int threads = ((E * H + 31) / 32) * 32;
      if (threads > max_threads) break;
      // the largest E for each thread count (fewest idle lanes)
      if ((E + 1) * H <= max_threads && (((E + 1) * H + 31) / 32) * 32 == threads) continue;
      if (threads == last_threads) continue;
      last_threads = threads;
      AmpConfig c;
      c.H = H; c.E_cta = E; c.threads = threads; c.regvar = rv;
      c.smem = (((size_t)E * tab_stride * (fp64 ? 8 : 4) + 7) & ~size_t(7)) + (size_t)threads * 16 + 16;
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, c.smem) != cudaSuccess || per_sm < 1)
        continue;
      c.grid = per_sm * num_sms;
      c.per_sm = per_sm;
      out.push_back(cap(c));
    }
    }
    return out;
  }
  if (hs_supported(p, fp64, H)) {
    for (AmpConfig c : hs_candidates(p, H, num_sms, max_smem, smem_per_sm)) out.push_back(cap(c));
    if (p.hs_only) return out;
  }
  if (hsp_supported(p, fp64, H)) {
    for (AmpConfig c : hsp_candidates(p, H, num_sms, max_smem, smem_per_sm)) out.push_back(cap(c));
    if (p.hsp_only) return out;
  }
  const int placements[4][2] = {{1, 1}, {1, 0}, {0, 1}, {0, 0}};
  for (auto& pl : placements) {
    if (p.n_colour == 0 && !pl[0]) continue;  // no colour accumulators: one placement axis
    int last_threads = -1;
    for (int E = 1; E * H <= kMaxThreads; ++E) {
      int threads = ((E * H + 31) / 32) * 32;
      if ((E + 1) * H <= kMaxThreads && (((E + 1) * H + 31) / 32) * 32 == threads) continue;
      if (threads == last_threads) continue;
      last_threads = threads;
      size_t sm = fp64 ? smem_bytes<double>(p, threads, E, pl[0], pl[1]) : smem_bytes<float>(p, threads, E, pl[0], pl[1]);
      if (sm > max_smem) break;
      int per_sm = (int)std::min<size_t>(smem_per_sm / std::max<size_t>(sm, 1), 2048 / threads);
      per_sm = std::min(per_sm, 32);
      if (per_sm < 1) continue;
      const int res = interp_resident(fp64, pl[0] != 0, pl[1] != 0, p.n_colour == 0 && !fp64, threads);
      if (res >= 1) per_sm = std::min(per_sm, res);
      AmpConfig c;
      c.H = H; c.E_cta = E; c.threads = threads; c.smem = sm;
      c.jamp_in_smem = pl[0] != 0; c.slots_in_smem = pl[1] != 0;
      c.grid = per_sm * num_sms;
      c.per_sm = per_sm;
      if (!p.fwd_only) out.push_back(cap(c));
      if (p.fwd && p.n_colour == 0 && !fp64) {
        // the same tile with the previous op's output forwarded in registers
        AmpConfig f = c;
        f.fwd = true;
        const int rf = interp_resident(false, true, pl[1] != 0, true, threads, true);
        if (rf >= 1) {
          f.per_sm = std::min(per_sm, rf);
          f.grid = f.per_sm * num_sms;
          out.push_back(cap(f));
        }
      }
      // with slots in global memory, fewer resident lanes per SM leave each lane
      // more of the L1 and L2 for its wavefunction slots (fewer DRAM trips)
      // against less latency hiding: the tuner times both sides
      if (!pl[1]) {
        int prev = per_sm;
        for (int k : {per_sm / 2, 2, 1}) {
          if (k < 1 || k >= prev) continue;
          AmpConfig r = c;
          r.per_sm = k;
          r.grid = k * num_sms;
          out.push_back(cap(r));
          prev = k;
        }
      }
    }
  }
  return out;
}

size_t jamp_scratch_bytes_needed(const DevProgram& p, bool fp64, const AmpConfig& c) {
  if (c.jamp_in_smem) return 0;
  const int JW = fp64 ? 2 : 4;
  return (size_t)c.grid * p.n_colour * JW * c.threads * (fp64 ? sizeof(double) : sizeof(float));
}

size_t slot_scratch_bytes_needed(const DevProgram& p, bool fp64, const AmpConfig& c) {
  if (c.helshare) return hs_arena_bytes(p, c);
  if (c.hsplit) return hsp_area_bytes(p, c);
  if (c.slots_in_smem) return 0;
  return (size_t)c.grid * p.n_slots * 8 * c.threads * (fp64 ? sizeof(double) : sizeof(float));
}

int carveout_percent(const AmpConfig& c) {
  static int smem_sm = 0;
  if (smem_sm == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || v <= 0)
      v = 228 * 1024;
    smem_sm = v;
  }
  const double need = (double)std::max(1, c.per_sm) * ((double)c.smem + 1024.0);  // 1 KB reserved per CTA
  return std::max(0, std::min(100, (int)std::ceil(100.0 * need / smem_sm) + 1));
}

template <typename R, bool J, bool S, bool O = false, bool F = false>
static cudaError_t launch_one(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {
  cudaError_t e = ensure_dynamic_smem((const void*)amp_kernel<R, J, S, O, F>, c.smem);
  if (e != cudaSuccess) return e;
  // the carveout is a preference: a value the driver refuses leaves the launch valid
  if (cudaFuncSetAttribute(amp_kernel<R, J, S, O, F>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           carveout_percent(c)) != cudaSuccess)
    cudaGetLastError();
  amp_kernel<R, J, S, O, F><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  return cudaGetLastError();
}

cudaError_t launch_amp(const DevProgram& p, bool fp64, const AmpConfig& c, const AmpLaunch& a,
                       cudaStream_t s) {
  if (c.grid <= 0) return cudaSuccess;
  cudaError_t err = cudaSuccess;
  if (c.helshare || c.hsplit) {
    if (fp64) return cudaErrorInvalidValue;
    err = c.helshare ? launch_amp_hs(p, c, a, s) : launch_amp_hsp(p, c, a, s);
    if (err == cudaSuccess) ++launch_counter();
    return err;
  }
  if (c.threads < 32 || c.threads > kMaxThreads || c.E_cta < 1 || c.E_cta * c.H > c.threads)
    return cudaErrorInvalidConfiguration;
  if (a.amp_out) {
    // diagram amplitudes out (no colour accumulators): FP32 interpreter only
    if (fp64 || p.n_colour != 0) return cudaErrorInvalidValue;
    if (c.fwd) {
      if (!p.fwd) return cudaErrorInvalidValue;
      err = c.slots_in_smem ? launch_one<float, true, true, true, true>(p, c, a, s)
                            : launch_one<float, true, false, true, true>(p, c, a, s);
    } else {
      err = c.slots_in_smem ? launch_one<float, true, true, true>(p, c, a, s) : launch_one<float, true, false, true>(p, c, a, s);
    }
  } else if (p.gen) {
    p.gen->launch(fp64, c.regvar, p, c, a, s);
    err = cudaGetLastError();
  } else if (fp64) {
    if (c.jamp_in_smem && c.slots_in_smem) err = launch_one<double, true, true>(p, c, a, s);
    else if (c.jamp_in_smem) err = launch_one<double, true, false>(p, c, a, s);
    else if (c.slots_in_smem) err = launch_one<double, false, true>(p, c, a, s);
    else err = launch_one<double, false, false>(p, c, a, s);
  } else {
    if (c.jamp_in_smem && c.slots_in_smem) err = launch_one<float, true, true>(p, c, a, s);
    else if (c.jamp_in_smem) err = launch_one<float, true, false>(p, c, a, s);
    else if (c.slots_in_smem) err = launch_one<float, false, true>(p, c, a, s);
    else err = launch_one<float, false, false>(p, c, a, s);
  }
  if (err == cudaSuccess) ++launch_counter();
  return err;
}

}  // namespace mea

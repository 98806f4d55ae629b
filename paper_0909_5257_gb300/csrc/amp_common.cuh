// Per-tile phases shared by the amplitude kernels (the table-driven
// interpreter in amp_kernel.cu and the straight-line per-process kernels the
// generator emits): FP64 preparation of the per-event tables (phase 0) and the
// fixed-order helicity sum with the event flags (phase 2).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "../../include/mea.h"
#include "heget.cuh"
#include "kernels.h"

namespace mea {
namespace {

// The mixed path's per-event relative error indicator, in units of FP32
// roundoff u = 2^-24:
//   ind = u * (kIndicatorBase + kappa),
//   kappa = sum_h |M_h|^2 kappa_h / sum_h |M_h|^2,  kappa_h = sum |c A| / sum |J|,
// kappa_h being the cancellation in helicity h's diagram sum into the colour
// amplitudes (Eq. (color-amplitude)); a relative perturbation u of every
// diagram amplitude moves |M|^2 by at most u kappa.  kIndicatorBase covers the
// rounding of the vertex and current evaluations that produce the amplitudes:
// measured on GB300 for every process through gg -> 5g, the mixed result's
// relative error against the FP64 path stays below 20-47 u whatever kappa
// (1 <= kappa <= 23 in those samples), and u (32 + kappa) bounds it for more
// than 99.7 % of the events.
constexpr double kRoundoff = 1.0 / 16777216.0;
constexpr double kIndicatorBase = 32.0;
__host__ __device__ __forceinline__ double error_indicator(double weighted_kappa, double sum) {
  return sum > 0.0 ? kRoundoff * (kIndicatorBase + weighted_kappa / sum) : 0.0;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Per-event table in shared memory (lane precision R), stride
// event_table_stride(): [8 per leg] polarisation basis or spinor block,
// [5 per mask] flowing-out momentum sum and 1/P^2, [8 per leg] the leg's FP64
// momentum split into two R parts (hi, lo) -- used by the FP32 path to form the
// invariants without the FP64 pipe.
__host__ __device__ __forceinline__ int event_table_stride(int n_ext, int n_masks) {
  return 16 * n_ext + 5 * n_masks;
}

// Leg item: polarisation bases and spinor blocks (directions and square roots,
// no cancellation: |p| + pz is taken as pT^2/(|p| - pz) when pz < 0) in the
// lane precision R.
template <typename R>
__device__ void prep_leg(const DevProgram& P, const double* mom, int k, R* et) {
  const int n_ext = P.n_ext;
  const double* p = mom + 4 * k;
  R* o = et + 8 * k;
  int type = P.leg_info[4 * k];
  R px = (R)p[1], py = (R)p[2], pz = (R)p[3];
  R kt2 = px * px + py * py;
  R kk = sqrt(kt2 + pz * pz);
  if (type == 0) {
    R kt = sqrt(kt2);
    R ct, st, cp, sp;
    if (kt > R(0)) { ct = pz / kk; st = kt / kk; cp = px / kt; sp = py / kt; }
    else { ct = pz < R(0) ? R(-1) : R(1); st = R(0); cp = R(1); sp = R(0); }
    o[0] = ct * cp; o[1] = ct * sp; o[2] = -st;
    o[3] = -sp; o[4] = cp; o[5] = R(0);
    o[6] = R(0); o[7] = R(0);
  } else {
    // chi_+ = (a, b) with a = sqrt((|p|+pz)/(2|p|)), b = (px + i py)/sqrt(2|p|(|p|+pz))
    R apz = (pz >= R(0)) ? kk + pz : kt2 / (kk - pz);
    R a, br, bi;
    if (apz > R(0)) {
      R nrm = R(1) / sqrt(R(2) * kk * apz);
      a = apz * nrm; br = px * nrm; bi = py * nrm;
    } else {  // exactly along -z: chi_+ = (0, 1)
      a = R(0); br = R(1); bi = R(0);
    }
    o[0] = sqrt(R(2) * (R)p[0]); o[1] = a; o[2] = br; o[3] = bi;
    o[4] = o[5] = o[6] = o[7] = R(0);
  }
  if constexpr (std::is_same<R, float>::value) {
    float* sp = et + 8 * n_ext + 5 * P.n_masks + 8 * k;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const float hi = (float)p[mu];
      sp[mu] = hi;
      sp[4 + mu] = (float)(p[mu] - (double)hi);
    }
  }
}

// Flowing-out momentum sum of the legs in msk as an unevaluated FP32 pair
// (hi + lo, two-sum compensated) from the split momenta of the table.
__device__ __forceinline__ void split_sum(const DevProgram& P, const float* et, uint32_t msk, float qh[4],
                                          float ql[4]) {
  const int n_ext = P.n_ext;
  const float* sp = et + 8 * n_ext + 5 * P.n_masks;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) { qh[mu] = 0.f; ql[mu] = 0.f; }
  for (int l = 0; l < n_ext; ++l)
    if (msk >> l & 1u) {
      const bool neg = P.leg_info[4 * l + 2] != 0;  // incoming legs enter with -p
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const float h = neg ? -sp[8 * l + mu] : sp[8 * l + mu];
        const float lo = neg ? -sp[8 * l + 4 + mu] : sp[8 * l + 4 + mu];
        float s, e;
        two_sum(qh[mu], h, s, e);
        qh[mu] = s;
        ql[mu] = __fadd_rn(ql[mu], __fadd_rn(e, lo));
      }
    }
}

// Minkowski square of an FP32 pair vector (q = qh + ql) to about 2^-46 of the
// squared components: exact squares of the high parts by FMA (two-product),
// their signed sum by two-sum, the cross terms 2 qh ql in FP32.
__device__ __forceinline__ float split_square(const float qh[4], const float ql[4]) {
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const float sg = mu == 0 ? 1.f : -1.f;
    const float pp = __fmul_rn(qh[mu], qh[mu]);
    const float pe = fmaf(qh[mu], qh[mu], -pp);
    float s, e;
    two_sum(hi, sg * pp, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, sg * fmaf(2.f * qh[mu], ql[mu], pe)));
  }
  return __fadd_rn(hi, lo);
}

// Mask item: flowing-out momentum of the line and 1/P^2.  The invariant P^2,
// where collinear kinematics cancel digits, is formed in FP64 on the FP64 path
// and from the split momenta in compensated FP32 (about 46 bits) on the FP32
// path.  Sets MEA_FLAG_QGUARD when an internal line has |P^2| below 1e-10 of
// the squared energy flowing through it.
template <typename R>
__device__ void prep_mask(const DevProgram& P, const double* mom, int row, R* et, unsigned int* evflag) {
  const int n_ext = P.n_ext;
  const uint32_t msk = P.masks[row];
  const int np = __popc(msk);
  R* o = et + 8 * n_ext + 5 * row;
  R q2r, esum;
  if constexpr (std::is_same<R, float>::value) {
    float qh[4], ql[4];
    split_sum(P, et, msk, qh, ql);
    for (int mu = 0; mu < 4; ++mu) o[mu] = __fadd_rn(qh[mu], ql[mu]);
    q2r = split_square(qh, ql);
    esum = 0.f;
    for (int l = 0; l < n_ext; ++l)
      if (msk >> l & 1u) esum += et[8 * n_ext + 5 * P.n_masks + 8 * l];
  } else {
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    esum = 0.0;
    for (int l = 0; l < n_ext; ++l)
      if (msk >> l & 1u) {
        double s = P.leg_info[4 * l + 2] ? -1.0 : 1.0;  // flowing-out momentum
        for (int mu = 0; mu < 4; ++mu) q[mu] += s * mom[4 * l + mu];
        esum += mom[4 * l];
      }
    for (int mu = 0; mu < 4; ++mu) o[mu] = q[mu];
    q2r = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
  }
  // internal lines only: a sum of n_ext - 1 legs is an external momentum (P^2 = 0)
  if (np > 1 && np < n_ext - 1 && !(fabs(q2r) >= R(1e-10) * esum * esum)) atomicOr(evflag, MEA_FLAG_QGUARD);
  o[4] = (np > 1) ? R(1) / q2r : R(0);
}

// Check item: momentum conservation, every component of (incoming - outgoing)
// against 1e-9 of the incoming energy (MEA_FLAG_MOMENTUM).
template <typename R>
__device__ void prep_check(const DevProgram& P, const double* mom, const R* et, unsigned int* evflag) {
  const int n_ext = P.n_ext;
  double worst = 0.0, scale;
  if constexpr (std::is_same<R, float>::value) {
    float qh[4], ql[4];
    split_sum(P, et, (1u << n_ext) - 1u, qh, ql);  // = -(incoming - outgoing)
    for (int mu = 0; mu < 4; ++mu) worst = fmax(worst, (double)fabsf(__fadd_rn(qh[mu], ql[mu])));
    const float* sp = et + 8 * n_ext + 5 * P.n_masks;
    scale = (double)sp[0] + (double)sp[8];
  } else {
    double bal[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < n_ext; ++l) {
      const double sg = P.leg_info[4 * l + 2] ? 1.0 : -1.0;
      for (int mu = 0; mu < 4; ++mu) bal[mu] += sg * mom[4 * l + mu];
    }
    for (int mu = 0; mu < 4; ++mu) worst = fmax(worst, fabs(bal[mu]));
    scale = mom[0] + mom[4];
  }
  if (!(worst <= 1e-9 * scale)) atomicOr(evflag, MEA_FLAG_MOMENTUM);
}

// Phase 0: the threads of the tile prepare the (event, leg) items, then -- after
// a barrier, since the FP32 path reads the split momenta -- the (event, mask)
// items and one momentum-conservation check per event.
template <typename R>
__device__ __forceinline__ void tile_prep(const DevProgram& P, const AmpLaunch& A, R* tab, int tab_stride,
                                          int64_t ev0, int64_t n, int E, int t, int L, unsigned int* evflag) {
  const bool listed = A.event_list != nullptr;
  const int n_ext = P.n_ext;
  for (int i = t; i < E * n_ext; i += L) {
    int e = i / n_ext, k = i - e * n_ext;
    int64_t ev = ev0 + e;
    if (ev < n) {
      int64_t gev = listed ? (int64_t)A.event_list[ev] : ev;
      prep_leg<R>(P, A.mom + (size_t)gev * n_ext * 4, k, tab + (size_t)e * tab_stride);
    }
  }
  __syncthreads();
  const int items = P.n_masks + 1;
  for (int i = t; i < E * items; i += L) {
    int e = i / items, k = i - e * items;
    int64_t ev = ev0 + e;
    if (ev < n) {
      int64_t gev = listed ? (int64_t)A.event_list[ev] : ev;
      const double* mom = A.mom + (size_t)gev * n_ext * 4;
      R* et = tab + (size_t)e * tab_stride;
      if (k < P.n_masks) prep_mask<R>(P, mom, k, et, evflag + e);
      else prep_check<R>(P, mom, et, evflag + e);
    }
  }
}

// Phase 2: thread e < E sums the H helicity lanes of its event in fixed order,
// applies the 1/4 helicity average, writes me2 and the flags, and appends
// flagged events to the re-evaluation list.
template <bool F32>
__device__ __forceinline__ void tile_finish(const AmpLaunch& A, int t, int E, int H, int64_t ev0, int64_t n,
                                            bool listed, const double* res, const float* kap,
                                            unsigned int* evflag) {
    if (t < E) {
      const uint8_t inflags = (uint8_t)evflag[t];
      evflag[t] = 0u;  // ready for the next tile (its prep follows a barrier)
      int64_t evr = ev0 + t;
      if (evr < n) {
        int64_t gev = listed ? (int64_t)A.event_list[evr] : evr;
        double s = 0.0, wk = 0.0;
        for (int hh = 0; hh < H; ++hh) {
          double v = res[t * H + hh];
          s += v;
          wk += v * (double)kap[t * H + hh];
        }
        double me = 0.25 * s;
        A.me2[gev] = me;
        uint8_t fl = inflags;
        if (!isfinite(me)) fl |= MEA_FLAG_NONFINITE;
        if (F32) {
          // relative error indicator (roundoff x (base + cancellation in J))
          const double ind = error_indicator(wk, s);
          if (!(ind <= (double)A.flag_threshold)) fl |= MEA_FLAG_CANCEL;
        }
        if (A.flags) {
          if (A.write_flags_mode == 0) A.flags[gev] = fl;
          // re-evaluation: keep why the event was flagged (cancellation, input
          // checks), take finiteness from the FP64 result
          else A.flags[gev] = (uint8_t)((A.flags[gev] & ~MEA_FLAG_NONFINITE) | MEA_FLAG_REEVALUATED | fl);
        }
        if (A.flag_list && (fl & (MEA_FLAG_CANCEL | MEA_FLAG_NONFINITE | MEA_FLAG_QGUARD))) {
          int slot = atomicAdd(A.flag_count, 1);
          A.flag_list[slot] = (int32_t)gev;
        }
      }
    }
}

}  // namespace
}  // namespace mea

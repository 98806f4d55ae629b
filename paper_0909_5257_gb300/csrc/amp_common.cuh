// Per-tile phases shared by the amplitude kernels (the table-driven
// interpreter in amp_kernel.cu and the straight-line per-process kernels the
// generator emits): FP64 preparation of the per-event tables (phase 0) and the
// fixed-order helicity sum with the event flags (phase 2).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mea.h"
#include "heget.cuh"
#include "kernels.h"

namespace mea {
namespace {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Preparation of one leg or one mask row of one event, shared by the event's
// helicity lanes.  The invariants P^2 of the momentum sums (the propagator
// denominators, where collinear kinematics cancel digits) are formed in FP64
// from the FP64 momenta; the polarisation bases and spinor blocks (directions
// and square roots, no cancellation: |p| + pz is taken as pT^2/(|p| - pz) when
// pz < 0) are computed in the lane precision R.
template <typename R>
__device__ void prep_item(const DevProgram& P, const double* mom, int k, R* tab) {
  const int n_ext = P.n_ext;
  if (k < n_ext) {
    const double* p = mom + 4 * k;
    R* o = tab + 8 * k;
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
  } else {
    int row = k - n_ext;
    uint32_t msk = P.masks[row];
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = 0; l < n_ext; ++l)
      if (msk >> l & 1u) {
        double s = P.leg_info[4 * l + 2] ? -1.0 : 1.0;  // flowing-out momentum
        for (int mu = 0; mu < 4; ++mu) q[mu] += s * mom[4 * l + mu];
      }
    R* o = tab + 8 * n_ext + 5 * row;
    double q2 = q[0] * q[0] - q[1] * q[1] - q[2] * q[2] - q[3] * q[3];
    for (int mu = 0; mu < 4; ++mu) o[mu] = (R)q[mu];
    o[4] = (__popc(msk) > 1) ? R(1) / (R)q2 : R(0);
  }
}

// Phase 0: every thread of the tile prepares (event, leg) and (event, mask)
// items in FP64 and stores them in the lane precision.
template <typename R>
__device__ __forceinline__ void tile_prep(const DevProgram& P, const AmpLaunch& A, R* tab, int tab_stride,
                                          int64_t ev0, int64_t n, int E, int t, int L) {
  const bool listed = A.event_list != nullptr;
  const int items = P.n_ext + P.n_masks;
  for (int i = t; i < E * items; i += L) {
    int e = i / items, k = i - e * items;
    int64_t ev = ev0 + e;
    if (ev < n) {
      int64_t gev = listed ? (int64_t)A.event_list[ev] : ev;
      prep_item<R>(P, A.mom + (size_t)gev * P.n_ext * 4, k, tab + (size_t)e * tab_stride);
    }
  }
}

// Phase 2: thread e < E sums the H helicity lanes of its event in fixed order,
// applies the 1/4 helicity average, writes me2 and the flags, and appends
// flagged events to the re-evaluation list.
template <bool F32>
__device__ __forceinline__ void tile_finish(const AmpLaunch& A, int t, int E, int H, int64_t ev0, int64_t n,
                                            bool listed, const double* res, const float* kap) {
    if (t < E) {
      int64_t evr = ev0 + t;
      if (evr < n) {
        int64_t gev = listed ? (int64_t)A.event_list[evr] : evr;
        double s = 0.0, wk = 0.0;
        for (int hh = 0; hh < H; ++hh) {
          double v = res[t * H + hh];
          s += v;
          wk += v * (double)kap[t * H + hh];
          if (A.pair_out) A.pair_out[gev * H + hh] = v;
        }
        double me = 0.25 * s;
        A.me2[gev] = me;
        uint8_t fl = 0;
        if (!isfinite(me)) fl |= MEA_FLAG_NONFINITE;
        if (F32) {
          // relative error indicator: FP32 unit roundoff x cancellation in J
          double ind = (s > 0.0) ? 5.96e-8 * wk / s : 0.0;
          if (!(ind <= (double)A.flag_threshold)) fl |= MEA_FLAG_CANCEL;
        }
        if (A.flags) {
          if (A.write_flags_mode == 0) A.flags[gev] = fl;
          else A.flags[gev] = (uint8_t)((A.flags[gev] & ~MEA_FLAG_CANCEL) | MEA_FLAG_REEVALUATED | fl);
        }
        if (A.flag_list && (fl & (MEA_FLAG_CANCEL | MEA_FLAG_NONFINITE))) {
          int slot = atomicAdd(A.flag_count, 1);
          A.flag_list[slot] = (int32_t)gev;
        }
      }
    }
}

}  // namespace
}  // namespace mea

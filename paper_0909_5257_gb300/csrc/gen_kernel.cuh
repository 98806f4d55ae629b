// Kernel template for the straight-line per-process bodies that codegen.cpp
// emits.  Same tile structure as the interpreter (amp_kernel.cu): FP64
// preparation of the per-event tables in shared memory, one lane per
// (event, helicity) running the process body with all wavefunctions and
// colour amplitudes in registers, fixed-order helicity sum.  Only the
// per-event tables and the lane results use shared memory.
#pragma once
#include <type_traits>

#include "amp_common.cuh"

namespace mea {
namespace {

constexpr int kGenMaxThreads = 256;

// J += (cr + i ci) a, two-sum compensated in FP32 (lo collects the rounding
// errors); mass accumulates sum |c a| for the cancellation indicator.
template <typename R>
__device__ __forceinline__ void jacc(cx<R>& hi, cx<R>& lo, float& mass, R cr, R ci, cx<R> a) {
  R xr = cr * a.r - ci * a.i;
  R xi = cr * a.i + ci * a.r;
  if constexpr (std::is_same<R, float>::value) {
    float s, e;
    two_sum(hi.r, xr, s, e);
    hi.r = s;
    lo.r += e;
    two_sum(hi.i, xi, s, e);
    hi.i = s;
    lo.i += e;
    mass += fabsf(xr) + fabsf(xi);
  } else {
    hi.r += xr;
    hi.i += xi;
  }
}

// J += a, two-sum compensated in FP32 (the coefficient is folded into a by
// the emitter; mass is accumulated once per amplitude).
template <typename R>
__device__ __forceinline__ void jadd(cx<R>& hi, cx<R>& lo, cx<R> a) {
  if constexpr (std::is_same<R, float>::value) {
    float s, e;
    two_sum(hi.r, a.r, s, e);
    hi.r = s;
    lo.r += e;
    two_sum(hi.i, a.i, s, e);
    hi.i = s;
    lo.i += e;
  } else {
    hi.r += a.r;
    hi.i += a.i;
  }
}

template <typename R>
__device__ __forceinline__ cx<R> neg(cx<R> a) {
  return cx<R>{-a.r, -a.i};
}

template <typename R>
__device__ __forceinline__ cx<R> jfin(cx<R> hi, cx<R> lo) {
  if constexpr (std::is_same<R, float>::value) return cx<R>{hi.r + lo.r, hi.i + lo.i};
  return hi;
}

// Register-cap variants: MINB resident CTAs of MAXT threads per SM cap a
// thread at 65536 / (MAXT MINB) registers.  Spilling part of the long
// straight-line body to L1 in exchange for more resident warps wins for the
// 3-jet bodies (measured on 2^20 events: gg>ggg 14.4 ms at 255 registers,
// 11.3 ms at 128; uu>uug 2.6 ms at 128, 2.25 ms at 85), so the FP32 bodies
// come at 128 (256 threads, MINB 2), 85 (256, 3) and 168 (192, 2) registers --
// the last halves the gg>ggg spill footprint (640 against 936 bytes per
// thread) so that it stays in L1 with 10 resident warps -- and the autotuner
// picks; the FP64 bodies come at 128.  A module that also held uncapped FP32
// variants measured 25-45 % slower on the same 128-register kernel, so none
// is built.
template <typename R, typename Body, int MINB, int MAXT>
__global__ void __launch_bounds__(MAXT, MINB) gen_kernel(const DevProgram P, const AmpLaunch A,
                                                                   const AmpConfig C) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool F32 = std::is_same<R, float>::value;
  const int L = blockDim.x;
  const int t = threadIdx.x;
  const int n_ext = P.n_ext, H = C.H, E = C.E_cta;
  const int tab_stride = event_table_stride(n_ext, P.n_masks);
  R* tab = reinterpret_cast<R*>(smem);
  size_t off = ((size_t)E * tab_stride * sizeof(R) + 7) & ~size_t(7);
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

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t ev0 = tile * E;
    __syncthreads();  // evflag cleared (first tile) / released by the previous finish
    tile_prep<R>(P, A, tab, tab_stride, ev0, n, E, t, L, evflag);
    __syncthreads();
    const int e = t / H, h = t - (t / H) * H;
    const int64_t ev = ev0 + e;
    const bool active = (t < E * H) && (ev < n);
    double val = 0.0;
    float kappa = 0.f;
    if (active) {
      const int64_t gev = listed ? (int64_t)A.event_list[ev] : ev;
      uint32_t lam = 0;
      for (int l = 0; l < n_ext; ++l) {
        int8_t v;
        if (A.hel_mode == 0) v = P.hel[h * n_ext + l];
        else if (A.hel_mode == 1) v = P.hel_all[h * n_ext + l];
        else v = A.hel_given[gev * n_ext + l];
        if (v > 0) lam |= 1u << l;
      }
      const R* et = tab + (size_t)e * tab_stride;
      Body::run(et, et + 8 * n_ext, lam, g, gg, P.cf_inv_den, val, kappa);
      if (!isfinite(val)) val = __longlong_as_double(0x7ff8000000000000ll);
    }
    res[t] = val;
    kap[t] = kappa;
    __syncthreads();
    tile_finish<F32>(A, t, E, H, ev0, n, listed, res, kap, evflag);
    __syncthreads();
  }
}

template <typename R, typename Body, int MINB, int MAXT>
void gen_launch_v(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {
  auto k = gen_kernel<R, Body, MINB, MAXT>;
  if (ensure_dynamic_smem((const void*)k, c.smem) != cudaSuccess) return;
  // the carveout is a preference: a value the driver refuses leaves the launch valid
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_percent(c)) != cudaSuccess)
    cudaGetLastError();
  k<<<c.grid, c.threads, c.smem, s>>>(p, a, c);
}

// Each kernel variant of a process -- the FP32 bodies (with vertex partials
// or one vertex call per diagram) at 128, 85 and 168 registers, numbered
// 2 * cap + body (kernels.h), and the FP64 body with partials at 128 -- is
// instantiated in a translation unit (device module) of its own by
// codegen.cpp, behind two plain functions: gen_launch_v and the kernel's
// address.  Separate units compile in parallel.
}  // namespace
}  // namespace mea

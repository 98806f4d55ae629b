// Amplitude stage with helicity sharing (amplitude-output mode, FP32): one
// warp per event.
//
// Every wavefunction of the process program depends on the helicities of the
// legs flowing into it and on nothing else of the helicity combination
// (helshare.h).  Per event the warp therefore evaluates each external state,
// off-shell current and vertex partial once per helicity pattern of its own
// legs -- its lanes take the 2^k variants of a k-leg wavefunction -- and each
// diagram amplitude once per summed helicity combination (lanes h, h + 32, ...),
// reading every input from the variant its own helicities select.  The
// arithmetic of each operation is the per-lane interpreter's (the same HELAS
// functions of heget.cuh on the same inputs), so the diagram amplitudes, their
// row maxima and the cancellation mass it writes for the tensor-core colour
// stages (jamp_gemm.cu, colour_gemm.cu) are those of amp_kernel.cu's
// amplitude-output mode.
//
// Per CTA: W warps = W events per tile.  Phase 0 (tile_prep, amp_common.cuh)
// fills the per-event tables (polarisation bases, spinor blocks, momentum sums
// and 1/P^2 from the compensated FP32 invariants, input checks) for the W
// events; then each warp runs the program for its event with its variants in
// its own region of global memory ([variant][8 reals], 32 bytes, 16-byte
// accesses); the variant index of an input is looked up in two shared-memory
// tables (bit extraction and deposit over the leg sets).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/mea.h"
#include "amp_common.cuh"
#include "heget.cuh"
#include "helshare.h"
#include "kernels.h"

namespace mea {
namespace {

union HsOpWords {
  int4 v[2];
  Op op;
};
union HsRec {
  int4 v;
  HsOp h;
};

__device__ __forceinline__ W4<float> ld_var(const float* arena, int idx) {
  const float* b = arena + (size_t)idx * 8;
  const float4 u = *reinterpret_cast<const float4*>(b);
  const float4 v = *reinterpret_cast<const float4*>(b + 4);
  W4<float> w;
  w.c[0] = {u.x, u.y}; w.c[1] = {u.z, u.w}; w.c[2] = {v.x, v.y}; w.c[3] = {v.z, v.w};
  return w;
}
__device__ __forceinline__ void st_var(float* arena, int idx, const W4<float>& w) {
  float* b = arena + (size_t)idx * 8;
  *reinterpret_cast<float4*>(b) = make_float4(w.c[0].r, w.c[0].i, w.c[1].r, w.c[1].i);
  *reinterpret_cast<float4*>(b + 4) = make_float4(w.c[2].r, w.c[2].i, w.c[3].r, w.c[3].i);
}

__device__ __forceinline__ bool hs_is_amp(int t) {
  return t == OP_AVVV || t == OP_AGGGG || t == OP_AIOV || t == OP_ADOT;
}

// Loads input k of the current op for the helicity bits lam: the variant of
// that input's legs that lam selects.
struct HsInputs {
  const float* arena;
  const uint8_t* pext;
  int NL;
  const HsOp& q;
  uint32_t lam;
  __device__ __forceinline__ W4<float> operator()(int k) const {
    return ld_var(arena, q.in_off[k] + pext[q.in_mask[k] * NL + lam]);
  }
};

// Split evaluation's per-lane inputs: the prologue variant that lam selects,
// or the transient current of the previous op (kHsTransient).
struct HsSplitInputs {
  const float* area;
  const uint8_t* pext;
  int NL;
  const HsOp& q;
  uint32_t lam;
  const W4<float>& tr;
  __device__ __forceinline__ W4<float> operator()(int k) const {
    if (q.in_off[k] == kHsTransient) return tr;
    return ld_var(area, q.in_off[k] + pext[q.in_mask[k] * NL + lam]);
  }
};

// The wavefunction a slot-producing op makes (lam: the helicity bits of the
// variant; external states read their own leg's bit).
template <class X>
__device__ __forceinline__ W4<float> hs_produce(const Op& op, const DevProgram& P, const X& x,
                                                const float* et, const float* mt, float g, float gg) {
  switch (op.type) {
    case OP_EXT: {
      const int l = op.leg;
      const int type = P.leg_info[4 * l], kind = P.leg_info[4 * l + 1];
      const bool in = P.leg_info[4 * l + 2] != 0;
      const float* o = et + 8 * l;
      const int h = (x.lam >> l & 1u) ? 1 : -1;
      if (type == 0) return ext_gluon<float>(o, o + 3, h, !in);
      return ext_spinor<float>(o[0], o[1], mk<float>(o[2], o[3]), h, kind);
    }
    case OP_JVV: {
      W4<float> a = x(0), b = x(1);
      return jvv<float>(a, b, mt + 5 * op.min[0], mt + 5 * op.min[1], mt[5 * op.mout + 4], g);
    }
    case OP_JGGG: {
      W4<float> a = x(0), b = x(1), c = x(2);
      return jggg<float>(a, b, c, mt[5 * op.mout + 4], gg);
    }
    case OP_FVI: {
      W4<float> f = x(0), v = x(1);
      const float* pq = mt + 5 * op.mout;
      return fvi<float>(f, v, pq, pq[4], g);
    }
    case OP_FVO: {
      W4<float> f = x(0), v = x(1);
      const float* pq = mt + 5 * op.mout;
      return fvo<float>(f, v, pq, pq[4], g);
    }
    case OP_JIO: {
      W4<float> f = x(0), o = x(1);
      return jio<float>(f, o, mt[5 * op.mout + 4], g);
    }
    case OP_PVVV: {
      W4<float> b = x(0), c = x(1);
      return vvv_part<float>(b, c, mt + 5 * op.min[0], mt + 5 * op.min[1], mt + 5 * op.min[2], g);
    }
    case OP_PGGGG: {
      W4<float> a = x(0), b = x(1), c = x(2);
      return gggg_part<float>(a, b, c, gg);
    }
    case OP_PIOV: {
      W4<float> a = x(0), b = x(1);
      return op.leg == 0 ? iov_part_i<float>(a, b, g) : (op.leg == 1 ? iov_part_o<float>(a, b, g) : iov_part_v<float>(a, b, g));
    }
    default:
      break;
  }
  W4<float> z;
  for (int k = 0; k < 4; ++k) z.c[k] = {0.f, 0.f};
  return z;
}

// The diagram amplitude of an amplitude op.
template <class X>
__device__ __forceinline__ cx<float> hs_amplitude(const Op& op, const X& x, const float* mt, float g,
                                                  float gg) {
  switch (op.type) {
    case OP_AVVV: {
      W4<float> a = x(0), b = x(1), c = x(2);
      return vvv_amp<float>(a, b, c, mt + 5 * op.min[0], mt + 5 * op.min[1], mt + 5 * op.min[2], g);
    }
    case OP_AGGGG: {
      W4<float> a = x(0), b = x(1), c = x(2), d = x(3);
      return gggg_amp<float>(a, b, c, d, gg);
    }
    case OP_AIOV: {
      W4<float> f = x(0), o = x(1), v = x(2);
      return iov_amp<float>(f, o, v, g);
    }
    case OP_ADOT: {
      W4<float> w = x(0), p = x(1);
      return part_contract<float>(w, p, (op.leg & 1u) != 0, (op.leg & 2u) != 0);
    }
    default:
      break;
  }
  return {0.f, 0.f};
}

// CAP 0: at most 4 warps per CTA and 64 registers per thread (32 resident
// warps per SM); CAP 1: up to 8 warps and the registers the compiler wants.
template <int NP, int CAP>
__global__ void __launch_bounds__(CAP == 0 ? 128 : 256, CAP == 0 ? 8 : 1)
    amp_hs_kernel(const DevProgram P, const AmpLaunch A, const AmpConfig C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_ext = P.n_ext, NL = 1 << n_ext, H = C.H, W = C.E_cta;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int tab_stride = event_table_stride(n_ext, P.n_masks);
  // shared memory: bit-extraction table [NL][NL], bit-deposit table [NL][NL],
  // per-event tables [W][tab_stride], input-check bits [W]
  uint8_t* pext_t = smem;
  uint8_t* pdep_t = smem + NL * NL;
  size_t off = ((size_t)2 * NL * NL + 15) & ~size_t(15);
  float* tab = reinterpret_cast<float*>(smem + off);
  off += (size_t)W * tab_stride * sizeof(float);
  off = (off + 15) & ~size_t(15);
  unsigned int* evflag = reinterpret_cast<unsigned int*>(smem + off);
  for (int i = t; i < NL * NL; i += blockDim.x) {
    // pext: the bits of x at the legs of S, packed in leg order;
    // pdep: bit k of x placed at the k-th leg of S
    const uint32_t S = (uint32_t)(i / NL), x = (uint32_t)(i % NL);
    uint32_t pe = 0, pd = 0;
    int k = 0;
    for (int l = 0; l < n_ext; ++l)
      if (S >> l & 1u) {
        if (x >> l & 1u) pe |= 1u << k;
        if (x >> k & 1u) pd |= 1u << l;
        ++k;
      }
    pext_t[i] = (uint8_t)pe;
    pdep_t[i] = (uint8_t)pd;
  }
  for (int i = t; i < W; i += blockDim.x) evflag[i] = 0u;

  // helicity bits of the amplitude lanes h = lane + 32 j
  uint32_t lam[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int h = lane + 32 * j;
    uint32_t b = 0;
    if (h < H)
      for (int l = 0; l < n_ext; ++l) {
        const int8_t v = A.hel_mode == 0 ? P.hel[h * n_ext + l] : P.hel_all[h * n_ext + l];
        if (v > 0) b |= 1u << l;
      }
    lam[j] = b;
  }

  float* arena = A.slot_scratch + ((size_t)blockIdx.x * W + w) * (size_t)P.hs_arena * 8;
  const int64_t n = A.n_events;
  const int64_t n_tiles = (n + W - 1) / W;
  const float g = (float)P.g;
  const float gg = (float)(P.g * P.g);
  const HsOpWords* ops = reinterpret_cast<const HsOpWords*>(P.ops);
  const int4* hs = reinterpret_cast<const int4*>(P.hs);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t ev0 = tile * W;
    __syncthreads();  // tables filled (first tile) / the previous tile's reads done
    tile_prep<float>(P, A, tab, tab_stride, ev0, n, W, t, blockDim.x, evflag);
    __syncthreads();
    const int64_t ev = ev0 + w;
    if (ev < n) {  // warp-uniform
      const float* et = tab + (size_t)w * tab_stride;
      const float* mt = et + 8 * n_ext;
      // per pass: row maxima of |Re A|, |Im A|, cancellation mass, finiteness
      float mx_re[NP], mx_im[NP], mass[NP];
      bool finite[NP];
#pragma unroll
      for (int j = 0; j < NP; ++j) { mx_re[j] = 0.f; mx_im[j] = 0.f; mass[j] = 0.f; finite[j] = true; }
      int d_amp = 0;
      // the records of op i + 1 are loaded while op i runs
      int4 nx0 = __ldg(&ops[0].v[0]), nx1 = __ldg(&ops[0].v[1]), nxq = __ldg(hs);
      for (int i = 0; i < P.n_ops; ++i) {
        HsOpWords ow;
        ow.v[0] = nx0;
        ow.v[1] = nx1;
        HsRec q;
        q.v = nxq;
        if (i + 1 < P.n_ops) {
          nx0 = __ldg(&ops[i + 1].v[0]);
          nx1 = __ldg(&ops[i + 1].v[1]);
          nxq = __ldg(hs + i + 1);
        }
        const Op& op = ow.op;
        if (!hs_is_amp(op.type)) {
          const int nv = 1 << __popc((uint32_t)q.h.out_mask);
          for (int v = lane; v < nv; v += 32) {
            const HsInputs x{arena, pext_t, NL, q.h, (uint32_t)pdep_t[q.h.out_mask * NL + v]};
            st_var(arena, q.h.out_off + v, hs_produce(op, P, x, et, mt, g, gg));
          }
          __syncwarp();  // the variants are read by other lanes from here on
        } else {
          const float wd = __ldg(P.amp_w + d_amp);
          float* col = A.amp_out + (size_t)d_amp * A.lda;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            const int h = lane + 32 * j;
            if (h < H) {
              const HsInputs x{arena, pext_t, NL, q.h, lam[j]};
              const cx<float> amp = hs_amplitude(op, x, mt, g, gg);
              const int64_t pair = ev * H + h;
              *reinterpret_cast<float2*>(col + 2 * pair) = make_float2(amp.r, amp.i);
              const float ar = fabsf(amp.r), ai = fabsf(amp.i);
              finite[j] = finite[j] && isfinite(ar) && isfinite(ai);
              mx_re[j] = fmaxf(mx_re[j], ar);
              mx_im[j] = fmaxf(mx_im[j], ai);
              mass[j] += wd * (ar + ai);
            }
          }
          ++d_amp;
        }
      }
      const float nan = __int_as_float(0x7fc00000);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int h = lane + 32 * j;
        if (h < H) {
          const int64_t pair = ev * H + h;
          A.amp_rowmax[2 * pair] = finite[j] ? mx_re[j] : nan;
          A.amp_rowmax[2 * pair + 1] = finite[j] ? mx_im[j] : nan;
          A.pair_kappa[pair] = mass[j];  // divided by sum |J| after the colour-amplitude stage
        }
      }
      // the helicity sum runs after the colour stages: hand over the input checks
      if (lane == 0) A.ev_flags[ev] = (uint8_t)evflag[w];
    }
    if (lane == 0) evflag[w] = 0u;  // cleared before the next tile's prep (after its barrier)
  }
}

template <int CAP>
const void* hs_kernel_for_cap(int H) {
  if (H <= 32) return (const void*)amp_hs_kernel<1, CAP>;
  if (H <= 64) return (const void*)amp_hs_kernel<2, CAP>;
  if (H <= 96) return (const void*)amp_hs_kernel<3, CAP>;
  return (const void*)amp_hs_kernel<4, CAP>;
}
const void* hs_kernel_for(int H, int cap) { return cap == 0 ? hs_kernel_for_cap<0>(H) : hs_kernel_for_cap<1>(H); }
constexpr int kHsCapWarps[2] = {4, 8};  // largest warps per CTA of each register variant

template <int CAP>
void hs_launch(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {
  if (c.H <= 32) amp_hs_kernel<1, CAP><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  else if (c.H <= 64) amp_hs_kernel<2, CAP><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  else if (c.H <= 96) amp_hs_kernel<3, CAP><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  else amp_hs_kernel<4, CAP><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
}

// Split helicity sharing (helshare.h, build_split_shared): a CTA owns a tile
// of E events x H helicity lanes, as the per-lane interpreter does.  Per tile:
// phase 0 the per-event tables (tile_prep); the prologue -- every wavefunction
// of at most n_ext - 3 legs once per helicity pattern of its legs, for the E
// events, level by level with one CTA barrier per level (its threads take the
// (event, op, variant) tasks of a level in turn) -- into the per-event area
// (shared memory when ASMEM, else the CTA's region of global memory); then
// each lane runs the rest of the program for its (event, helicity): the
// currents of n_ext - 2 legs into one register-held transient, read by the
// next op, and the diagram amplitudes, written out as in the per-lane
// interpreter's amplitude-output mode.
template <bool ASMEM>
__global__ void __launch_bounds__(512) amp_hsp_kernel(const DevProgram P, const AmpLaunch A, const AmpConfig C) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_ext = P.n_ext, NL = 1 << n_ext, H = C.H, E = C.E_cta;
  const int t = threadIdx.x, L = blockDim.x;
  const int tab_stride = event_table_stride(n_ext, P.n_masks);
  const size_t area_stride = (size_t)P.hsp_area * 8;  // floats per event
  // shared memory: bit-extraction table [NL][NL], bit-deposit table [NL][NL],
  // (ASMEM) the areas [E][area][8 reals], per-event tables [E][tab_stride],
  // input-check bits [E]
  uint8_t* pext_t = smem;
  uint8_t* pdep_t = smem + NL * NL;
  size_t off = ((size_t)2 * NL * NL + 15) & ~size_t(15);
  float* area_base;
  if (ASMEM) {
    area_base = reinterpret_cast<float*>(smem + off);
    off += (size_t)E * area_stride * sizeof(float);
  } else {
    area_base = A.slot_scratch + (size_t)blockIdx.x * E * area_stride;
  }
  float* tab = reinterpret_cast<float*>(smem + off);
  off += (size_t)E * tab_stride * sizeof(float);
  off = (off + 15) & ~size_t(15);
  unsigned int* evflag = reinterpret_cast<unsigned int*>(smem + off);
  for (int i = t; i < NL * NL; i += L) {
    const uint32_t S = (uint32_t)(i / NL), x = (uint32_t)(i % NL);
    uint32_t pe = 0, pd = 0;
    int k = 0;
    for (int l = 0; l < n_ext; ++l)
      if (S >> l & 1u) {
        if (x >> l & 1u) pe |= 1u << k;
        if (x >> k & 1u) pd |= 1u << l;
        ++k;
      }
    pext_t[i] = (uint8_t)pe;
    pdep_t[i] = (uint8_t)pd;
  }
  for (int i = t; i < E; i += L) evflag[i] = 0u;

  const int e = t / H, h = t - (t / H) * H;  // this lane's (event in tile, helicity)
  const bool lane_ok = t < E * H;
  uint32_t lam = 0;
  if (lane_ok)
    for (int l = 0; l < n_ext; ++l) {
      const int8_t v = A.hel_mode == 0 ? P.hel[h * n_ext + l] : P.hel_all[h * n_ext + l];
      if (v > 0) lam |= 1u << l;
    }
  const int64_t n = A.n_events;
  const int64_t n_tiles = (n + E - 1) / E;
  const float g = (float)P.g;
  const float gg = (float)(P.g * P.g);
  const HsOpWords* all_ops = reinterpret_cast<const HsOpWords*>(P.ops);
  const int4* all_rec = reinterpret_cast<const int4*>(P.hsp_rec);
  const HsOpWords* mops = reinterpret_cast<const HsOpWords*>(P.hsp_main_ops);
  const int4* mrec = reinterpret_cast<const int4*>(P.hsp_main_rec);

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t ev0 = tile * E;
    const int e_here = (int)((n - ev0 < E) ? (n - ev0) : E);
    __syncthreads();  // tables filled (first tile) / the previous tile's reads done
    tile_prep<float>(P, A, tab, tab_stride, ev0, n, E, t, L, evflag);
    __syncthreads();
    // ---- prologue, level by level
    int begin = 0;
    for (int lv = 0; lv < P.hsp_levels; ++lv) {
      const int end = P.hsp_level_end[lv];
      const int nt = end - begin;
      for (int i = t; i < e_here * nt; i += L) {
        const int pe = i / nt;
        const uint32_t task = __ldg(P.hsp_tasks + begin + (i - pe * nt));
        const int oi = (int)(task >> 8), v = (int)(task & 0xffu);
        HsOpWords ow;
        ow.v[0] = __ldg(&all_ops[oi].v[0]);
        ow.v[1] = __ldg(&all_ops[oi].v[1]);
        HsRec q;
        q.v = __ldg(all_rec + oi);
        float* ar = area_base + (size_t)pe * area_stride;
        const float* et = tab + (size_t)pe * tab_stride;
        const HsInputs x{ar, pext_t, NL, q.h, (uint32_t)pdep_t[q.h.out_mask * NL + v]};
        st_var(ar, q.h.out_off + v, hs_produce(ow.op, P, x, et, et + 8 * n_ext, g, gg));
      }
      begin = end;
      __syncthreads();  // the level's variants are read by every lane from here on
    }
    // ---- one (event, helicity) per lane
    const int64_t ev = ev0 + e;
    if (lane_ok && e < e_here) {
      const float* et = tab + (size_t)e * tab_stride;
      const float* mt = et + 8 * n_ext;
      const float* ar = area_base + (size_t)e * area_stride;
      const int64_t pair = ev * H + h;
      float mx_re = 0.f, mx_im = 0.f, mass = 0.f;
      bool finite = true;
      int d_amp = 0;
      W4<float> tr;
      for (int k = 0; k < 4; ++k) tr.c[k] = {0.f, 0.f};
      int4 nx0 = __ldg(&mops[0].v[0]), nx1 = __ldg(&mops[0].v[1]), nxq = __ldg(mrec);
      for (int i = 0; i < P.hsp_n_main; ++i) {
        HsOpWords ow;
        ow.v[0] = nx0;
        ow.v[1] = nx1;
        HsRec q;
        q.v = nxq;
        if (i + 1 < P.hsp_n_main) {
          nx0 = __ldg(&mops[i + 1].v[0]);
          nx1 = __ldg(&mops[i + 1].v[1]);
          nxq = __ldg(mrec + i + 1);
        }
        const Op& op = ow.op;
        const HsSplitInputs x{ar, pext_t, NL, q.h, lam, tr};
        if (!hs_is_amp(op.type)) {
          tr = hs_produce(op, P, x, et, mt, g, gg);
        } else {
          const cx<float> amp = hs_amplitude(op, x, mt, g, gg);
          *reinterpret_cast<float2*>(A.amp_out + (size_t)d_amp * A.lda + 2 * pair) = make_float2(amp.r, amp.i);
          const float a_r = fabsf(amp.r), a_i = fabsf(amp.i);
          finite = finite && isfinite(a_r) && isfinite(a_i);
          mx_re = fmaxf(mx_re, a_r);
          mx_im = fmaxf(mx_im, a_i);
          mass += __ldg(P.amp_w + d_amp) * (a_r + a_i);
          ++d_amp;
        }
      }
      const float nan = __int_as_float(0x7fc00000);
      A.amp_rowmax[2 * pair] = finite ? mx_re : nan;
      A.amp_rowmax[2 * pair + 1] = finite ? mx_im : nan;
      A.pair_kappa[pair] = mass;  // divided by sum |J| after the colour-amplitude stage
    }
    __syncthreads();
    if (t < E) {
      // the helicity sum runs after the colour stages: hand over the input checks
      if (t < e_here) A.ev_flags[ev0 + t] = (uint8_t)evflag[t];
      evflag[t] = 0u;
    }
  }
}

}  // namespace

bool hs_supported(const DevProgram& p, bool fp64, int H) {
  return !fp64 && p.hs != nullptr && p.hs_arena > 0 && p.n_colour == 0 && H >= 1 && H <= 128 && p.n_ext <= 7;
}

size_t hs_smem_bytes(const DevProgram& p, int warps) {
  const int NL = 1 << p.n_ext;
  size_t b = ((size_t)2 * NL * NL + 15) & ~size_t(15);
  b += (size_t)warps * event_table_stride(p.n_ext, p.n_masks) * sizeof(float);
  b = (b + 15) & ~size_t(15);
  return b + (size_t)warps * sizeof(unsigned int) + 16;
}

size_t hs_arena_bytes(const DevProgram& p, const AmpConfig& c) {
  return (size_t)c.grid * c.E_cta * (size_t)p.hs_arena * 8 * sizeof(float);
}

// CTAs of W warps that registers, threads and shared memory allow on one SM
// (the kernel's register count is read with cudaFuncGetAttributes; nothing
// is changed).
int hs_resident(const DevProgram& p, int H, int cap, int warps, size_t smem_per_sm) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, hs_kernel_for(H, cap)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int regs_warp = ((std::max(fa.numRegs, 1) + 7) / 8) * 8 * 32;
  const int by_regs = 65536 / std::max(regs_warp * warps, 1);
  const size_t sm = hs_smem_bytes(p, warps) + 1024;
  const int by_smem = (int)(smem_per_sm / sm);
  return std::max(0, std::min({by_regs, by_smem, 2048 / (warps * 32), 32}));
}

std::vector<AmpConfig> hs_candidates(const DevProgram& p, int H, int num_sms, size_t max_smem,
                                     size_t smem_per_sm) {
  // 64 registers: 2 or 4 warps per CTA; uncapped: 4 or 8; at full and half
  // residency
  std::vector<AmpConfig> out;
  for (int cap = 0; cap < 2; ++cap)
    for (int W : {2, 4, 8}) {
      if (W > kHsCapWarps[cap] || W < kHsCapWarps[cap] / 2) continue;
      const size_t sm = hs_smem_bytes(p, W);
      if (sm > max_smem) continue;
      const int res = hs_resident(p, H, cap, W, smem_per_sm);
      if (res < 1) continue;
      int prev = 0;
      for (int k : {res, res / 2}) {
        if (k < 1 || k == prev) continue;
        prev = k;
        AmpConfig c;
        c.H = H;
        c.E_cta = W;
        c.threads = 32 * W;
        c.smem = sm;
        c.jamp_in_smem = true;
        c.slots_in_smem = false;
        c.helshare = true;
        c.regvar = cap;
        c.per_sm = k;
        c.grid = k * num_sms;
        out.push_back(c);
      }
    }
  return out;
}

AmpConfig hs_plan(const DevProgram& p, int H, int num_sms, size_t max_smem, size_t smem_per_sm) {
  // the uncapped variant (the tuner's choice on every process measured), four
  // warps per CTA, as many CTAs per SM as can be resident
  std::vector<AmpConfig> c = hs_candidates(p, H, num_sms, max_smem, smem_per_sm);
  for (const AmpConfig& x : c)
    if (x.regvar == 1 && x.E_cta == 4) return x;
  if (!c.empty()) return c.front();
  AmpConfig none;
  none.grid = 0;
  return none;
}

// ---- split evaluation (amp_hsp_kernel)
bool hsp_supported(const DevProgram& p, bool fp64, int H) {
  return !fp64 && p.hsp_main_ops != nullptr && p.hsp_area > 0 && p.n_colour == 0 && H >= 1 && H <= 512 &&
         p.n_ext <= 7;
}

size_t hsp_smem_bytes(const DevProgram& p, int events, bool area_in_smem) {
  const int NL = 1 << p.n_ext;
  size_t b = ((size_t)2 * NL * NL + 15) & ~size_t(15);
  if (area_in_smem) b += (size_t)events * p.hsp_area * 8 * sizeof(float);
  b += (size_t)events * event_table_stride(p.n_ext, p.n_masks) * sizeof(float);
  b = (b + 15) & ~size_t(15);
  return b + (size_t)events * sizeof(unsigned int) + 16;
}

size_t hsp_area_bytes(const DevProgram& p, const AmpConfig& c) {
  return c.slots_in_smem ? 0 : (size_t)c.grid * c.E_cta * (size_t)p.hsp_area * 8 * sizeof(float);
}

std::vector<AmpConfig> hsp_candidates(const DevProgram& p, int H, int num_sms, size_t max_smem,
                                      size_t smem_per_sm) {
  std::vector<AmpConfig> out;
  for (int sm_area = 1; sm_area >= 0; --sm_area) {
    const void* k = sm_area ? (const void*)amp_hsp_kernel<true> : (const void*)amp_hsp_kernel<false>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    int last_threads = -1;
    for (int E = 1; E * H <= 512; ++E) {
      const int threads = ((E * H + 31) / 32) * 32;
      // the largest E for each thread count (fewest idle lanes)
      if ((E + 1) * H <= 512 && (((E + 1) * H + 31) / 32) * 32 == threads) continue;
      if (threads == last_threads) continue;
      last_threads = threads;
      const size_t sm = hsp_smem_bytes(p, E, sm_area != 0);
      if (sm > max_smem) break;
      const int warps = threads / 32;
      const int regs_warp = ((std::max(fa.numRegs, 1) + 7) / 8) * 8 * 32;
      const int res = std::min({65536 / std::max(regs_warp * warps, 1), (int)(smem_per_sm / (sm + 1024)),
                                2048 / threads, 32});
      if (res < 1) continue;
      int prev = 0;
      for (int r : {res, res / 2}) {
        if (r < 1 || r == prev) continue;
        prev = r;
        AmpConfig c;
        c.H = H;
        c.E_cta = E;
        c.threads = threads;
        c.smem = sm;
        c.jamp_in_smem = true;
        c.slots_in_smem = sm_area != 0;  // the prologue area in shared memory
        c.hsplit = true;
        c.per_sm = r;
        c.grid = r * num_sms;
        out.push_back(c);
      }
    }
  }
  return out;
}

cudaError_t launch_amp_hsp(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {
  if (!hsp_supported(p, false, c.H) || !a.amp_out || (!c.slots_in_smem && !a.slot_scratch) || a.event_list ||
      a.hel_mode == 2)
    return cudaErrorInvalidValue;
  if (c.threads < 32 || c.threads > 512 || c.threads % 32 != 0 || c.E_cta < 1 || c.E_cta * c.H > c.threads ||
      c.smem != hsp_smem_bytes(p, c.E_cta, c.slots_in_smem))
    return cudaErrorInvalidConfiguration;
  const void* k = c.slots_in_smem ? (const void*)amp_hsp_kernel<true> : (const void*)amp_hsp_kernel<false>;
  cudaError_t e = ensure_dynamic_smem(k, c.smem);
  if (e != cudaSuccess) return e;
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_percent(c)) != cudaSuccess)
    cudaGetLastError();
  if (c.slots_in_smem) amp_hsp_kernel<true><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  else amp_hsp_kernel<false><<<c.grid, c.threads, c.smem, s>>>(p, a, c);
  return cudaGetLastError();
}

cudaError_t launch_amp_hs(const DevProgram& p, const AmpConfig& c, const AmpLaunch& a, cudaStream_t s) {
  if (!hs_supported(p, false, c.H) || !a.amp_out || !a.slot_scratch || a.event_list || a.hel_mode == 2)
    return cudaErrorInvalidValue;
  if (c.regvar < 0 || c.regvar > 1 || c.E_cta < 1 || c.E_cta > kHsCapWarps[c.regvar] || c.threads != 32 * c.E_cta)
    return cudaErrorInvalidConfiguration;
  const void* k = hs_kernel_for(c.H, c.regvar);
  cudaError_t e = ensure_dynamic_smem(k, c.smem);
  if (e != cudaSuccess) return e;
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, carveout_percent(c)) != cudaSuccess)
    cudaGetLastError();
  if (c.regvar == 0) hs_launch<0>(p, c, a, s);
  else hs_launch<1>(p, c, a, s);
  return cudaGetLastError();
}

}  // namespace mea

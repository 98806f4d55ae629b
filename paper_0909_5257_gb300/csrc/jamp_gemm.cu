// Colour amplitudes J_alpha = sum_d c_{alpha d} A_d (Eq. (color-amplitude))
// as an exact integer contraction on the tensor cores.
//
// The amplitude kernel writes every Feynman-diagram amplitude A_d of every
// (event, helicity) pair in FP32.  All colour coefficients of the processes
// handled here are real, c = cfac * n with small integers n.  Per row r (the
// real or the imaginary parts of one pair) the amplitudes are scaled by a
// power of two, x = A * 2^(q - e_r) with 2^(e_r - 1) <= max_d |A_rd| < 2^e_r,
// so that |x| < 2^q, and split into three integer digits
//     x = h + m 2^-(q+1) + l 2^-2(q+1) + O(2^-(2q+3)),   |h|, |m|, |l| <= 2^q,
// each exact in FP16 (q <= 11).  tcgen05.mma kind::f16 then forms
// H = sum_d n_d h_d, M = sum_d n_d m_d, L = sum_d n_d l_d in three FP32
// tensor-memory accumulators over the whole diagram sum: every product and
// every partial sum is an integer below sum_d |n_{alpha d}| 2^q < 2^24, so the
// accumulation is exact whatever order or internal rounding the tensor core
// uses.  The epilogue recombines cfac * 2^(e_r - q) (H + M 2^-(q+1) +
// L 2^-2(q+1)) with two FP32 FMAs (within an ulp of the exact value).  The
// only other error is the digit truncation, below 2^-(3q+3) of the row
// maximum: the colour amplitudes come out as the FP32-rounded exact sum of the
// FP32 diagram amplitudes (the compensated summation of the paper's Sec. 3.2
// step 3 with nothing left to compensate).
//
// Tile: 128 rows (64 pairs) x nc colour columns, K in chunks of 64 diagrams,
// two shared-memory stages so that the digit conversion of chunk k+1 overlaps
// the MMAs of chunk k.  Every wait is bounded; on expiry the kernel records an
// error in *status, drains its MMAs with one more bounded wait, frees its
// tensor memory and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <numeric>

#include "jamp_gemm.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace mea {
namespace {

using namespace tc;

constexpr int kThreads = 512;  // 16 warps convert; warps 0..3 own TMEM lanes 0..127 in the epilogue
constexpr int kTileVec = kThreads >= 1024 ? 1 : 1024 / kThreads;  // 16-byte tile vectors per thread (nc <= 128)
constexpr int kM = 128;
constexpr int kKC = 64;
constexpr int kStageA = kM * kKC * 2;  // one FP16 digit plane of A
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMaxNC = 128;            // 3 accumulators of nc columns in 512 TMEM columns; 4 tile vectors per thread

__host__ __device__ constexpr size_t stage_bytes(int nc) { return (size_t)3 * kStageA + (size_t)nc * kKC * 2; }

__global__ void __launch_bounds__(kThreads) jamp_gemm_kernel(JampGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int NC = g.nc;
  const size_t SB = stage_bytes(NC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SB);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);
  float* rscale = reinterpret_cast<float*>(tslot + 4);  // [128] 2^(q - e_r)
  float* rowabs = rscale + kM;                          // [128] sum |J| of the row in this split

  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(3 * NC)) tmem_cols <<= 1;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) tmem_alloc(tslot, tmem_cols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t d_h = tmem, d_m = tmem + (uint32_t)NC, d_l = tmem + (uint32_t)(2 * NC);

  uint32_t phase[2] = {0u, 0u};
  int outstanding[2] = {0, 0};  // commits on each stage's barrier not yet waited for
  const int64_t n_rows = 2 * g.n_pairs;
  const int64_t n_mt = (n_rows + kM - 1) / kM;
  const int n_kc = g.kpad / kKC;
  const uint32_t idesc = make_idesc(kM, NC);
  const float w1 = ldexpf(1.f, g.q + 1);  // digit base
  const float inv_w1 = 1.f / w1, inv_w2 = inv_w1 * inv_w1;  // powers of two

  auto wait_stage = [&](int st) {
    if (outstanding[st] == 0) return;
    if (!*abort_flag) {
      if (!mbar_wait(&bar[st], phase[st])) {
        atomicExch(abort_flag, 1);
        if (g.status) atomicExch(g.status, 1);
        return;  // left outstanding: drained once more before TMEM is freed
      }
    } else {
      return;
    }
    phase[st] ^= 1u;
    outstanding[st] = 0;
  };

  for (int64_t w = blockIdx.x; w < n_mt * g.n_splits; w += gridDim.x) {
    const int64_t mt = w / g.n_splits;
    const int split = (int)(w - mt * g.n_splits);
    const int64_t row0 = mt * kM;
    const int n0 = split * NC;
    if (t < kM) {
      const int64_t r = row0 + t;
      float mx = (r < n_rows) ? g.rowmax[r] : 0.f;
      float sc;
      if (!isfinite(mx)) {
        sc = __int_as_float(0x7fc00000);  // a non-finite row stays non-finite (flagged later)
      } else {
        int e = 0;
        if (mx > 0.f) frexpf(mx, &e);
        sc = ldexpf(1.f, max(-120, min(120, g.q - e)));
      }
      rscale[t] = sc;
      rowabs[t] = 0.f;
    }
    __syncthreads();

    // Register prefetch: each thread holds its 2 x 8 amplitudes of the next
    // two chunks (two buffers, used alternately) and the coefficient-tile
    // vectors of the next chunk; a chunk's loads are issued right after the
    // buffer they replace is converted, so they have two chunks' time to land.
    const int row = t & (kM - 1);
    const int64_t r = row0 + row;
    const bool row_ok = r < n_rows;
    typedef float ABuf[kKC / 8 / (kThreads / kM)][8];
    ABuf pa0, pa1;  // amplitudes of the chunks two apart: prefetched two chunks ahead
    uint4 pb[kTileVec];
    const int nb = NC * kKC / 8;  // 16-byte vectors per coefficient tile
    const float* arow = g.A + r;
    auto prefetch_a = [&](int kc, ABuf& pa) {
      const bool full = (kc + 1) * kKC <= g.kd;
#pragma unroll
      for (int j = 0; j < kKC / 8 / (kThreads / kM); ++j) {
        const int kg = (t >> 7) + j * (kThreads / kM);
        const float* src = arow + (size_t)(kc * kKC + kg * 8) * g.lda;
        if (full) {
#pragma unroll
          for (int i = 0; i < 8; ++i) pa[j][i] = row_ok ? __ldg(src + (size_t)i * g.lda) : 0.f;
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int d = kc * kKC + kg * 8 + i;
            pa[j][i] = (row_ok && d < g.kd) ? __ldg(src + (size_t)i * g.lda) : 0.f;
          }
        }
      }
    };
    auto prefetch_b = [&](int kc) {
      const uint4* src = reinterpret_cast<const uint4*>(g.tiles + ((size_t)split * n_kc + kc) * NC * kKC);
#pragma unroll
      for (int j = 0; j < kTileVec; ++j) {
        const int i = t + j * kThreads;
        if (i < nb) pb[j] = __ldg(src + i);
      }
    };
    prefetch_a(0, pa0);
    if (n_kc > 1) prefetch_a(1, pa1);
    prefetch_b(0);
    auto step = [&](int kc, ABuf& pa) {
      const int st = kc & 1;
      wait_stage(st);  // the MMAs that read this stage two chunks ago are done
      unsigned char* a_h = smem + st * SB;
      unsigned char* a_m = a_h + kStageA;
      unsigned char* a_l = a_m + kStageA;
      unsigned char* b_t = a_l + kStageA;
      // A digits: thread -> (row, 8 consecutive diagrams); global reads are
      // coalesced over rows, shared stores are whole 16-byte core-matrix rows
      {
        const float sc = rscale[row];
#pragma unroll
        for (int j = 0; j < kKC / 8 / (kThreads / kM); ++j) {
          const int kg = (t >> 7) + j * (kThreads / kM);
          __align__(16) __half2 hv[4], mv[4], lv[4];
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            float h[2], mm[2], l[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              // x = a sc, r1 = (x - h) w1, r2 = (r1 - m) w1: every product by
              // the powers of two sc and w1 and every difference of a value and
              // its nearest integer is exact, so each FMA below rounds once,
              // where adding 1.5 * 2^23 rounds to the nearest integer
              const float a = pa[j][i + u];
              h[u] = __fsub_rn(__fmaf_rn(a, sc, kRoundMagic), kRoundMagic);
              const float y1 = __fmaf_rn(a, sc, -h[u]);  // x - h
              mm[u] = __fsub_rn(__fmaf_rn(y1, w1, kRoundMagic), kRoundMagic);
              const float y2 = __fmaf_rn(y1, w1, -mm[u]);  // r1 - m
              l[u] = __fsub_rn(__fmaf_rn(y2, w1, kRoundMagic), kRoundMagic);
            }
            // integers of at most 2^q <= 2048 in magnitude: exact in FP16
            hv[i / 2] = __floats2half2_rn(h[0], h[1]);
            mv[i / 2] = __floats2half2_rn(mm[0], mm[1]);
            lv[i / 2] = __floats2half2_rn(l[0], l[1]);
          }
          const uint32_t off = canon_off(row, kg * 8, kKC);
          *reinterpret_cast<uint4*>(a_h + off) = *reinterpret_cast<const uint4*>(hv);
          *reinterpret_cast<uint4*>(a_m + off) = *reinterpret_cast<const uint4*>(mv);
          *reinterpret_cast<uint4*>(a_l + off) = *reinterpret_cast<const uint4*>(lv);
        }
      }
      // B: the precomputed canonical tile of coefficient integers
      {
        uint4* dst = reinterpret_cast<uint4*>(b_t);
#pragma unroll
        for (int j = 0; j < kTileVec; ++j) {
          const int i = t + j * kThreads;
          if (i < nb) dst[i] = pb[j];
        }
      }
      if (kc + 2 < n_kc) prefetch_a(kc + 2, pa);
      if (kc + 1 < n_kc) prefetch_b(kc + 1);
      fence_async_smem();
      fence_before();
      __syncthreads();
      fence_after();
      if (!*abort_flag) {
        if (t == 0) {
          const uint32_t lbo = 128, sbo = (kKC / 8) * 128;
          for (int ks = 0; ks < kKC / 16; ++ks) {
            const uint32_t koff = (uint32_t)(ks * 2 * 128);
            const uint64_t db = make_desc(smem_u32(b_t) + koff, lbo, sbo);
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_f16(d_l, make_desc(smem_u32(a_l) + koff, lbo, sbo), db, idesc, acc);
            mma_f16(d_m, make_desc(smem_u32(a_m) + koff, lbo, sbo), db, idesc, acc);
            mma_f16(d_h, make_desc(smem_u32(a_h) + koff, lbo, sbo), db, idesc, acc);
          }
          mma_commit(&bar[st]);
        }
        outstanding[st] = 1;
      }
    };
    for (int kc = 0; kc < n_kc; kc += 2) {
      step(kc, pa0);
      if (kc + 1 < n_kc) step(kc + 1, pa1);
    }
    // all MMAs of this tile: the last chunk's commit covers every earlier one,
    // but each barrier's phases are consumed in order
    if (n_kc >= 2) wait_stage((n_kc - 2) & 1);
    wait_stage((n_kc - 1) & 1);
    fence_after();
    if (warp < 4 && !*abort_flag) {
      const int64_t r = row0 + t;
      const float back = (float)g.cfac / rscale[t];  // cfac (1 or 2) times a power of two
      const uint32_t lane = (uint32_t)(warp * 32) << 16;
      float* jrow = g.J + (size_t)r * g.ldj;
      float sabs = 0.f;
      for (int c0 = 0; c0 < NC && n0 + c0 < g.m; c0 += 16) {
        float vh[16], vm[16], vl[16];
        tmem_ld16(d_h + lane + (uint32_t)c0, vh);
        tmem_ld16(d_m + lane + (uint32_t)c0, vm);
        tmem_ld16(d_l + lane + (uint32_t)c0, vl);
        if (r < n_rows) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int a = n0 + c0 + i;
            if (a < g.m) {
              // h + m/2^(q+1) + l/2^2(q+1): the inner FMA is exact up to one rounding and the
              // l term lies below the last digit of m, so v is within an ulp of the exact sum
              const float v = fmaf(vl[i], inv_w2, fmaf(vm[i], inv_w1, vh[i])) * back;
              jrow[a] = v;
              sabs += fabsf(v);
            }
          }
        }
      }
      rowabs[t] = sabs;
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (t < kM / 2 && g.jabs) {
      const int64_t p = row0 / 2 + t;
      if (p < g.n_pairs) g.jabs[(size_t)split * g.n_pairs + p] = rowabs[2 * t] + rowabs[2 * t + 1];
    }
  }
  // an expired wait: one more bounded wait for each stage's MMAs before the
  // tensor memory they write is released
  for (int st = 0; st < 2; ++st)
    if (outstanding[st]) mbar_wait(&bar[st], phase[st]);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

}  // namespace

JampMap build_jamp_map(const Program& p) {
  JampMap M;
  M.m = p.n_jamp;
  int kd = 0;
  int g = 0;
  bool real = true;
  for (const Op& op : p.ops) {
    if (!is_amp_op(op.type)) continue;
    ++kd;
    for (uint32_t k = 0; k < op.col_count; ++k) {
      const ColEntry& c = p.col[op.col_begin + k];
      if (c.im != 0) real = false;
      g = std::gcd(g, std::abs((int)c.re));
    }
  }
  M.kd = kd;
  if (!real || kd == 0 || M.m <= 0 || g == 0) return M;
  M.cfac = g;
  M.nc = std::min(kMaxNC, ((M.m + 15) / 16) * 16);
  M.n_splits = (M.m + M.nc - 1) / M.nc;
  // balance the splits: the smallest multiple of 16 that still needs n_splits
  M.nc = std::min(M.nc, (((M.m + M.n_splits - 1) / M.n_splits) + 15) / 16 * 16);
  M.kpad = ((kd + kKC - 1) / kKC) * kKC;
  std::vector<int> colw(M.m, 0);
  M.weight.assign(kd, 0.f);
  const int n_kc = M.kpad / kKC;
  M.tiles.assign((size_t)M.n_splits * n_kc * M.nc * kKC, __float2half(0.f));
  int d = 0;
  for (const Op& op : p.ops) {
    if (!is_amp_op(op.type)) continue;
    for (uint32_t k = 0; k < op.col_count; ++k) {
      const ColEntry& c = p.col[op.col_begin + k];
      const int n = c.re / g;
      const int a = c.alpha;
      colw[a] += std::abs(n);
      M.weight[d] += (float)std::abs((int)c.re);
      const int split = a / M.nc, row = a - split * M.nc;
      const int kc = d / kKC, kk = d - kc * kKC;
      __half* tile = M.tiles.data() + ((size_t)split * n_kc + kc) * M.nc * kKC;
      const float prev = __half2float(*reinterpret_cast<__half*>(reinterpret_cast<char*>(tile) + tc::canon_off(row, kk, kKC)));
      *reinterpret_cast<__half*>(reinterpret_cast<char*>(tile) + tc::canon_off(row, kk, kKC)) =
          __float2half((float)(prev + n));
    }
    ++d;
  }
  const int wmax = *std::max_element(colw.begin(), colw.end());
  // exact accumulation: sum_d |n_{alpha d}| 2^q < 2^24 for every alpha, and 2^q <= 2048 (FP16 integers)
  int q = 11;
  while (q > 0 && (double)wmax * std::ldexp(1.0, q) >= 16777216.0) --q;
  M.q = q;
  // every tile entry must itself be a small integer (coefficients of one diagram in one colour add up)
  for (const __half& h : M.tiles)
    if (std::fabs(__half2float(h)) > 2048.f) return M;
  M.ok = q >= 8;  // digit truncation below 2^-27 of the row maximum
  return M;
}

size_t jamp_gemm_smem(int nc) { return 2 * stage_bytes(nc) + 16 + 16 + (size_t)kM * 8 + 16; }

cudaError_t launch_jamp_gemm(const JampGemmArgs& a, int num_sms, cudaStream_t s) {
  if (a.n_pairs <= 0) return cudaSuccess;
  if (a.nc < 16 || a.nc > kMaxNC || a.nc % 16 != 0 || a.kpad % kKC != 0) return cudaErrorInvalidValue;
  const size_t sm = jamp_gemm_smem(a.nc);
  cudaError_t e = ensure_dynamic_smem((const void*)jamp_gemm_kernel, sm);
  if (e != cudaSuccess) return e;
  const int64_t work = ((2 * a.n_pairs + kM - 1) / kM) * a.n_splits;
  int tmem = 32;
  while (tmem < 3 * a.nc) tmem *= 2;
  int per_sm = std::max(1, std::min<int>(512 / tmem, (int)((227u << 10) / sm)));
  const int grid = (int)std::min<int64_t>(work, (int64_t)num_sms * per_sm);
  jamp_gemm_kernel<<<grid, kThreads, sm, s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

}  // namespace mea

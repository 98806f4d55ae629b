// Colour contraction on the tensor cores (Eq. (color-averaged-amplitude)):
// for every (event, helicity) pair p with colour amplitudes J_p (FP32, from
// the colour-amplitude stage)
//     val_p = 1/D * sum_{ab} J_a K_ab J_b^*  =  1/D * [ Jr.(K Jr) + Ji.(K Ji) ]
// with the integer colour matrix K (N = K / D).  The rows (Jr, Ji) of 64 pairs
// form the M = 128 rows of one tile; Z = J K runs as tcgen05.mma kind::f16
// with FP32 accumulation in tensor memory:
//   * each row is scaled by a power of two and split J = J_hi + J_mid + J_lo
//     into three FP16 parts (33 significant bits together, more than FP32's 24);
//   * K is an integer matrix; it is split K = K_hi + K_lo with K_hi = fp16(K)
//     (exact when |K| <= 2048, then K_lo = 0 and those products are skipped);
//   * Z = (J_hi + J_mid + J_lo) K_hi + (J_hi + J_mid) K_lo with FP32
//     accumulation in tensor memory, restarted for every 64-wide K chunk: the
//     tensor core's FP32 accumulation is biased over long sums (measured: a
//     systematic 2e-6 relative shift of |M|^2 at m = 720 when one accumulator
//     spans all of K), so each chunk's partial Z is read out (tcgen05.ld) and
//     sum_a J_a Z_a is accumulated across chunks against the unscaled FP32 J
//     with the compensated dot product Dot2 in FP32 (twice the working
//     precision; the FP64 pipe of this part is 64 times slower), after which
//     the row scale is undone.
// Pipeline (one iteration per (column block, K chunk)): the J chunk of the
// next iteration is prefetched into registers and its K tiles copied
// asynchronously (cp.async) into the other shared-memory stage while the
// tensor core works; the MMAs of iteration i write one of two tensor-memory
// buffers while the epilogue of iteration i-1 reads the other.  Operands are
// staged in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices); the K tiles are laid out that way once per process
// (build_colour_tiles).  Every wait is bounded: on expiry the kernel records an
// error in *status, drains its own MMAs with a bounded wait, frees its tensor
// memory and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "colour_gemm.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace mea {
namespace {

using namespace tc;

constexpr int kThreads = 256;  // 8 warps convert; warps w and w+4 share TMEM lanes 32(w%4).. in the epilogue
constexpr int kM = 128;        // tile rows (64 pairs x {re, im})
constexpr int kKC = 64;        // K elements per stage
constexpr int kPlaneA = kM * kKC * 2;

__host__ __device__ constexpr size_t stage_bytes(int nc) { return (size_t)3 * kPlaneA + (size_t)2 * nc * kKC * 2; }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared (TMA), completing `bytes` on the mbarrier
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) colour_gemm_kernel(ColourGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int NC = g.nc;
  const size_t SB = stage_bytes(NC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SB);  // [2] MMA commits of the two TMEM buffers
  uint64_t* kbar = bar + 2;                                      // [2] K tiles landed in each stage
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);
  float* rscale = reinterpret_cast<float*>(tslot + 4);           // [128] per-row scale 2^-e
  // scratch that lives in stage 1's first operand plane while no MMA reads it:
  // row-maximum halves at the start of a tile, per-(row, half) values at its end
  float* rmax = reinterpret_cast<float*>(smem + SB);                     // [256]
  double* part = reinterpret_cast<double*>(smem + SB + kThreads * 4);    // [256]

  {
    // the layout above must fit the dynamic shared memory of this launch
    uint32_t dyn = 0;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if ((size_t)dyn < (size_t)(reinterpret_cast<unsigned char*>(rscale + kM) - smem)) {
      if (t == 0 && g.status) atomicExch(g.status, 2);
      return;  // before any barrier, copy or tensor-memory use
    }
  }
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(2 * NC)) tmem_cols <<= 1;
  uint32_t kphase[2] = {0u, 0u};  // thread 0: next phase of each stage's K-tile barrier
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&kbar[0], 1);
    mbar_init(&kbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) tmem_alloc(tslot, tmem_cols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  uint32_t phase[2] = {0u, 0u};
  int outstanding[2] = {0, 0};
  const int m = g.m, ldj = g.ldj;
  const int64_t n_rows = 2 * g.n_pairs;
  const int64_t n_tiles = (n_rows + kM - 1) / kM;
  const int n_kc = g.kp / kKC, n_nb = g.np / NC;
  const int n_it = n_kc * n_nb;
  const uint32_t idesc = make_idesc(kM, NC);
  const bool use_blo = g.b_lo != nullptr;
  const int row = t & (kM - 1);
  const int half = t >> 7;  // conversion: k groups of this thread; epilogue: column half

  auto wait_buf = [&](int b) -> bool {
    if (!outstanding[b]) return true;
    if (*abort_flag) return false;
    if (!mbar_wait(&bar[b], phase[b])) {
      atomicExch(abort_flag, 1);
      if (g.status) atomicExch(g.status, 1);
      return false;  // left outstanding: drained once more before TMEM is freed
    }
    phase[b] ^= 1u;
    outstanding[b] = 0;
    return true;
  };

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kM;
    const int64_t r = row0 + row;
    const bool row_ok = r < n_rows;
    const float* jrow = g.J + r * ldj;
    // J is read in 16-byte vectors of one row: the row starts are 16-byte
    // aligned (ldj is a multiple of 16, checked at launch), and a vector that
    // starts below m ends within the row (at most ldj); entries at m and
    // beyond are never used
    const float4* jrow4 = reinterpret_cast<const float4*>(jrow);
    // per-row power-of-two scale so that the largest |J| lands near 2^14
    {
      float mx = 0.f;
      if (row_ok)
        for (int k4 = half; 4 * k4 < m; k4 += 2) {
          const float4 v = jrow4[k4];
          const int k = 4 * k4;
          mx = fmaxf(mx, fabsf(v.x));
          if (k + 1 < m) mx = fmaxf(mx, fabsf(v.y));
          if (k + 2 < m) mx = fmaxf(mx, fabsf(v.z));
          if (k + 3 < m) mx = fmaxf(mx, fabsf(v.w));
        }
      rmax[t] = mx;
      __syncthreads();
      if (t < kM) {
        mx = fmaxf(rmax[t], rmax[t + kM]);
        int e = 0;
        if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);
        rscale[t] = ldexpf(1.f, max(-120, min(120, 14 - e)));
      }
      __syncthreads();
    }
    const float sc = rscale[row];
    float acc_hi = 0.f, acc_lo = 0.f;  // Dot2 of this thread's (row, column half)
    float pj[4][8];                    // prefetched J chunk: 4 groups of 8 columns

    auto prefetch = [&](int it) {
      const int kc = it % n_kc;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk0 = kc * kKC + (half + 2 * j) * 8;
        float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
        if (row_ok && kk0 < m) {
          v0 = jrow4[kk0 / 4];
          v1 = jrow4[kk0 / 4 + 1];
        }
        const float v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i) pj[j][i] = (kk0 + i < m) ? v[i] : 0.f;
      }
    };
    // K tiles of iteration it into stage st: one thread issues 1-D bulk copies
    // (TMA) of the precomputed contiguous tiles, completing on kbar[st]; the
    // stage's previous MMAs were waited for (epilogue of it-1, same thread)
    auto copy_tiles = [&](int it, int st) {
      if (t != 0 || *abort_flag) return;
      const int nb = it / n_kc, kc = it % n_kc;
      unsigned char* b_hi = smem + st * SB + 3 * kPlaneA;
      unsigned char* b_lo = b_hi + (size_t)NC * kKC * 2;
      const size_t tile_off = ((size_t)nb * n_kc + kc) * NC * kKC;
      const uint32_t bytes = (uint32_t)(NC * kKC * 2);
      mbar_expect_tx(&kbar[st], use_blo ? 2 * bytes : bytes);
      bulk_g2s(b_hi, g.b_hi + tile_off, bytes, &kbar[st]);
      if (use_blo) bulk_g2s(b_lo, g.b_lo + tile_off, bytes, &kbar[st]);
    };
    // epilogue of iteration it (buffer it % 2): this thread's row, its half of the columns
    auto epilogue = [&](int it) {
      const int b = it & 1;
      if (!wait_buf(b)) return;
      fence_after();
      const int n0 = (it / n_kc) * NC;
      const uint32_t lane = (uint32_t)((warp & 3) * 32) << 16;
      const uint32_t base = tmem + (uint32_t)(b * NC) + lane;
      for (int c0 = half * (NC / 2); c0 < (half + 1) * (NC / 2); c0 += 16) {
        float jvals[16];
        {
          float4 v[4] = {};
          if (row_ok && n0 + c0 < m) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = jrow4[(n0 + c0) / 4 + q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            jvals[4 * q] = v[q].x;
            jvals[4 * q + 1] = v[q].y;
            jvals[4 * q + 2] = v[q].z;
            jvals[4 * q + 3] = v[q].w;
          }
        }
        float z[16];
        tmem_ld16(base + (uint32_t)c0, z);
        if (row_ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int a = n0 + c0 + i;
            if (a < m) {
              // Dot2 (Ogita, Rump, Oishi 2005): exact product error by FMA,
              // two-sum of the running value, errors collected in acc_lo
              const float jv = jvals[i];
              const float p = __fmul_rn(jv, z[i]);
              const float pe = fmaf(jv, z[i], -p);
              const float s = __fadd_rn(acc_hi, p);
              const float bb = __fsub_rn(s, acc_hi);
              const float se = __fadd_rn(__fsub_rn(acc_hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
              acc_hi = s;
              acc_lo = __fadd_rn(acc_lo, __fadd_rn(se, pe));
            }
          }
        }
      }
      fence_before();
    };

    prefetch(0);
    copy_tiles(0, 0);
    for (int it = 0; it < n_it; ++it) {
      const int st = it & 1;
      unsigned char* a_hi = smem + st * SB;
      unsigned char* a_mid = a_hi + kPlaneA;
      unsigned char* a_lo = a_mid + kPlaneA;
      unsigned char* b_hi = a_lo + kPlaneA;
      unsigned char* b_lo = b_hi + (size_t)NC * kKC * 2;
      // J digits into this stage (free: its MMAs, iteration it-2, were waited
      // for by the epilogue of it-2 during iteration it-1)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kg = half + 2 * j;
        __align__(16) __half hv[8], mv[8], lv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float x = __fmul_rn(pj[j][i], sc);
          const __half h = __float2half_rn(x);
          const float r1 = __fsub_rn(x, __half2float(h));
          const __half md = __float2half_rn(r1);
          hv[i] = h;
          mv[i] = md;
          lv[i] = __float2half_rn(__fsub_rn(r1, __half2float(md)));
        }
        const uint32_t off = canon_off(row, kg * 8, kKC);
        *reinterpret_cast<uint4*>(a_hi + off) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(a_mid + off) = *reinterpret_cast<const uint4*>(mv);
        *reinterpret_cast<uint4*>(a_lo + off) = *reinterpret_cast<const uint4*>(lv);
      }
      fence_async_smem();
      fence_before();
      __syncthreads();
      fence_after();
      if (t == 0 && !*abort_flag) {
        // this stage's K tiles
        if (!mbar_wait(&kbar[st], kphase[st])) {
          atomicExch(abort_flag, 1);
          if (g.status) atomicExch(g.status, 1);
        }
        kphase[st] ^= 1u;
      }
      if (!*abort_flag) {
        if (t == 0) {
          const uint32_t lbo = 128, sbo = (kKC / 8) * 128;
          const uint32_t d = tmem + (uint32_t)(st * NC);
          for (int ks = 0; ks < kKC / 16; ++ks) {
            const uint32_t koff = (uint32_t)(ks * 2 * 128);
            const uint64_t dah = make_desc(smem_u32(a_hi) + koff, lbo, sbo);
            const uint64_t dam = make_desc(smem_u32(a_mid) + koff, lbo, sbo);
            const uint64_t dal = make_desc(smem_u32(a_lo) + koff, lbo, sbo);
            const uint64_t dbh = make_desc(smem_u32(b_hi) + koff, lbo, sbo);
            const uint64_t dbl = make_desc(smem_u32(b_lo) + koff, lbo, sbo);
            const uint32_t first = (ks == 0) ? 0u : 1u;  // fresh accumulator for every K chunk
            // smallest terms first
            mma_f16(d, dal, dbh, idesc, first);
            if (use_blo) {
              mma_f16(d, dam, dbl, idesc, 1u);
              mma_f16(d, dah, dbl, idesc, 1u);
            }
            mma_f16(d, dam, dbh, idesc, 1u);
            mma_f16(d, dah, dbh, idesc, 1u);
          }
          mma_commit(&bar[st]);
        }
        outstanding[st] = 1;
      }
      if (it > 0) epilogue(it - 1);
      if (it + 1 < n_it) {
        prefetch(it + 1);
        copy_tiles(it + 1, st ^ 1);
      }
    }
    if (n_it > 0) epilogue(n_it - 1);
    // row value = (J . Z) / scale ; pair value = (re row + im row) / D
    part[t] = ((double)acc_hi + (double)acc_lo) / (double)sc;
    fence_before();
    __syncthreads();
    fence_after();
    if (t < kM / 2) {
      const int64_t p = tile * (kM / 2) + t;
      const int a = 2 * t, b = 2 * t + 1;
      if (p < g.n_pairs) g.pairval[p] = (part[a] + part[a + kM] + part[b] + part[b + kM]) * g.inv_den;
    }
    __syncthreads();
  }
  // an expired wait: give the outstanding MMAs one more bounded wait before
  // the tensor memory they write is released
  for (int b = 0; b < 2; ++b)
    if (outstanding[b]) mbar_wait(&bar[b], phase[b]);
  // K-tile copies still in flight (only after an expired wait) land before the
  // CTA's shared memory goes away
  if (t == 0 && *abort_flag)
    for (int b = 0; b < 2; ++b) {
      mbar_wait(&kbar[b], 0u);
      mbar_wait(&kbar[b], 1u);
    }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// Probe of the timeout path: waits on an mbarrier that nothing arrives on,
// with the same bounded wait as the kernels above, and records the expiry in
// *status exactly as they do.
__global__ void wait_probe_kernel(int* status, uint32_t limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit) && status) atomicExch(status, 1);
}

}  // namespace

cudaError_t launch_wait_probe(int* status, uint32_t spin_limit, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(status, spin_limit);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

ColourTiles build_colour_tiles(const std::vector<int64_t>& K, int m) {
  ColourTiles T;
  T.m = m;
  const int nb = (m + 255) / 256;
  T.nc = ((m + nb - 1) / nb + 31) / 32 * 32;  // column halves of the epilogue are multiples of 16
  T.np = nb * T.nc;
  T.kp = ((m + kKC - 1) / kKC) * kKC;
  const int n_kc = T.kp / kKC;
  const size_t per_tile = (size_t)T.nc * kKC;
  T.hi.assign((size_t)nb * n_kc * per_tile, __float2half(0.f));
  T.lo.assign(T.hi.size(), __float2half(0.f));
  T.exact = true;
  for (int a = 0; a < T.np; ++a)
    for (int k = 0; k < T.kp; ++k) {
      const int b = a / T.nc, row = a - b * T.nc, kc = k / kKC, kk = k - kc * kKC;
      double v = (a < m && k < m) ? (double)K[(size_t)a * m + k] : 0.0;
      const __half h = __float2half_rn((float)v);
      const double rest = v - (double)__half2float(h);
      const __half l = __float2half_rn((float)rest);
      if (rest != 0.0) T.exact = false;
      const size_t base = ((size_t)b * n_kc + kc) * per_tile;
      const uint32_t off = tc::canon_off(row, kk, kKC) / 2;
      T.hi[base + off] = h;
      T.lo[base + off] = l;
    }
  return T;
}

// two stages, 4 mbarriers (32 B), TMEM slot and abort flag (16 B), row scales (512 B)
size_t colour_gemm_smem(int nc) { return 2 * stage_bytes(nc) + 32 + 16 + (size_t)kM * 4 + 64; }

cudaError_t launch_colour_gemm(const ColourGemmArgs& a, int num_sms, cudaStream_t s) {
  if (a.n_pairs <= 0) return cudaSuccess;
  if (a.nc < 32 || a.nc > 256 || a.nc % 32 != 0 || a.kp % kKC != 0 || a.np % a.nc != 0) return cudaErrorInvalidValue;
  // the kernel reads J in 16-byte vectors within rows of ldj >= m entries
  if (a.ldj % 16 != 0 || a.m > a.ldj || (reinterpret_cast<uintptr_t>(a.J) & 15) != 0) return cudaErrorInvalidValue;
  size_t sm = colour_gemm_smem(a.nc);
  cudaError_t e = ensure_dynamic_smem((const void*)colour_gemm_kernel, sm);
  if (e != cudaSuccess) return e;
  int64_t tiles = (2 * a.n_pairs + kM - 1) / kM;
  int tmem = 32;
  while (tmem < 2 * a.nc) tmem *= 2;
  const int per_sm = std::max(1, std::min<int>(512 / tmem, (int)((227u << 10) / sm)));
  int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms * per_sm);
  colour_gemm_kernel<<<grid, kThreads, sm, s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

}  // namespace mea

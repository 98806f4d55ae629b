// Colour contraction on the tensor cores (Eq. (color-averaged-amplitude)):
// for every (event, helicity) pair p with colour amplitudes J_p (FP32, from
// the amplitude kernel)
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
// Operands are staged in shared memory in the canonical no-swizzle K-major
// layout (8-row x 16-byte core matrices).  Every wait is bounded: on expiry
// the kernel records an error in *status, drains its own MMAs with a bounded
// wait, frees its tensor memory and returns.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "colour_gemm.h"
#include "kernels.h"
#include "tc_common.cuh"

namespace mea {
namespace {

constexpr int kThreads = 128;   // 4 warps: TMEM lanes 0..127 = tile rows
constexpr int kM = 128;         // tile rows (64 pairs x {re, im})
constexpr int kKC = 64;         // K elements per shared-memory stage
using namespace tc;

__global__ void __launch_bounds__(kThreads) colour_gemm_kernel(ColourGemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // layout: A_hi, A_mid, A_lo [128 x KC], B_hi, B_lo [NC x KC], bars, tmem slot, scales
  const int t = threadIdx.x;
  const int warp = t >> 5;
  const int NC = g.nc;
  unsigned char* a_hi = smem;
  unsigned char* a_mid = a_hi + kM * kKC * 2;
  unsigned char* a_lo = a_mid + kM * kKC * 2;
  unsigned char* b_hi = a_lo + kM * kKC * 2;
  unsigned char* b_lo = b_hi + NC * kKC * 2;
  uint64_t* bar = reinterpret_cast<uint64_t*>(b_lo + NC * kKC * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  float* rscale = reinterpret_cast<float*>(tslot + 4);  // [128] per-row scale 2^-e
  int* abort_flag = reinterpret_cast<int*>(rscale + kM);
  double* rowbuf = reinterpret_cast<double*>(abort_flag + 2);  // [128] row values

  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)g.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  int pending = -1;  // phase of a wait that expired (drained once more before freeing TMEM)
  const int m = g.m, ldj = g.ldj;
  const int64_t n_rows = 2 * g.n_pairs;
  const int64_t n_tiles = (n_rows + kM - 1) / kM;
  const uint32_t idesc = make_idesc(kM, NC);
  const bool use_blo = g.b_lo != nullptr;

  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t row0 = tile * kM;
    // per-row power-of-two scale so that the largest |J| lands near 2^14
    {
      const int64_t r = row0 + t;
      float mx = 0.f;
      if (r < n_rows) {
        const float* jr = g.J + r * ldj;
        for (int k = 0; k < m; ++k) mx = fmaxf(mx, fabsf(jr[k]));
      }
      int e = 0;
      if (mx > 0.f && isfinite(mx)) { frexpf(mx, &e); }
      rscale[t] = ldexpf(1.f, max(-120, min(120, 14 - e)));
    }
    float acc_hi = 0.f, acc_lo = 0.f;  // this thread's row: sum_a J_a Z_a (scaled), compensated
    for (int n0 = 0; n0 < g.np; n0 += NC) {
      for (int k0 = 0; k0 < g.kp; k0 += kKC) {
        __syncthreads();  // previous MMAs and epilogue reads are done before overwriting
        // A tiles: 128 rows x KC columns, three FP16 parts of the scaled J
        for (int idx = t; idx < kM * kKC; idx += kThreads) {
          int row = idx / kKC, k = idx - (idx / kKC) * kKC;
          int64_t r = row0 + row;
          int kk = k0 + k;
          float x = 0.f;
          if (r < n_rows && kk < m) x = g.J[r * ldj + kk] * rscale[row];
          __half hi = __float2half_rn(x);
          float r1 = x - __half2float(hi);
          __half mid = __float2half_rn(r1);
          __half lo = __float2half_rn(r1 - __half2float(mid));
          uint32_t off = canon_off(row, k, kKC);
          *reinterpret_cast<__half*>(a_hi + off) = hi;
          *reinterpret_cast<__half*>(a_mid + off) = mid;
          *reinterpret_cast<__half*>(a_lo + off) = lo;
        }
        // B tiles: rows n0..n0+NC of the (symmetric) colour matrix, K columns k0..
        for (int idx = t; idx < NC * kKC; idx += kThreads) {
          int row = idx / kKC, k = idx - (idx / kKC) * kKC;
          int nn = n0 + row, kk = k0 + k;
          __half hi = __float2half_rn(0.f), lo = hi;
          if (nn < m && kk < m) {
            hi = g.b_hi[(size_t)nn * m + kk];
            if (use_blo) lo = g.b_lo[(size_t)nn * m + kk];
          }
          uint32_t off = canon_off(row, k, kKC);
          *reinterpret_cast<__half*>(b_hi + off) = hi;
          *reinterpret_cast<__half*>(b_lo + off) = lo;
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();
        if (t == 0 && !*abort_flag) {
          const uint32_t lbo = 128, sbo_a = (kKC / 8) * 128, sbo_b = (kKC / 8) * 128;
          for (int ks = 0; ks < kKC / 16; ++ks) {
            uint32_t koff = (uint32_t)(ks * 2 * 128);
            uint64_t dah = make_desc(smem_u32(a_hi) + koff, lbo, sbo_a);
            uint64_t dam = make_desc(smem_u32(a_mid) + koff, lbo, sbo_a);
            uint64_t dal = make_desc(smem_u32(a_lo) + koff, lbo, sbo_a);
            uint64_t dbh = make_desc(smem_u32(b_hi) + koff, lbo, sbo_b);
            uint64_t dbl = make_desc(smem_u32(b_lo) + koff, lbo, sbo_b);
            uint32_t first = (ks == 0) ? 0u : 1u;  // fresh accumulator for every K chunk
            // smallest terms first
            mma_f16(tmem, dal, dbh, idesc, first);
            if (use_blo) {
              mma_f16(tmem, dam, dbl, idesc, 1u);
              mma_f16(tmem, dah, dbl, idesc, 1u);
            }
            mma_f16(tmem, dam, dbh, idesc, 1u);
            mma_f16(tmem, dah, dbh, idesc, 1u);
          }
          mma_commit(bar);
        }
        if (!*abort_flag) {
          if (!mbar_wait(bar, phase)) {
            atomicExch(abort_flag, 1);
            pending = (int)phase;
            if (g.status) atomicExch(g.status, 1);
          }
        }
        phase ^= 1u;
        fence_after();
        // epilogue of this K chunk: this thread owns TMEM lane t (its row)
        if (!*abort_flag) {
          const int64_t r = row0 + t;
          const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
          for (int c0 = 0; c0 < NC && n0 + c0 < m; c0 += 16) {
            float z[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, z);
            if (r < n_rows) {
              const float* jr = g.J + r * ldj + n0 + c0;
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (n0 + c0 + i < m) {
                  // Dot2 (Ogita, Rump, Oishi 2005): exact product error by FMA,
                  // two-sum of the running value, errors collected in acc_lo
                  const float p = __fmul_rn(jr[i], z[i]);
                  const float pe = fmaf(jr[i], z[i], -p);
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
      }
      __syncthreads();
      fence_after();
    }
    // row value = (J . Z) / scale ; pair value = (re row + im row) / D
    {
      double* rowval = rowbuf;
      rowval[t] = ((double)acc_hi + (double)acc_lo) / (double)rscale[t];
      __syncthreads();
      if (t < kM / 2) {
        int64_t p = tile * (kM / 2) + t;
        if (p < g.n_pairs) g.pairval[p] = (rowval[2 * t] + rowval[2 * t + 1]) * g.inv_den;
      }
      __syncthreads();
    }
  }
  // an expired wait: give the outstanding MMAs one more bounded wait before
  // the tensor memory they write is released
  if (pending >= 0) mbar_wait(bar, (uint32_t)pending);
  // free tensor memory (after every tcgen05.ld has completed)
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)g.tmem_cols)
                 : "memory");
}

}  // namespace

size_t colour_gemm_smem(int nc) {
  return (size_t)kM * kKC * 2 * 3 + (size_t)nc * kKC * 2 * 2 + 64 + kM * 4 + 16 + kM * 8;
}

cudaError_t launch_colour_gemm(const ColourGemmArgs& a, int num_sms, cudaStream_t s) {
  if (a.n_pairs <= 0) return cudaSuccess;
  size_t sm = colour_gemm_smem(a.nc);
  cudaError_t e = cudaFuncSetAttribute(colour_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int64_t tiles = (2 * a.n_pairs + kM - 1) / kM;
  int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms);
  colour_gemm_kernel<<<grid, kThreads, sm, s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

}  // namespace mea

// Tensor-core colour contraction (tcgen05, kind::f16 split precision).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mea {

struct ColourGemmArgs {
  const float* J = nullptr;      // [2*n_pairs][ldj] FP32 colour amplitudes, rows (re, im) per pair
  int64_t n_pairs = 0;
  int m = 0;                     // colour basis size
  int ldj = 0;                   // row stride of J (elements)
  int kp = 0, np = 0;            // K and N extents padded to 64 and to a multiple of nc
  int nc = 0;                    // N columns per tensor-memory chunk (multiple of 16, <= 256)
  int tmem_cols = 0;             // power of two >= max(32, nc)
  const __half* b_hi = nullptr;  // [m][m] fp16(K)
  const __half* b_lo = nullptr;  // [m][m] K - fp16(K), or nullptr when fp16(K) is exact
  double inv_den = 0;            // 1 / D
  double* pairval = nullptr;     // [n_pairs] output: J K J^* / D per pair
  int* status = nullptr;         // set to 1 when a bounded wait expired
};

size_t colour_gemm_smem(int nc);
cudaError_t launch_colour_gemm(const ColourGemmArgs& a, int num_sms, cudaStream_t s);

}  // namespace mea

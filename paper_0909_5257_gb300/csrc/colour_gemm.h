// Tensor-core colour contraction (tcgen05, kind::f16 split precision).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace mea {

// The integer colour matrix K laid out once per process as the kernel's
// operand tiles: column blocks of nc (a multiple of 32, <= 256) times K chunks
// of 64, each tile nc x 64 FP16 in the canonical no-swizzle K-major layout;
// hi = fp16(K), lo = K - hi (all zero, and exact = true, when |K| <= 2048).
struct ColourTiles {
  int m = 0, nc = 0, np = 0, kp = 0;
  bool exact = true;
  std::vector<__half> hi, lo;  // [np / nc][kp / 64][nc x 64]
};
ColourTiles build_colour_tiles(const std::vector<int64_t>& K, int m);

struct ColourGemmArgs {
  const float* J = nullptr;      // [2*n_pairs][ldj] FP32 colour amplitudes, rows (re, im) per pair
  int64_t n_pairs = 0;
  int m = 0;                     // colour amplitudes per row
  int ldj = 0;                   // row stride of J (elements)
  int kp = 0, np = 0, nc = 0;    // from ColourTiles
  const __half* b_hi = nullptr;  // device copy of ColourTiles::hi
  const __half* b_lo = nullptr;  // device copy of ColourTiles::lo, or nullptr when exact
  double inv_den = 0;            // 1 / D
  double* pairval = nullptr;     // [n_pairs] output: J K J^* / D per pair
  int* status = nullptr;         // set to 1 when a bounded wait expired
};

// One-warp kernel whose bounded mbarrier wait expires (nothing arrives):
// exercises the timeout reporting of the tensor-core kernels without a hang.
cudaError_t launch_wait_probe(int* status, uint32_t spin_limit, cudaStream_t s);

size_t colour_gemm_smem(int nc);
cudaError_t launch_colour_gemm(const ColourGemmArgs& a, int num_sms, cudaStream_t s);

}  // namespace mea

// Colour amplitudes from Feynman-diagram amplitudes on the tensor cores.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "generator.h"

namespace mea {

// Host-side description of the diagram -> colour-amplitude map
// J_alpha = sum_d c_{alpha d} A_d of a program (Eq. (color-amplitude)), with
// every coefficient real: c = cfac * n, n a small integer.
struct JampMap {
  bool ok = false;          // false: some coefficient is not real (path unavailable)
  int kd = 0;               // diagrams (K)
  int m = 0;                // colour amplitudes (N)
  int nc = 0;               // N columns per CTA (multiple of 16, 3 * nc <= 512)
  int n_splits = 0;         // ceil(m / nc)
  int kpad = 0;             // kd rounded up to 64
  int q = 0;                // digit bound 2^q (see jamp_gemm.cu)
  double cfac = 1;          // common factor of the coefficients
  std::vector<__half> tiles;  // [n_splits][kpad/64][nc x 64] canonical K-major fp16 tiles of n
  std::vector<float> weight;  // [kd] sum_alpha |c_{alpha d}| (cancellation indicator)
};

JampMap build_jamp_map(const Program& p);

struct JampGemmArgs {
  const float* A = nullptr;      // [kd][lda]: A[d*lda + 2p] = Re A_d, [.. + 1] = Im A_d of pair p
  int64_t lda = 0;
  const float* rowmax = nullptr;  // [2*n_pairs] max_d |A| of each row (NaN when a row is not finite)
  int64_t n_pairs = 0;
  int kd = 0, kpad = 0, m = 0, nc = 0, n_splits = 0, q = 0;
  double cfac = 1;
  const __half* tiles = nullptr;  // device copy of JampMap::tiles
  float* J = nullptr;             // [2*n_pairs][ldj] output rows (re, im) per pair
  int ldj = 0;
  float* jabs = nullptr;          // [n_splits][n_pairs]: sum |J| over the split's columns
  int* status = nullptr;          // set to 1 when a bounded wait expired
};

size_t jamp_gemm_smem(int nc);
cudaError_t launch_jamp_gemm(const JampGemmArgs& a, int num_sms, cudaStream_t s);

}  // namespace mea

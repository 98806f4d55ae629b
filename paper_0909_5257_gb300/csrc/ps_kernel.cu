// Synthetic phase-space generation on the device (input generator): one thread
// per event runs the shared seeded generator of phasespace.h (Philox4x32-10
// counters, sqrt(s_hat) log-uniform, RAMBO, jet cuts with redraw), so the
// device and host generators produce the same events.
#include <cuda_runtime.h>

#include "../phasespace/phasespace.h"
#include "kernels.h"

namespace mea {
namespace {

__global__ void ps_kernel(ps_config cfg, uint64_t first, int64_t n, double* mom, int32_t* att) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int n_ext = 2 + cfg.n_final;
  double (*m)[4] = reinterpret_cast<double (*)[4]>(mom + (size_t)i * n_ext * 4);
  int a = ps_generate_event(&cfg, first + (uint64_t)i, m);
  if (att) att[i] = a;
}

}  // namespace

cudaError_t launch_phase_space(const PsConfigDev& c, uint64_t first_event, int64_t n, double* mom,
                               int32_t* attempts, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ps_config cfg;
  cfg.seed = c.seed;
  cfg.n_final = c.n_final;
  cfg.rs_lo = c.rs_lo;
  cfg.rs_hi = c.rs_hi;
  cfg.pt_min = c.pt_min;
  cfg.eta_max = c.eta_max;
  cfg.dr_min = c.dr_min;
  const int threads = 128;
  int64_t blocks = (n + threads - 1) / threads;
  ps_kernel<<<(unsigned)blocks, threads, 0, s>>>(cfg, first_event, n, mom, attempts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

}  // namespace mea

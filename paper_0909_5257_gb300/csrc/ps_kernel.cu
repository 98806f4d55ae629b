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

// VEGAS points of events first .. first + n - 1 (ps_vegas_event).
__global__ void vegas_kernel(ps_config cfg, const double* edges, int nb, uint64_t first, int64_t n, double* mom,
                             double* weight, unsigned char* bins) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int n_ext = 2 + cfg.n_final;
  const int dims = ps_rambo_dims(cfg.n_final);
  double (*m)[4] = reinterpret_cast<double (*)[4]>(mom + (size_t)i * n_ext * 4);
  weight[i] = ps_vegas_event(&cfg, edges, nb, first + (uint64_t)i, m, bins + (size_t)i * dims);
}

// Partonic cross-section sums over a chunk: per block, in a fixed order, the
// sums of f and f^2 with f = me2 for accepted points (attempt index >= 0) and
// 0 otherwise, and the number of phase-space points drawn (attempt index + 1,
// or all PS_MAX_ATTEMPTS when none was accepted) and of accepted points;
// part_a holds (drawn, accepted) pairs.
__global__ void xsec_sum_kernel(const double* me2, const int32_t* att, int64_t n, double* part_f,
                                double* part_f2, long long* part_a) {
  __shared__ double sf[256], sf2[256];
  __shared__ long long sa[256], sn[256];
  const int t = threadIdx.x;
  double f = 0.0, f2 = 0.0;
  long long a = 0, acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + t; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = att[i];
    if (k >= 0) {
      const double v = me2[i];
      f += v;
      f2 += v * v;
      a += k + 1;
      ++acc;
    } else {
      a += PS_MAX_ATTEMPTS;
    }
  }
  sf[t] = f; sf2[t] = f2; sa[t] = a; sn[t] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) { sf[t] += sf[t + w]; sf2[t] += sf2[t + w]; sa[t] += sa[t + w]; sn[t] += sn[t + w]; }
    __syncthreads();
  }
  if (t == 0) {
    part_f[blockIdx.x] = sf[0];
    part_f2[blockIdx.x] = sf2[0];
    part_a[2 * blockIdx.x] = sa[0];
    part_a[2 * blockIdx.x + 1] = sn[0];
  }
}

}  // namespace

cudaError_t launch_xsec_sums(const double* me2, const int32_t* att, int64_t n, double* part_f, double* part_f2,
                             long long* part_a, int blocks, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  xsec_sum_kernel<<<blocks, 256, 0, s>>>(me2, att, n, part_f, part_f2, part_a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

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
  cfg.ptij_min = c.ptij_min;
  const int threads = 128;
  int64_t blocks = (n + threads - 1) / threads;
  ps_kernel<<<(unsigned)blocks, threads, 0, s>>>(cfg, first_event, n, mom, attempts);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

cudaError_t launch_vegas_points(const PsConfigDev& c, const double* edges, int nb, uint64_t first_event, int64_t n,
                                double* mom, double* weight, unsigned char* bins, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ps_config cfg;
  cfg.seed = c.seed;
  cfg.n_final = c.n_final;
  cfg.rs_lo = c.rs_lo;
  cfg.rs_hi = c.rs_hi;
  cfg.pt_min = c.pt_min;
  cfg.eta_max = c.eta_max;
  cfg.dr_min = c.dr_min;
  cfg.ptij_min = c.ptij_min;
  const int threads = 128;
  const int64_t blocks = (n + threads - 1) / threads;
  vegas_kernel<<<(unsigned)blocks, threads, 0, s>>>(cfg, edges, nb, first_event, n, mom, weight, bins);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++launch_counter();
  return e;
}

}  // namespace mea

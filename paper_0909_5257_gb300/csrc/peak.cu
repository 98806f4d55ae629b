// Measured arithmetic peaks of the FP32 and FP64 pipes (C ABI, declared in
// include/mea.h): the denominators of the rooflines of the ALU-bound
// amplitude kernels.  Every thread runs kChains independent fused
// multiply-add chains (enough independent work per lane to cover the FMA
// latency), the grid fills every SM several times over, and the launch is
// timed with CUDA events after a warm-up launch.  One FMA counts two FLOPs.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/mea.h"
#include "kernels.h"
#include "process.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

template <typename R>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, R a, R b, R* sink) {
  R x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (R)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (R)-1.2345) sink[blockIdx.x] = s;  // never true: keeps the chains alive
}

template <typename R>
cudaError_t time_chain(int num_sms, double target_flop, cudaStream_t s, double* tflops, double* ms_out) {
  const int grid = num_sms * kBlocksPerSm;
  const double per_iter = (double)grid * kThreads * kChains * 4 * 2;
  const int iters = (int)std::max(1.0, std::min(2.0e9, target_flop / per_iter));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    fma_chain_kernel<R><<<grid, kThreads, 0, s>>>(std::max(1, iters / 8), (R)0.9999999, (R)1e-7, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_chain_kernel<R><<<grid, kThreads, 0, s>>>(iters, (R)0.9999999, (R)1e-7, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) {
    mea::launch_counter() += 2;
    *ms_out = ms;
    *tflops = per_iter * iters / (ms * 1e-3) / 1e12;
  }
  return e;
}

}  // namespace

extern "C" {

mea_status mea_measure_alu_peak(int fp64, double seconds, double* tflops, double* ms) {
  if (!tflops || !ms || !(seconds > 0.0) || seconds > 10.0)
    return mea::set_error(MEA_E_ARG, "mea_measure_alu_peak: bad arguments");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return mea::set_error(MEA_E_CUDA, std::string("mea_measure_alu_peak: ") + cudaGetErrorString(e));
  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return mea::set_error(MEA_E_CUDA, std::string("mea_measure_alu_peak: ") + cudaGetErrorString(e));
  // size the timed launch for about `seconds` at a nominal rate (FP32 80, FP64 1.3 TFLOP/s)
  const double nominal = fp64 ? 1.3e12 : 80e12;
  e = fp64 ? time_chain<double>(sms, nominal * seconds, s, tflops, ms)
           : time_chain<float>(sms, nominal * seconds, s, tflops, ms);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return mea::set_error(MEA_E_CUDA, std::string("mea_measure_alu_peak: ") + cudaGetErrorString(e));
  return MEA_OK;
}

}  // extern "C"

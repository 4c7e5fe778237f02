// FP64 arithmetic rate of the device, measured: the roofline denominator of
// the kernels bound by the FP64 units (the FP64 relaxation, K1).  No
// counterpart in the paper.
//
// Every thread runs eight independent chains of a = a * b + c (one DFMA per
// step; b < 1 keeps the values bounded) over `steps` steps; a grid of four
// 256-thread CTAs per SM keeps 32 warps on every SM, so the chains' latency is
// hidden and the FP64 pipe is the bound.  The sums are stored so that no
// chain is removed.
#include "../../include/hms.h"
#include "hms_internal.cuh"

namespace hms {
namespace {

constexpr int PROBE_NT = 256, PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_NT) k_fp64_fma_loop(double* out, int steps, double b, double c) {
  double a[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) t += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace
}  // namespace hms

extern "C" hms_status hms_measure_fp64_rate(int32_t device, double* gflops) {
  using namespace hms;
  if (!gflops) return HMS_ERR_ARG;
  *gflops = 0.0;
  if (cudaSetDevice(device) != cudaSuccess) return HMS_ERR_ARG;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return HMS_ERR_CUDA;
  const int grid = 4 * nsm, steps = 1 << 14;
  double* out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hms_status st = HMS_ERR_CUDA;
  if (cudaMalloc(&out, (size_t)grid * PROBE_NT * sizeof(double)) != cudaSuccess) return HMS_ERR_OOM;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    for (int k = 0; k < 3; ++k) k_fp64_fma_loop<<<grid, PROBE_NT, 0, s>>>(out, steps, 0.999999, 1e-6);
    cudaEventRecord(e0, s);
    const int reps = 5;
    for (int k = 0; k < reps; ++k) k_fp64_fma_loop<<<grid, PROBE_NT, 0, s>>>(out, steps, 0.999999, 1e-6);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double flops = 2.0 * PROBE_CHAINS * (double)steps * (double)grid * PROBE_NT * reps;
      if (ms > 0.f) {
        *gflops = flops / ((double)ms * 1e-3) * 1e-9;
        st = HMS_OK;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  return st;
}

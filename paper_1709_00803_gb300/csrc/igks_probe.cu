// igks_probe.cu -- measured FP64 arithmetic rate of the GPU, the denominator of the ALU
// roofline of the flux kernel (which is bound by the FP64 pipe, not by HBM).
//
// Every thread runs eight independent chains of fused multiply-adds, so the pipe sees
// eight independent instructions per warp between any two that depend on each other;
// the grid is eight blocks of 256 threads per SM. The result is the best of three timed
// launches after one warm-up, in TFLOP/s (one FMA = two flops).
#include <cuda_runtime.h>

#include "../../include/igks.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) k_fp64_probe(int iters, double a, double b, double* sink) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) x[c] = 1e-3 * (threadIdx.x + c);
  for (int k = 0; k < iters; k++) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" int igks_fp64_probe(int32_t device, double* tflops) {
  if (!tflops) return IGKS_EINVAL;
  *tflops = 0.0;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return IGKS_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return IGKS_ECUDA;
  int sms = 0;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = IGKS_OK;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = IGKS_ECUDA;
  } else {
    const int blocks = 8 * sms, iters = 4096;
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * PROBE_THREADS * blocks;
    double best = 0.0;
    for (int r = 0; r < 4 && rc == IGKS_OK; r++) {
      cudaEventRecord(e0, s);
      k_fp64_probe<<<blocks, PROBE_THREADS, 0, s>>>(iters, 0.9999999, 1e-7, nullptr);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        rc = IGKS_ECUDA;
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && ms > 0.0f) best = fmax(best, flops / (ms * 1e-3) / 1e12);
    }
    *tflops = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return rc;
}

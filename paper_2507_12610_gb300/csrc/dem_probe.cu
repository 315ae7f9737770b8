// Throughput probe of the FP64 pipe: the denominator of the roofline of the
// DEM_FP64 step, whose contact law and integration are bound by double
// precision arithmetic.  A measurement utility beside the library, not part
// of the timestep.
//
// Every SM gets eight blocks of 256 threads (the most resident threads an SM
// holds); each thread runs eight independent chains of fused multiply-adds
// x <- x a + b, so issue never waits on a result.  The count of FMAs divided
// by the CUDA-event time of the launch is the rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "dem.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int64_t iters, double a, double b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (double)(k + 1) + 1e-9 * (double)threadIdx.x;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[t] = s;
}

}  // namespace

extern "C" int dem_probe_fp64_fma(int64_t iters, void* stream, double* fma_per_s) {
  if (iters <= 0 || !fma_per_s) return DEM_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DEM_ERR_CUDA;
  const int blocks = 8 * sms, threads = 256;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * (size_t)blocks * threads) != cudaSuccess)
    return DEM_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  int rc = DEM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess) rc = DEM_ERR_CUDA;
  if (rc == DEM_OK && cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    rc = DEM_ERR_CUDA;
  }
  if (rc == DEM_OK) {
    float best = 0.f;
    for (int rep = 0; rep < 3 && rc == DEM_OK; ++rep) {  // first launch warms up
      cudaEventRecord(e0, st);
      k_fp64_fma<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-6);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = DEM_ERR_CUDA;
      else if (rep > 0 && (best == 0.f || ms < best))
        best = ms;
    }
    if (rc == DEM_OK)
      *fma_per_s = (double)blocks * threads * kChains * (double)iters / (best * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaFree(out);
  return rc;
}

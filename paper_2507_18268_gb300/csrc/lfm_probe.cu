// Measured FP64 fused multiply-add rate of the device (lfm_measure_fp64_fma_rate in
// include/lapfoam.h): the issue-rate roofline of the FP64 form, whose steps need about 14
// FP64 instructions per cell and PCG iteration against 160 bytes.
//
// Every thread runs kChains independent multiply-add chains (enough in flight to cover the
// pipe's latency); the grid puts kBlocksPerSm blocks on every SM. The chains contract to a
// fixed point (x = a x + b, 0 < a < 1), so values stay finite whatever the trip count.
#include <cuda_runtime.h>

#include "lfm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) fma_rate_kernel(double* sink, int trips, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int i = 0; i < trips; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == 12345.0) sink[0] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" int lfm_measure_fp64_fma_rate(int device, double* fma_per_s) {
  if (!fma_per_s) return lfm::set_last_error(LFM_EINVAL, "lfm_measure_fp64_fma_rate: fma_per_s is NULL");
  *fma_per_s = 0.0;
  int prev = -1, sms = 0, count = 0;
  // checked before cudaSetDevice, whose failure would stay in the runtime's last-error slot
  // and surface at the caller's next launch check
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return lfm::set_last_error(LFM_EINVAL, "lfm_measure_fp64_fma_rate: device %d not available", device);
  }
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return lfm::set_last_error(LFM_ECUDA, "lfm_measure_fp64_fma_rate: cannot select device %d", device);
  }
  int rc = LFM_OK;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  const int trips = 8192;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&sink, sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    rc = lfm::set_last_error(LFM_ECUDA, "lfm_measure_fp64_fma_rate: set-up failed");
  } else {
    const int blocks = sms * kBlocksPerSm;
    const double fmas = (double)blocks * kThreads * kChains * (double)trips;
    float best = 0.0f;
    for (int rep = 0; rep < 4 && rc == LFM_OK; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, s);
      fma_rate_kernel<<<blocks, kThreads, 0, s>>>(sink, trips, 0.999999, 1e-7);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = lfm::set_last_error(LFM_ECUDA, "lfm_measure_fp64_fma_rate: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
    }
    if (rc == LFM_OK && best > 0.0f) *fma_per_s = fmas / (1e-3 * (double)best);
  }
  if (rc != LFM_OK) cudaGetLastError();
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return rc;
}

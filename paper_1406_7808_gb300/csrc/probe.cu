// Peak fused multiply-add issue rate of the current device, float64 or
// float32: the denominator of the roofline of the float64-pipe-bound stencil
// kernels, measured instead of derived from a lane count and a clock.
//
// Every thread runs kChains independent FMA chains x = fma(a, x, c) with a
// and c kernel parameters (the operand form the solver's kernels use), so the
// pipe, not the dependency latency, bounds the rate; the grid fills every SM
// with resident blocks; the chains' sum is stored so nothing is optimised
// away.  The rate is lane operations (one FMA on one lane counts one) per
// second over the event-timed launch.
#include <cuda_runtime.h>

#include "srfmg.h"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T a, T c, int iters, T* out) {
  T x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = T(threadIdx.x + j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = fma(a, x[j], c);
  }
  T s = x[0];
#pragma unroll
  for (int j = 1; j < kChains; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(double* rate, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SR_ERR_NO_DEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SR_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_probe<T>, kProbeThreads, 0) !=
      cudaSuccess)
    return SR_ERR_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const int iters = sizeof(T) == 8 ? 2048 : 32768;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kProbeThreads) != cudaSuccess) {
    cudaGetLastError();
    return SR_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SR_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SR_ERR_CUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && rc == SR_OK; ++rep) {  // first launch warms up
    cudaEventRecord(e0, s);
    k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(T(0.999999), T(1e-7), iters, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = SR_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (rc == SR_OK && best > 0.f)
    *rate = (double)blocks * kProbeThreads * iters * kChains / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int sr_probe_fma_rate(int bits, double* lane_ops_per_s, void* stream) {
  if (!lane_ops_per_s || (bits != 64 && bits != 32)) return SR_ERR_INVALID;
  *lane_ops_per_s = 0.0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SR_ERR_NO_DEVICE;
  }
  return bits == 64 ? probe<double>(lane_ops_per_s, (cudaStream_t)stream)
                    : probe<float>(lane_ops_per_s, (cudaStream_t)stream);
}

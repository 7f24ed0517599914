// Throughput probes for the blend's roofline: the FP32 pipe (independent
// fused multiply-add chains) and the exp2 pipe (independent ex2.approx
// chains), run over every SM of the device. The blend's work is counted in
// FP32 lane operations (an FMA is one) and exp2 evaluations, so the probes
// report those per second.
#include "lfd_internal.h"

namespace lfd {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeIters = 4096;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(float seed, float* sink) {
  float v[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) v[c] = seed + (float)(threadIdx.x + c);
  const float m = 0.999f, a = 1e-3f;
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = fmaf(v[c], m, a);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += v[c];
  if (s == 12345.f) sink[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ex2(float seed, float* sink) {
  float v[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) v[c] = seed + 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < kProbeIters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) v[c] = ex2_approx(v[c]) - 1.f;  // stays in (-0.5, 1)
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += v[c];
  if (s == 12345.f) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace lfd

using namespace lfd;

extern "C" LFD_API int lfd_measure_alu_peaks(double* fp32_ops_per_s, double* ex2_per_s, void* stream) {
  if (!fp32_ops_per_s || !ex2_per_s) return LFD_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_ffma, kProbeThreads, 0) != cudaSuccess)
    return LFD_ERR_CUDA;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1) * 4;
  float* sink = nullptr;
  cudaEvent_t e[3] = {};
  int rc = LFD_OK;
  if (cudaMalloc(&sink, (size_t)blocks * sizeof(float)) != cudaSuccess) return LFD_ERR_OOM;
  for (cudaEvent_t& x : e)
    if (cudaEventCreate(&x) != cudaSuccess) rc = LFD_ERR_CUDA;
  float ms_f = 0.f, ms_e = 0.f;
  if (rc == LFD_OK) {
    // one untimed round of each, then the timed ones
    k_probe_ffma<<<blocks, kProbeThreads, 0, s>>>(0.5f, sink);
    k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(0.25f, sink);
    cudaEventRecord(e[0], s);
    k_probe_ffma<<<blocks, kProbeThreads, 0, s>>>(0.5f, sink);
    cudaEventRecord(e[1], s);
    k_probe_ex2<<<blocks, kProbeThreads, 0, s>>>(0.25f, sink);
    cudaEventRecord(e[2], s);
    note_launches(4);
    if (cudaEventSynchronize(e[2]) != cudaSuccess || cudaEventElapsedTime(&ms_f, e[0], e[1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms_e, e[1], e[2]) != cudaSuccess)
      rc = LFD_ERR_CUDA;
  }
  for (cudaEvent_t& x : e)
    if (x) cudaEventDestroy(x);
  cudaFree(sink);
  if (rc != LFD_OK) return rc;
  const double n = (double)blocks * kProbeThreads * kProbeChains * kProbeIters;
  *fp32_ops_per_s = n / (ms_f * 1e-3);
  *ex2_per_s = n / (ms_e * 1e-3);
  return LFD_OK;
}

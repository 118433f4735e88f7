// FP32 FMA throughput probe (include/pulsar_probe.h): the denominator of the
// render passes' arithmetic roofline, measured rather than assumed.
#include "pulsar_internal.cuh"
#include "pulsar_probe.h"

namespace pulsar {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;          // independent FMA chains per thread
constexpr int kProbeBlocksPerSm = 8;     // 64 resident warps per SM

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float* sink, int iters, float b, float c) {
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == -1.0f) *sink = s;   // never true for the inputs used (b, c > 0)
}

}  // namespace
}  // namespace pulsar

using namespace pulsar;

extern "C" pulsar_status pulsar_probe_fma_throughput(float* sink, int iters, double* flops_per_s,
                                                     float* ms, void* stream) {
  if (!sink || iters < 1) return PULSAR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PULSAR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PULSAR_ERR_CUDA;
  const unsigned blocks = (unsigned)sms * kProbeBlocksPerSm;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PULSAR_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PULSAR_ERR_CUDA;
  }
  // one untimed launch, then the timed one
  fma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
  cudaEventRecord(e0, st);
  fma_probe_kernel<<<blocks, kProbeThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || t <= 0.0f) return PULSAR_ERR_CUDA;
  const double flops = 2.0 * kProbeChains * (double)iters * kProbeThreads * blocks;
  if (flops_per_s) *flops_per_s = flops / (t * 1e-3);
  if (ms) *ms = t;
  return PULSAR_OK;
}

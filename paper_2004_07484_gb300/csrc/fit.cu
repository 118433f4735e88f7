// The optimisation loop's kernels (include/pulsar_fit.h): image loss and its
// gradient, and a multi-tensor Adam step (Sec. 3.4; Adam as in Kingma & Ba,
// Algorithm 1).  Both are streaming, HBM-bound passes: coalesced, one read
// and at most one write of every value, grids sized in multiples of the SM
// count.
#include <cmath>

#include "pulsar_fit.h"
#include "pulsar_internal.cuh"

namespace pulsar {
namespace {

constexpr int kLossThreads = 256;
constexpr int kLossBlocks = PULSAR_LOSS_SCRATCH_FLOATS;   // at most one partial per CTA

__device__ __forceinline__ float loss_term(int kind, float d, float scale, float& g) {
  if (kind == PULSAR_LOSS_L2) {
    g = 2.0f * scale * d;
    return d * d;
  }
  g = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
  return fabsf(d);
}

// Grid-stride pass: per element d = F - T, the gradient, and this CTA's sum
// of loss terms (unscaled) in scratch[blockIdx.x].
__global__ void __launch_bounds__(kLossThreads) loss_partials_kernel(int kind, const float* __restrict__ image,
                                                                     const float* __restrict__ target, int64_t n,
                                                                     float scale, float* __restrict__ grad,
                                                                     float* __restrict__ scratch, int vec) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sh[kLossThreads / 32];
  float acc = 0.0f;
  const int64_t stride = (int64_t)gridDim.x * kLossThreads;
  const int64_t first = (int64_t)blockIdx.x * kLossThreads + threadIdx.x;
  int64_t tail_begin = 0;
  if (vec) {
    const int64_t n4 = n >> 2;
    const float4* F4 = reinterpret_cast<const float4*>(image);
    const float4* T4 = reinterpret_cast<const float4*>(target);
    float4* G4 = reinterpret_cast<float4*>(grad);
    for (int64_t i = first; i < n4; i += stride) {
      const float4 f = __ldg(F4 + i), t = __ldg(T4 + i);
      float4 g;
      acc += loss_term(kind, f.x - t.x, scale, g.x);
      acc += loss_term(kind, f.y - t.y, scale, g.y);
      acc += loss_term(kind, f.z - t.z, scale, g.z);
      acc += loss_term(kind, f.w - t.w, scale, g.w);
      if (grad) G4[i] = g;
    }
    tail_begin = n4 << 2;
  }
  for (int64_t i = tail_begin + first; i < n; i += stride) {
    float g;
    acc += loss_term(kind, __ldg(image + i) - __ldg(target + i), scale, g);
    if (grad) grad[i] = g;
  }
  acc = warp_sum(acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int w = 0; w < kLossThreads / 32; ++w) s += sh[w];
    scratch[blockIdx.x] = s;
  }
}

// One CTA: the partials summed in a fixed order (FP64), times scale.
__global__ void __launch_bounds__(kLossBlocks) loss_total_kernel(const float* __restrict__ scratch, int parts,
                                                                 float scale, float* __restrict__ loss) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[kLossBlocks];
  sh[threadIdx.x] = threadIdx.x < (unsigned)parts ? (double)scratch[threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = kLossBlocks / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = (float)(sh[0] * (double)scale);
}

constexpr int kAdamThreads = 256;
constexpr int kAdamPerThread = 8;
constexpr int kAdamChunk = kAdamThreads * kAdamPerThread;

struct AdamPack {
  pulsar_adam_tensor t[PULSAR_ADAM_MAX_TENSORS];
  int64_t block_begin[PULSAR_ADAM_MAX_TENSORS + 1];   // first CTA of each tensor, then the total
  int n;
  float beta1, beta2, eps;
  int zero_grad;
};

// One thread: t += 1 and the bias-corrected step factors of the new step.
__global__ void adam_tick_kernel(pulsar_adam_state* st, float lr, float beta1, float beta2) {
  pdl_wait();
  pdl_trigger();
  const int t = st->t + 1;
  st->t = t;
  const double bc1 = 1.0 - pow((double)beta1, (double)t);
  const double bc2 = 1.0 - pow((double)beta2, (double)t);
  st->step_size = (float)((double)lr / bc1);
  st->inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
}

// CTA b updates kAdamChunk consecutive elements of the tensor whose CTA range
// holds b; each thread takes every kAdamThreads-th element of the chunk.
__global__ void __launch_bounds__(kAdamThreads) adam_update_kernel(const AdamPack pk,
                                                                   const pulsar_adam_state* __restrict__ st) {
  pdl_wait();
  pdl_trigger();
  const int64_t b = blockIdx.x;
  int k = 0;
  while (k + 1 < pk.n && pk.block_begin[k + 1] <= b) ++k;
  const pulsar_adam_tensor& T = pk.t[k];
  const float step_size = st->step_size, inv_sqrt_bc2 = st->inv_sqrt_bc2;
  const int64_t base = (b - pk.block_begin[k]) * kAdamChunk + threadIdx.x;
#pragma unroll
  for (int j = 0; j < kAdamPerThread; ++j) {
    const int64_t i = base + (int64_t)j * kAdamThreads;
    if (i < T.n) {
      const float g = T.grad[i];
      const float m = pk.beta1 * T.m[i] + (1.0f - pk.beta1) * g;
      const float v = pk.beta2 * T.v[i] + (1.0f - pk.beta2) * (g * g);
      float p = T.param[i] - step_size * m / (sqrtf(v) * inv_sqrt_bc2 + pk.eps);
      p = fminf(fmaxf(p, T.lo), T.hi);
      T.m[i] = m;
      T.v[i] = v;
      T.param[i] = p;
      if (pk.zero_grad) T.grad[i] = 0.0f;
    }
  }
}

}  // namespace
}  // namespace pulsar

using namespace pulsar;

extern "C" pulsar_status pulsar_image_loss(int kind, const float* image, const float* target, int64_t n,
                                           float scale, float* grad, float* loss, float* scratch,
                                           void* stream) {
  if ((kind != PULSAR_LOSS_L2 && kind != PULSAR_LOSS_L1) || n < 0) return PULSAR_ERR_INVALID_ARG;
  if (n > 0 && (!image || !target || !scratch)) return PULSAR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), st) != cudaSuccess) return PULSAR_ERR_CUDA;
    return PULSAR_OK;
  }
  const auto aligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const int vec = aligned(image) && aligned(target) && (!grad || aligned(grad)) ? 1 : 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PULSAR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PULSAR_ERR_CUDA;
  const int64_t work = vec ? (n + 3) / 4 : n;
  const int64_t want = (work + kLossThreads - 1) / kLossThreads;
  const int per_sm = kLossBlocks / (sms > 0 ? sms : 1);   // whole waves of CTAs over the SMs
  const int cap = per_sm > 0 ? per_sm * sms : kLossBlocks;
  const int blocks = (int)(want < cap ? want : cap);
  cudaError_t e = launch_pdl(loss_partials_kernel, dim3(blocks), dim3(kLossThreads), 0, st, kind, image, target,
                             n, scale, grad, scratch, vec);
  if (e == cudaSuccess && loss)
    e = launch_pdl(loss_total_kernel, dim3(1), dim3(kLossBlocks), 0, st, (const float*)scratch, blocks, scale, loss);
  return e == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}

extern "C" pulsar_status pulsar_adam_step(int n_tensors, const pulsar_adam_tensor* tensors,
                                          const pulsar_adam_hyper* hyper, pulsar_adam_state* state,
                                          void* stream) {
  if (n_tensors < 1 || n_tensors > PULSAR_ADAM_MAX_TENSORS || !tensors || !hyper || !state)
    return PULSAR_ERR_INVALID_ARG;
  const pulsar_adam_hyper& h = *hyper;
  if (!(h.lr >= 0.0f) || !(h.beta1 >= 0.0f && h.beta1 < 1.0f) || !(h.beta2 >= 0.0f && h.beta2 < 1.0f) ||
      !(h.eps >= 0.0f))
    return PULSAR_ERR_INVALID_ARG;
  AdamPack pk;
  pk.n = n_tensors;
  pk.beta1 = h.beta1;
  pk.beta2 = h.beta2;
  pk.eps = h.eps;
  pk.zero_grad = h.zero_grad ? 1 : 0;
  int64_t blocks = 0;
  for (int k = 0; k < n_tensors; ++k) {
    const pulsar_adam_tensor& T = tensors[k];
    if (T.n < 0 || !(T.lo <= T.hi)) return PULSAR_ERR_INVALID_ARG;
    if (T.n > 0 && (!T.param || !T.grad || !T.m || !T.v)) return PULSAR_ERR_INVALID_ARG;
    pk.t[k] = T;
    pk.block_begin[k] = blocks;
    blocks += (T.n + kAdamChunk - 1) / kAdamChunk;
  }
  pk.block_begin[n_tensors] = blocks;
  if (blocks > 0x7fffffff) return PULSAR_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_pdl(adam_tick_kernel, dim3(1), dim3(1), 0, st, state, h.lr, h.beta1, h.beta2);
  if (e == cudaSuccess && blocks > 0)
    e = launch_pdl(adam_update_kernel, dim3((unsigned)blocks), dim3(kAdamThreads), 0, st, pk,
                   (const pulsar_adam_state*)state);
  return e == cudaSuccess ? PULSAR_OK : PULSAR_ERR_CUDA;
}

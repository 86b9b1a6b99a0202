// Summed L1 / L2 image loss and its gradient dL/dC, the input of the backward
// pass.  One HBM pass: image and target are read and dL/dC written as float4s
// when all three are 16-byte aligned (a scalar loop takes the ragged tail and
// unaligned arrays).  Each thread sums four values in FP32 before adding them
// to its FP64 accumulator, so the FP64 adds (slow on this GPU) are a quarter
// of the values; the CTA sums go to one FP64 atomic each.
#include "common.cuh"

namespace gsr {

constexpr int kLossThreads = 256;

__device__ __forceinline__ float loss_term(float d, int kind, float& g) {
  if (kind == GS_LOSS_L1) {
    g = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    return fabsf(d);
  }
  g = 2.f * d;
  return d * d;
}

__global__ void __launch_bounds__(kLossThreads) loss_kernel(const float* __restrict__ img,
                                                           const float* __restrict__ tgt,
                                                           int64_t n, int kind, int vec,
                                                           float* __restrict__ grad,
                                                           double* __restrict__ loss) {
  __shared__ double s_w[kLossThreads / 32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kLossThreads;
  const int64_t t0 = blockIdx.x * (int64_t)kLossThreads + threadIdx.x;
  const int64_t n4 = vec ? n / 4 : 0;
  const float4* img4 = reinterpret_cast<const float4*>(img);
  const float4* tgt4 = reinterpret_cast<const float4*>(tgt);
  float4* grad4 = reinterpret_cast<float4*>(grad);
  for (int64_t i = t0; i < n4; i += stride) {
    const float4 a = img4[i], b = tgt4[i];
    float4 g;
    const float s = loss_term(a.x - b.x, kind, g.x) + loss_term(a.y - b.y, kind, g.y) +
                    loss_term(a.z - b.z, kind, g.z) + loss_term(a.w - b.w, kind, g.w);
    acc += (double)s;
    if (grad) grad4[i] = g;
  }
  for (int64_t i = 4 * n4 + t0; i < n; i += stride) {
    float g;
    acc += (double)loss_term(img[i] - tgt[i], kind, g);
    if (grad) grad[i] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) t += s_w[w];
    atomicAdd(loss, t);
  }
}

cudaError_t launch_loss(const float* img, const float* tgt, int64_t n, int kind, float* grad,
                        double* loss, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int vec = (((uintptr_t)img | (uintptr_t)tgt | (uintptr_t)grad) & 15) == 0;
  int64_t blocks = ((vec ? n / 4 : n) + kLossThreads - 1) / kLossThreads;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  if (blocks < 1) blocks = 1;
  loss_kernel<<<(int)blocks, kLossThreads, 0, st>>>(img, tgt, n, kind, vec, grad, loss);
  return cudaGetLastError();
}

}  // namespace gsr

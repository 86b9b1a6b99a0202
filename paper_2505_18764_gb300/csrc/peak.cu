// Measurement helper, not part of the method: the FP32 FMA rate this GPU
// sustains, the ceiling of the FP32-bound raster kernels.  Every thread runs
// eight independent FMA chains (enough to cover the FMA latency at full
// occupancy); the result is stored so the chains are not optimised away.
#include "common.cuh"

namespace gsr {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

__global__ void __launch_bounds__(kPeakThreads) fma_rate_kernel(int iters, float* out) {
  float x[kPeakChains];
  const float m = 0.9999f + 1e-7f * (float)(threadIdx.x & 7);
  const float c = 1e-6f * (float)(blockIdx.x & 15);
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) x[k] = fmaf(x[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == 1234.5f) out[blockIdx.x] = s;   // practically never true; keeps the chains live
}

int record_error(int code, const char* msg);  // sets gs_last_error() (api.cu)

}  // namespace gsr

using namespace gsr;

extern "C" int gs_fp32_fma_rate(int32_t iters, double* tflops, gs_stream_t stream) {
  if (iters <= 0 || !tflops) return record_error(GS_ERR_INVALID_ARG, "iters must be > 0, tflops non-null");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel, kPeakThreads, 0);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    fma_rate_kernel<<<grid, kPeakThreads, 0, st>>>(iters / 8 + 1, nullptr);   // warm-up
    cudaEventRecord(a, st);
    fma_rate_kernel<<<grid, kPeakThreads, 0, st>>>(iters, nullptr);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return record_error(GS_ERR_CUDA, cudaGetErrorString(e));
  const double flops = 2.0 * kPeakChains * (double)iters * grid * kPeakThreads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return GS_OK;
}

// Compositing of depth slabs.
//
// Front-to-back blending (Eq. 2) is associative over contiguous runs of the
// depth order: a slab k rendered on its own, starting from T = 1, gives the
// colour C_k and transmittance T_k of its fragments, and the image is the
// "over" composite C = C_0 + T_0 (C_1 + T_1 (C_2 + ...)), T = T_0 T_1 ...
// For the backward of slab k this kernel also gives t_front_k = T_0 ... T_{k-1}
// (the slab's colour enters the image scaled by it) and behind_k, the
// composite of the slabs after k (C' of the slab's first fragment includes
// T_k behind_k).  One thread per pixel; every array is coalesced.
#include "common.cuh"

namespace gsr {

__global__ void __launch_bounds__(256) slab_composite_kernel(
    const void* __restrict__ states, int fmt, int n_slabs, int64_t npix, float* __restrict__ image,
    float* __restrict__ trans, float* __restrict__ t_front, float* __restrict__ behind) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    // back to front: behind_{n-1} = 0, behind_{k-1} = C_k + T_k behind_k
    float b0 = 0.f, b1 = 0.f, b2 = 0.f, tprod = 1.f;
    for (int k = n_slabs - 1; k >= 0; --k) {
      if (behind) {
        float* bk = behind + ((int64_t)k * npix + p) * 3;
        bk[0] = b0;
        bk[1] = b1;
        bk[2] = b2;
      }
      const float4 s = load_state(states, fmt, (size_t)((int64_t)k * npix + p));
      b0 = fmaf(s.w, b0, s.x);
      b1 = fmaf(s.w, b1, s.y);
      b2 = fmaf(s.w, b2, s.z);
      tprod *= s.w;
    }
    if (image) {
      image[3 * p] = b0;
      image[3 * p + 1] = b1;
      image[3 * p + 2] = b2;
    }
    if (trans) trans[p] = tprod;
    if (t_front) {
      float tf = 1.f;
      for (int k = 0; k < n_slabs; ++k) {
        t_front[(int64_t)k * npix + p] = tf;
        tf *= load_state(states, fmt, (size_t)((int64_t)k * npix + p)).w;
      }
    }
  }
}

cudaError_t launch_slab_composite(const void* states, int fmt, int n_slabs, int64_t npix,
                                  float* image, float* trans, float* t_front, float* behind,
                                  int num_sms, cudaStream_t st) {
  if (npix == 0) return cudaSuccess;
  int64_t blocks = (npix + 255) / 256;
  if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
  slab_composite_kernel<<<(int)blocks, 256, 0, st>>>(states, fmt, n_slabs, npix, image, trans,
                                                      t_front, behind);
  return cudaGetLastError();
}

}  // namespace gsr

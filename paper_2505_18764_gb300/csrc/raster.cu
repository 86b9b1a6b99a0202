// Forward and backward rasterization over 16x16 pixel blocks.
//
// One CTA per block, one thread per pixel.  The block's (depth-ordered) splat
// list is staged into shared memory 256 records at a time; every thread then
// walks the same splat sequence, so all 256 fragments a block produces for a
// splat are evaluated by the CTA at the same moment.  That is the CUDA
// counterpart of the paper's ordered fragment processing: a pixel is owned by
// one thread, so no interlock is needed (the race that programmable blending
// guards against cannot occur), and fragments of one splat are always
// together in a warp and a CTA (the "cohesion" of Sec. 3.2.2 holds by
// construction).
//
// Forward (Eq. 2, Sec. 2.1.2): alpha = min(0.99, o exp(power)), fragments with
// alpha < 1/255 skipped, T-culling skips fragment i iff T_i < t_cull
// (Procedure 1; the same rule in both passes, so the backward is the exact
// gradient of the image the forward produced).
//
// Backward (Procedure 1): (C', T) start at (stored C, 1); per fragment
// dL/dc = g alpha T (Eq. 3), dL/dalpha = g . (c T - C') / (1 - alpha) (Eq. 7),
// then C' -= T alpha c (Eq. 6) and T *= 1 - alpha (Eq. 5).  The chain rule to
// the 2D splat parameters follows; the nine per-fragment values are reduced
// per splat (Procedure 2's role) by a warp transpose-reduce and a cross-warp
// shared-memory sum, so one vector atomic triple per (splat, block) reaches
// global memory.
#include "common.cuh"

namespace gsr {

constexpr int kBatch = 256;   // records staged per round

// Each warp owns a 16x2 strip of the block (lanes 0-15 the upper row, 16-31
// the lower).  After a batch of records is staged, every lane tests one splat
// against its warp's strip (strip_may_hit); the ballots give each warp a
// bitmask of the splats that can touch its strip, and the warp walks only
// those, in depth order.
__device__ __forceinline__ void stage_batch(const uint32_t* __restrict__ pair_ranks,
                                            const SplatRec* __restrict__ rec, uint32_t s,
                                            uint32_t end, float4* s_a, float4* s_b, float4* s_c,
                                            uint32_t* s_rank) {
  const uint32_t i = s + threadIdx.x;
  if (i < end) {
    const uint32_t r = pair_ranks[i];
    s_rank[threadIdx.x] = r;
    const SplatRec R = rec[r];
    s_a[threadIdx.x] = R.a;
    s_b[threadIdx.x] = R.b;
    s_c[threadIdx.x] = R.c;
  }
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlockPixels) raster_fwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ pair_ranks,
    const SplatRec* __restrict__ rec, int W, int H, int gw, float t_cull, int fmt,
    float* __restrict__ image, void* __restrict__ state, uint32_t* __restrict__ last_out,
    uint32_t* __restrict__ ncontrib) {
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_rank[kBatch];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bx = blockIdx.x % gw, by = blockIdx.x / gw;
  const int x = bx * kBlock + (lane & 15), y = by * kBlock + 2 * warp + (lane >> 4);
  const bool inside = x < W && y < H;
  const uint2 range = ranges[blockIdx.x];
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const float xs = (float)(bx * kBlock) + 0.5f, ys = (float)(by * kBlock + 2 * warp) + 0.5f;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  uint32_t last = kNone, n = 0;
  bool done = !inside;
  for (uint32_t s = range.x; s < range.y; s += kBatch) {
    if (__syncthreads_and(done)) break;
    stage_batch(pair_ranks, rec, s, range.y, s_a, s_b, s_c, s_rank);
    __syncthreads();
    const int cnt = min((uint32_t)kBatch, range.y - s);
    for (int k = 0; k * 32 < cnt; ++k) {
      const int jt = k * 32 + lane;
      uint32_t m = __ballot_sync(0xffffffffu, jt < cnt && strip_may_hit(s_a[jt], s_b[jt], xs, ys));
      if (__all_sync(0xffffffffu, done)) break;
      while (m) {
        const int j = k * 32 + __ffs(m) - 1;
        m &= m - 1;
        if (done) continue;
        const float4 a = s_a[j];
        const float4 b = s_b[j];
        float y1, y2;
        const float q = frag_q(px, py, a, b, y1, y2);
        if (q > b.y) continue;             // alpha < 1/255
        const float4 c = s_c[j];
        float G, at;
        const float alpha = frag_alpha(c.w, q, G, at);
        const float w = __fmul_rn(alpha, T);
        C0 = __fmaf_rn(w, c.x, C0);
        C1 = __fmaf_rn(w, c.y, C1);
        C2 = __fmaf_rn(w, c.z, C2);
        T = next_T(T, alpha);
        last = s_rank[j];
        ++n;
        if (T < t_cull) done = true;       // every later fragment is T-culled
      }
    }
  }
  if (inside) {
    const size_t pix = (size_t)y * W + x;
    if (image) {
      image[3 * pix + 0] = C0;
      image[3 * pix + 1] = C1;
      image[3 * pix + 2] = C2;
    }
    store_state(state, fmt, pix, C0, C1, C2, T);
    last_out[pix] = last;
    if (ncontrib) ncontrib[pix] = n;
  }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// Sum of nine values over the warp, scattered so that each even lane ends with
// one total: 12 shuffles instead of 45 for nine butterflies.  Lane l holds the
// value with index  (b1 + 2 b2) + 3 b3 + 5 b4  (bits of l), valid when
// b1 + 2 b2 < 3, (b1 + 2 b2) + 3 b3 < 5 and the index < 9.
__device__ __forceinline__ float warp_transpose_reduce9(const float v[9], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float k1[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float lo = v[i];
    const float hi = (i + 5 < 9) ? v[i + 5] : 0.f;
    k1[i] = (b4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b4 ? lo : hi, 16);
  }
  float k2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float lo = k1[i];
    const float hi = (i + 3 < 5) ? k1[i + 3] : 0.f;
    k2[i] = (b3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
  }
  float k3[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float lo = k2[i];
    const float hi = (i + 2 < 3) ? k2[i + 2] : 0.f;
    k3[i] = (b2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 4);
  }
  const float k4 = (b1 ? k3[1] : k3[0]) + __shfl_xor_sync(0xffffffffu, b1 ? k3[0] : k3[1], 2);
  return k4 + __shfl_xor_sync(0xffffffffu, k4, 1);
}

__device__ __forceinline__ int transpose_slot(int lane) {
  const int b1 = (lane >> 1) & 1, b2 = (lane >> 2) & 1, b3 = (lane >> 3) & 1, b4 = (lane >> 4) & 1;
  const int i2 = b1 + 2 * b2;
  const int i1 = i2 + 3 * b3;
  const int v = i1 + 5 * b4;
  return ((lane & 1) == 0 && i2 < 3 && i1 < 5 && v < 9) ? v : -1;
}

template <int MODE>
__global__ void __launch_bounds__(kBlockPixels) raster_bwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ pair_ranks,
    const SplatRec* __restrict__ rec, int W, int H, int gw, float t_cull, int fmt,
    const void* __restrict__ state, const uint32_t* __restrict__ last_in,
    const float* __restrict__ dLdC, float* __restrict__ g2d, int threshold) {
  constexpr int kWarps = kBlockPixels / 32;
  __shared__ float4 s_a[kBatch];
  __shared__ float4 s_b[kBatch];
  __shared__ float4 s_c[kBatch];
  __shared__ uint32_t s_rank[kBatch];
  __shared__ __align__(16) float s_part[32][kWarps][12];
  __shared__ uint32_t s_mask[kWarps];
  __shared__ uint32_t s_end;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bx = blockIdx.x % gw, by = blockIdx.x / gw;
  const int x = bx * kBlock + (lane & 15), y = by * kBlock + 2 * warp + (lane >> 4);
  const bool inside = x < W && y < H;
  const uint2 range = ranges[blockIdx.x];
  const float px = (float)x + 0.5f, py = (float)y + 0.5f;
  const float xs = (float)(bx * kBlock) + 0.5f, ys = (float)(by * kBlock + 2 * warp) + 0.5f;
  const int slot = transpose_slot(lane);

  float Cp0 = 0.f, Cp1 = 0.f, Cp2 = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  uint32_t my_end = 0;
  if (inside) {
    const size_t pix = (size_t)y * W + x;
    const float4 st = load_state(state, fmt, pix);
    Cp0 = st.x; Cp1 = st.y; Cp2 = st.z;
    g0 = dLdC[3 * pix]; g1 = dLdC[3 * pix + 1]; g2 = dLdC[3 * pix + 2];
    const uint32_t l = last_in[pix];
    my_end = (l == kNone) ? 0u : l + 1u;
  }
  if (tid == 0) s_end = 0;
  // padding slots 9..11 of the partial sums stay zero
  for (int i = tid; i < 32 * kWarps; i += kBlockPixels) {
    float* p = &s_part[0][0][0] + i * 12;
    p[9] = 0.f; p[10] = 0.f; p[11] = 0.f;
  }
  __syncthreads();
  if (my_end) atomicMax(&s_end, my_end);
  float T = 1.f;
  bool done = my_end == 0;
  __syncthreads();
  const uint32_t block_end = s_end;  // depth ranks >= this contribute nowhere in the block

  for (uint32_t s = range.x; s < range.y; s += kBatch) {
    if (__syncthreads_and(done)) break;
    stage_batch(pair_ranks, rec, s, range.y, s_a, s_b, s_c, s_rank);
    __syncthreads();
    if (s_rank[0] >= block_end) break;   // uniform: ranks ascend within the block
    const int cnt = min((uint32_t)kBatch, range.y - s);
    for (int k = 0; k * 32 < cnt; ++k) {
      const int jt = k * 32 + lane;
      uint32_t m = __ballot_sync(0xffffffffu, jt < cnt && strip_may_hit(s_a[jt], s_b[jt], xs, ys));
      if (__all_sync(0xffffffffu, done)) m = 0u;
      if (MODE != GS_REDUCE_NAIVE && lane == 0) s_mask[warp] = m;
      while (m) {
        const int jj = __ffs(m) - 1;
        m &= m - 1;
        const int j = k * 32 + jj;
        float v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = 0.f;
        bool frag = false;
        if (!done) {
          if (s_rank[j] >= my_end) {
            done = true;                   // past this pixel's last fragment
          } else {
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            float y1, y2;
            const float q = frag_q(px, py, a, b, y1, y2);
            if (q <= b.y) {
              frag = true;
              const float4 c = s_c[j];
              float G, at;
              const float alpha = frag_alpha(c.w, q, G, at);
              const float oma = __fsub_rn(1.0f, alpha);
              const float wT = __fmul_rn(alpha, T);
              // Eq. 3
              v[5] = g0 * wT;
              v[6] = g1 * wT;
              v[7] = g2 * wT;
              // Eq. 7 with C'_i before its update
              const float dLda = (g0 * (c.x * T - Cp0) + g1 * (c.y * T - Cp1) + g2 * (c.z * T - Cp2)) *
                                 __frcp_rn(oma);
              // Eq. 6, Eq. 5
              Cp0 -= wT * c.x;
              Cp1 -= wT * c.y;
              Cp2 -= wT * c.z;
              T = next_T(T, alpha);
              if (T < t_cull) done = true;
              // alpha = min(0.99, o G): no gradient through the clamp
              const float d_at = at < kAlphaMax ? dLda : 0.f;
              v[8] = G * d_at;
              // z = Sigma^-1 d = L^-T L^-1 d, in units of 1 / (2 ln 2):
              // dpower/dmu_2D = z and dpower/dSigma_2D = z z^T / 2
              const float w = at * d_at;
              const float z1 = b.x * y2;
              const float z0 = a.z * y1 - a.w * z1;
              v[0] = w * z0;
              v[1] = w * z1;
              v[2] = w * z0 * z0;
              v[3] = w * z0 * z1;
              v[4] = w * z1 * z1;
            }
          }
        }
        float* gdst = g2d + (size_t)s_rank[j] * 12;
        if (MODE == GS_REDUCE_NAIVE) {
          if (frag) {
            red_add_v4(gdst, v[0], v[1], v[2], v[3]);
            red_add_v4(gdst + 4, v[4], v[5], v[6], v[7]);
            red_add_v4(gdst + 8, v[8], 0.f, 0.f, 0.f);
          }
        } else {
          const uint32_t active = __ballot_sync(0xffffffffu, frag);
          const bool reduce = active != 0u && __popc(active) >= threshold;
          float tot = 0.f;
          if (active != 0u && !reduce) {    // few lanes: add directly (Sec. 3.2.3)
            if (frag) {
              red_add_v4(gdst, v[0], v[1], v[2], v[3]);
              red_add_v4(gdst + 4, v[4], v[5], v[6], v[7]);
              red_add_v4(gdst + 8, v[8], 0.f, 0.f, 0.f);
            }
          } else if (reduce) {
            tot = warp_transpose_reduce9(v, lane);
          }
          if (slot >= 0) s_part[jj][warp][slot] = tot;
        }
      }
      if (MODE != GS_REDUCE_NAIVE) {
        __syncthreads();
        if (MODE == GS_REDUCE_BLOCK) {
          // one thread per (splat, float4 group): sum the warps that looked at it
          if (tid < 32 * 3) {
            const int jj = tid / 3, q = tid % 3;
            if (k * 32 + jj < cnt) {
              float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int w = 0; w < kWarps; ++w) {
                if ((s_mask[w] >> jj) & 1u) {
                  const float4 p = *reinterpret_cast<const float4*>(&s_part[jj][w][4 * q]);
                  acc.x += p.x; acc.y += p.y; acc.z += p.z; acc.w += p.w;
                }
              }
              if (acc.x != 0.f || acc.y != 0.f || acc.z != 0.f || acc.w != 0.f)
                red_add_v4(g2d + (size_t)s_rank[k * 32 + jj] * 12 + 4 * q, acc.x, acc.y, acc.z, acc.w);
            }
          }
        } else {
          // GS_REDUCE_WARP: each warp adds its own partial sums
          if ((s_mask[warp] >> lane) & 1u) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const float4 p = *reinterpret_cast<const float4*>(&s_part[lane][warp][4 * q]);
              if (p.x != 0.f || p.y != 0.f || p.z != 0.f || p.w != 0.f)
                red_add_v4(g2d + (size_t)s_rank[k * 32 + lane] * 12 + 4 * q, p.x, p.y, p.z, p.w);
            }
          }
        }
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Summed L1 / L2 image loss and its gradient.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ img,
                                                   const float* __restrict__ tgt, int64_t n,
                                                   int kind, float* __restrict__ grad,
                                                   double* __restrict__ loss) {
  __shared__ double s_w[8];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = img[i] - tgt[i];
    float g;
    if (kind == GS_LOSS_L1) {
      acc += fabsf(d);
      g = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
    } else {
      acc += (double)d * d;
      g = 2.f * d;
    }
    if (grad) grad[i] = g;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
    atomicAdd(loss, t);
  }
}

cudaError_t launch_raster_fwd(const uint2* ranges, const uint32_t* pair_ranks, const SplatRec* rec,
                              int W, int H, int gw, int gh, float t_cull, int fmt, float* image,
                              void* state, uint32_t* last, uint32_t* ncontrib, cudaStream_t st) {
  const int blocks = gw * gh;
  if (blocks == 0) return cudaSuccess;
  raster_fwd_kernel<<<blocks, kBlockPixels, 0, st>>>(ranges, pair_ranks, rec, W, H, gw, t_cull, fmt,
                                                     image, state, last, ncontrib);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const uint2* ranges, const uint32_t* pair_ranks, const SplatRec* rec,
                              int W, int H, int gw, int gh, float t_cull, int fmt,
                              const void* state, const uint32_t* last, const float* dLdC,
                              float* g2d, int mode, int threshold, cudaStream_t st) {
  const int blocks = gw * gh;
  if (blocks == 0) return cudaSuccess;
  if (mode == GS_REDUCE_NAIVE)
    raster_bwd_kernel<GS_REDUCE_NAIVE><<<blocks, kBlockPixels, 0, st>>>(
        ranges, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
  else if (mode == GS_REDUCE_WARP)
    raster_bwd_kernel<GS_REDUCE_WARP><<<blocks, kBlockPixels, 0, st>>>(
        ranges, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
  else
    raster_bwd_kernel<GS_REDUCE_BLOCK><<<blocks, kBlockPixels, 0, st>>>(
        ranges, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* img, const float* tgt, int64_t n, int kind, float* grad,
                        double* loss, int num_sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  if (blocks > num_sms * 4) blocks = num_sms * 4;
  if (blocks < 1) blocks = 1;
  loss_kernel<<<(int)blocks, 256, 0, st>>>(img, tgt, n, kind, grad, loss);
  return cudaGetLastError();
}

}  // namespace gsr

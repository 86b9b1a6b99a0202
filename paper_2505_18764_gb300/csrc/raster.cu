// Forward and backward rasterization over 16x16 pixel blocks.
//
// One CTA of 128 threads per block; each thread owns two pixels of one column
// (rows r and r + 2 of its warp's 16x4 band), so every warp covers a compact
// 16x4 footprint with two independent per-pixel dependency chains per lane.
// The block's depth-ordered splat list is staged into shared memory 256
// records at a time (asynchronous copies, double-buffered); every thread walks
// the same splat sequence, so all fragments a block produces for one splat
// are evaluated together.  That is the CUDA counterpart of the paper's ordered
// fragment processing: a pixel belongs to one thread, so no interlock is
// needed (the race programmable blending guards against cannot occur), and a
// splat's fragments are always together in a warp and a CTA (the "cohesion"
// of Sec. 3.2.3 holds by construction).  Each warp first tests the staged
// splats against its footprint (rect_may_hit) and then walks only those that
// can touch it.
//
// Forward (Eq. 2, Sec. 2.1.2): alpha = min(0.99, o exp(power)), fragments with
// alpha < 1/255 skipped, T-culling skips fragment i iff T_i < t_cull
// (Procedure 1; the same rule in both passes, so the backward is the exact
// gradient of the image the forward produced).
//
// Backward (Procedure 1): (C', T) start at (stored C, 1); per fragment
// dL/dc = g alpha T (Eq. 3), dL/dalpha = g . (c T - C') / (1 - alpha) (Eq. 7),
// then C' -= T alpha c (Eq. 6) and T *= 1 - alpha (Eq. 5).  The chain rule to
// the 2D splat parameters follows; the nine per-fragment values of a thread's
// two pixels are added, reduced over the warp by a transpose-reduce and over
// the CTA's warps in shared memory, so one vector-atomic triple per
// (splat, block) reaches global memory (Procedure 2's role).
#include "common.cuh"

namespace gsr {

constexpr int kThreads = 128;                 // 4 warps, two pixels each per lane
constexpr int kWarps = kThreads / 32;
constexpr int kBatch = 256;                   // records staged per round
constexpr int kRecPerThread = kBatch / kThreads;

struct Stage {
  float4 a[kBatch];
  float4 b[kBatch];
  float4 c[kBatch];
  uint32_t rank[kBatch];
};

// Issue the copies of batch [s, min(s + kBatch, end)) into `st`; `rk` holds the
// depth ranks of this thread's records (loaded one batch earlier).
__device__ __forceinline__ void stage_issue(Stage& st, const SplatRec* __restrict__ rec,
                                            uint32_t s, uint32_t end,
                                            const uint32_t (&rk)[kRecPerThread]) {
#pragma unroll
  for (int u = 0; u < kRecPerThread; ++u) {
    const int t = threadIdx.x + u * kThreads;
    if (s + t < end) {
      const SplatRec* g = rec + rk[u];
      cp_async16(&st.a[t], &g->a);
      cp_async16(&st.b[t], &g->b);
      cp_async16(&st.c[t], &g->c);
      st.rank[t] = rk[u];
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ void load_ranks(const uint32_t* __restrict__ pair_ranks, uint32_t s,
                                           uint32_t end, uint32_t (&rk)[kRecPerThread]) {
#pragma unroll
  for (int u = 0; u < kRecPerThread; ++u) {
    const uint32_t i = s + threadIdx.x + u * kThreads;
    rk[u] = i < end ? pair_ranks[i] : 0u;
  }
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
struct PixelFwd {
  float T, C0, C1, C2;
  uint32_t last, n;
  bool done;
};

__device__ __forceinline__ void blend(PixelFwd& p, float alpha, const float4& c, uint32_t rank,
                                      float t_cull) {
  const float w = __fmul_rn(alpha, p.T);
  p.C0 = __fmaf_rn(w, c.x, p.C0);
  p.C1 = __fmaf_rn(w, c.y, p.C1);
  p.C2 = __fmaf_rn(w, c.z, p.C2);
  p.T = next_T(p.T, alpha);
  p.last = rank;
  ++p.n;
  if (p.T < t_cull) p.done = true;   // every later fragment is T-culled
}

__device__ __forceinline__ void write_fwd(const PixelFwd& p, int x, int y, int W, int H, int fmt,
                                          float* image, void* state, uint32_t* last_out,
                                          uint32_t* ncontrib) {
  if (x >= W || y >= H) return;
  const size_t pix = (size_t)y * W + x;
  if (image) {
    image[3 * pix + 0] = p.C0;
    image[3 * pix + 1] = p.C1;
    image[3 * pix + 2] = p.C2;
  }
  store_state(state, fmt, pix, p.C0, p.C1, p.C2, p.T);
  last_out[pix] = p.last;
  if (ncontrib) ncontrib[pix] = p.n;
}

__global__ void __launch_bounds__(kThreads) raster_fwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pair_ranks, const SplatRec* __restrict__ rec, int W, int H, int gw,
    float t_cull, int fmt, float* __restrict__ image, void* __restrict__ state,
    uint32_t* __restrict__ last_out, uint32_t* __restrict__ ncontrib) {
  __shared__ Stage stg[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = order[blockIdx.x];   // longest lists first
  const int bx = tile % gw, by = tile / gw;
  const int x = bx * kBlock + (lane & 15);
  const int ya = by * kBlock + 4 * warp + (lane >> 4), yb = ya + 2;
  const float px = (float)x + 0.5f, pya = (float)ya + 0.5f, pyb = (float)yb + 0.5f;
  const float xs = (float)(bx * kBlock) + 0.5f, ys = (float)(by * kBlock + 4 * warp) + 0.5f;
  const uint2 range = ranges[tile];
  PixelFwd pa{1.f, 0.f, 0.f, 0.f, kNone, 0u, !(x < W && ya < H)};
  PixelFwd pb{1.f, 0.f, 0.f, 0.f, kNone, 0u, !(x < W && yb < H)};

  uint32_t rk[kRecPerThread];
  load_ranks(pair_ranks, range.x, range.y, rk);
  if (range.x < range.y) stage_issue(stg[0], rec, range.x, range.y, rk);
  load_ranks(pair_ranks, range.x + kBatch, range.y, rk);
  int cur = 0;
  for (uint32_t s = range.x; s < range.y; s += kBatch, cur ^= 1) {
    cp_async_wait_all();
    if (__syncthreads_and(pa.done && pb.done)) break;
    if (s + kBatch < range.y) {     // next batch in flight while this one is blended
      stage_issue(stg[cur ^ 1], rec, s + kBatch, range.y, rk);
      load_ranks(pair_ranks, s + 2 * kBatch, range.y, rk);
    }
    const Stage& S = stg[cur];
    const int cnt = min((uint32_t)kBatch, range.y - s);
    for (int k = 0; k * 32 < cnt; ++k) {
      if (__all_sync(0xffffffffu, pa.done && pb.done)) break;
      const int jt = k * 32 + lane;
      uint32_t m = __ballot_sync(0xffffffffu,
                                 jt < cnt && rect_may_hit(S.a[jt], S.b[jt], xs, ys, 15.f, 3.f));
      while (m) {
        const int j = k * 32 + __ffs(m) - 1;
        m &= m - 1u;
        const float4 a = S.a[j];
        const float4 b = S.b[j];
        float y1, y2;
        const float qa = frag_q(px, pya, a, b, y1, y2);
        const float qb = frag_q(px, pyb, a, b, y1, y2);
        const bool ha = !pa.done && qa <= b.y;   // alpha >= 1/255
        const bool hb = !pb.done && qb <= b.y;
        if (!(ha || hb)) continue;
        const float4 c = S.c[j];
        const uint32_t rank = S.rank[j];
        float G, at;
        if (ha) blend(pa, frag_alpha(c.w, qa, G, at), c, rank, t_cull);
        if (hb) blend(pb, frag_alpha(c.w, qb, G, at), c, rank, t_cull);
      }
    }
  }
  cp_async_wait_all();
  write_fwd(pa, x, ya, W, H, fmt, image, state, last_out, ncontrib);
  write_fwd(pb, x, yb, W, H, fmt, image, state, last_out, ncontrib);
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

struct PixelBwd {
  float Cp0, Cp1, Cp2, T, g0, g1, g2;
  uint32_t end;   // depth rank after the pixel's last fragment
  bool done;
};

__device__ __forceinline__ void load_pixel_bwd(PixelBwd& p, int x, int y, int W, int H, int fmt,
                                               const void* state, const uint32_t* last_in,
                                               const float* dLdC) {
  p.Cp0 = p.Cp1 = p.Cp2 = 0.f;
  p.g0 = p.g1 = p.g2 = 0.f;
  p.T = 1.f;
  p.end = 0;
  if (x < W && y < H) {
    const size_t pix = (size_t)y * W + x;
    const float4 st = load_state(state, fmt, pix);
    p.Cp0 = st.x; p.Cp1 = st.y; p.Cp2 = st.z;
    p.g0 = dLdC[3 * pix]; p.g1 = dLdC[3 * pix + 1]; p.g2 = dLdC[3 * pix + 2];
    const uint32_t l = last_in[pix];
    p.end = (l == kNone) ? 0u : l + 1u;
  }
  p.done = p.end == 0;
}

// One fragment of Procedure 1 plus the chain rule to the 2D parameters; the
// nine values are added into v.
__device__ __forceinline__ void grad_fragment(PixelBwd& p, float q, float y1, float y2,
                                              const float4& a, const float4& b, const float4& c,
                                              float t_cull, float v[9]) {
  float G, at;
  const float alpha = frag_alpha(c.w, q, G, at);
  const float oma = __fsub_rn(1.0f, alpha);
  const float wT = __fmul_rn(alpha, p.T);
  // Eq. 3
  v[5] += p.g0 * wT;
  v[6] += p.g1 * wT;
  v[7] += p.g2 * wT;
  // Eq. 7 with C'_i before its update
  const float dLda = (p.g0 * (c.x * p.T - p.Cp0) + p.g1 * (c.y * p.T - p.Cp1) +
                      p.g2 * (c.z * p.T - p.Cp2)) * __fdividef(1.0f, oma);
  // Eq. 6, Eq. 5
  p.Cp0 -= wT * c.x;
  p.Cp1 -= wT * c.y;
  p.Cp2 -= wT * c.z;
  p.T = next_T(p.T, alpha);
  if (p.T < t_cull) p.done = true;
  // alpha = min(0.99, o G): no gradient through the clamp
  const float d_at = at < kAlphaMax ? dLda : 0.f;
  v[8] += G * d_at;
  // z = Sigma^-1 d = L^-T L^-1 d, in units of 1 / (2 ln 2):
  // dpower/dmu_2D = z and dpower/dSigma_2D = z z^T / 2
  const float w = at * d_at;
  const float z1 = b.x * y2;
  const float z0 = a.z * y1 - a.w * z1;
  const float wz0 = w * z0, wz1 = w * z1;
  v[0] += wz0;
  v[1] += wz1;
  v[2] += wz0 * z0;
  v[3] += wz0 * z1;
  v[4] += wz1 * z1;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ pair_ranks, const SplatRec* __restrict__ rec, int W, int H, int gw,
    float t_cull, int fmt, const void* __restrict__ state, const uint32_t* __restrict__ last_in,
    const float* __restrict__ dLdC, float* __restrict__ g2d, int threshold) {
  __shared__ Stage stg[2];
  __shared__ __align__(16) float s_part[32][kWarps][12];
  __shared__ uint32_t s_mask[kWarps];
  __shared__ uint32_t s_end;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t tile = order[blockIdx.x];   // longest lists first
  const int bx = tile % gw, by = tile / gw;
  const int x = bx * kBlock + (lane & 15);
  const int ya = by * kBlock + 4 * warp + (lane >> 4), yb = ya + 2;
  const float px = (float)x + 0.5f, pya = (float)ya + 0.5f, pyb = (float)yb + 0.5f;
  const float xs = (float)(bx * kBlock) + 0.5f, ys = (float)(by * kBlock + 4 * warp) + 0.5f;
  const uint2 range = ranges[tile];
  const int slot = transpose_slot(lane);

  PixelBwd pa, pb;
  load_pixel_bwd(pa, x, ya, W, H, fmt, state, last_in, dLdC);
  load_pixel_bwd(pb, x, yb, W, H, fmt, state, last_in, dLdC);
  if (tid == 0) s_end = 0;
  // padding slots 9..11 of the partial sums stay zero
  for (int i = tid; i < 32 * kWarps; i += kThreads) {
    float* p = &s_part[0][0][0] + i * 12;
    p[9] = 0.f; p[10] = 0.f; p[11] = 0.f;
  }
  __syncthreads();
  const uint32_t mine = max(pa.end, pb.end);
  if (mine) atomicMax(&s_end, mine);
  __syncthreads();
  const uint32_t block_end = s_end;  // depth ranks >= this contribute nowhere in the block

  uint32_t rk[kRecPerThread];
  load_ranks(pair_ranks, range.x, range.y, rk);
  if (range.x < range.y) stage_issue(stg[0], rec, range.x, range.y, rk);
  load_ranks(pair_ranks, range.x + kBatch, range.y, rk);
  int cur = 0;
  for (uint32_t s = range.x; s < range.y; s += kBatch, cur ^= 1) {
    cp_async_wait_all();
    if (__syncthreads_and(pa.done && pb.done)) break;
    const Stage& S = stg[cur];
    if (S.rank[0] >= block_end) break;   // uniform: ranks ascend within the block
    if (s + kBatch < range.y) {
      stage_issue(stg[cur ^ 1], rec, s + kBatch, range.y, rk);
      load_ranks(pair_ranks, s + 2 * kBatch, range.y, rk);
    }
    const int cnt = min((uint32_t)kBatch, range.y - s);
    for (int k = 0; k * 32 < cnt; ++k) {
      const int jt = k * 32 + lane;
      uint32_t m = __ballot_sync(0xffffffffu,
                                 jt < cnt && rect_may_hit(S.a[jt], S.b[jt], xs, ys, 15.f, 3.f));
      if (__all_sync(0xffffffffu, pa.done && pb.done)) m = 0u;
      if (MODE != GS_REDUCE_NAIVE && lane == 0) s_mask[warp] = m;
      while (m) {
        const int jj = __ffs(m) - 1;
        m &= m - 1u;
        const int j = k * 32 + jj;
        const uint32_t rank = S.rank[j];
        float v[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) v[q] = 0.f;
        bool frag = false;
        if (!(pa.done && pb.done)) {
          const float4 a = S.a[j];
          const float4 b = S.b[j];
          float y1a, y2a, y1b, y2b;
          const float qa = frag_q(px, pya, a, b, y1a, y2a);
          const float qb = frag_q(px, pyb, a, b, y1b, y2b);
          if (rank >= pa.end) pa.done = true;   // past this pixel's last fragment
          if (rank >= pb.end) pb.done = true;
          const bool ha = !pa.done && qa <= b.y;
          const bool hb = !pb.done && qb <= b.y;
          if (ha || hb) {
            const float4 c = S.c[j];
            frag = true;
            if (ha) grad_fragment(pa, qa, y1a, y2a, a, b, c, t_cull, v);
            if (hb) grad_fragment(pb, qb, y1b, y2b, a, b, c, t_cull, v);
          }
        }
        float* gdst = g2d + (size_t)rank * 12;
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
          if (active != 0u && !reduce) {    // few lanes: add directly (Sec. 3.2.4)
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
                red_add_v4(g2d + (size_t)S.rank[k * 32 + jj] * 12 + 4 * q, acc.x, acc.y, acc.z,
                           acc.w);
            }
          }
        } else {
          // GS_REDUCE_WARP: each warp adds its own partial sums
          if ((s_mask[warp] >> lane) & 1u) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const float4 p = *reinterpret_cast<const float4*>(&s_part[lane][warp][4 * q]);
              if (p.x != 0.f || p.y != 0.f || p.z != 0.f || p.w != 0.f)
                red_add_v4(g2d + (size_t)S.rank[k * 32 + lane] * 12 + 4 * q, p.x, p.y, p.z, p.w);
            }
          }
        }
        __syncthreads();
      }
    }
  }
  cp_async_wait_all();
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

cudaError_t launch_raster_fwd(const uint2* ranges, const uint32_t* order, const uint32_t* pair_ranks,
                              const SplatRec* rec, int W, int H, int gw, int gh, float t_cull,
                              int fmt, float* image, void* state, uint32_t* last,
                              uint32_t* ncontrib, cudaStream_t st) {
  const int blocks = gw * gh;
  if (blocks == 0) return cudaSuccess;
  raster_fwd_kernel<<<blocks, kThreads, 0, st>>>(ranges, order, pair_ranks, rec, W, H, gw, t_cull,
                                                 fmt, image, state, last, ncontrib);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const uint2* ranges, const uint32_t* order, const uint32_t* pair_ranks,
                              const SplatRec* rec, int W, int H, int gw, int gh, float t_cull,
                              int fmt, const void* state, const uint32_t* last, const float* dLdC,
                              float* g2d, int mode, int threshold, cudaStream_t st) {
  const int blocks = gw * gh;
  if (blocks == 0) return cudaSuccess;
  if (mode == GS_REDUCE_NAIVE)
    raster_bwd_kernel<GS_REDUCE_NAIVE><<<blocks, kThreads, 0, st>>>(
        ranges, order, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
  else if (mode == GS_REDUCE_WARP)
    raster_bwd_kernel<GS_REDUCE_WARP><<<blocks, kThreads, 0, st>>>(
        ranges, order, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
  else
    raster_bwd_kernel<GS_REDUCE_BLOCK><<<blocks, kThreads, 0, st>>>(
        ranges, order, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d, threshold);
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

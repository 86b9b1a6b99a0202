// Device-side definitions shared by the kernels of the splat rasterizer.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/gsr.h"

namespace gsr {

constexpr int kBlock = 16;                 // pixel block edge (16x16 = 256 threads)
constexpr int kBlockPixels = kBlock * kBlock;
constexpr uint32_t kNone = 0xFFFFFFFFu;    // "no splat" rank / culled key
constexpr float kAlphaMax = 0.99f;         // opacity clamp
constexpr float kDilation = 0.3f;          // EWA low-pass filter added to Sigma_2D
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr int kMaxShDegree = 3;

// Device status bits (workspace header word 0).
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

// Bounded spins: a look-back that waits longer than this many polls gives up,
// records kStatusTimeout and continues with what it has (never hangs).
constexpr uint32_t kSpinLimit = 1u << 22;

// Workspace header layout (u32 words).
struct Header {
  uint32_t status;
  uint32_t visible;        // V
  uint32_t pairs;          // P (clamped to the capacity)
  uint32_t pairs_wanted;   // P before clamping
  uint32_t live_pairs;     // pairs whose block the ellipse reaches (the rest are dropped)
  uint32_t pair_base;      // first (global) pair index of the current chunk
  uint32_t pad0[2];
  uint32_t tile_counter[16];  // dynamic tile ids: [0..3] depth-sort passes, [4..7] pair passes,
                              // [8] bin scan, [9..] standalone sort
  uint32_t depth_hist[4][256];
  uint32_t pair_hist[4][256];
  uint32_t n_items;            // raster work items (warp footprints) of the last binning
  uint32_t raster_next[2];     // next item to take: [0] forward, [1] backward
  uint32_t spare[61];
};

// Projected splat record, 48 B (three float4):
//   a = (mu_x, mu_y, i11, k), b = (i22, tau, mu_x_lo, mu_y_lo), c = (r, g, b, o)
// The Gaussian's exponent uses the inverse Cholesky factor of Sigma_2D:
//   q = y1^2 + y2^2,  y1 = i11 dx,  y2 = i22 (dy - k dx),  q = -log2(e) * power,
// i.e. k = s01 / s00, i11 = c / sqrt(s00), i22 = c sqrt(s00 / det) with
// c = sqrt(log2(e) / 2).  Unlike the conic form a dx^2 + 2 b dx dy + c dy^2,
// whose terms cancel along a needle's long axis (error ~ eigenvalue ratio x
// FP32 epsilon), this form loses only ~ its square root.  tau = log2(255 o):
// a fragment exists iff q <= tau (alpha >= 1/255).
// The screen centre is a float-float pair mu + mu_lo: at 1000-pixel
// coordinates one FP32 ulp is 6e-5 px, which over a hundred fragments moves a
// pixel's colour by ~1e-4; the pair keeps dx, dy exact to FP32 rounding of dx.
struct __align__(16) SplatRec {
  float4 a, b, c;
};

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// Fragment arithmetic.  Forward and backward must take identical decisions
// (alpha floor, T-culling) and recompute bit-identical T, so every operation
// here uses explicitly rounded intrinsics, which the compiler never contracts
// or reorders.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float frag_q(float px, float py, const float4& a, const float4& b,
                                        float& y1, float& y2) {
  const float dx = __fsub_rn(__fsub_rn(px, a.x), b.z);
  const float dy = __fsub_rn(__fsub_rn(py, a.y), b.w);
  y1 = __fmul_rn(a.z, dx);
  y2 = __fmul_rn(b.x, __fmaf_rn(-a.w, dx, dy));
  return __fmaf_rn(y1, y1, __fmul_rn(y2, y2));
}

// frag_q for the two pixels (px, pya) and (px, pyb) of one column: dx and y1
// are common, and each q is bit-identical to frag_q's.
__device__ __forceinline__ void frag_q2(float px, float pya, float pyb, const float4& a,
                                        const float4& b, float& y1, float& y2a, float& y2b,
                                        float& qa, float& qb) {
  const float dx = __fsub_rn(__fsub_rn(px, a.x), b.z);
  const float dya = __fsub_rn(__fsub_rn(pya, a.y), b.w);
  const float dyb = __fsub_rn(__fsub_rn(pyb, a.y), b.w);
  y1 = __fmul_rn(a.z, dx);
  y2a = __fmul_rn(b.x, __fmaf_rn(-a.w, dx, dya));
  y2b = __fmul_rn(b.x, __fmaf_rn(-a.w, dx, dyb));
  qa = __fmaf_rn(y1, y1, __fmul_rn(y2a, y2a));
  qb = __fmaf_rn(y1, y1, __fmul_rn(y2b, y2b));
}

// frag_alpha for a fragment that may be absent: a miss gets G = 0, so alpha,
// alpha T and every term derived from them are exact zeros and T * (1 - alpha)
// leaves T unchanged.
__device__ __forceinline__ float frag_alpha_masked(bool hit, float opacity, float q, float& G,
                                                   float& at) {
  G = hit ? ex2_approx(-q) : 0.0f;
  at = __fmul_rn(opacity, G);
  return fminf(kAlphaMax, at);
}

__device__ __forceinline__ float frag_alpha(float opacity, float q, float& G, float& at) {
  G = ex2_approx(-q);
  at = __fmul_rn(opacity, G);
  return fminf(kAlphaMax, at);
}

__device__ __forceinline__ float next_T(float T, float alpha) {
  return __fmul_rn(T, __fsub_rn(1.0f, alpha));
}

// Can any pixel centre of the rectangle [x0, x0 + wx] x [y0, y0 + wy] (pixel
// centres) hold a fragment of this splat?  q is convex, so its minimum over
// the rectangle is 0 if the splat's centre lies inside, else on one of the four
// edges, each a one-dimensional minimum at a clamped vertex.  The margin keeps
// the test conservative against the rounding of frag_q (it only decides what
// to skip).
__device__ __forceinline__ bool rect_may_hit(const float4& a, const float4& b, float x0, float y0,
                                             float wx, float wy) {
  const float X0 = (x0 - a.x) - b.z, X1 = X0 + wx;
  const float Y0 = (y0 - a.y) - b.w, Y1 = Y0 + wy;
  if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
  const float i11 = a.z, k = a.w, i22 = b.x;
  const float ki = k * i22;
  // row vertex dx = slope * dy; an approximate quotient moves the evaluated point by
  // ~1e-7 of its offset, which changes q by far less than the margin below
  const float slope = __fdividef(ki * i22, fmaf(i11, i11, ki * ki));
  const float lim = b.y + 0.01f + 1e-3f * b.y;
  float best = INFINITY;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const float Y = e ? Y1 : Y0;                         // horizontal edge
    const float dx = fminf(fmaxf(slope * Y, X0), X1);
    const float y1 = i11 * dx, y2 = i22 * (Y - k * dx);
    best = fminf(best, fmaf(y1, y1, y2 * y2));
    const float X = e ? X1 : X0;                         // vertical edge: vertex dy = k dx
    const float dy = fminf(fmaxf(k * X, Y0), Y1);
    const float z1 = i11 * X, z2 = i22 * (dy - k * X);
    best = fminf(best, fmaf(z1, z1, z2 * z2));
  }
  return best <= lim;
}

__device__ __forceinline__ bool block_may_hit(const float4& a, const float4& b, float x0,
                                              float y0) {
  return rect_may_hit(a, b, x0, y0, 15.0f, 15.0f);
}

// Asynchronous 16-byte global -> shared copies (bypassing L1) and their fences.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Float-float ("double-float") arithmetic from error-free transformations
// (Knuth's two-sum, FMA-based two-product); used once per splat to place the
// screen centre to ~1e-12 relative without FP64.
// ---------------------------------------------------------------------------
struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ FF ff_norm(float hi, float lo) {  // |hi| >= |lo|
  const float s = __fadd_rn(hi, lo);
  return {s, __fsub_rn(lo, __fsub_rn(s, hi))};
}
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.hi, y.hi);
  return ff_norm(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_add_f(FF x, float b) {
  const FF s = ff_two_sum(x.hi, b);
  return ff_norm(s.hi, __fadd_rn(s.lo, x.lo));
}
__device__ __forceinline__ FF ff_mul_f(FF x, float b) {
  const FF p = ff_two_prod(x.hi, b);
  return ff_norm(p.hi, __fmaf_rn(x.lo, b, p.lo));
}
__device__ __forceinline__ FF ff_div(FF x, FF y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const FF qy = ff_mul_f(y, q1);
  const FF r = ff_add(x, FF{-qy.hi, -qy.lo});
  return ff_norm(q1, __fdiv_rn(r.hi, y.hi));
}
// sum_j a_j b_j + c, compensated
__device__ __forceinline__ FF ff_dot3_add(const float* a, float b0, float b1, float b2, float c) {
  FF s = ff_two_prod(a[0], b0);
  s = ff_add(s, ff_two_prod(a[1], b1));
  s = ff_add(s, ff_two_prod(a[2], b2));
  return ff_add_f(s, c);
}

// ---------------------------------------------------------------------------
// State formats (Sec. 3.3).  Round to nearest even on store.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint16_t to_unorm16(float x) {
  return (uint16_t)__float2uint_rn(__saturatef(x) * 65535.0f);
}
__device__ __forceinline__ uint8_t to_unorm8(float x) {
  return (uint8_t)__float2uint_rn(__saturatef(x) * 255.0f);
}

__device__ __forceinline__ void store_state(void* state, int fmt, size_t pix, float r, float g,
                                            float b, float T) {
  switch (fmt) {
    case GS_STATE_FP16: {
      __half2 lo = __floats2half2_rn(r, g);
      __half2 hi = __floats2half2_rn(b, T);
      uint2 v;
      v.x = *reinterpret_cast<uint32_t*>(&lo);
      v.y = *reinterpret_cast<uint32_t*>(&hi);
      reinterpret_cast<uint2*>(state)[pix] = v;
      break;
    }
    case GS_STATE_UNORM16: {
      uint2 v;
      v.x = (uint32_t)to_unorm16(r) | ((uint32_t)to_unorm16(g) << 16);
      v.y = (uint32_t)to_unorm16(b) | ((uint32_t)to_unorm16(T) << 16);
      reinterpret_cast<uint2*>(state)[pix] = v;
      break;
    }
    case GS_STATE_UNORM8: {
      uint32_t v = (uint32_t)to_unorm8(r) | ((uint32_t)to_unorm8(g) << 8) |
                   ((uint32_t)to_unorm8(b) << 16) | ((uint32_t)to_unorm8(T) << 24);
      reinterpret_cast<uint32_t*>(state)[pix] = v;
      break;
    }
    default:
      reinterpret_cast<float4*>(state)[pix] = make_float4(r, g, b, T);
  }
}

__device__ __forceinline__ float4 load_state(const void* state, int fmt, size_t pix) {
  switch (fmt) {
    case GS_STATE_FP16: {
      uint2 v = reinterpret_cast<const uint2*>(state)[pix];
      __half2 lo = *reinterpret_cast<__half2*>(&v.x);
      __half2 hi = *reinterpret_cast<__half2*>(&v.y);
      float2 a = __half22float2(lo), b = __half22float2(hi);
      return make_float4(a.x, a.y, b.x, b.y);
    }
    case GS_STATE_UNORM16: {
      uint2 v = reinterpret_cast<const uint2*>(state)[pix];
      const float s = 1.0f / 65535.0f;
      return make_float4((v.x & 0xFFFFu) * s, (v.x >> 16) * s, (v.y & 0xFFFFu) * s, (v.y >> 16) * s);
    }
    case GS_STATE_UNORM8: {
      uint32_t v = reinterpret_cast<const uint32_t*>(state)[pix];
      const float s = 1.0f / 255.0f;
      return make_float4((v & 0xFFu) * s, ((v >> 8) & 0xFFu) * s, ((v >> 16) & 0xFFu) * s,
                         (v >> 24) * s);
    }
    default:
      return reinterpret_cast<const float4*>(state)[pix];
  }
}

// ---------------------------------------------------------------------------
// Relaxed GPU-scope loads/stores for look-back status words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Vector reduction into global memory (sm_90+): four float adds in one op.
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, Condon-Shortley phase, index l^2+l+m.
// Constants are the normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
// (times sqrt 2 for m != 0) folded into the Cartesian polynomial forms.
// ---------------------------------------------------------------------------
struct ShConst {
  static constexpr float c0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
  static constexpr float c1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
  static constexpr float c2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
  static constexpr float c2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
  static constexpr float c2c = 0.5462742152960396f;   // sqrt(15/(16 pi))
  static constexpr float c3a = 0.5900435899266435f;   // sqrt(35/(32 pi))
  static constexpr float c3b = 2.890611442640554f;    // sqrt(105/(4 pi))
  static constexpr float c3c = 0.4570457994644658f;   // sqrt(21/(32 pi))
  static constexpr float c3d = 0.3731763325901154f;   // sqrt(7/(16 pi))
  static constexpr float c3e = 1.445305721320277f;    // sqrt(105/(16 pi))
};

// Y[k] for a unit direction (x, y, z).
__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float* Y) {
  Y[0] = ShConst::c0;
  if (deg < 1) return;
  Y[1] = -ShConst::c1 * y;
  Y[2] = ShConst::c1 * z;
  Y[3] = -ShConst::c1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
  Y[4] = ShConst::c2a * xy;
  Y[5] = -ShConst::c2a * yz;
  Y[6] = ShConst::c2b * (3.0f * zz - 1.0f);
  Y[7] = -ShConst::c2a * xz;
  Y[8] = ShConst::c2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -ShConst::c3a * y * (3.0f * xx - yy);
  Y[10] = ShConst::c3b * xy * z;
  Y[11] = -ShConst::c3c * y * (5.0f * zz - 1.0f);
  Y[12] = ShConst::c3d * z * (5.0f * zz - 3.0f);
  Y[13] = -ShConst::c3c * x * (5.0f * zz - 1.0f);
  Y[14] = ShConst::c3e * z * (xx - yy);
  Y[15] = -ShConst::c3a * x * (xx - 3.0f * yy);
}

// Gradient of each polynomial above with respect to (x, y, z): dY[k][3].
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, float* dY) {
  for (int i = 0; i < 48; ++i) dY[i] = 0.0f;
  if (deg < 1) return;
  dY[1 * 3 + 1] = -ShConst::c1;
  dY[2 * 3 + 2] = ShConst::c1;
  dY[3 * 3 + 0] = -ShConst::c1;
  if (deg < 2) return;
  dY[4 * 3 + 0] = ShConst::c2a * y;
  dY[4 * 3 + 1] = ShConst::c2a * x;
  dY[5 * 3 + 1] = -ShConst::c2a * z;
  dY[5 * 3 + 2] = -ShConst::c2a * y;
  dY[6 * 3 + 2] = ShConst::c2b * 6.0f * z;
  dY[7 * 3 + 0] = -ShConst::c2a * z;
  dY[7 * 3 + 2] = -ShConst::c2a * x;
  dY[8 * 3 + 0] = ShConst::c2c * 2.0f * x;
  dY[8 * 3 + 1] = -ShConst::c2c * 2.0f * y;
  if (deg < 3) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  dY[9 * 3 + 0] = -ShConst::c3a * 6.0f * x * y;
  dY[9 * 3 + 1] = -ShConst::c3a * (3.0f * xx - 3.0f * yy);
  dY[10 * 3 + 0] = ShConst::c3b * y * z;
  dY[10 * 3 + 1] = ShConst::c3b * x * z;
  dY[10 * 3 + 2] = ShConst::c3b * x * y;
  dY[11 * 3 + 1] = -ShConst::c3c * (5.0f * zz - 1.0f);
  dY[11 * 3 + 2] = -ShConst::c3c * 10.0f * y * z;
  dY[12 * 3 + 2] = ShConst::c3d * (15.0f * zz - 3.0f);
  dY[13 * 3 + 0] = -ShConst::c3c * (5.0f * zz - 1.0f);
  dY[13 * 3 + 2] = -ShConst::c3c * 10.0f * x * z;
  dY[14 * 3 + 0] = ShConst::c3e * 2.0f * x * z;
  dY[14 * 3 + 1] = -ShConst::c3e * 2.0f * y * z;
  dY[14 * 3 + 2] = ShConst::c3e * (xx - yy);
  dY[15 * 3 + 0] = -ShConst::c3a * (3.0f * xx - 3.0f * yy);
  dY[15 * 3 + 1] = ShConst::c3a * 6.0f * x * y;
}

}  // namespace gsr

// Per-splat projection (forward) and its chain rule (backward).
//
// Forward (Sec. 2.1.1 Eq. 1, Sec. 2.1.2): t = W mu + w; cull tz <= znear;
// Sigma_3D = R S S^T R^T; Sigma_2D = J W Sigma_3D W^T J^T + 0.3 I;
// conic = Sigma_2D^-1; mu_2D = (fx tx/tz + cx, fy ty/tz + cy); SH colour; the
// alpha >= 1/255 ellipse's bounding box (the screen quad the paper rasterizes)
// and an off-screen / opacity-floor cull.  Writes the 48-B record, the box's
// 16x16 pixel blocks, the depth
// key (FP32 bits of tz, or 0xFFFFFFFF when culled), the visible count and the
// four 8-bit digit histograms the depth sort needs.
//
// Backward: from the per-splat 2D gradients accumulated by the backward raster
// (mu_2D, conic, colour, opacity) to mean, scale, quaternion, opacity and SH
// gradients, added into the caller's buffers.
#include "common.cuh"

namespace gsr {

struct CamDev {
  float R[9];
  float t[3];
  float campos[3];
  float fx, fy, cx, cy;
  int W, H;
  float znear;
};

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z);
  R[1] = 2.f * (x * y - w * z);
  R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z);
  R[4] = 1.f - 2.f * (x * x + z * z);
  R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y);
  R[7] = 2.f * (y * z + w * x);
  R[8] = 1.f - 2.f * (x * x + y * y);
}

// Shared by forward and backward: everything up to Sigma_2D.  Sigma_2D is
// formed as N N^T + 0.3 I with N = J W R S (2x3) and its determinant as the
// sum of the squared 2x2 minors of N (Cauchy-Binet) plus the dilation terms:
// no step subtracts nearly equal numbers, so needle-shaped splats (eigenvalue
// ratios of 1e4 and more) keep their short axis to FP32 precision.
struct ProjState {
  float t[3];
  float qn[4], rq;       // normalised quaternion, 1/|q|
  float R[9];            // rotation
  float M[9];            // R diag(s)
  float Tm[6];           // J W (2x3)
  float N[6];            // Tm M (2x3)
  float s00, s01, s11;   // Sigma_2D
  float det;             // det Sigma_2D
};

// a d - b c with one rounding (FMA-based, Kahan)
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
  const float w = b * c;
  const float e = fmaf(-b, c, w);
  const float f = fmaf(a, d, -w);
  return f + e;
}

__device__ __forceinline__ bool project_core(const CamDev& cam, float mx, float my, float mz,
                                             float4 q, float sx, float sy, float sz,
                                             ProjState& ps) {
  ps.t[0] = ff_dot3_add(&cam.R[0], mx, my, mz, cam.t[0]).hi;
  ps.t[1] = ff_dot3_add(&cam.R[3], mx, my, mz, cam.t[1]).hi;
  ps.t[2] = ff_dot3_add(&cam.R[6], mx, my, mz, cam.t[2]).hi;
  if (!(ps.t[2] > cam.znear)) return false;
  const float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  if (!(qq > 0.f)) return false;
  ps.rq = rsqrtf(qq);
  ps.qn[0] = q.x * ps.rq;
  ps.qn[1] = q.y * ps.rq;
  ps.qn[2] = q.z * ps.rq;
  ps.qn[3] = q.w * ps.rq;
  quat_to_rot(ps.qn[0], ps.qn[1], ps.qn[2], ps.qn[3], ps.R);
  const float s[3] = {sx, sy, sz};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) ps.M[i * 3 + j] = ps.R[i * 3 + j] * s[j];
  const float iz = 1.f / ps.t[2];
  const float J00 = cam.fx * iz, J02 = -cam.fx * ps.t[0] * iz * iz;
  const float J11 = cam.fy * iz, J12 = -cam.fy * ps.t[1] * iz * iz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {   // Tm = J W
    ps.Tm[j] = J00 * cam.R[j] + J02 * cam.R[6 + j];
    ps.Tm[3 + j] = J11 * cam.R[3 + j] + J12 * cam.R[6 + j];
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)    // N = Tm M
      ps.N[i * 3 + j] = ps.Tm[i * 3 + 0] * ps.M[j] + ps.Tm[i * 3 + 1] * ps.M[3 + j] +
                        ps.Tm[i * 3 + 2] * ps.M[6 + j];
  const float* N = ps.N;
  const float n0 = fmaf(N[0], N[0], fmaf(N[1], N[1], N[2] * N[2]));
  const float n1 = fmaf(N[3], N[3], fmaf(N[4], N[4], N[5] * N[5]));
  ps.s00 = n0 + kDilation;
  ps.s11 = n1 + kDilation;
  ps.s01 = fmaf(N[0], N[3], fmaf(N[1], N[4], N[2] * N[5]));
  const float m01 = det2(N[0], N[1], N[3], N[4]);
  const float m02 = det2(N[0], N[2], N[3], N[5]);
  const float m12 = det2(N[1], N[2], N[4], N[5]);
  ps.det = fmaf(m01, m01, fmaf(m02, m02, m12 * m12)) + kDilation * (n0 + n1) + kDilation * kDilation;
  return true;
}

// One splat's SH coefficients, 3 (DEG + 1)^2 floats.  When a row is a whole
// number of 16-byte words (SH degree 1 or 3) and the array is 16-byte aligned,
// it is read as float4s: a quarter of the memory instructions.
template <int DEG>
struct ShRow {
  static constexpr int kN = 3 * (DEG + 1) * (DEG + 1);
  static constexpr bool kVec = kN % 4 == 0;
  float v[kN];
  __device__ __forceinline__ void load(const float* __restrict__ p, bool vec) {
    if (kVec && vec) {
      const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
      for (int i = 0; i < kN / 4; ++i) {
        const float4 t = q[i];
        v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kN; ++i) v[i] = p[i];
    }
  }
};

// ---------------------------------------------------------------------------
// Forward projection.
//
// Only a fraction of the splats is visible, scattered over the index range,
// so a warp that ran the full projection on 32 consecutive splats would
// execute it whenever one lane needed it.  Each warp therefore first runs a
// cheap, conservative test on 32 consecutive splats (mean, opacity, scale:
// near plane, opacity floor, and a screen test with an upper bound of the
// ellipse's extent) and queues the survivors in shared memory; every time 32
// are queued it projects them with all lanes busy.  The depth keys stay
// indexed by splat id, so the sort sees them in index order.
// Persistent grid-stride loop so that each CTA flushes its shared-memory digit
// histograms to global memory once.
// ---------------------------------------------------------------------------
constexpr int kProjThreads = 256;
constexpr int kProjWarps = kProjThreads / 32;

// Cheap test: false only for splats the full projection would cull.
__device__ __forceinline__ bool may_be_visible(const CamDev& cam, float mx, float my, float mz,
                                               float o, float sx, float sy, float sz) {
  if (!(o * 255.0f >= 1.0f)) return false;
  const float tz = ff_dot3_add(&cam.R[6], mx, my, mz, cam.t[2]).hi;   // as in project_core
  if (!(tz > cam.znear)) return false;
  const float tx = fmaf(cam.R[0], mx, fmaf(cam.R[1], my, fmaf(cam.R[2], mz, cam.t[0])));
  const float ty = fmaf(cam.R[3], mx, fmaf(cam.R[4], my, fmaf(cam.R[5], mz, cam.t[1])));
  const float iz = 1.f / tz;
  const float ax = tx * iz, ay = ty * iz;
  // |J|_2^2 <= |J|_F^2 and |W R S|_2 = max scale bound the largest eigenvalue of Sigma_2D
  const float F2 = (cam.fx * cam.fx * fmaf(ax, ax, 1.f) + cam.fy * cam.fy * fmaf(ay, ay, 1.f)) * iz * iz;
  const float smax = fmaxf(fabsf(sx), fmaxf(fabsf(sy), fabsf(sz)));
  const float k = fmaxf(0.f, 2.0f * kLn2 * log2f(255.0f * o));
  const float r = sqrtf(k * fmaf(F2, smax * smax, kDilation)) * 1.01f + 1.0f;
  const float ux = fmaf(cam.fx, ax, cam.cx), uy = fmaf(cam.fy, ay, cam.cy);
  const float mx_ = 1.0f + 1e-4f * fabsf(ux), my_ = 1.0f + 1e-4f * fabsf(uy);
  return ux + r >= 0.5f - mx_ && ux - r <= (float)cam.W - 0.5f + mx_ &&
         uy + r >= 0.5f - my_ && uy - r <= (float)cam.H - 0.5f + my_;
}

// The full projection of splat i: returns its depth key (kNone when culled)
// and writes its record and block box.  DEG is the SH degree (0..3).
template <int DEG>
__device__ __forceinline__ uint32_t project_splat(
    int i, const float* __restrict__ means, const float* __restrict__ scales,
    const float4* __restrict__ quats, const float* __restrict__ opac, const float* __restrict__ sh,
    bool sh_vec, const CamDev& cam, int clamp01, SplatRec* __restrict__ rec,
    uint2* __restrict__ boxes) {
  const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
  const float o = opac[i];
  ProjState ps;
  bool ok = o * 255.0f >= 1.0f;   // opacity floor: alpha <= o < 1/255 everywhere
  if (ok) ok = project_core(cam, mx, my, mz, quats[i], scales[3 * i], scales[3 * i + 1],
                            scales[3 * i + 2], ps);
  if (ok) ok = ps.det > 0.f;
  if (!ok) return kNone;
  // screen centre in float-float: t = W mu + w and mu_2D = f t_xy / t_z + c
  const FF tx = ff_dot3_add(&cam.R[0], mx, my, mz, cam.t[0]);
  const FF ty = ff_dot3_add(&cam.R[3], mx, my, mz, cam.t[1]);
  const FF tz = ff_dot3_add(&cam.R[6], mx, my, mz, cam.t[2]);
  const FF fux = ff_add_f(ff_mul_f(ff_div(tx, tz), cam.fx), cam.cx);
  const FF fuy = ff_add_f(ff_mul_f(ff_div(ty, tz), cam.fy), cam.cy);
  const float ux = fux.hi, uy = fuy.hi;
  // power >= -ln(255 o)  <=>  d^T Q d <= k = 2 ln(255 o); the ellipse's box
  // has half-widths sqrt(k Sigma_00), sqrt(k Sigma_11).  A small relative
  // and absolute widening keeps every fragment the FP32 raster accepts.
  const float thr = -log2f(255.0f * o);
  const float k = fmaxf(0.f, -2.0f * kLn2 * thr);
  const float ex = sqrtf(k * ps.s00) * 1.002f + 0.02f;
  const float ey = sqrtf(k * ps.s11) * 1.002f + 0.02f;
  // any pixel centre (x + 0.5, y + 0.5) inside the box?
  const float x0 = ceilf(ux - ex - 0.5f), x1 = floorf(ux + ex - 0.5f);
  const float y0 = ceilf(uy - ey - 0.5f), y1 = floorf(uy + ey - 0.5f);
  if (!(x0 <= x1 && y0 <= y1 && x1 >= 0.f && y1 >= 0.f && x0 <= (float)(cam.W - 1) &&
        y0 <= (float)(cam.H - 1)))
    return kNone;
  // 16x16 blocks of the pixel-centre box (clamped to the image)
  const int bx0 = (int)fmaxf(x0, 0.f) >> 4, bx1 = (int)fminf(x1, (float)(cam.W - 1)) >> 4;
  const int by0 = (int)fmaxf(y0, 0.f) >> 4, by1 = (int)fminf(y1, (float)(cam.H - 1)) >> 4;
  boxes[i] = make_uint2((uint32_t)bx0 | ((uint32_t)by0 << 16),
                        (uint32_t)(bx1 - bx0 + 1) | ((uint32_t)(by1 - by0 + 1) << 16));
  // colour from SH at the view direction
  float vx = mx - cam.campos[0], vy = my - cam.campos[1], vz = mz - cam.campos[2];
  const float rn = rsqrtf(vx * vx + vy * vy + vz * vz);
  vx *= rn; vy *= rn; vz *= rn;
  constexpr int K = (DEG + 1) * (DEG + 1);
  float Y[16];
  sh_eval(DEG, vx, vy, vz, Y);
  float col[3] = {0.5f, 0.5f, 0.5f};
  if (K == 16 && sh_vec) {
    // degree 3: the 48 coefficients in three rounds of four float4 loads, the
    // rounds kept apart so that at most 16 are live (the kernel then fits four
    // CTAs per SM); each channel still adds its terms in coefficient order
    const float4* q = reinterpret_cast<const float4*>(sh + (size_t)i * K * 3);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float v[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 t = q[4 * ch + u];
        v[4 * u] = t.x; v[4 * u + 1] = t.y; v[4 * u + 2] = t.z; v[4 * u + 3] = t.w;
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) col[(16 * ch + e) % 3] += v[e] * Y[(16 * ch + e) / 3];
      asm volatile("" ::: "memory");
    }
  } else {
    ShRow<DEG> row;
    row.load(sh + (size_t)i * K * 3, sh_vec);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
      col[0] += row.v[kk * 3 + 0] * Y[kk];
      col[1] += row.v[kk * 3 + 1] * Y[kk];
      col[2] += row.v[kk * 3 + 2] * Y[kk];
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    col[c] = fmaxf(0.f, col[c]);
    if (clamp01) col[c] = fminf(1.f, col[c]);
  }
  // inverse Cholesky factor of Sigma_2D, scaled so that
  // q = (i11 dx)^2 + (i22 (dy - k dx))^2 = -log2(e) * power
  const float sc = 0.84932180028801904f;   // sqrt(log2(e) / 2)
  SplatRec r;
  r.a = make_float4(ux, uy, sc * rsqrtf(ps.s00), ps.s01 / ps.s00);
  r.b = make_float4(sc * sqrtf(ps.s00 / ps.det), -thr, fux.lo, fuy.lo);
  r.c = make_float4(col[0], col[1], col[2], o);
  rec[i] = r;
  return __float_as_uint(ps.t[2]);
}

template <int DEG>
__global__ void __launch_bounds__(kProjThreads, 4) project_fwd_kernel(
    const float* __restrict__ means, const float* __restrict__ scales,
    const float4* __restrict__ quats, const float* __restrict__ opac,
    const float* __restrict__ sh, int n, CamDev cam, int clamp01, int sh_vec,
    SplatRec* __restrict__ rec, uint2* __restrict__ boxes, uint32_t* __restrict__ keys,
    Header* __restrict__ hdr, uint2* __restrict__ ranges, int n_ranges,
    uint32_t* __restrict__ epoch) {
  __shared__ uint32_t s_hist[4][256];
  __shared__ int s_queue[kProjWarps][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a new view: look-back status words of earlier views stop matching
  if (blockIdx.x == 0 && threadIdx.x == 0) *epoch += 1u;
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  // zero the block ranges for this view (rebuilt by the binning stage)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_ranges; i += gridDim.x * blockDim.x)
    ranges[i] = make_uint2(0, 0);
  __syncthreads();
  int* q = s_queue[warp];
  int queued = 0;                       // warp-uniform
  uint32_t local_visible = 0;
  auto project_queued = [&](int count) {
    if (lane < count) {
      const int i = q[lane];
      const uint32_t key = project_splat<DEG>(i, means, scales, quats, opac, sh, sh_vec != 0, cam,
                                              clamp01, rec, boxes);
      keys[i] = key;
      if (key != kNone) {
        local_visible++;
        atomicAdd(&s_hist[0][key & 0xFF], 1u);
        atomicAdd(&s_hist[1][(key >> 8) & 0xFF], 1u);
        atomicAdd(&s_hist[2][(key >> 16) & 0xFF], 1u);
        atomicAdd(&s_hist[3][key >> 24], 1u);
      }
    }
  };
  const int64_t warps_total = (int64_t)gridDim.x * kProjWarps;
  // the cheap test's inputs of the warp's next 32 splats are loaded one step
  // ahead, so their DRAM latency overlaps the current step
  struct Cheap { float mx, my, mz, o, sx, sy, sz; };
  auto load_cheap = [&](int64_t b) {
    Cheap c{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int64_t i = b + lane;
    if (i < n) {
      c.mx = means[3 * i]; c.my = means[3 * i + 1]; c.mz = means[3 * i + 2];
      c.o = opac[i];
      c.sx = scales[3 * i]; c.sy = scales[3 * i + 1]; c.sz = scales[3 * i + 2];
    }
    return c;
  };
  int64_t base = ((int64_t)blockIdx.x * kProjWarps + warp) * 32;
  Cheap cur = load_cheap(base);
  for (; base < n; base += warps_total * 32) {
    const Cheap nxt = load_cheap(base + warps_total * 32);
    const int i = (int)base + lane;
    bool cand = false;
    if (i < n) cand = may_be_visible(cam, cur.mx, cur.my, cur.mz, cur.o, cur.sx, cur.sy, cur.sz);
    if (i < n && !cand) keys[i] = kNone;
    const uint32_t m = __ballot_sync(0xffffffffu, cand);
    if (cand) q[queued + __popc(m & lanemask_lt())] = i;
    queued += __popc(m);
    __syncwarp();
    if (queued >= 32) {
      project_queued(32);
      __syncwarp();
      queued -= 32;
      if (lane < queued) q[lane] = q[32 + lane];
      __syncwarp();
    }
    cur = nxt;
  }
  project_queued(queued);
  // visible count: warp-aggregate, one atomic per warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) local_visible += __shfl_xor_sync(0xffffffffu, local_visible, off);
  if (lane == 0 && local_visible) atomicAdd(&hdr->visible, local_visible);
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&hdr->depth_hist[0][0] + i, v);
  }
}

// ---------------------------------------------------------------------------
// Backward projection: the chain rule from the raster's per-splat sums to the
// splat parameters.  g2d holds 12 floats per depth rank: the sums over the
// splat's fragments of w z_hat and w z_hat z_hat^T (z_hat = Sigma_2D^-1 d in
// units of 1 / (2 ln 2), w = alpha dL/dalpha), then dL/d(rgb) and dL/do;
// they are converted here to dL/dmu_2D and dL/dSigma_2D.
//
// Only the splats that some fragment gave a gradient need the chain rule,
// and they are a fraction of the depth-ranked list.  As in the forward pass,
// each warp first reads the sums of 32 consecutive ranks, queues the ranks
// with a non-zero sum in shared memory, and handles 32 queued splats at a
// time with all lanes busy.
//
// The splats of a batch sit at scattered ids, so one lane per splat reading
// its own rows would make every memory instruction touch 32 cache lines.
// Instead the warp moves the rows between global and shared memory together:
// consecutive lanes take consecutive words of the batch's rows (a mean is 3
// floats, an SH row 3 (DEG+1)^2), so an instruction touches about 32 / (row
// length) lines.  Each lane then computes from its row in shared memory and
// leaves its gradients there, and the warp adds them to the gradient arrays
// the same way (every id occurs once, so the read-modify-writes do not race).
// ---------------------------------------------------------------------------
constexpr int kProjBwdThreads = 128;
constexpr int kProjBwdWarps = kProjBwdThreads / 32;

// One splat's row in shared memory (floats): [0, 3) mean, then dL/dmean;
// [3, 6) scale, then dL/dscale; [8, 8 + kSh) SH coefficients, then dL/dsh.
// The pitch is an odd number of 16-byte words, so 32 lanes reading float4s of
// their own rows hit distinct banks.
template <int DEG>
struct BwdRow {
  static constexpr int kSh = 3 * (DEG + 1) * (DEG + 1);
  static constexpr int kShOff = 8;
  static constexpr int kRound = (kShOff + kSh + 3) / 4 * 4;
  static constexpr int kPitch = (kRound / 4) % 2 == 1 ? kRound : kRound + 4;
  static constexpr bool kVec = kSh % 4 == 0;
};

// gd += sum_k w_k dY_k / d(x, y, z) for the polynomials of sh_eval, with no
// per-coefficient array (every term is used once).
template <int DEG>
__device__ __forceinline__ void sh_grad_dot(float x, float y, float z, const float* w, float* gd) {
  if (DEG < 1) return;
  gd[0] -= ShConst::c1 * w[3];
  gd[1] -= ShConst::c1 * w[1];
  gd[2] += ShConst::c1 * w[2];
  if (DEG < 2) return;
  gd[0] += ShConst::c2a * (y * w[4] - z * w[7]) + 2.0f * ShConst::c2c * x * w[8];
  gd[1] += ShConst::c2a * (x * w[4] - z * w[5]) - 2.0f * ShConst::c2c * y * w[8];
  gd[2] += 6.0f * ShConst::c2b * z * w[6] - ShConst::c2a * (y * w[5] + x * w[7]);
  if (DEG < 3) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  const float a = 3.0f * xx - 3.0f * yy, b = 5.0f * zz - 1.0f;
  gd[0] += -ShConst::c3a * (6.0f * x * y * w[9] + a * w[15]) + ShConst::c3b * y * z * w[10] -
           ShConst::c3c * b * w[13] + 2.0f * ShConst::c3e * x * z * w[14];
  gd[1] += ShConst::c3a * (6.0f * x * y * w[15] - a * w[9]) + ShConst::c3b * x * z * w[10] -
           ShConst::c3c * b * w[11] - 2.0f * ShConst::c3e * y * z * w[14];
  gd[2] += ShConst::c3b * x * y * w[10] - 10.0f * ShConst::c3c * z * (y * w[11] + x * w[13]) +
           ShConst::c3d * (15.0f * zz - 3.0f) * w[12] + ShConst::c3e * (xx - yy) * w[14];
}

// The warp's rows of `len` floats at src[id_j * len] (j < count; id_j in lane
// j's `id`) into rows[j * pitch + off], consecutive lanes on consecutive words.
template <int LEN, int PITCH>
__device__ __forceinline__ void gather_rows(float* rows, int off, const float* __restrict__ src,
                                            uint32_t id, int count, int lane) {
#pragma unroll 4
  for (int t = 0; t < LEN; ++t) {
    const int i = t * 32 + lane, j = i / LEN, c = i % LEN;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count) rows[j * PITCH + off + c] = src[(size_t)idj * LEN + c];
  }
}

// dst[id_j * len + c] += rows[j * pitch + off + c] (STORE: =), laid out as gather_rows.
template <int LEN, int PITCH, bool STORE = false>
__device__ __forceinline__ void scatter_add_rows(const float* rows, int off,
                                                 float* __restrict__ dst, uint32_t id, int count,
                                                 int lane) {
#pragma unroll 4
  for (int t = 0; t < LEN; ++t) {
    const int i = t * 32 + lane, j = i / LEN, c = i % LEN;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count) {
      if (STORE)
        dst[(size_t)idj * LEN + c] = rows[j * PITCH + off + c];
      else
        dst[(size_t)idj * LEN + c] += rows[j * PITCH + off + c];
    }
  }
}

// As the two above for rows of LEN4 16-byte words (both sides 16-byte aligned).
template <int LEN4, int PITCH>
__device__ __forceinline__ void gather_rows4(float* rows, int off, const float* __restrict__ src,
                                             uint32_t id, int count, int lane) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll 4
  for (int t = 0; t < LEN4; ++t) {
    const int i = t * 32 + lane, j = i / LEN4, c = i % LEN4;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count)
      *reinterpret_cast<float4*>(rows + j * PITCH + off + 4 * c) = s4[(size_t)idj * LEN4 + c];
  }
}

template <int LEN4, int PITCH, bool STORE = false>
__device__ __forceinline__ void scatter_add_rows4(const float* rows, int off,
                                                  float* __restrict__ dst, uint32_t id, int count,
                                                  int lane) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 4
  for (int t = 0; t < LEN4; ++t) {
    const int i = t * 32 + lane, j = i / LEN4, c = i % LEN4;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count) {
      const float4 g = *reinterpret_cast<const float4*>(rows + j * PITCH + off + 4 * c);
      if (STORE) {
        d4[(size_t)idj * LEN4 + c] = g;
      } else {
        float4 v = d4[(size_t)idj * LEN4 + c];
        v.x += g.x; v.y += g.y; v.z += g.z; v.w += g.w;
        d4[(size_t)idj * LEN4 + c] = v;
      }
    }
  }
}

// The chain rule for one splat: its row (mean, scale, SH) in shared memory,
// its quaternion and its 2D sums given.  dL/dmean, dL/dscale and dL/dsh go
// back into the row; dL/dq is returned.
template <int DEG>
__device__ __forceinline__ float4 project_bwd_splat(float* row, const float4 quat, const float4 ga,
                                                    const float4 gb, const CamDev& cam,
                                                    int clamp01) {
  using Row = BwdRow<DEG>;
  constexpr int K = (DEG + 1) * (DEG + 1);
  const float mx = row[0], my = row[1], mz = row[2];
  const float sx = row[3], sy = row[4], sz = row[5];
  ProjState ps;
  project_core(cam, mx, my, mz, quat, sx, sy, sz, ps);
  // 2D gradients in natural units: dL/dmu_2D = 2 ln2 (v0, v1) and
  // dL/dSigma_2D = 2 ln2^2 [[v2, v3], [v3, v4]]
  const float gmu2x = 2.f * kLn2 * ga.x, gmu2y = 2.f * kLn2 * ga.y;
  const float gs_scale = 2.f * kLn2 * kLn2;
  const float GS00 = gs_scale * ga.z, GS01 = gs_scale * ga.w, GS11 = gs_scale * gb.x;
  float gmu[3] = {0.f, 0.f, 0.f};

  // colour: rgb = clamp(sum_k sh_k Y_k(d) + 0.5), d = (mu - campos) / |mu - campos|
  {
    const float vx = mx - cam.campos[0], vy = my - cam.campos[1], vz = mz - cam.campos[2];
    const float rn = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float dx = vx * rn, dy = vy * rn, dz = vz * rn;
    float Y[16];
    sh_eval(DEG, dx, dy, dz, Y);
    float* shr = row + Row::kShOff;
    float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
    for (int k = 0; k < K; ++k) {
      raw[0] += shr[k * 3 + 0] * Y[k];
      raw[1] += shr[k * 3 + 1] * Y[k];
      raw[2] += shr[k * 3 + 2] * Y[k];
    }
    const float grgb[3] = {gb.y, gb.z, gb.w};
    float graw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool pass = raw[c] > 0.f && (!clamp01 || raw[c] < 1.f);
      graw[c] = pass ? grgb[c] : 0.f;
    }
    // read the coefficients again below rather than hold them in registers
    asm volatile("" ::: "memory");
    if (DEG > 0) {
      // through the view direction: w_k = sh_k . graw, dL/dd = sum_k w_k dY_k/dd
      float w[K];
#pragma unroll
      for (int k = 0; k < K; ++k)
        w[k] = shr[k * 3 + 0] * graw[0] + shr[k * 3 + 1] * graw[1] + shr[k * 3 + 2] * graw[2];
      float gd[3] = {0.f, 0.f, 0.f};
      sh_grad_dot<DEG>(dx, dy, dz, w, gd);
      const float dd = gd[0] * dx + gd[1] * dy + gd[2] * dz;
      gmu[0] += (gd[0] - dx * dd) * rn;
      gmu[1] += (gd[1] - dy * dd) * rn;
      gmu[2] += (gd[2] - dz * dd) * rn;
    }
    // dL/dsh_k = Y_k graw replaces the coefficients
#pragma unroll
    for (int i = 0; i < Row::kSh; ++i) shr[i] = Y[i / 3] * graw[i % 3];
  }

  // Sigma_2D = N N^T + 0.3 I:  G_N = 2 G_S N;  N = Tm M:  G_Tm = G_N M^T, G_M = Tm^T G_N
  const float* N = ps.N;
  const float* T = ps.Tm;
  float GN[6];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    GN[j] = 2.f * (GS00 * N[j] + GS01 * N[3 + j]);
    GN[3 + j] = 2.f * (GS01 * N[j] + GS11 * N[3 + j]);
  }
  float GT[2][3];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      GT[i][k] = GN[i * 3] * ps.M[k * 3] + GN[i * 3 + 1] * ps.M[k * 3 + 1] + GN[i * 3 + 2] * ps.M[k * 3 + 2];
  // Tm = J W:  G_J = G_Tm W^T (only J00, J02, J11, J12 depend on t)
  const float* W = cam.R;
  const float GJ00 = GT[0][0] * W[0] + GT[0][1] * W[1] + GT[0][2] * W[2];
  const float GJ02 = GT[0][0] * W[6] + GT[0][1] * W[7] + GT[0][2] * W[8];
  const float GJ11 = GT[1][0] * W[3] + GT[1][1] * W[4] + GT[1][2] * W[5];
  const float GJ12 = GT[1][0] * W[6] + GT[1][1] * W[7] + GT[1][2] * W[8];
  const float tx = ps.t[0], ty = ps.t[1], tz = ps.t[2];
  const float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
  float gt[3];
  gt[0] = GJ02 * (-cam.fx * iz2) + gmu2x * cam.fx * iz;
  gt[1] = GJ12 * (-cam.fy * iz2) + gmu2y * cam.fy * iz;
  gt[2] = GJ00 * (-cam.fx * iz2) + GJ02 * (2.f * cam.fx * tx * iz3) + GJ11 * (-cam.fy * iz2) +
          GJ12 * (2.f * cam.fy * ty * iz3) - gmu2x * cam.fx * tx * iz2 - gmu2y * cam.fy * ty * iz2;
#pragma unroll
  for (int j = 0; j < 3; ++j) gmu[j] += W[j] * gt[0] + W[3 + j] * gt[1] + W[6 + j] * gt[2];

  // M_kj = R_kj s_j:  dL/ds_j = sum_k G_M_kj R_kj,  G_R_kj = G_M_kj s_j
  const float s[3] = {sx, sy, sz};
  float gs[3] = {0.f, 0.f, 0.f};
  float GR[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float gm = T[k] * GN[j] + T[3 + k] * GN[3 + j];
      gs[j] += ps.R[k * 3 + j] * gm;
      GR[k * 3 + j] = gm * s[j];
    }
  // R(q_hat) -> q_hat -> q
  const float w = ps.qn[0], x = ps.qn[1], y = ps.qn[2], z = ps.qn[3];
  float gq[4];
  gq[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
  gq[1] = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] +
                 w * GR[7] - 2.f * x * GR[8]);
  gq[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] +
                 z * GR[7] - 2.f * y * GR[8]);
  gq[3] = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] +
                 y * GR[5] + x * GR[6] + y * GR[7]);
  const float qd = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    row[j] = gmu[j];
    row[3 + j] = gs[j];
  }
  return make_float4((gq[0] - w * qd) * ps.rq, (gq[1] - x * qd) * ps.rq,
                     (gq[2] - y * qd) * ps.rq, (gq[3] - z * qd) * ps.rq);
}

// One batch of `count` (<= 32) queued ranks, lane j holding rank r.  STORE:
// the rows are written instead of added to.
template <int DEG, bool STORE>
__device__ __forceinline__ void project_bwd_batch(
    float* rows, uint32_t r, int count, int lane, const float* __restrict__ means,
    const float* __restrict__ scales, const float4* __restrict__ quats,
    const float* __restrict__ sh, bool sh_vec, bool dq_vec, const CamDev& cam, int clamp01,
    const uint32_t* __restrict__ sorted_ids, const float4* __restrict__ g2d,
    float* __restrict__ d_means, float* __restrict__ d_scales, float* __restrict__ d_quats,
    float* __restrict__ d_opac, float* __restrict__ d_sh, uint32_t* __restrict__ live_list,
    uint32_t* __restrict__ list_state) {
  using Row = BwdRow<DEG>;
  constexpr int P = Row::kPitch;
  const bool mine = lane < count;
  const uint32_t id = mine ? sorted_ids[r] : 0u;
  if (STORE) {   // the rows this view writes: the next store-mode view zeroes them first
    uint32_t at0 = 0;
    if (lane == 0) at0 = atomicAdd(&list_state[0], (uint32_t)count);
    at0 = __shfl_sync(0xffffffffu, at0, 0);
    if (mine) live_list[at0 + lane] = id;
  }
  float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, quat = ga;
  float gop = 0.f;
  if (mine) {
    ga = g2d[3 * r];
    gb = g2d[3 * r + 1];
    gop = reinterpret_cast<const float*>(g2d)[12 * r + 8];
    quat = quats[id];
  }
  gather_rows<3, P>(rows, 0, means, id, count, lane);
  gather_rows<3, P>(rows, 3, scales, id, count, lane);
  if constexpr (Row::kVec) {   // float4 copies only where a row is whole 16-byte words
    if (sh_vec)
      gather_rows4<Row::kSh / 4, P>(rows, Row::kShOff, sh, id, count, lane);
    else
      gather_rows<Row::kSh, P>(rows, Row::kShOff, sh, id, count, lane);
  } else {
    gather_rows<Row::kSh, P>(rows, Row::kShOff, sh, id, count, lane);
  }
  __syncwarp();
  if (mine) {
    const float4 gq = project_bwd_splat<DEG>(rows + lane * P, quat, ga, gb, cam, clamp01);
    if (STORE) {
      if (dq_vec) {
        reinterpret_cast<float4*>(d_quats)[id] = gq;
      } else {
        d_quats[4 * id + 0] = gq.x;
        d_quats[4 * id + 1] = gq.y;
        d_quats[4 * id + 2] = gq.z;
        d_quats[4 * id + 3] = gq.w;
      }
      d_opac[id] = gop;
    } else {
      if (dq_vec) {
        float4* dq = reinterpret_cast<float4*>(d_quats) + id;
        float4 q4 = *dq;
        q4.x += gq.x; q4.y += gq.y; q4.z += gq.z; q4.w += gq.w;
        *dq = q4;
      } else {
        d_quats[4 * id + 0] += gq.x;
        d_quats[4 * id + 1] += gq.y;
        d_quats[4 * id + 2] += gq.z;
        d_quats[4 * id + 3] += gq.w;
      }
      d_opac[id] += gop;
    }
  }
  __syncwarp();
  // keep the gradient rows' loads below the chain rule: hoisted above it they
  // would hold a row's worth of registers through it
  asm volatile("" ::: "memory");
  scatter_add_rows<3, P, STORE>(rows, 0, d_means, id, count, lane);
  scatter_add_rows<3, P, STORE>(rows, 3, d_scales, id, count, lane);
  if constexpr (Row::kVec) {
    if (sh_vec)
      scatter_add_rows4<Row::kSh / 4, P, STORE>(rows, Row::kShOff, d_sh, id, count, lane);
    else
      scatter_add_rows<Row::kSh, P, STORE>(rows, Row::kShOff, d_sh, id, count, lane);
  } else {
    scatter_add_rows<Row::kSh, P, STORE>(rows, Row::kShOff, d_sh, id, count, lane);
  }
  __syncwarp();   // the rows are reused by the next batch
}

template <int DEG>
__device__ __forceinline__ void zero_splat_rows(uint32_t id, int count, int lane, int sh_vec,
                                                int dq_vec, float* __restrict__ d_means,
                                                float* __restrict__ d_scales,
                                                float* __restrict__ d_quats,
                                                float* __restrict__ d_opac, float* __restrict__ d_sh);

// STORE (a request's gradient alone): every visible splat's rows are written,
// the chain rule's for splats with a gradient and zeros for the others.
template <int DEG, bool STORE>
__global__ void __launch_bounds__(kProjBwdThreads, 5) project_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ scales,
    const float4* __restrict__ quats, const float* __restrict__ sh, int sh_vec, int dq_vec,
    CamDev cam, int clamp01, const uint32_t* __restrict__ sorted_ids,
    const float4* __restrict__ g2d, const Header* __restrict__ hdr, float* __restrict__ d_means,
    float* __restrict__ d_scales, float* __restrict__ d_quats, float* __restrict__ d_opac,
    float* __restrict__ d_sh, uint32_t* __restrict__ live_list, uint32_t* __restrict__ list_state) {
  constexpr int P = BwdRow<DEG>::kPitch;
  // STORE with a valid list: every non-zero row was on it and has been zeroed
  // (zero_listed_kernel), so the rows without a gradient need nothing
  const bool zero_nonlive = STORE && list_state[1] == 0u;
  // adding: the list no longer covers every non-zero row (nothing here reads it)
  if (!STORE && blockIdx.x == 0 && threadIdx.x == 0) list_state[1] = 0u;
  __shared__ __align__(16) float s_rows[kProjBwdWarps][32 * P];
  __shared__ uint32_t s_queue[kProjBwdWarps][64];
  const int lane = threadIdx.x & 31;
  float* rows = s_rows[threadIdx.x >> 5];
  uint32_t* queue = s_queue[threadIdx.x >> 5];
  int queued = 0;
  const uint32_t V = hdr->visible;
  const float* g = reinterpret_cast<const float*>(g2d);
  // base is the same for the whole warp, so every lane runs every iteration
  for (uint32_t base = blockIdx.x * kProjBwdThreads + (threadIdx.x & ~31u); base < V;
       base += gridDim.x * kProjBwdThreads) {
    const uint32_t r = base + lane;
    bool live = false;
    if (r < V) {
      const float4 ga = g2d[3 * r], gb = g2d[3 * r + 1];
      live = ga.x != 0.f || ga.y != 0.f || ga.z != 0.f || ga.w != 0.f || gb.x != 0.f ||
             gb.y != 0.f || gb.z != 0.f || gb.w != 0.f || g[12 * r + 8] != 0.f;
    }
    const unsigned m = __ballot_sync(0xffffffffu, live);
    if (zero_nonlive) {   // rows of visible splats without a gradient: zeros
      const unsigned z = __ballot_sync(0xffffffffu, r < V && !live);
      if (z) {
        const uint32_t zid = (z >> lane) & 1u ? sorted_ids[r] : 0u;
        // compacted: lane j takes the id of the j-th lane to zero
        const int cnt = __popc(z);
        const int src = lane < cnt ? (int)__fns(z, 0u, lane + 1) : 0;
        const uint32_t cid = __shfl_sync(0xffffffffu, zid, src);
        zero_splat_rows<DEG>(cid, cnt, lane, sh_vec, dq_vec, d_means, d_scales, d_quats, d_opac,
                             d_sh);
      }
    }
    if (live) queue[queued + __popc(m & lanemask_lt())] = r;
    queued += __popc(m);
    __syncwarp();
    if (queued >= 32) {
      queued -= 32;
      project_bwd_batch<DEG, STORE>(rows, queue[queued + lane], 32, lane, means, scales, quats,
                                    sh, sh_vec, dq_vec, cam, clamp01, sorted_ids, g2d, d_means,
                                    d_scales, d_quats, d_opac, d_sh, live_list, list_state);
    }
  }
  if (queued > 0)
    project_bwd_batch<DEG, STORE>(rows, lane < queued ? queue[lane] : 0u, queued, lane, means,
                                  scales, quats, sh, sh_vec, dq_vec, cam, clamp01, sorted_ids, g2d,
                                  d_means, d_scales, d_quats, d_opac, d_sh, live_list, list_state);
}

// Zeroing of the gradient rows of the last depth order's splats (the rows a
// backward on that view adds to), with the same warp-wide row layout as the
// copies above: an instruction writes consecutive words of the warp's rows.
template <int LEN>
__device__ __forceinline__ void zero_rows(float* __restrict__ dst, uint32_t id, int count,
                                          int lane) {
#pragma unroll 4
  for (int t = 0; t < LEN; ++t) {
    const int i = t * 32 + lane, j = i / LEN, c = i % LEN;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count) dst[(size_t)idj * LEN + c] = 0.f;
  }
}

template <int LEN4>
__device__ __forceinline__ void zero_rows4(float* __restrict__ dst, uint32_t id, int count,
                                           int lane) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll 4
  for (int t = 0; t < LEN4; ++t) {
    const int i = t * 32 + lane, j = i / LEN4, c = i % LEN4;
    const uint32_t idj = __shfl_sync(0xffffffffu, id, j);
    if (j < count) d4[(size_t)idj * LEN4 + c] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

template <int DEG>
__device__ __forceinline__ void zero_splat_rows(uint32_t id, int count, int lane, int sh_vec,
                                                int dq_vec, float* __restrict__ d_means,
                                                float* __restrict__ d_scales,
                                                float* __restrict__ d_quats,
                                                float* __restrict__ d_opac, float* __restrict__ d_sh) {
  constexpr int kSh = 3 * (DEG + 1) * (DEG + 1);
  zero_rows<3>(d_means, id, count, lane);
  zero_rows<3>(d_scales, id, count, lane);
  zero_rows<1>(d_opac, id, count, lane);
  if (dq_vec)
    zero_rows4<1>(d_quats, id, count, lane);
  else
    zero_rows<4>(d_quats, id, count, lane);
  if (kSh % 4 == 0 && sh_vec)
    zero_rows4<(kSh % 4 == 0 ? kSh / 4 : 1)>(d_sh, id, count, lane);
  else
    zero_rows<kSh>(d_sh, id, count, lane);
}

template <int DEG>
__global__ void __launch_bounds__(256) zero_touched_kernel(
    const uint32_t* __restrict__ sorted_ids, const Header* __restrict__ hdr, int sh_vec,
    int dq_vec, float* __restrict__ d_means, float* __restrict__ d_scales,
    float* __restrict__ d_quats, float* __restrict__ d_opac, float* __restrict__ d_sh) {
  const uint32_t V = hdr->visible;
  const int lane = threadIdx.x & 31;
  // base is the same for the whole warp
  for (uint32_t base = blockIdx.x * 256u + (threadIdx.x & ~31u); base < V;
       base += gridDim.x * 256u) {
    const int count = (int)min(32u, V - base);
    const uint32_t id = lane < count ? sorted_ids[base + lane] : 0u;
    zero_splat_rows<DEG>(id, count, lane, sh_vec, dq_vec, d_means, d_scales, d_quats, d_opac,
                         d_sh);
  }
}

// Rows of the splats the previous depth order held (prev_sorted_ids, prev_V of
// them) that the current projection culled (keys 0xFFFFFFFF): the splats that
// left the view.  With the current view's rows written by a store-mode
// backward, the arrays then hold the current view's gradient alone.
template <int DEG>
__global__ void __launch_bounds__(256) zero_left_kernel(
    const uint32_t* __restrict__ prev_sorted_ids, const uint32_t* __restrict__ prev_V,
    const uint32_t* __restrict__ keys, uint32_t n, int sh_vec, int dq_vec,
    float* __restrict__ d_means, float* __restrict__ d_scales, float* __restrict__ d_quats,
    float* __restrict__ d_opac, float* __restrict__ d_sh, const uint32_t* __restrict__ list_state) {
  if (list_state[1] != 0u) return;   // a valid list covers these rows (zero_listed_kernel)
  const uint32_t V = min(*prev_V, n);
  const int lane = threadIdx.x & 31;
  for (uint32_t base = blockIdx.x * 256u + (threadIdx.x & ~31u); base < V;
       base += gridDim.x * 256u) {
    const uint32_t r = base + lane;
    uint32_t id = r < V ? prev_sorted_ids[r] : 0u;
    const bool left = r < V && id < n && keys[id] == kNone;
    const unsigned z = __ballot_sync(0xffffffffu, left);
    if (!z) continue;
    const int cnt = __popc(z);
    const int src = lane < cnt ? (int)__fns(z, 0u, lane + 1) : 0;
    id = __shfl_sync(0xffffffffu, id, src);
    zero_splat_rows<DEG>(id, cnt, lane, sh_vec, dq_vec, d_means, d_scales, d_quats, d_opac, d_sh);
  }
}

// The rows of the splats the last store-mode view wrote (live_list), zeroed
// before this view's are written: with a valid list (list_state[1]) those are
// the only rows that can be non-zero.
template <int DEG>
__global__ void __launch_bounds__(256) zero_listed_kernel(
    const uint32_t* __restrict__ live_list, const uint32_t* __restrict__ list_state, uint32_t n,
    int sh_vec, int dq_vec, float* __restrict__ d_means, float* __restrict__ d_scales,
    float* __restrict__ d_quats, float* __restrict__ d_opac, float* __restrict__ d_sh) {
  if (list_state[1] == 0u) return;
  const uint32_t count = min(list_state[0], n);
  const int lane = threadIdx.x & 31;
  for (uint32_t base = blockIdx.x * 256u + (threadIdx.x & ~31u); base < count;
       base += gridDim.x * 256u) {
    const uint32_t r = base + lane;
    uint32_t id = r < count ? live_list[r] : 0u;
    const unsigned z = __ballot_sync(0xffffffffu, r < count && id < n);   // (ids of this scene)
    if (!z) continue;
    const int cnt = __popc(z);
    const int src = lane < cnt ? (int)__fns(z, 0u, lane + 1) : 0;
    id = __shfl_sync(0xffffffffu, id, src);
    zero_splat_rows<DEG>(id, cnt, lane, sh_vec, dq_vec, d_means, d_scales, d_quats, d_opac, d_sh);
  }
}

__global__ void copy_word_kernel(const uint32_t* src, uint32_t* dst) { *dst = *src; }

}  // namespace gsr

// Host launchers (called from api.cu)
namespace gsr {

CamDev make_cam(const gs_camera& c) {
  CamDev d;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) d.R[i * 3 + j] = c.viewmat[i * 4 + j];
    d.t[i] = c.viewmat[i * 4 + 3];
    d.campos[i] = c.campos[i];
  }
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
  d.W = c.width; d.H = c.height; d.znear = c.znear;
  return d;
}

cudaError_t launch_project_fwd(const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, int n, int deg,
                               const gs_camera& cam, int clamp01, SplatRec* rec, uint2* boxes,
                               uint32_t* keys, Header* hdr, uint2* ranges, int n_ranges,
                               uint32_t* epoch, int num_sms, cudaStream_t st) {
  int blocks = (n + kProjThreads - 1) / kProjThreads;
  const int cap = num_sms * 4;  // persistent: one wave, four CTAs per SM (the launch bound)
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const float4* q4 = reinterpret_cast<const float4*>(quats);
  const CamDev cd = make_cam(cam);
  const int sh_vec = ((uintptr_t)sh & 15) == 0;
#define GS_PROJECT_FWD(D)                                                                        \
  project_fwd_kernel<D><<<blocks, kProjThreads, 0, st>>>(means, scales, q4, opac, sh, n, cd,     \
                                                         clamp01, sh_vec, rec, boxes, keys, hdr, \
                                                         ranges, n_ranges, epoch)
  switch (deg) {
    case 0: GS_PROJECT_FWD(0); break;
    case 1: GS_PROJECT_FWD(1); break;
    case 2: GS_PROJECT_FWD(2); break;
    default: GS_PROJECT_FWD(3); break;
  }
#undef GS_PROJECT_FWD
  return cudaGetLastError();
}

cudaError_t launch_project_bwd(const float* means, const float* scales, const float* quats,
                               const float* opac, const float* sh, int n_cap, int deg,
                               const gs_camera& cam, int clamp01, const uint32_t* sorted_ids,
                               const float* g2d, const Header* hdr, float* d_means,
                               float* d_scales, float* d_quats, float* d_opac, float* d_sh,
                               int num_sms, cudaStream_t st, int store, uint32_t* live_list,
                               uint32_t* list_state) {
  (void)opac;
  int blocks = (n_cap + kProjBwdThreads - 1) / kProjBwdThreads;
  if (blocks == 0) return cudaSuccess;
  if (blocks > num_sms * 16) blocks = num_sms * 16;
  const int sh_vec = ((uintptr_t)sh & 15) == 0 && ((uintptr_t)d_sh & 15) == 0;
  const int dq_vec = ((uintptr_t)d_quats & 15) == 0;
  const CamDev cd = make_cam(cam);
  const float4* q4 = reinterpret_cast<const float4*>(quats);
  const float4* g4 = reinterpret_cast<const float4*>(g2d);
#define GS_PROJECT_BWD(D)                                                                      \
  if (store)                                                                                   \
    project_bwd_kernel<D, true><<<blocks, kProjBwdThreads, 0, st>>>(                           \
        means, scales, q4, sh, sh_vec, dq_vec, cd, clamp01, sorted_ids, g4, hdr, d_means,      \
        d_scales, d_quats, d_opac, d_sh, live_list, list_state);                               \
  else                                                                                         \
    project_bwd_kernel<D, false><<<blocks, kProjBwdThreads, 0, st>>>(                          \
        means, scales, q4, sh, sh_vec, dq_vec, cd, clamp01, sorted_ids, g4, hdr, d_means,      \
        d_scales, d_quats, d_opac, d_sh, live_list, list_state)
  switch (deg) {
    case 0: GS_PROJECT_BWD(0); break;
    case 1: GS_PROJECT_BWD(1); break;
    case 2: GS_PROJECT_BWD(2); break;
    default: GS_PROJECT_BWD(3); break;
  }
#undef GS_PROJECT_BWD
  return cudaGetLastError();
}

cudaError_t launch_copy_word(const uint32_t* src, uint32_t* dst, cudaStream_t st) {
  copy_word_kernel<<<1, 1, 0, st>>>(src, dst);
  return cudaGetLastError();
}

cudaError_t launch_zero_left(int n, int deg, const uint32_t* prev_sorted_ids,
                             const uint32_t* prev_V, const uint32_t* keys, float* d_means,
                             float* d_scales, float* d_quats, float* d_opac, float* d_sh,
                             int num_sms, cudaStream_t st, const uint32_t* list_state) {
  int blocks = (n + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  const int sh_vec = ((uintptr_t)d_sh & 15) == 0;
  const int dq_vec = ((uintptr_t)d_quats & 15) == 0;
#define GS_ZERO_LEFT(D)                                                                         \
  zero_left_kernel<D><<<blocks, 256, 0, st>>>(prev_sorted_ids, prev_V, keys, (uint32_t)n,       \
                                              sh_vec, dq_vec, d_means, d_scales, d_quats, d_opac, \
                                              d_sh, list_state)
  switch (deg) {
    case 0: GS_ZERO_LEFT(0); break;
    case 1: GS_ZERO_LEFT(1); break;
    case 2: GS_ZERO_LEFT(2); break;
    default: GS_ZERO_LEFT(3); break;
  }
#undef GS_ZERO_LEFT
  return cudaGetLastError();
}

cudaError_t launch_zero_listed(int n, int deg, const uint32_t* live_list,
                               const uint32_t* list_state, float* d_means, float* d_scales,
                               float* d_quats, float* d_opac, float* d_sh, int num_sms,
                               cudaStream_t st) {
  int blocks = (n + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  const int sh_vec = ((uintptr_t)d_sh & 15) == 0;
  const int dq_vec = ((uintptr_t)d_quats & 15) == 0;
#define GS_ZERO_LISTED(D)                                                                       \
  zero_listed_kernel<D><<<blocks, 256, 0, st>>>(live_list, list_state, (uint32_t)n, sh_vec,      \
                                                dq_vec, d_means, d_scales, d_quats, d_opac, d_sh)
  switch (deg) {
    case 0: GS_ZERO_LISTED(0); break;
    case 1: GS_ZERO_LISTED(1); break;
    case 2: GS_ZERO_LISTED(2); break;
    default: GS_ZERO_LISTED(3); break;
  }
#undef GS_ZERO_LISTED
  return cudaGetLastError();
}

cudaError_t launch_zero_touched(int n_cap, int deg, const uint32_t* sorted_ids,
                                const Header* hdr, float* d_means, float* d_scales,
                                float* d_quats, float* d_opac, float* d_sh, int num_sms,
                                cudaStream_t st) {
  int blocks = (n_cap + 255) / 256;
  if (blocks == 0) return cudaSuccess;
  if (blocks > num_sms * 8) blocks = num_sms * 8;
  const int sh_vec = ((uintptr_t)d_sh & 15) == 0;
  const int dq_vec = ((uintptr_t)d_quats & 15) == 0;
#define GS_ZERO_TOUCHED(D)                                                                      \
  zero_touched_kernel<D><<<blocks, 256, 0, st>>>(sorted_ids, hdr, sh_vec, dq_vec, d_means,      \
                                                 d_scales, d_quats, d_opac, d_sh)
  switch (deg) {
    case 0: GS_ZERO_TOUCHED(0); break;
    case 1: GS_ZERO_TOUCHED(1); break;
    case 2: GS_ZERO_TOUCHED(2); break;
    default: GS_ZERO_TOUCHED(3); break;
  }
#undef GS_ZERO_TOUCHED
  return cudaGetLastError();
}

}  // namespace gsr

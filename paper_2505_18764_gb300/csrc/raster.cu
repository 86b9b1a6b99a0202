// Forward and backward rasterization.
//
// Work is cut into warp-sized items.  An item is a rectangle of pixels (the
// warp's footprint) inside one 16x16 block; the warp walks that block's
// depth-ordered splat list on its own, staging 32 records at a time into a
// private ring in shared memory (asynchronous copies, a few groups in
// flight), so warps never wait for one another.  A block is cut into four
// 8x8 quadrants with two pixels per lane (rows r and r + 4), or, when its
// list is long, into eight 8x4 footprints with one pixel per lane, or, when
// it is very long, into sixteen 4x4 footprints on half a warp: a block under
// a pile of small splats is then walked by more warps, each meeting fewer
// candidates, instead of setting the launch time on its own.  (Square
// quadrants meet ~10% fewer splats than 16x4 bands of the same area.)
// Persistent CTAs take items from a counter: the forward in the order the
// binning wrote them (longest lists first), the backward costliest first by
// the forward's measured time per item (fragment density, not list length,
// decides most of it).
//
// That is the CUDA counterpart of the paper's ordered fragment processing: a
// pixel belongs to one lane, which meets the block's splats in depth order, so
// no interlock is needed (the race programmable blending guards against cannot
// occur), and a splat's fragments in a footprint are evaluated together by one
// warp (the "cohesion" of Sec. 3.2.3 holds by construction).  Each warp first
// tests the staged splats against its footprint (rect_may_hit) and then walks
// only those that can touch it.
//
// Forward (Eq. 2, Sec. 2.1.2): alpha = min(0.99, o exp(power)), fragments with
// alpha < 1/255 skipped, T-culling skips fragment i iff T_i < t_cull
// (Procedure 1; the same rule in both passes, so the backward is the exact
// gradient of the image the forward produced).
//
// Backward (Procedure 1): (C', T) start at (stored C, 1); per fragment
// dL/dc = g alpha T (Eq. 3), dL/dalpha = g . (c T - C') / (1 - alpha) (Eq. 7),
// then C' -= T alpha c (Eq. 6) and T *= 1 - alpha (Eq. 5).  The chain rule to
// the 2D splat parameters follows; the nine per-fragment values of a lane's
// pixels are added, summed over the warp through shared memory in batches of
// four candidates, and one vector-atomic triple per (splat, footprint) reaches
// global memory (Procedure 2's role).  Both passes take their candidates two
// per step, evaluating what does not depend on the pixel's running state for
// both before the depth-ordered updates.
#include "common.cuh"

namespace gsr {

constexpr int kThreads = 128;                 // 4 independent warps per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kFwdStages = 4;                 // groups of 32 records in flight per warp: forward
constexpr int kBwdStages = 2;                 // backward (a group takes it far longer)
constexpr unsigned kFull = 0xffffffffu;

// Item encoding: block << 5 | code; code 0..3 = 8x8 quadrant (two pixels per
// lane), 8..15 = 8x4 cell (one pixel per lane), 16..31 = 4x4 cell (one pixel
// on each of lanes 0..15).
constexpr uint32_t kCell8Code = 8u, kCell4Code = 16u;

template <int STAGES>
struct WarpRing {
  static constexpr int kStages = STAGES;
  float4 a[STAGES][32];
  float4 b[STAGES][32];
  float4 c[STAGES][32];
  uint32_t rank[STAGES][32];
};
using FwdRing = WarpRing<kFwdStages>;
using BwdRing = WarpRing<kBwdStages>;

// Copy the records of list entries [i - lane, i - lane + 32) (this lane's is i)
// into ring slot `slot`; `rk` is this lane's depth rank, loaded beforehand.
// Every call commits one copy group, empty or not, so wait_group counts slots.
template <class Ring>
__device__ __forceinline__ void ring_issue(Ring& R, int slot, const SplatRec* __restrict__ rec,
                                           uint32_t i, uint32_t end, uint32_t rk, int lane) {
  if (i < end) {
    const SplatRec* g = rec + rk;
    cp_async16(&R.a[slot][lane], &g->a);
    cp_async16(&R.b[slot][lane], &g->b);
    cp_async16(&R.c[slot][lane], &g->c);
    R.rank[slot][lane] = rk;
  }
  cp_async_commit();
}

// Fill all slots with the first kStages groups of [beg, end).
template <class Ring>
__device__ __forceinline__ void ring_start(Ring& R, const SplatRec* __restrict__ rec,
                                           const uint32_t* __restrict__ pair_ranks, uint32_t beg,
                                           uint32_t end, int lane) {
  constexpr int S = Ring::kStages;
  uint32_t rk[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const uint32_t i = beg + 32u * s + lane;
    rk[s] = i < end ? __ldg(pair_ranks + i) : 0u;
  }
#pragma unroll
  for (int s = 0; s < S; ++s) ring_issue(R, s, rec, beg + 32u * s + lane, end, rk[s], lane);
}

// Next item index for this warp (one atomic per warp), or >= n_items when none are left.
__device__ __forceinline__ uint32_t next_item(uint32_t* counter, int lane) {
  uint32_t idx = 0;
  if (lane == 0) idx = atomicAdd(counter, 1u);
  return __shfl_sync(kFull, idx, 0);
}

// Block and top-left pixel of an item; returns the footprint width (16, 8 or 4).
__device__ __forceinline__ int item_origin(uint32_t it, int gw, int& block, int& x0, int& y0) {
  block = (int)(it >> 5);
  const int code = (int)(it & 31u);
  const int bx = block % gw, by = block / gw;
  x0 = bx * kBlock;
  y0 = by * kBlock;
  if (code < (int)kCell8Code) {
    x0 += 8 * (code & 1);
    y0 += 8 * (code >> 1);
    return 16;
  }
  if (code < (int)kCell4Code) {
    const int c = code - (int)kCell8Code;
    x0 += 8 * (c & 1);
    y0 += 4 * (c >> 1);
    return 8;
  }
  const int c = code - (int)kCell4Code;
  x0 += 4 * (c & 3);
  y0 += 4 * (c >> 2);
  return 4;
}

// This lane's pixels: COLS = 16 stands for an 8x8 quadrant with two pixels
// per lane, (x, ya) and (x, ya + 4); COLS = 8 or 4, a footprint COLS wide and 4
// high with one pixel per lane (lanes beyond a 4x4 footprint own none).
template <int COLS>
__device__ __forceinline__ void lane_pixels(int x0, int y0, int lane, int& x, int& ya, bool& own) {
  x = x0 + (COLS == 16 ? lane % 8 : lane % COLS);
  ya = y0 + (COLS == 16 ? lane / 8 : lane / COLS);
  own = COLS != 4 || lane < 16;
}

// The pixel-centre rectangle (x0, y0, wx, wy) of the warp's pixels still in
// play (act_a: the lane's pixel (x, ya); act_b: (x, yb)): the forward tests a
// group's candidates against it instead of the whole footprint, so once pixels
// are T-culled the candidates that can only reach them are not walked (the
// densest blocks, whose items end the launch, are T-culled almost everywhere).
// At least one lane must have a pixel in play.  (In the backward, with pixels
// past their last fragment, the same test cost more than it saved.)
__device__ __forceinline__ void active_rect(bool act_a, bool act_b, int x, int ya, int yb,
                                            float& x0, float& y0, float& wx, float& wy) {
  const bool any = act_a || act_b;
  const int lx = any ? x : 0x7fffffff, hx = any ? x : -1;
  const int ly = act_a ? ya : (act_b ? yb : 0x7fffffff);
  const int hy = act_b ? yb : (act_a ? ya : -1);
  const int xmin = __reduce_min_sync(kFull, lx), xmax = __reduce_max_sync(kFull, hx);
  const int ymin = __reduce_min_sync(kFull, ly), ymax = __reduce_max_sync(kFull, hy);
  x0 = (float)xmin + 0.5f;
  y0 = (float)ymin + 0.5f;
  wx = (float)(xmax - xmin);
  wy = (float)(ymax - ymin);
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
struct PixelFwd {
  float T, C0, C1, C2;
  uint32_t last, n;
  bool done;
};

// One fragment (hit false would make it an exact no-op: alpha = 0 leaves C and
// T unchanged).
__device__ __forceinline__ void blend(PixelFwd& p, bool hit, float alpha, const float4& c,
                                      uint32_t rank, float t_cull) {
  const float w = __fmul_rn(alpha, p.T);
  p.C0 = __fmaf_rn(w, c.x, p.C0);
  p.C1 = __fmaf_rn(w, c.y, p.C1);
  p.C2 = __fmaf_rn(w, c.z, p.C2);
  p.T = next_T(p.T, alpha);
  p.last = hit ? rank : p.last;
  p.n += hit ? 1u : 0u;
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

// One warp, one footprint COLS x 4 (two pixels per lane when COLS = 16).
// resume: the pixel continues from the colour, transmittance, last rank and
// count stored by the previous chunk (memory-efficiency mode).
__device__ __forceinline__ void resume_fwd(PixelFwd& p, int x, int y, int W, int fmt,
                                           const void* state, const uint32_t* last_out,
                                           const uint32_t* ncontrib, float t_cull) {
  const size_t pix = (size_t)y * W + x;
  const float4 st = load_state(state, fmt, pix);
  p.C0 = st.x; p.C1 = st.y; p.C2 = st.z; p.T = st.w;
  p.last = last_out[pix];
  p.n = ncontrib ? ncontrib[pix] : 0u;
  p.done = p.T < t_cull;
}

// Returns (warp-uniform) how many of the footprint's pixels in the image end
// T-culled (the memory-efficiency mode's per-block count).
template <int COLS>
__device__ __forceinline__ uint32_t fwd_item(FwdRing& R, const SplatRec* __restrict__ rec,
                                         const uint32_t* __restrict__ pair_ranks, uint2 range,
                                         int x0, int y0, int lane, int W, int H, float t_cull,
                                         int fmt, float* image, void* state, uint32_t* last_out,
                                         uint32_t* ncontrib, int resume) {
  constexpr int NPX = COLS == 16 ? 2 : 1;
  int x, ya;
  bool own;
  lane_pixels<COLS>(x0, y0, lane, x, ya, own);
  const int yb = ya + 4;
  const float px = (float)x + 0.5f, pya = (float)ya + 0.5f, pyb = (float)yb + 0.5f;
  PixelFwd pa{1.f, 0.f, 0.f, 0.f, kNone, 0u, !(own && x < W && ya < H)};
  PixelFwd pb{1.f, 0.f, 0.f, 0.f, kNone, 0u, NPX == 1 || !(x < W && yb < H)};
  if (resume) {
    if (!pa.done) resume_fwd(pa, x, ya, W, fmt, state, last_out, ncontrib, t_cull);
    if (!pb.done) resume_fwd(pb, x, yb, W, fmt, state, last_out, ncontrib, t_cull);
  }
  const bool wa = own && x < W && ya < H, wb = NPX == 2 && x < W && yb < H;

  const uint32_t beg = range.x, end = range.y;
  if (beg < end) ring_start(R, rec, pair_ranks, beg, end, lane);
  int slot = 0;
  if (COLS == 4) {
    // 4x4 cells (long lists): two groups per round, so the round's fixed work
    // (waits, active rectangle, votes, refills) is spread over 64 entries
    auto walk = [&](int s, uint32_t m) {
      while (m) {
        const int j1 = __ffs(m) - 1;
        m &= m - 1u;
        const bool two = m != 0u;
        const int j2 = two ? __ffs(m) - 1 : j1;
        if (two) m &= m - 1u;
        const float4 a1 = R.a[s][j1], b1 = R.b[s][j1];
        const float4 a2 = R.a[s][j2], b2 = R.b[s][j2];
        float y1, y2;
        const float qa1 = frag_q(px, pya, a1, b1, y1, y2);
        const float qa2 = frag_q(px, pya, a2, b2, y1, y2);
        const float4 c1 = R.c[s][j1], c2 = R.c[s][j2];
        const uint32_t rank1 = R.rank[s][j1], rank2 = R.rank[s][j2];
        float G, at;
        const float alpha1 = frag_alpha(c1.w, qa1, G, at), alpha2 = frag_alpha(c2.w, qa2, G, at);
        if (!pa.done && qa1 <= b1.y) blend(pa, true, alpha1, c1, rank1, t_cull);
        if (two && !pa.done && qa2 <= b2.y) blend(pa, true, alpha2, c2, rank2, t_cull);
      }
    };
    for (uint32_t gs = beg; gs < end; gs += 64u, slot ^= 2) {
      const uint32_t ip0 = gs + 32u * kFwdStages + lane, ip1 = ip0 + 32u;
      const uint32_t rk0 = ip0 < end ? __ldg(pair_ranks + ip0) : 0u;
      const uint32_t rk1 = ip1 < end ? __ldg(pair_ranks + ip1) : 0u;
      cp_async_wait_group<kFwdStages - 2>();
      __syncwarp();
      if (__all_sync(kFull, pa.done)) break;
      const uint32_t cnt0 = min(32u, end - gs);
      const uint32_t cnt1 = gs + 32u < end ? min(32u, end - gs - 32u) : 0u;
      float rx, ry, rw, rh;
      active_rect(!pa.done, false, x, ya, yb, rx, ry, rw, rh);
      const uint32_t m0 = __ballot_sync(kFull, (uint32_t)lane < cnt0 &&
                                                   rect_may_hit(R.a[slot][lane], R.b[slot][lane],
                                                                rx, ry, rw, rh));
      const uint32_t m1 = __ballot_sync(kFull, (uint32_t)lane < cnt1 &&
                                                   rect_may_hit(R.a[slot + 1][lane],
                                                                R.b[slot + 1][lane], rx, ry, rw, rh));
      walk(slot, m0);
      walk(slot + 1, m1);
      __syncwarp();   // every lane is done with both slots before they are refilled
      ring_issue(R, slot, rec, ip0, end, rk0, lane);
      ring_issue(R, slot + 1, rec, ip1, end, rk1, lane);
    }
  }
  for (uint32_t gs = COLS == 4 ? end : beg; gs < end; gs += 32u, slot = (slot + 1) & (kFwdStages - 1)) {
    const uint32_t ip = gs + 32u * kFwdStages + lane;      // this lane's entry of the refill
    const uint32_t rk_next = ip < end ? __ldg(pair_ranks + ip) : 0u;
    cp_async_wait_group<kFwdStages - 1>();
    __syncwarp();
    if (__all_sync(kFull, pa.done && pb.done)) break;
    const uint32_t cnt = min(32u, end - gs);
    float rx, ry, rw, rh;
    active_rect(!pa.done, NPX == 2 && !pb.done, x, ya, yb, rx, ry, rw, rh);
    uint32_t m = __ballot_sync(kFull, (uint32_t)lane < cnt &&
                                          rect_may_hit(R.a[slot][lane], R.b[slot][lane], rx, ry,
                                                       rw, rh));
    // two candidates at a time: their q and alpha do not depend on the pixel's
    // state, so both are evaluated before the first blends (the second's hit
    // is decided after the first may have T-culled the pixel)
    while (m) {
      const int j1 = __ffs(m) - 1;
      m &= m - 1u;
      const bool two = m != 0u;
      const int j2 = two ? __ffs(m) - 1 : j1;
      if (two) m &= m - 1u;
      const float4 a1 = R.a[slot][j1], b1 = R.b[slot][j1];
      const float4 a2 = R.a[slot][j2], b2 = R.b[slot][j2];
      float y1, y2a, y2b = 0.f, qa1, qb1 = 0.f, qa2, qb2 = 0.f;
      if (NPX == 2) {
        frag_q2(px, pya, pyb, a1, b1, y1, y2a, y2b, qa1, qb1);
        frag_q2(px, pya, pyb, a2, b2, y1, y2a, y2b, qa2, qb2);
      } else {
        qa1 = frag_q(px, pya, a1, b1, y1, y2a);
        qa2 = frag_q(px, pya, a2, b2, y1, y2a);
      }
      const float4 c1 = R.c[slot][j1], c2 = R.c[slot][j2];
      const uint32_t rank1 = R.rank[slot][j1], rank2 = R.rank[slot][j2];
      float G, at;
      const float alpha_a1 = frag_alpha(c1.w, qa1, G, at), alpha_a2 = frag_alpha(c2.w, qa2, G, at);
      float alpha_b1 = 0.f, alpha_b2 = 0.f;
      if (NPX == 2) {
        alpha_b1 = frag_alpha(c1.w, qb1, G, at);
        alpha_b2 = frag_alpha(c2.w, qb2, G, at);
      }
      if (!pa.done && qa1 <= b1.y) blend(pa, true, alpha_a1, c1, rank1, t_cull);
      if (NPX == 2 && !pb.done && qb1 <= b1.y) blend(pb, true, alpha_b1, c1, rank1, t_cull);
      if (two && !pa.done && qa2 <= b2.y) blend(pa, true, alpha_a2, c2, rank2, t_cull);
      if (NPX == 2 && two && !pb.done && qb2 <= b2.y) blend(pb, true, alpha_b2, c2, rank2, t_cull);
    }
    __syncwarp();   // every lane is done with the slot before it is refilled
    ring_issue(R, slot, rec, ip, end, rk_next, lane);
  }
  cp_async_wait_all();
  __syncwarp();
  if (wa) write_fwd(pa, x, ya, W, H, fmt, image, state, last_out, ncontrib);
  if (wb) write_fwd(pb, x, yb, W, H, fmt, image, state, last_out, ncontrib);
  return (uint32_t)__popc(__ballot_sync(kFull, wa && pa.T < t_cull)) +
         (uint32_t)__popc(__ballot_sync(kFull, wb && pb.T < t_cull));
}

__global__ void __launch_bounds__(kThreads) raster_fwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ items,
    const Header* __restrict__ hdr, uint32_t* __restrict__ next, uint32_t* __restrict__ item_cost,
    const uint32_t* __restrict__ pair_ranks, const SplatRec* __restrict__ rec, int W, int H, int gw,
    float t_cull, int fmt, float* __restrict__ image, void* __restrict__ state,
    uint32_t* __restrict__ last_out, uint32_t* __restrict__ ncontrib, int resume,
    uint32_t* __restrict__ block_done, uint32_t* __restrict__ done_px, uint32_t chunk) {
  __shared__ FwdRing rings[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  FwdRing& R = rings[warp];
  const uint32_t n_items = hdr->n_items;
  for (uint32_t idx = next_item(next, lane); idx < n_items; idx = next_item(next, lane)) {
    int block, x0, y0;
    const int cols = item_origin(items[idx], gw, block, x0, y0);
    const uint2 range = ranges[block];
    const long long t0 = clock64();
    uint32_t culled;
    if (cols == 16)
      culled = fwd_item<16>(R, rec, pair_ranks, range, x0, y0, lane, W, H, t_cull, fmt, image,
                            state, last_out, ncontrib, resume);
    else if (cols == 8)
      culled = fwd_item<8>(R, rec, pair_ranks, range, x0, y0, lane, W, H, t_cull, fmt, image,
                           state, last_out, ncontrib, resume);
    else
      culled = fwd_item<4>(R, rec, pair_ranks, range, x0, y0, lane, W, H, t_cull, fmt, image,
                           state, last_out, ncontrib, resume);
    if (lane == 0) item_cost[idx] = (uint32_t)min(clock64() - t0, (long long)0xFFFFFFFF);
    // memory-efficiency mode: the item that completes the count of the block's
    // T-culled pixels marks the block done after this chunk
    if (block_done && lane == 0 && culled) {
      const int bx = block % gw, by = block / gw;
      const uint32_t valid = (uint32_t)(min(kBlock, W - bx * kBlock) * min(kBlock, H - by * kBlock));
      // (the earliest such chunk stays: later chunks count the same pixels again)
      if (atomicAdd(done_px + block, culled) + culled == valid) atomicMin(block_done + block, chunk);
    }
  }
}

// ---------------------------------------------------------------------------
// Backward
//
// Procedure 1 carries C' (three channels) to form dL/dalpha_i = g . (c_i T_i -
// C'_i) / (1 - alpha_i) (Eq. 7).  Only the dot product with g enters, so each
// pixel carries D = g . C' instead: D_1 = g . C (stored colour), and Eq. 6
// dotted with g gives D_{i+1} = D_i - T_i alpha_i (g . c_i).  Then
// dL/dalpha_i = (T_i (g . c_i) - D_i) / (1 - alpha_i): the same quantity with
// one running number per pixel instead of three.
// ---------------------------------------------------------------------------

// Reduced candidates are summed over the warp in batches of kBatch through
// shared memory: each lane stores its nine values of a candidate in column
// rows; after kBatch candidates, 18 lanes each add up 16 rows of one column
// (values 0-3 or 4-7 of a candidate, or value 8 of all four) and one shuffle
// joins the two halves.  Per candidate that is about a third of the
// instructions of a shuffle transpose-reduce.
constexpr int kBatch = 4;
constexpr int kColStride = 41;   // float4 per column: 32 rows, 4 of padding between the halves,
                                 // 41 = 1 mod 8 so that columns start in different bank groups

struct GradBatch {
  float4 col[9 * kColStride];
  uint32_t rank[kBatch];
};

// Row position of lane `lane` in a column: rows 16..31 sit four float4 later,
// so that the two halves read in one step fall in different bank groups.
__device__ __forceinline__ int batch_row(int lane) { return lane + ((lane >> 4) << 2); }

__device__ __forceinline__ void batch_put(GradBatch& B, int s, int lane, uint32_t rank,
                                          const float v[9]) {
  const int row = batch_row(lane);
  B.col[(2 * s) * kColStride + row] = make_float4(v[0], v[1], v[2], v[3]);
  B.col[(2 * s + 1) * kColStride + row] = make_float4(v[4], v[5], v[6], v[7]);
  reinterpret_cast<float*>(&B.col[8 * kColStride + row])[s] = v[8];
  B.rank[s] = rank;   // every lane stores the same value: no branch
}

// Sums of the batch's first n candidates, added to their accumulators.
__device__ __forceinline__ void batch_flush(GradBatch& B, int n, int lane, float* g2d) {
  __syncwarp();
  const int c = min(lane & 15, 8), half = lane >> 4;
  const float4* src = &B.col[c * kColStride + half * 20];
  // 16 rows as packed pairs, four running sums (a shorter dependency chain)
  float2 lo[4], hi[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float4 v = src[r];
    lo[r] = make_float2(v.x, v.y);
    hi[r] = make_float2(v.z, v.w);
  }
#pragma unroll
  for (int r = 4; r < 16; ++r) {
    const float4 v = src[r];
    lo[r & 3] = __fadd2_rn(lo[r & 3], make_float2(v.x, v.y));
    hi[r & 3] = __fadd2_rn(hi[r & 3], make_float2(v.z, v.w));
  }
  const float2 l = __fadd2_rn(__fadd2_rn(lo[0], lo[1]), __fadd2_rn(lo[2], lo[3]));
  const float2 h = __fadd2_rn(__fadd2_rn(hi[0], hi[1]), __fadd2_rn(hi[2], hi[3]));
  float4 acc = make_float4(l.x, l.y, h.x, h.y);
  acc.x += __shfl_xor_sync(kFull, acc.x, 16);
  acc.y += __shfl_xor_sync(kFull, acc.y, 16);
  acc.z += __shfl_xor_sync(kFull, acc.z, 16);
  acc.w += __shfl_xor_sync(kFull, acc.w, 16);
  if (lane < 8) {
    const int s = lane >> 1;
    if (s < n) red_add_v4(g2d + (size_t)B.rank[s] * 12 + 4 * (lane & 1), acc.x, acc.y, acc.z, acc.w);
  } else if (lane == 8) {   // value 8 of each candidate
    atomicAdd(g2d + (size_t)B.rank[0] * 12 + 8, acc.x);
    if (n > 1) atomicAdd(g2d + (size_t)B.rank[1] * 12 + 8, acc.y);
    if (n > 2) atomicAdd(g2d + (size_t)B.rank[2] * 12 + 8, acc.z);
    if (n > 3) atomicAdd(g2d + (size_t)B.rank[3] * 12 + 8, acc.w);
  }
  __syncwarp();   // the columns are free again
}

__device__ __forceinline__ void red_add9(float* dst, const float v[9]) {
  red_add_v4(dst, v[0], v[1], v[2], v[3]);
  red_add_v4(dst + 4, v[4], v[5], v[6], v[7]);
  red_add_v4(dst + 8, v[8], 0.f, 0.f, 0.f);
}

// Candidate `rank`'s nine values v of this lane (frag: the lane had a
// fragment): added directly when fewer than `threshold` lanes have one (the
// balancing threshold of Sec. 3.2.4), else put in the batch (nb: candidates
// waiting in it).
template <int MODE>
__device__ __forceinline__ void reduce_candidate(const float v[9], bool frag, uint32_t rank,
                                                 GradBatch& B, int& nb, float* g2d,
                                                 int threshold, int lane) {
  if (MODE != GS_REDUCE_WARP) {
    if (frag) red_add9(g2d + (size_t)rank * 12, v);
  } else {
    const uint32_t active = __ballot_sync(kFull, frag);
    if (active != 0u) {
      if (__popc(active) < threshold) {
        if (frag) red_add9(g2d + (size_t)rank * 12, v);
      } else {
        batch_put(B, nb, lane, rank, v);
        if (++nb == kBatch) {
          batch_flush(B, kBatch, lane, g2d);
          nb = 0;
        }
      }
    }
  }
}

struct PixelBwd {
  float D, T, g0, g1, g2;   // D = g . C'
  uint32_t end;             // depth rank after the pixel's last fragment
};

// Per-pixel inputs of the backward beyond the state: chunk_state (memory-
// efficiency mode: with chunk_in, (D, T) continue from the previous chunk
// instead of (g . stored C, 1)) and, for a depth slab, t_front (the
// transmittance of the slabs in front: the slab's colour enters the image as
// t_front C_slab, so its image gradient is t_front g) and behind (the colour
// composited from the slabs behind: the colour seen from the slab's start is
// C_slab + T_slab behind, which is where C' starts).  Null pointers stand for
// t_front = 1 and behind = 0.
struct BwdExtra {
  const float4* chunk_state;
  int chunk_in;
  const float* t_front;
  const float* behind;
};

__device__ __forceinline__ void load_pixel_bwd(PixelBwd& p, bool valid, int x, int y, int W,
                                               int fmt, const void* state,
                                               const uint32_t* last_in, const float* dLdC,
                                               const BwdExtra& ex) {
  p.D = 0.f;
  p.g0 = p.g1 = p.g2 = 0.f;
  p.T = 1.f;
  p.end = 0;
  if (valid) {
    const size_t pix = (size_t)y * W + x;
    p.g0 = dLdC[3 * pix]; p.g1 = dLdC[3 * pix + 1]; p.g2 = dLdC[3 * pix + 2];
    if (ex.t_front) {
      const float tf = ex.t_front[pix];
      p.g0 *= tf; p.g1 *= tf; p.g2 *= tf;
    }
    if (ex.chunk_in) {
      const float4 cs = ex.chunk_state[pix];
      p.D = cs.x;
      p.T = cs.y;
    } else {
      float4 st = load_state(state, fmt, pix);
      if (ex.behind) {
        st.x = fmaf(st.w, ex.behind[3 * pix], st.x);
        st.y = fmaf(st.w, ex.behind[3 * pix + 1], st.y);
        st.z = fmaf(st.w, ex.behind[3 * pix + 2], st.z);
      }
      p.D = p.g0 * st.x + p.g1 * st.y + p.g2 * st.z;
    }
    const uint32_t l = last_in[pix];
    p.end = (l == kNone) ? 0u : l + 1u;
  }
}

// One fragment of Procedure 1 plus the chain rule to the 2D parameters, in two
// halves.  frag_pre takes what does not depend on the pixel's running state
// (alpha, 1 / (1 - alpha), g . c, the whitened offset z), frag_post the rest:
// the two halves of two candidates can then be interleaved, the second
// candidate's first half filling the first candidate's latencies.  The nine
// values go to v.  The pixel's fragments are exactly the hits below its end
// rank: the forward stopped after the fragment that took T under t_cull, so
// Procedure 1's cull test needs no second evaluation.  A missed pixel (hit
// false) runs the same code with G = 0: every term is an exact zero and the
// state is unchanged.
struct FragPre {
  float G, at, alpha, oma, inv, gc, z0, z1;
};

__device__ __forceinline__ void frag_pre(const PixelBwd& p, bool hit, float q, float y1, float y2,
                                         const float4& a, const float4& b, const float4& c,
                                         FragPre& r) {
  r.alpha = frag_alpha_masked(hit, c.w, q, r.G, r.at);
  r.oma = __fsub_rn(1.0f, r.alpha);
  r.inv = __fdividef(1.0f, r.oma);
  r.gc = p.g0 * c.x + p.g1 * c.y + p.g2 * c.z;
  // z = Sigma^-1 d = L^-T L^-1 d, in units of 1 / (2 ln 2):
  // dpower/dmu_2D = z and dpower/dSigma_2D = z z^T / 2
  r.z1 = b.x * y2;
  r.z0 = a.z * y1 - a.w * r.z1;
}

__device__ __forceinline__ void frag_post(PixelBwd& p, const FragPre& r, float v[9]) {
  const float wT = r.alpha * p.T;
  // Eq. 3
  v[5] = p.g0 * wT;
  v[6] = p.g1 * wT;
  v[7] = p.g2 * wT;
  // Eq. 7 with D_i = g . C'_i before its update, then Eq. 6 and Eq. 5
  const float dLda = (p.T * r.gc - p.D) * r.inv;
  p.D -= wT * r.gc;
  p.T = next_T(p.T, r.alpha);
  // alpha = min(0.99, o G): no gradient through the clamp
  const float d_at = r.at < kAlphaMax ? dLda : 0.f;
  v[8] = r.G * d_at;
  const float w = r.at * d_at;
  const float wz0 = w * r.z0, wz1 = w * r.z1;
  v[0] = wz0;
  v[1] = wz1;
  v[2] = wz0 * r.z0;
  v[3] = wz0 * r.z1;
  v[4] = wz1 * r.z1;
}

__device__ __forceinline__ void grad_fragment(PixelBwd& p, bool hit, float q, float y1, float y2,
                                              const float4& a, const float4& b, const float4& c,
                                              float v[9]) {
  FragPre r;
  frag_pre(p, hit, q, y1, y2, a, b, c, r);
  frag_post(p, r, v);
}

// One warp, one footprint COLS x 4 with one pixel per lane (COLS = 8 or 4).
template <int COLS, int MODE>
__device__ __forceinline__ void bwd_item(BwdRing& R, GradBatch& B,
                                         const SplatRec* __restrict__ rec,
                                         const uint32_t* __restrict__ pair_ranks, uint2 range,
                                         int x0, int y0, int lane, int W, int H, int fmt,
                                         const void* state, const uint32_t* last_in,
                                         const float* dLdC, float* g2d, int threshold,
                                         const BwdExtra& ex, float4* chunk_state, int chunk_out) {
  int x, ya;
  bool own;
  lane_pixels<COLS>(x0, y0, lane, x, ya, own);
  const float px = (float)x + 0.5f, pya = (float)ya + 0.5f;
  const float xs = (float)x0 + 0.5f, ys = (float)y0 + 0.5f;
  PixelBwd pa;
  const bool va = own && x < W && ya < H;
  load_pixel_bwd(pa, va, x, ya, W, fmt, state, last_in, dLdC, ex);
  // depth ranks >= this contribute nowhere in the footprint
  const uint32_t warp_end = __reduce_max_sync(kFull, pa.end);

  const uint32_t beg = range.x, end = warp_end > 0u ? range.y : range.x;
  if (beg < end) ring_start(R, rec, pair_ranks, beg, end, lane);
  int slot = 0, nb = 0;
  for (uint32_t gs = beg; gs < end; gs += 32u, slot = (slot + 1) & (kBwdStages - 1)) {
    const uint32_t ip = gs + 32u * kBwdStages + lane;
    const uint32_t rk_next = ip < end ? __ldg(pair_ranks + ip) : 0u;
    cp_async_wait_group<kBwdStages - 1>();
    __syncwarp();
    if (R.rank[slot][0] >= warp_end) break;   // ranks ascend along the list
    const uint32_t cnt = min(32u, end - gs);
    uint32_t m = __ballot_sync(kFull, (uint32_t)lane < cnt &&
                                          rect_may_hit(R.a[slot][lane], R.b[slot][lane], xs, ys,
                                                       (float)(COLS - 1), 3.f));
    // Two candidates per step (the second may be absent): both are tested, then
    // the first halves of both fragments are taken before the second halves,
    // which follow the depth order.
    while (m) {
      const int j0 = __ffs(m) - 1;
      m &= m - 1u;
      const bool two = m != 0u;
      const int j1 = two ? __ffs(m) - 1 : j0;
      m &= m - 1u;
      const uint32_t rank0 = R.rank[slot][j0], rank1 = R.rank[slot][j1];
      const float4 a0 = R.a[slot][j0], b0 = R.b[slot][j0];
      const float4 a1 = R.a[slot][j1], b1 = R.b[slot][j1];
      float y10, y20, y11, y21;
      const float q0 = frag_q(px, pya, a0, b0, y10, y20);
      const float q1 = frag_q(px, pya, a1, b1, y11, y21);
      const bool h0 = rank0 < pa.end && q0 <= b0.y;
      const bool h1 = two && rank1 < pa.end && q1 <= b1.y;
      const float4 c0 = R.c[slot][j0], c1 = R.c[slot][j1];
      const bool u0 = __any_sync(kFull, h0), u1 = __any_sync(kFull, h1);
      float v0[9], v1[9];
      if (u0 && u1) {
        FragPre r0, r1;
        frag_pre(pa, h0, q0, y10, y20, a0, b0, c0, r0);
        frag_pre(pa, h1, q1, y11, y21, a1, b1, c1, r1);
        frag_post(pa, r0, v0);
        frag_post(pa, r1, v1);
        reduce_candidate<MODE>(v0, h0, rank0, B, nb, g2d, threshold, lane);
        reduce_candidate<MODE>(v1, h1, rank1, B, nb, g2d, threshold, lane);
      } else if (u0) {
        grad_fragment(pa, h0, q0, y10, y20, a0, b0, c0, v0);
        reduce_candidate<MODE>(v0, h0, rank0, B, nb, g2d, threshold, lane);
      } else if (u1) {
        grad_fragment(pa, h1, q1, y11, y21, a1, b1, c1, v1);
        reduce_candidate<MODE>(v1, h1, rank1, B, nb, g2d, threshold, lane);
      }
    }
    __syncwarp();   // every lane is done with the slot before it is refilled
    ring_issue(R, slot, rec, ip, end, rk_next, lane);
  }
  cp_async_wait_all();
  if (nb > 0) batch_flush(B, nb, lane, g2d);
  __syncwarp();
  if (chunk_out && va) chunk_state[(size_t)ya * W + x] = make_float4(pa.D, pa.T, 0.f, 0.f);
}

// ---------------------------------------------------------------------------
// The two pixels of a lane in an 8x8 quadrant, (x, ya) and (x, ya + 4), walked as
// packed FP32 pairs: each operation below is one FP32x2 instruction that
// rounds both halves exactly as the scalar operation does, so a candidate
// costs about half the issue slots of two scalar walks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// q at both pixels, bit-identical to frag_q2 (dx and y1 are common).
__device__ __forceinline__ float2 frag_q_pair(float px, float2 py, const float4& a,
                                              const float4& b, float& y1, float2& y2) {
  const float dx = __fsub_rn(__fsub_rn(px, a.x), b.z);
  const float2 dy = __fadd2_rn(__fadd2_rn(py, f2(-a.y)), f2(-b.w));   // x - y == x + (-y)
  y1 = __fmul_rn(a.z, dx);
  y2 = __fmul2_rn(f2(b.x), __ffma2_rn(f2(-a.w), f2(dx), dy));
  return __ffma2_rn(f2(y1), f2(y1), __fmul2_rn(y2, y2));
}

struct PairBwd {
  float2 nD;              // -D = -g . C' of the two pixels
  float2 T, g0, g1, g2;
  uint32_t end_a, end_b;  // depth rank after each pixel's last fragment
};

__device__ __forceinline__ PairBwd pack_pair(const PixelBwd& a, const PixelBwd& b) {
  PairBwd p;
  p.nD = make_float2(-a.D, -b.D);
  p.T = make_float2(a.T, b.T);
  p.g0 = make_float2(a.g0, b.g0);
  p.g1 = make_float2(a.g1, b.g1);
  p.g2 = make_float2(a.g2, b.g2);
  p.end_a = a.end;
  p.end_b = b.end;
  return p;
}

// One candidate of Procedure 1 at both pixels of a lane, in the two halves of
// frag_pre and frag_post; t[k] holds the two pixels' contributions to value k.
struct PairPre {
  float2 G, at, alpha, oma, inv, gc, z0, z1;
};

__device__ __forceinline__ void pair_pre(const PairBwd& p, bool ha, bool hb, float2 q, float y1,
                                         float2 y2, const float4& a, const float4& b,
                                         const float4& c, PairPre& r) {
  r.G = make_float2(ha ? ex2_approx(-q.x) : 0.0f, hb ? ex2_approx(-q.y) : 0.0f);
  r.at = __fmul2_rn(f2(c.w), r.G);
  r.alpha = make_float2(fminf(kAlphaMax, r.at.x), fminf(kAlphaMax, r.at.y));
  r.oma = __ffma2_rn(r.alpha, f2(-1.0f), f2(1.0f));   // 1 - alpha, rounded once
  r.inv = make_float2(__fdividef(1.0f, r.oma.x), __fdividef(1.0f, r.oma.y));
  r.gc = __ffma2_rn(p.g0, f2(c.x), __ffma2_rn(p.g1, f2(c.y), __fmul2_rn(p.g2, f2(c.z))));
  // z = Sigma^-1 d (see frag_pre)
  r.z1 = __fmul2_rn(f2(b.x), y2);
  r.z0 = __ffma2_rn(f2(-a.w), r.z1, f2(a.z * y1));
}

__device__ __forceinline__ void pair_post(PairBwd& p, const PairPre& r, float2 t[9]) {
  const float2 wT = __fmul2_rn(r.alpha, p.T);
  // Eq. 3
  t[5] = __fmul2_rn(p.g0, wT);
  t[6] = __fmul2_rn(p.g1, wT);
  t[7] = __fmul2_rn(p.g2, wT);
  // Eq. 7 with D_i before its update: (T g . c - D) / (1 - alpha)
  const float2 dLda = __fmul2_rn(__ffma2_rn(p.T, r.gc, p.nD), r.inv);
  // Eq. 6 (dotted with g), Eq. 5
  p.nD = __ffma2_rn(wT, r.gc, p.nD);
  p.T = __fmul2_rn(p.T, r.oma);
  // alpha = min(0.99, o G): no gradient through the clamp
  const float2 d_at = make_float2(r.at.x < kAlphaMax ? dLda.x : 0.0f,
                                  r.at.y < kAlphaMax ? dLda.y : 0.0f);
  t[8] = __fmul2_rn(r.G, d_at);
  // weighted by dL/dpower
  const float2 w = __fmul2_rn(r.at, d_at);
  t[0] = __fmul2_rn(w, r.z0);
  t[1] = __fmul2_rn(w, r.z1);
  t[2] = __fmul2_rn(t[0], r.z0);
  t[3] = __fmul2_rn(t[0], r.z1);
  t[4] = __fmul2_rn(t[1], r.z1);
}

// The values of a lane: its two pixels' contributions added.
__device__ __forceinline__ void pair_post_sum(PairBwd& p, const PairPre& r, float v[9]) {
  float2 t[9];
  pair_post(p, r, t);
#pragma unroll
  for (int k = 0; k < 9; ++k) v[k] = t[k].x + t[k].y;
}

// GS_REDUCE_FRAGMENT: each pixel's fragment adds its own values to the
// splat's accumulators (the per-fragment atomics of the ablation).
__device__ __forceinline__ void pair_fragment_atomics(PairBwd& p, const PairPre& r, bool ha,
                                                      bool hb, uint32_t rank, float* g2d) {
  float2 t[9];
  pair_post(p, r, t);
  float va9[9], vb9[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    va9[k] = t[k].x;
    vb9[k] = t[k].y;
  }
  if (ha) red_add9(g2d + (size_t)rank * 12, va9);
  if (hb) red_add9(g2d + (size_t)rank * 12, vb9);
}

// One candidate at both pixels, to the reduction of the mode.
template <int MODE>
__device__ __forceinline__ void pair_one(PairBwd& p, bool ha, bool hb, float2 q, float y1,
                                         float2 y2, const float4& a, const float4& b,
                                         const float4& c, uint32_t rank, GradBatch& B, int& nb,
                                         float* g2d, int threshold, int lane) {
  PairPre r;
  pair_pre(p, ha, hb, q, y1, y2, a, b, c, r);
  if (MODE == GS_REDUCE_FRAGMENT) {
    pair_fragment_atomics(p, r, ha, hb, rank, g2d);
  } else {
    float v[9];
    pair_post_sum(p, r, v);
    reduce_candidate<MODE>(v, ha || hb, rank, B, nb, g2d, threshold, lane);
  }
}

// The 8x8 quadrant (two pixels per lane) with the pixel pair packed.
template <int MODE>
__device__ __forceinline__ void bwd_item_pair(BwdRing& R, GradBatch& B,
                                              const SplatRec* __restrict__ rec,
                                              const uint32_t* __restrict__ pair_ranks,
                                              uint2 range, int x0, int y0, int lane, int W,
                                              int H, int fmt, const void* state,
                                              const uint32_t* last_in, const float* dLdC,
                                              float* g2d, int threshold, const BwdExtra& ex,
                                              float4* chunk_state, int chunk_out) {
  int x, ya;
  bool own;
  lane_pixels<16>(x0, y0, lane, x, ya, own);
  const int yb = ya + 4;
  const float px = (float)x + 0.5f;
  const float2 py = make_float2((float)ya + 0.5f, (float)yb + 0.5f);
  const float xs = (float)x0 + 0.5f, ys = (float)y0 + 0.5f;
  const bool va = x < W && ya < H, vb = x < W && yb < H;
  PairBwd pp;
  {
    PixelBwd pa, pb;
    load_pixel_bwd(pa, va, x, ya, W, fmt, state, last_in, dLdC, ex);
    load_pixel_bwd(pb, vb, x, yb, W, fmt, state, last_in, dLdC, ex);
    pp = pack_pair(pa, pb);
  }
  // depth ranks >= this contribute nowhere in the footprint
  const uint32_t warp_end = __reduce_max_sync(kFull, max(pp.end_a, pp.end_b));

  const uint32_t beg = range.x, end = warp_end > 0u ? range.y : range.x;
  if (beg < end) ring_start(R, rec, pair_ranks, beg, end, lane);
  int slot = 0, nb = 0;
  for (uint32_t gs = beg; gs < end; gs += 32u, slot = (slot + 1) & (kBwdStages - 1)) {
    const uint32_t ip = gs + 32u * kBwdStages + lane;
    const uint32_t rk_next = ip < end ? __ldg(pair_ranks + ip) : 0u;
    cp_async_wait_group<kBwdStages - 1>();
    __syncwarp();
    if (R.rank[slot][0] >= warp_end) break;   // ranks ascend along the list
    const uint32_t cnt = min(32u, end - gs);
    uint32_t m = __ballot_sync(kFull, (uint32_t)lane < cnt &&
                                          rect_may_hit(R.a[slot][lane], R.b[slot][lane], xs, ys,
                                                       7.f, 7.f));
    // Two candidates per step, as in bwd_item.
    while (m) {
      const int j0 = __ffs(m) - 1;
      m &= m - 1u;
      const bool two = m != 0u;
      const int j1 = two ? __ffs(m) - 1 : j0;
      m &= m - 1u;
      const uint32_t rank0 = R.rank[slot][j0], rank1 = R.rank[slot][j1];
      const float4 a0 = R.a[slot][j0], b0 = R.b[slot][j0];
      const float4 a1 = R.a[slot][j1], b1 = R.b[slot][j1];
      float y10, y11;
      float2 y20, y21;
      const float2 q0 = frag_q_pair(px, py, a0, b0, y10, y20);
      const float2 q1 = frag_q_pair(px, py, a1, b1, y11, y21);
      const bool ha0 = rank0 < pp.end_a && q0.x <= b0.y;
      const bool hb0 = rank0 < pp.end_b && q0.y <= b0.y;
      const bool ha1 = two && rank1 < pp.end_a && q1.x <= b1.y;
      const bool hb1 = two && rank1 < pp.end_b && q1.y <= b1.y;
      const float4 c0 = R.c[slot][j0], c1 = R.c[slot][j1];
      const bool u0 = __any_sync(kFull, ha0 || hb0), u1 = __any_sync(kFull, ha1 || hb1);
      if (u0 && u1) {
        PairPre r0, r1;
        pair_pre(pp, ha0, hb0, q0, y10, y20, a0, b0, c0, r0);
        pair_pre(pp, ha1, hb1, q1, y11, y21, a1, b1, c1, r1);
        if (MODE == GS_REDUCE_FRAGMENT) {
          pair_fragment_atomics(pp, r0, ha0, hb0, rank0, g2d);
          pair_fragment_atomics(pp, r1, ha1, hb1, rank1, g2d);
        } else {
          float v0[9], v1[9];
          pair_post_sum(pp, r0, v0);
          pair_post_sum(pp, r1, v1);
          reduce_candidate<MODE>(v0, ha0 || hb0, rank0, B, nb, g2d, threshold, lane);
          reduce_candidate<MODE>(v1, ha1 || hb1, rank1, B, nb, g2d, threshold, lane);
        }
      } else if (u0) {
        pair_one<MODE>(pp, ha0, hb0, q0, y10, y20, a0, b0, c0, rank0, B, nb, g2d, threshold, lane);
      } else if (u1) {
        pair_one<MODE>(pp, ha1, hb1, q1, y11, y21, a1, b1, c1, rank1, B, nb, g2d, threshold, lane);
      }
    }
    __syncwarp();   // every lane is done with the slot before it is refilled
    ring_issue(R, slot, rec, ip, end, rk_next, lane);
  }
  cp_async_wait_all();
  if (nb > 0) batch_flush(B, nb, lane, g2d);
  __syncwarp();
  if (chunk_out) {
    if (va) chunk_state[(size_t)ya * W + x] = make_float4(-pp.nD.x, pp.T.x, 0.f, 0.f);
    if (vb) chunk_state[(size_t)yb * W + x] = make_float4(-pp.nD.y, pp.T.y, 0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Backward, back to front (opts backward_order = GS_BWD_BACK_TO_FRONT)
//
// Each pixel starts at its last fragment with T = the stored final
// transmittance and walks towards the front: T_i = T_{i+1} / (1 - alpha_i)
// recovers the transmittance in front of fragment i, and S, the colour of the
// fragments behind it, gives Eq. 4 directly:
//   dL/dalpha_i = g . (c_i T_i - S_i / (1 - alpha_i)),  S_{i-1} = S_i + T_i alpha_i c_i.
// The fragment set is the forward's (every hit at or before the last rank).
// ---------------------------------------------------------------------------
struct PixelBack {
  float S0, S1, S2, T, g0, g1, g2;
  uint32_t end;
};

// A depth slab (see BwdExtra) starts S at the colour behind the slab's last
// fragment, T_slab behind, and scales g by t_front.
__device__ __forceinline__ void load_pixel_back(PixelBack& p, bool valid, int x, int y, int W,
                                                int fmt, const void* state,
                                                const uint32_t* last_in, const float* dLdC,
                                                const BwdExtra& ex) {
  p.S0 = p.S1 = p.S2 = 0.f;
  p.g0 = p.g1 = p.g2 = 0.f;
  p.T = 1.f;
  p.end = 0;
  if (valid) {
    const size_t pix = (size_t)y * W + x;
    p.T = load_state(state, fmt, pix).w;
    p.g0 = dLdC[3 * pix]; p.g1 = dLdC[3 * pix + 1]; p.g2 = dLdC[3 * pix + 2];
    if (ex.t_front) {
      const float tf = ex.t_front[pix];
      p.g0 *= tf; p.g1 *= tf; p.g2 *= tf;
    }
    if (ex.behind) {
      p.S0 = p.T * ex.behind[3 * pix];
      p.S1 = p.T * ex.behind[3 * pix + 1];
      p.S2 = p.T * ex.behind[3 * pix + 2];
    }
    const uint32_t l = last_in[pix];
    p.end = (l == kNone) ? 0u : l + 1u;
  }
}

__device__ __forceinline__ void grad_fragment_back(PixelBack& p, float q, float y1, float y2,
                                                   const float4& a, const float4& b,
                                                   const float4& c, float v[9]) {
  float G, at;
  const float alpha = frag_alpha(c.w, q, G, at);
  const float oma = __fsub_rn(1.0f, alpha);
  const float Ti = __fdiv_rn(p.T, oma);
  const float wT = __fmul_rn(alpha, Ti);
  v[5] += p.g0 * wT;
  v[6] += p.g1 * wT;
  v[7] += p.g2 * wT;
  const float inv = __fdividef(1.0f, oma);
  const float dLda = p.g0 * (c.x * Ti - p.S0 * inv) + p.g1 * (c.y * Ti - p.S1 * inv) +
                     p.g2 * (c.z * Ti - p.S2 * inv);
  p.S0 += wT * c.x;
  p.S1 += wT * c.y;
  p.S2 += wT * c.z;
  p.T = Ti;
  const float d_at = at < kAlphaMax ? dLda : 0.f;
  v[8] += G * d_at;
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

// First index in [lo, hi) whose depth rank is >= r (hi if none): a 32-way
// search, one coalesced probe per lane and step.
__device__ __forceinline__ uint32_t first_rank_at_least(const uint32_t* __restrict__ pair_ranks,
                                                        uint32_t lo, uint32_t hi, uint32_t r,
                                                        int lane) {
  while (hi - lo > 32u) {
    const uint32_t step = (hi - lo + 31u) / 32u;
    const uint32_t p = lo + (uint32_t)lane * step;
    const bool ge = p >= hi || __ldg(pair_ranks + p) >= r;
    const uint32_t b = __ballot_sync(kFull, ge);
    if (b == 0u) {
      lo = lo + 31u * step + 1u;
      continue;
    }
    const uint32_t f = (uint32_t)(__ffs(b) - 1);
    const uint32_t nhi = min(lo + f * step, hi);
    lo = f > 0u ? lo + (f - 1u) * step + 1u : lo;
    hi = nhi;
  }
  const uint32_t p = lo + (uint32_t)lane;
  const bool ge = p >= hi || __ldg(pair_ranks + p) >= r;
  const uint32_t b = __ballot_sync(kFull, ge);
  return b ? min(lo + (uint32_t)(__ffs(b) - 1), hi) : hi;
}

// Entries [glo, ghi) of group k when walking [beg, stop) backwards in 32s.
__device__ __forceinline__ void back_group(uint32_t k, uint32_t beg, uint32_t stop, uint32_t& glo,
                                           uint32_t& ghi) {
  const uint64_t off = 32ull * k;
  ghi = stop - beg > off ? stop - (uint32_t)off : beg;
  glo = ghi - beg > 32u ? ghi - 32u : beg;
}

template <int COLS, int MODE>
__device__ __forceinline__ void bwd_item_back(BwdRing& R, GradBatch& B,
                                              const SplatRec* __restrict__ rec,
                                              const uint32_t* __restrict__ pair_ranks,
                                              uint2 range, int x0, int y0, int lane, int W, int H,
                                              int fmt, const void* state,
                                              const uint32_t* last_in, const float* dLdC,
                                              float* g2d, int threshold, const BwdExtra& ex) {
  constexpr int NPX = COLS == 16 ? 2 : 1;
  int x, ya;
  bool own;
  lane_pixels<COLS>(x0, y0, lane, x, ya, own);
  const int yb = ya + 4;
  const float px = (float)x + 0.5f, pya = (float)ya + 0.5f, pyb = (float)yb + 0.5f;
  const float xs = (float)x0 + 0.5f, ys = (float)y0 + 0.5f;
  PixelBack pa, pb;
  load_pixel_back(pa, own && x < W && ya < H, x, ya, W, fmt, state, last_in, dLdC, ex);
  if (NPX == 2) {
    load_pixel_back(pb, x < W && yb < H, x, yb, W, fmt, state, last_in, dLdC, ex);
  } else {
    pb.S0 = pb.S1 = pb.S2 = 0.f;
    pb.g0 = pb.g1 = pb.g2 = 0.f;
    pb.T = 1.f;
    pb.end = 0u;
  }
  const uint32_t warp_end = __reduce_max_sync(kFull, max(pa.end, pb.end));
  if (warp_end == 0u) return;
  const uint32_t beg = range.x;
  const uint32_t stop = first_rank_at_least(pair_ranks, range.x, range.y, warp_end, lane);
  // prologue: the last kBwdStages groups before `stop`
#pragma unroll
  for (int s = 0; s < kBwdStages; ++s) {
    uint32_t glo, ghi;
    back_group((uint32_t)s, beg, stop, glo, ghi);
    const uint32_t i = glo + (uint32_t)lane;
    const uint32_t rk = i < ghi ? __ldg(pair_ranks + i) : 0u;
    ring_issue(R, s, rec, i, ghi, rk, lane);
  }
  int slot = 0, nb = 0;
  for (uint32_t k = 0;; ++k, slot = (slot + 1) & (kBwdStages - 1)) {
    uint32_t glo, ghi;
    back_group(k, beg, stop, glo, ghi);
    if (glo >= ghi) break;
    uint32_t nlo, nhi;
    back_group(k + kBwdStages, beg, stop, nlo, nhi);
    const uint32_t ip = nlo + (uint32_t)lane;
    const uint32_t rk_next = ip < nhi ? __ldg(pair_ranks + ip) : 0u;
    cp_async_wait_group<kBwdStages - 1>();
    __syncwarp();
    const uint32_t cnt = ghi - glo;
    uint32_t m = __ballot_sync(kFull, (uint32_t)lane < cnt &&
                                          rect_may_hit(R.a[slot][lane], R.b[slot][lane], xs, ys,
                                                       COLS == 16 ? 7.f : (float)(COLS - 1), COLS == 16 ? 7.f : 3.f));
    while (m) {
      const int j = 31 - __clz(m);   // deepest first
      m &= ~(1u << j);
      const uint32_t rank = R.rank[slot][j];
      float v[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = 0.f;
      const float4 a = R.a[slot][j];
      const float4 b = R.b[slot][j];
      float y1a, y2a, y1b = 0.f, y2b = 0.f, qb = 0.f;
      const float qa = frag_q(px, pya, a, b, y1a, y2a);
      if (NPX == 2) qb = frag_q(px, pyb, a, b, y1b, y2b);
      const bool ha = rank < pa.end && qa <= b.y;
      const bool hb = NPX == 2 && rank < pb.end && qb <= b.y;
      if (ha || hb) {
        const float4 c = R.c[slot][j];
        if (ha) grad_fragment_back(pa, qa, y1a, y2a, a, b, c, v);
        if (NPX == 2 && hb) grad_fragment_back(pb, qb, y1b, y2b, a, b, c, v);
      }
      reduce_candidate<MODE>(v, ha || hb, rank, B, nb, g2d, threshold, lane);
    }
    __syncwarp();
    ring_issue(R, slot, rec, ip, nhi, rk_next, lane);
  }
  cp_async_wait_all();
  if (nb > 0) batch_flush(B, nb, lane, g2d);
  __syncwarp();
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) raster_bwd_kernel(
    const uint2* __restrict__ ranges, const uint32_t* __restrict__ items,
    const Header* __restrict__ hdr, uint32_t* __restrict__ next,
    const uint32_t* __restrict__ pair_ranks, const SplatRec* __restrict__ rec, int W, int H, int gw,
    float t_cull, int fmt, const void* __restrict__ state, const uint32_t* __restrict__ last_in,
    const float* __restrict__ dLdC, float* __restrict__ g2d, int threshold, int back,
    float4* __restrict__ chunk_state, int chunk_in, int chunk_out,
    const float* __restrict__ t_front, const float* __restrict__ behind) {
  __shared__ BwdRing rings[kWarps];
  const BwdExtra ex{chunk_state, chunk_in, t_front, behind};
  __shared__ GradBatch batches[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  BwdRing& R = rings[warp];
  GradBatch& B = batches[warp];
  const uint32_t n_items = hdr->n_items;
  for (uint32_t idx = next_item(next, lane); idx < n_items; idx = next_item(next, lane)) {
    int block, x0, y0;
    const int cols = item_origin(items[idx], gw, block, x0, y0);
    const uint2 range = ranges[block];
    if (back) {
      if (cols == 16)
        bwd_item_back<16, MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                                last_in, dLdC, g2d, threshold, ex);
      else if (cols == 8)
        bwd_item_back<8, MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                               last_in, dLdC, g2d, threshold, ex);
      else
        bwd_item_back<4, MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                               last_in, dLdC, g2d, threshold, ex);
      continue;
    }
    if (cols == 16)
      bwd_item_pair<MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                          last_in, dLdC, g2d, threshold, ex, chunk_state, chunk_out);
    else if (cols == 8)
      bwd_item<8, MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                        last_in, dLdC, g2d, threshold, ex, chunk_state, chunk_out);
    else
      bwd_item<4, MODE>(R, B, rec, pair_ranks, range, x0, y0, lane, W, H, fmt, state,
                        last_in, dLdC, g2d, threshold, ex, chunk_state, chunk_out);
  }
}

// The forward's items reordered costliest first: a counting sort by
// log-bucket of the measured cost (4 buckets per octave).  Any cost values
// give a permutation of the items, so stale costs only cost time.
constexpr int kCostBuckets = 128;

__device__ __forceinline__ int cost_bucket(uint32_t c) {
  if (c == 0) return kCostBuckets - 1;
  const int lg = 31 - __clz(c);
  const int frac = lg >= 2 ? (int)((c >> (lg - 2)) & 3) : 0;
  return kCostBuckets - 2 - min(lg * 4 + frac, kCostBuckets - 2);
}

constexpr int kOrderThreads = 1024;
constexpr int kOrderWarps = kOrderThreads / 32;

__global__ void __launch_bounds__(kOrderThreads) item_order_kernel(
    const uint32_t* __restrict__ items, const uint32_t* __restrict__ cost,
    const Header* __restrict__ hdr, uint32_t* __restrict__ out) {
  // per-warp bucket counts, then per-warp placement cursors
  __shared__ uint32_t s_cnt[kOrderWarps][kCostBuckets];
  __shared__ uint32_t s_part[kCostBuckets / 32];
  const uint32_t n = hdr->n_items;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kOrderWarps * kCostBuckets; i += kOrderThreads)
    (&s_cnt[0][0])[i] = 0u;
  __syncthreads();
#pragma unroll 4
  for (uint32_t i = threadIdx.x; i < n; i += kOrderThreads)
    atomicAdd(&s_cnt[warp][cost_bucket(cost[i])], 1u);
  __syncthreads();
  // exclusive scan in (bucket, warp) order; thread b < kCostBuckets owns bucket b
  uint32_t tot = 0;
  if (threadIdx.x < kCostBuckets) {
    for (int w = 0; w < kOrderWarps; ++w) tot += s_cnt[w][threadIdx.x];
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (threadIdx.x < kCostBuckets && lane == 31) s_part[warp] = incl;
  __syncthreads();
  if (threadIdx.x < kCostBuckets) {
    uint32_t run = incl - tot;
    for (int w = 0; w < warp; ++w) run += s_part[w];
    for (int w = 0; w < kOrderWarps; ++w) {
      const uint32_t c = s_cnt[w][threadIdx.x];
      s_cnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll 4
  for (uint32_t i = threadIdx.x; i < n; i += kOrderThreads)
    out[atomicAdd(&s_cnt[warp][cost_bucket(cost[i])], 1u)] = items[i];
}

namespace {
// Resident CTAs per SM of `kernel` at kThreads.
template <typename K>
int resident_per_sm(K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return per_sm;
}
}  // namespace

constexpr int kFwdMaxCtasPerSm = 5;

cudaError_t launch_raster_fwd(const uint2* ranges, const uint32_t* items, const Header* hdr,
                              uint32_t* next, uint32_t* item_cost, const uint32_t* pair_ranks,
                              const SplatRec* rec,
                              int W, int H, int gw, int gh, float t_cull, int fmt, float* image,
                              void* state, uint32_t* last, uint32_t* ncontrib, int resume,
                              uint32_t* block_done, uint32_t* done_px, uint32_t chunk,
                              int num_sms, cudaStream_t st) {
  if (gw * gh == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  // At most five CTAs (20 warps) per SM although eight fit: the launch ends when
  // the few items of the densest blocks (started first) end, and with fewer
  // warps sharing their schedulers those run faster.  On the 3M-splat scene at
  // 1256x828: 8 CTAs 0.297 ms, 6 0.282, 5 0.271, 4 0.271, 3 0.325.
  static const int per_sm = min(resident_per_sm(raster_fwd_kernel), kFwdMaxCtasPerSm);
  const int grid = per_sm * num_sms;
  raster_fwd_kernel<<<grid, kThreads, 0, st>>>(ranges, items, hdr, next, item_cost, pair_ranks, rec,
                                               W, H, gw, t_cull, fmt, image, state, last, ncontrib,
                                               resume, block_done, done_px, chunk);
  return cudaGetLastError();
}

// The backward's item order (costliest first) from the forward's item times.
cudaError_t launch_item_order(const uint32_t* fwd_items, const uint32_t* item_cost,
                              const Header* hdr, uint32_t* items, cudaStream_t st) {
  item_order_kernel<<<1, kOrderThreads, 0, st>>>(fwd_items, item_cost, hdr, items);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const uint2* ranges, const uint32_t* fwd_items,
                              const uint32_t* item_cost, uint32_t* items, const Header* hdr,
                              uint32_t* next, const uint32_t* pair_ranks, const SplatRec* rec,
                              int W, int H, int gw, int gh, float t_cull, int fmt,
                              const void* state, const uint32_t* last, const float* dLdC,
                              float* g2d, int mode, int threshold, int back, float4* chunk_state,
                              int chunk_in, int chunk_out, const float* t_front,
                              const float* behind, int num_sms, cudaStream_t st,
                              int order_done) {
  if (gw * gh == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  if (!order_done) {   // else launch_item_order ran already (on another stream)
    item_order_kernel<<<1, kOrderThreads, 0, st>>>(fwd_items, item_cost, hdr, items);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (mode == GS_REDUCE_NAIVE) {
    static const int per_sm = resident_per_sm(raster_bwd_kernel<GS_REDUCE_NAIVE>);
    const int grid = per_sm * num_sms;
    raster_bwd_kernel<GS_REDUCE_NAIVE><<<grid, kThreads, 0, st>>>(
        ranges, items, hdr, next, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d,
        threshold, back, chunk_state, chunk_in, chunk_out, t_front, behind);
  } else if (mode == GS_REDUCE_FRAGMENT) {
    static const int per_sm = resident_per_sm(raster_bwd_kernel<GS_REDUCE_FRAGMENT>);
    const int grid = per_sm * num_sms;
    raster_bwd_kernel<GS_REDUCE_FRAGMENT><<<grid, kThreads, 0, st>>>(
        ranges, items, hdr, next, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d,
        threshold, back, chunk_state, chunk_in, chunk_out, t_front, behind);
  } else {
    static const int per_sm = resident_per_sm(raster_bwd_kernel<GS_REDUCE_WARP>);
    const int grid = per_sm * num_sms;
    raster_bwd_kernel<GS_REDUCE_WARP><<<grid, kThreads, 0, st>>>(
        ranges, items, hdr, next, pair_ranks, rec, W, H, gw, t_cull, fmt, state, last, dLdC, g2d,
        threshold, back, chunk_state, chunk_in, chunk_out, t_front, behind);
  }
  return cudaGetLastError();
}

}  // namespace gsr

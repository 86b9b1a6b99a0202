// Quad coverage -> (16x16 block, depth rank) pairs, in depth order.
//
// The paper rasterizes each depth-sorted splat as a screen quad bounding its
// alpha >= 1/255 ellipse (Sec. 1, Sec. 2.2) into fixed O(N) buffers.  Here the
// quad's pixel-centre box is turned into the list of 16x16 pixel blocks it
// touches.  Two passes:
//   count: per tile of 1024 depth ranks, gathers each splat's record into
//      depth order (the raster reads records by rank), zeroes its backward
//      accumulators, counts its blocks and scans the counts across tiles with a
//      decoupled look-back (tagged 64-bit status words, bounded waits), giving
//      every rank its first pair index;
//   emit: each CTA writes whole runs of 2048 consecutive pairs (binary searches
//      over the ranks' first pair indices find the run's splats, then each
//      pair's), so the work is even even though the nearest splats are the
//      largest on screen; it also accumulates the 8-bit digit histograms of the
//      block ids that the stable pair sort by block needs (depth order survives
//      within a block).
// The pairs a view needs may exceed the workspace's capacity.  Normally the
// shortfall is recorded and the view fails with GS_ERR_CAPACITY.  In the
// memory-efficiency mode the depth ranks are cut into chunks whose pairs fit
// (chunk k holds the splats whose first pair index lies in [k B, (k + 1) B),
// B = capacity - blocks, so no chunk exceeds the capacity) and each chunk is
// emitted, sorted and rasterized in turn, front to back; a block whose pixels
// are all T-culled after chunk j gets no pairs in the chunks after j (they
// would hold no fragment), which in dense views drops most of the pairs.
#include "common.cuh"

namespace gsr {

constexpr int kBinThreads = 256;
constexpr int kBinItems = 4;
constexpr int kBinTile = kBinThreads * kBinItems;  // 1024 ranks
constexpr unsigned long long kBinAgg = 1ull << 30;
constexpr unsigned long long kBinPre = 2ull << 30;
constexpr unsigned long long kBinCount = (1ull << 30) - 1;
constexpr int kEmitPer = 8;                   // steps of 32 pairs in one warp task
constexpr int kEmitTask = 32 * kEmitPer;       // pairs of one warp task of the emission (256)
constexpr int kChunkWhole = 0, kChunkBudget = 1, kChunkSlab = 2;   // chunk_setup_kernel modes
static_assert(kChunkWhole == 0 && kChunkBudget == 1,
              "the whole-view and budget modes are the workspace's chunked flag (0 or 1)");

// Pass 1: one tile of 1024 depth ranks per step of a persistent loop.
__global__ void __launch_bounds__(kBinThreads) bin_count_kernel(
    const uint32_t* __restrict__ sorted_ids, const SplatRec* __restrict__ rec,
    const uint2* __restrict__ boxes_by_id, SplatRec* __restrict__ rec_sorted,
    float4* __restrict__ g2d, Header* __restrict__ hdr,
    unsigned long long* __restrict__ scan_status, const uint32_t* __restrict__ epoch,
    uint32_t* __restrict__ offsets, uint2* __restrict__ boxes, uint32_t pair_cap, int chunked,
    uint32_t* __restrict__ run_first, uint32_t run_cap) {
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_cnt[kBinTile];
  __shared__ uint32_t s_warp[kBinThreads / 32];
  __shared__ unsigned long long s_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t V = hdr->visible;
  const uint32_t ntiles = (V + kBinTile - 1) / kBinTile;
  const uint32_t tag = *epoch;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&hdr->tile_counter[8], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) break;
    const uint32_t base = tile * kBinTile;
    // ids and boxes first: the tile's pair count needs only the boxes, so it is
    // published before the records move, and later tiles find it sooner
    uint32_t idv[kBinItems];
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
      const uint32_t r = base + k * kBinThreads + tid;
      idv[k] = r < V ? sorted_ids[r] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
      const int j = k * kBinThreads + tid;
      const uint32_t r = base + j;
      uint32_t cnt = 0;
      if (r < V) {
        const uint2 box = boxes_by_id[idv[k]];   // every visible splat covers >= 1 block
        boxes[r] = box;
        cnt = (box.y & 0xFFFFu) * (box.y >> 16);
      }
      s_cnt[j] = cnt;
    }
    __syncthreads();
    // exclusive scan of the 1024 counts in rank order: 4 contiguous per thread
    uint32_t c4[kBinItems], sum = 0;
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
      c4[k] = s_cnt[tid * kBinItems + k];
      sum += c4[k];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t wbefore = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kBinThreads / 32; ++w) {
      const uint32_t v = s_warp[w];
      if (w < warp) wbefore += v;
      total += v;
    }
    unsigned long long* my = scan_status + tile;
    const unsigned long long tot = min((unsigned long long)total, kBinCount);
    if (tid == 0)
      st_relaxed64(my, ((unsigned long long)tag << 32) | (tile == 0 ? kBinPre : kBinAgg) | tot);
    // gather the records into depth order and zero the backward accumulators
    // while lower tiles publish
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
      const uint32_t r = base + k * kBinThreads + tid;
      // the warp's 32 consecutive ranks move their 48-byte records together:
      // consecutive lanes take consecutive 16-byte words of the 32 records
      const uint32_t r0 = r - (uint32_t)lane;
      const float4* src = reinterpret_cast<const float4*>(rec);
      float4* dst = reinterpret_cast<float4*>(rec_sorted);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const int w = t * 32 + lane, q = w / 3, part = w % 3;
        const uint32_t idq = __shfl_sync(0xffffffffu, idv[k], q);
        if (r0 + q < V) dst[(size_t)(r0 + q) * 3 + part] = src[(size_t)idq * 3 + part];
      }
      if (r < V) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        g2d[3 * (size_t)r] = z;
        g2d[3 * (size_t)r + 1] = z;
        g2d[3 * (size_t)r + 2] = z;
      }
    }
    // tile offset by decoupled look-back over lower tiles, 32 of them per round
    // trip (lane l reads tile j - l)
    if (warp == 0) {
      unsigned long long excl = 0;
      if (tile > 0) {
        int64_t j = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (j >= 0) {
          const int64_t t = j - lane;
          const unsigned long long s = t >= 0 ? ld_relaxed64(scan_status + t) : 0ull;
          const bool ready = t >= 0 && (uint32_t)(s >> 32) == tag && (s & (3ull << 30)) != 0;
          const uint32_t waiting = __ballot_sync(0xffffffffu, t >= 0 && !ready);
          const uint32_t prefix = __ballot_sync(0xffffffffu, ready && (s & (3ull << 30)) == kBinPre);
          const int first_wait = waiting ? __ffs(waiting) - 1 : 32;
          const int first_pre = prefix ? __ffs(prefix) - 1 : 32;
          // lanes before the first unpublished word are consumed; a prefix ends the walk
          const int take = first_pre < first_wait ? first_pre + 1 : first_wait;
          unsigned long long c = (lane < take && t >= 0) ? (s & kBinCount) : 0ull;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
          excl += c;
          if (first_pre < first_wait) break;
          if (take == 0) {
            if (++spins > kSpinLimit) {
              if (lane == 0) atomicOr(&hdr->status, kStatusTimeout);
              break;
            }
            continue;
          }
          j -= take;
        }
        if (lane == 0)
          st_relaxed64(my, ((unsigned long long)tag << 32) | kBinPre | min(excl + tot, kBinCount));
      }
      if (lane == 0) s_off = excl;
    }
    if (tid == 0) {
      const unsigned long long excl = s_off;
      if (base + kBinTile >= V) {  // last tile: total pair count
        const unsigned long long want = excl + total;
        hdr->pairs_wanted = (uint32_t)min(want, (unsigned long long)0xFFFFFFFFu);
        hdr->pairs = (uint32_t)min(want, (unsigned long long)pair_cap);
        if (want > pair_cap && !chunked) atomicOr(&hdr->status, kStatusCapacity);
      }
    }
    __syncthreads();
    // global exclusive offsets (saturated at 2^32 - 1)
    unsigned long long run = s_off + wbefore + x - sum;
#pragma unroll
    for (int k = 0; k < kBinItems; ++k) {
      const uint32_t r = base + tid * kBinItems + k;
      if (r < V) {
        offsets[r] = (uint32_t)min(run, (unsigned long long)0xFFFFFFFFu);
        // run table: this rank holds pair m kEmitTask for each such m in its range
        for (unsigned long long m = (run + kEmitTask - 1) / kEmitTask;
             m * kEmitTask < run + c4[k] && m < run_cap; ++m)
          run_first[m] = r;
      }
      run += c4[k];
    }
    __syncthreads();
  }
}

// Last rank r in [0, V) with offsets[r] <= p (offsets ascend; offsets[0] = 0),
// found by the whole warp: each round the 32 lanes probe 32 evenly spaced
// ranks of the interval, and the ballot of "offsets <= p" (a prefix of the
// lanes) narrows it 32-fold, so a search over V ranks takes log32 V dependent
// loads instead of log2 V.  Every lane returns the answer.
__device__ __forceinline__ uint32_t warp_rank_of_pair(const uint32_t* __restrict__ offsets,
                                                      uint32_t V, uint32_t p, int lane) {
  uint32_t lo = 0, hi = V;   // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t idx = lo + (uint32_t)(lane + 1) * step;
    const bool le = idx < hi && offsets[idx] <= p;
    const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xffffffffu, le));
    hi = min(hi, lo + (cnt + 1) * step);
    lo += cnt * step;
  }
  return lo;
}

// Chunk k of the view: pair indices [pair_base, pair_base + pairs) and the
// per-chunk state the emission and the pair sort start from.  mode
// kChunkWhole: one chunk, the first `capacity` pairs; kChunkBudget (the
// memory-efficiency mode): the splats whose first pair index lies in
// [k B, (k + 1) B); kChunkSlab: depth slab k of B, the ranks
// [k V / B, (k + 1) V / B) (a slab whose pairs exceed the capacity records
// kStatusCapacity and keeps the first `capacity`).  It also advances the
// epoch: the pair sort's look-back words of any earlier chunk or binning then
// carry a stale tag and are never taken for this one's.
__global__ void __launch_bounds__(256) chunk_setup_kernel(const uint32_t* __restrict__ offsets,
                                                          Header* __restrict__ hdr,
                                                          uint32_t* __restrict__ epoch, uint32_t k,
                                                          uint32_t B, uint32_t pair_cap,
                                                          int mode, uint2* __restrict__ ranges,
                                                          int nblocks, uint32_t* __restrict__ block_done,
                                                          uint32_t* __restrict__ done_px,
                                                          int reset_done) {
  const uint32_t V = hdr->visible, total = hdr->pairs_wanted;
  if (threadIdx.x == 0) {
    uint32_t lo = 0, hi = min(total, pair_cap);
    if (mode == kChunkSlab) {
      const uint32_t r0 = (uint32_t)((unsigned long long)k * V / B);
      const uint32_t r1 = (uint32_t)((unsigned long long)(k + 1) * V / B);
      lo = r0 < V ? offsets[r0] : total;
      hi = r1 < V ? offsets[r1] : total;
      if (hi - lo > pair_cap) {
        atomicOr(&hdr->status, kStatusCapacity);
        hi = lo + pair_cap;
      }
    } else if (mode == kChunkBudget) {
      // first rank whose first pair index is >= t
      auto first_at = [&](unsigned long long t) -> uint32_t {
        if (t >= total) return total;
        uint32_t a = 0, b = V;   // answer in [a, b]
        while (a < b) {
          const uint32_t mid = a + (b - a) / 2;
          if (offsets[mid] >= t) b = mid; else a = mid + 1;
        }
        return a < V ? offsets[a] : total;
      };
      lo = first_at((unsigned long long)k * B);
      hi = first_at((unsigned long long)(k + 1) * B);
    }
    *epoch += 1u;
    hdr->pair_base = lo;
    hdr->pairs = hi - lo;
    hdr->live_pairs = 0;
    for (int q = 4; q < 8; ++q) hdr->tile_counter[q] = 0;
  }
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&hdr->pair_hist[0][0])[i] = 0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) ranges[i] = make_uint2(0, 0);
  if (done_px)
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) done_px[i] = 0u;
  if (block_done && reset_done)
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) block_done[i] = kNone;
}

// The ellipse q <= lim of one splat against rows of 16x16 blocks.  With (X, Y)
// the offset of a pixel centre from the splat's centre, q = (i11 X)^2 +
// (i22 (Y - k X))^2; at a fixed Y, q <= lim holds for |X - s Y| <=
// sqrt(alpha lim - (i11 i22 Y)^2) / alpha, alpha = i11^2 + (k i22)^2, s =
// k i22^2 / alpha.  The boundary's largest X, sqrt(lim) / i11, lies at Y = k
// times it and its smallest at the mirror point; X along the boundary is
// concave in Y, so over a band of rows the extremes are taken at those two Y
// clamped into the band.  A block of the row is reached iff its columns meet
// [X_min, X_max]: the same set as the minimum of q over the block's rectangle
// against lim (rect_may_hit), evaluated once per row instead of once per block.
// lim carries rect_may_hit's margin and the range is widened by a further
// 0.1% + 0.01 px, so rounding never drops a block with a fragment; non-finite
// values keep every column.
struct RowTest {
  float ax, bz, ay, bw;                 // centre, float-float
  float slope, ia, alim, d2, ys, ye;

  __device__ __forceinline__ void init(const float4& a, const float4& b) {
    ax = a.x;
    bz = b.z;
    ay = a.y;
    bw = b.w;
    const float i11 = a.z, k = a.w, i22 = b.x;
    const float lim = b.y + 0.01f + 1e-3f * b.y;
    const float ki = k * i22;
    const float alpha = fmaf(i11, i11, ki * ki);
    ia = __fdividef(1.0f, alpha);
    slope = ki * i22 * ia;
    alim = alpha * lim;
    const float d = i11 * i22;
    d2 = d * d;
    ys = k * __fdividef(sqrtf(lim), i11);
    ye = fmaf(__fdividef(sqrtf(alim), d), 1.001f, 0.01f);   // |Y| extent, widened
  }
  // Columns [c_lo, c_hi] of block row `by` that the ellipse may reach (empty
  // when c_lo > c_hi).
  __device__ __forceinline__ void row(int by, int& c_lo, int& c_hi) const {
    const float Y0 = ((float)(by * kBlock) + 0.5f - ay) - bw;
    const float Y1 = Y0 + (float)(kBlock - 1);
    if (Y0 > ye || Y1 < -ye) {
      c_lo = 1;
      c_hi = 0;
      return;
    }
    const float yh = fminf(fmaxf(ys, Y0), Y1), yl = fminf(fmaxf(-ys, Y0), Y1);
    const float xh = fmaf(slope, yh, sqrtf(fmaxf(0.0f, alim - d2 * yh * yh)) * ia);
    const float xl = fmaf(slope, yl, -sqrtf(fmaxf(0.0f, alim - d2 * yl * yl)) * ia);
    const float m = fmaf(1e-3f, xh - xl, 0.01f);
    // column c spans X in [X0, X0 + 15], X0 = (16 c + 0.5 - a.x) - b.z
    const float cx = ax + bz;
    const float lo = (xl - m + cx - 15.5f) * (1.0f / kBlock);
    const float hi = (xh + m + cx - 0.5f) * (1.0f / kBlock);
    c_lo = (int)ceilf(fmaxf(lo, -1.0f));     // NaN -> -1, every column kept
    c_hi = (int)floorf(fminf(hi, 65536.0f));
  }
};

// Pass 2: every warp takes tasks of kEmitTask consecutive pairs of the chunk
// (so the work is even however the pairs are spread over splats) and works on
// its own: it stages the offsets and boxes of the ranks its pairs belong to in
// its own shared memory, with no barrier shared with the other warps.
__global__ void __launch_bounds__(kBinThreads, 4) bin_emit_kernel(
    const uint32_t* __restrict__ offsets, const uint2* __restrict__ boxes,
    const SplatRec* __restrict__ rec_sorted, Header* __restrict__ hdr,
    uint32_t* __restrict__ pair_keys, uint32_t* __restrict__ pair_vals, int gw, int gh,
    int pair_passes, const uint32_t* __restrict__ block_done, uint32_t chunk,
    const uint32_t* __restrict__ run_first, uint32_t run_cap) {
  constexpr int kWarps = kBinThreads / 32;
  __shared__ uint32_t s_offw[kWarps][kEmitTask + 1];
  __shared__ uint2 s_boxw[kWarps][kEmitTask + 1];
  __shared__ uint32_t s_hist[4][256];
  __shared__ uint32_t s_unit[kWarps][kEmitTask];   // per warp: (rank << 21) | block row
  __shared__ uint32_t s_iv[kWarps][kEmitTask];     // its columns: lo | (hi + 1) << 16
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 4 * 256; i += kBinThreads) (&s_hist[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t P = hdr->pairs, V = hdr->visible, pbase = hdr->pair_base;
  const uint32_t ntasks = (P + kEmitTask - 1) / kEmitTask;
  // run-table entries written by the binning's first pass
  const uint32_t nb = (uint32_t)min((unsigned long long)run_cap,
                                    ((unsigned long long)hdr->pairs_wanted + kEmitTask - 1) / kEmitTask);
  uint32_t* s_off = s_offw[warp];
  uint2* s_box = s_boxw[warp];
  uint32_t live = 0;
  for (uint32_t task = blockIdx.x * kWarps + warp; task < ntasks; task += gridDim.x * kWarps) {
    const uint32_t p0 = pbase + task * kEmitTask;         // global pair indices [p0, p1)
    const uint32_t p1 = pbase + min(P, (task + 1) * kEmitTask);
    // the ranks of the task's first and last pairs: from the run table where it
    // has them (the rank of pair m kEmitTask; for the last pair, the rank
    // holding the next table pair, an upper bound), else by a warp search
    const uint32_t m0 = p0 / kEmitTask, m1 = (p1 - 1) / kEmitTask + 1;
    const uint32_t r0 = (p0 % kEmitTask == 0 && m0 < nb) ? run_first[m0]
                                                          : warp_rank_of_pair(offsets, V, p0, lane);
    const uint32_t r1 = m1 < nb ? run_first[m1] : warp_rank_of_pair(offsets, V, p1 - 1, lane);
    // ranks overlapping [p0, p1): each has >= 1 pair, so at most kEmitTask of
    // them, and the upper bound adds at most one
    const uint32_t nr = min(r1 - r0 + 1, (uint32_t)kEmitTask + 1);
    __syncwarp();   // the previous task is done with the warp's arrays
    for (uint32_t i = lane; i < nr; i += 32) {
      s_off[i] = offsets[r0 + i];
      s_box[i] = boxes[r0 + i];
    }
    __syncwarp();
    // The task's pairs in kEmitPer steps of 32 consecutive pairs.  First every
    // pair finds its rank, row and column, and the first pair of each box row
    // in the task registers the row as a unit; then each lane tests one unit
    // against the splat's ellipse (RowTest), so a row costs one test however
    // many blocks it has; then every pair reads its unit's columns.
    const uint32_t wp0 = p0;
    {
      uint32_t unit_mask[kEmitPer], bxy[kEmitPer], lov[kEmitPer];
      uint32_t nunits = 0;
      int lo_base = 0;   // staged rank 0 (r0) holds the task's first pair
#pragma unroll
      for (int st = 0; st < kEmitPer; ++st) {
        const uint32_t q = wp0 + 32u * st;
        const uint32_t p = q + (uint32_t)lane;
        const bool valid = p < p1;
        // ranks starting inside this step: lane j looks at the j-th rank after
        // lo_base (the rank of the pair before the step, or of its first pair
        // in the first step); a rank starting at lane v counts for lanes >= v
        const int j = lo_base + 1 + lane;
        const uint32_t v = j < (int)nr ? s_off[j] - q : 32u;
        const uint32_t starts = __reduce_or_sync(0xffffffffu,
                                                 (v < 32u && (st > 0 || v > 0u)) ? 1u << v : 0u);
        const int lo = lo_base + __popc(starts & (lanemask_lt() | (1u << lane)));
        lo_base = __shfl_sync(0xffffffffu, lo, 31);
        const uint32_t pc = valid ? p : p1 - 1;
        const uint2 box = s_box[lo];
        const uint32_t w = max(box.y & 0xFFFFu, 1u), h = max(box.y >> 16, 1u);
        const uint32_t k = pc - s_off[lo];
        // k / w and k % w through a float quotient corrected by one step (k and
        // w below 2^22, so the estimate is off by at most one): no integer division
        uint32_t qd = (uint32_t)__fdividef((float)k, (float)w);
        int32_t rem = (int32_t)k - (int32_t)(qd * w);
        if (rem < 0) {
          --qd;
          rem += (int32_t)w;
        } else if (rem >= (int32_t)w) {
          ++qd;
          rem -= (int32_t)w;
        }
        const uint32_t row = min(qd, h - 1);   // stays inside the box
        const uint32_t bx = (box.x & 0xFFFFu) + (uint32_t)rem, by = (box.x >> 16) + row;
        bxy[st] = (by << 16) | bx;
        lov[st] = valid ? (uint32_t)lo : kNone;
        const bool lead = valid && (rem == 0 || (st == 0 && lane == 0));
        const uint32_t m = __ballot_sync(0xffffffffu, lead);
        unit_mask[st] = m;
        if (lead) s_unit[warp][nunits + __popc(m & lanemask_lt())] = ((uint32_t)lo << 21) | by;
        nunits += __popc(m);
      }
      __syncwarp();
      for (uint32_t u = (uint32_t)lane; u < nunits; u += 32) {
        const uint32_t dsc = s_unit[warp][u];
        const SplatRec& R = rec_sorted[r0 + (dsc >> 21)];
        RowTest rt;
        rt.init(R.a, R.b);
        int c_lo, c_hi;
        rt.row((int)(dsc & 0x1FFFFFu), c_lo, c_hi);
        c_lo = min(max(c_lo, 0), 65535);     // block columns are below 65536
        c_hi = min(max(c_hi, -1), 65534);
        s_iv[warp][u] = (uint32_t)c_lo | ((uint32_t)(c_hi + 1) << 16);
      }
      __syncwarp();
      uint32_t before = 0;
#pragma unroll
      for (int st = 0; st < kEmitPer; ++st) {
        if (lov[st] != kNone) {
          const uint32_t m = unit_mask[st];
          const uint32_t u = before + __popc(m & lanemask_lt()) + ((m >> lane) & 1u) - 1u;
          const uint32_t iv = s_iv[warp][u];
          const uint32_t bx = bxy[st] & 0xFFFFu, by = bxy[st] >> 16;
          const uint32_t blk = by * (uint32_t)gw + bx;
          // blocks of the box that the ellipse misses get the key 0xFFFFFFFF,
          // which the first pass of the pair sort drops; so do, in the memory-
          // efficiency mode, blocks every pixel of which an earlier chunk left
          // T-culled (they take no more fragments)
          const bool hit = bx >= (iv & 0xFFFFu) && bx + 1u <= (iv >> 16) &&
                           !(block_done && block_done[blk] < chunk);
          const uint32_t dst = wp0 + 32u * st + (uint32_t)lane - pbase;
          pair_keys[dst] = hit ? blk : kNone;
          pair_vals[dst] = r0 + lov[st];
          if (hit) {
            ++live;
            for (int q = 0; q < pair_passes; ++q) atomicAdd(&s_hist[q][(blk >> (8 * q)) & 0xFF], 1u);
          }
        }
        before += __popc(unit_mask[st]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
  if ((tid & 31) == 0 && live) atomicAdd(&hdr->live_pairs, live);
  __syncthreads();
  for (int i = tid; i < pair_passes * 256; i += kBinThreads) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&hdr->pair_hist[0][0] + i, v);
  }
}

// Block ranges [start, end) in the live pairs sorted by block id.  ranges must
// be zero beforehand (the chunk setup clears them).  Each thread reads eight
// consecutive keys as two 16-byte words (more bytes in flight than one key per
// thread) plus the key on either side.
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ keys,
                                                     const Header* __restrict__ hdr,
                                                     uint2* __restrict__ ranges, uint32_t nblocks) {
  const uint32_t P = hdr->live_pairs;
  const uint32_t n8 = (P + 7) / 8;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n8; g += gridDim.x * blockDim.x) {
    const uint32_t i0 = 8 * g;
    uint32_t k[8];
    if (i0 + 8 <= P) {   // keys is 256-byte aligned
      const uint4 u = reinterpret_cast<const uint4*>(keys)[2 * g];
      const uint4 v = reinterpret_cast<const uint4*>(keys)[2 * g + 1];
      k[0] = u.x; k[1] = u.y; k[2] = u.z; k[3] = u.w;
      k[4] = v.x; k[5] = v.y; k[6] = v.z; k[7] = v.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) k[j] = i0 + j < P ? keys[i0 + j] : kNone;
    }
    const uint32_t before = i0 > 0 ? keys[i0 - 1] : kNone;
    const uint32_t after = i0 + 8 < P ? keys[i0 + 8] : kNone;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t kk = k[j];
      if (kk >= nblocks) continue;   // also the slots past P
      if ((j ? k[j - 1] : before) != kk) ranges[kk].x = i0 + j;
      if ((j < 7 ? k[j + 1] : after) != kk) ranges[kk].y = i0 + j + 1;
    }
  }
}

// Longest-list-first launch order of the pixel blocks: a counting sort of the
// blocks by a logarithmic bucket of their list length (descending), in one
// CTA.  CTAs are dispatched roughly in launch order, so the heaviest blocks
// start first and the raster's tail shrinks.  The order inside a bucket only
// affects scheduling, never a result.
constexpr int kOrderBuckets = 128;

__device__ __forceinline__ int length_bucket(uint32_t len) {
  if (len == 0) return kOrderBuckets - 1;
  const int lg = 31 - __clz(len);                       // floor(log2 len), 0..31
  const int frac = lg >= 2 ? (int)((len >> (lg - 2)) & 3) : 0;  // 4 sub-buckets per octave
  return kOrderBuckets - 2 - min(lg * 4 + frac, kOrderBuckets - 2);  // long lists first
}

// Raster work items, longest lists first: a counting sort of the blocks by
// length bucket, each block writing its items contiguously: four 8x8 quadrants,
// eight 8x4 cells when its list has at least `split` entries, sixteen 4x4
// cells from 8 `split` entries on (raster.cu has the encoding).  The item
// count goes to the header.
__device__ __forceinline__ uint32_t block_items(uint32_t len, uint32_t split) {
  return len >= 8u * (uint64_t)split ? 16u : (len >= split ? 8u : 4u);
}

constexpr int kBlockOrderThreads = 1024;
constexpr int kBlockOrderWarps = kBlockOrderThreads / 32;
constexpr int kBlockOrderPer = 8;   // blocks per thread held in registers (8192 blocks)

__global__ void __launch_bounds__(kBlockOrderThreads) block_order_kernel(
    const uint2* __restrict__ ranges, int nblocks, uint32_t split, uint32_t* __restrict__ items,
    Header* __restrict__ hdr) {
  // per-warp item counts per bucket, then per-warp placement cursors
  __shared__ uint32_t s_cnt[kBlockOrderWarps][kOrderBuckets];
  __shared__ uint32_t s_part[kOrderBuckets / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kBlockOrderWarps * kOrderBuckets; i += kBlockOrderThreads)
    (&s_cnt[0][0])[i] = 0u;
  __syncthreads();
  // the lengths of this thread's blocks (any beyond kBlockOrderPer per thread are re-read)
  uint32_t len_r[kBlockOrderPer];
#pragma unroll
  for (int k = 0; k < kBlockOrderPer; ++k) {
    const int b = threadIdx.x + k * kBlockOrderThreads;
    len_r[k] = b < nblocks ? ranges[b].y - ranges[b].x : 0u;
  }
  auto len_of = [&](int b, int k) {
    return k < kBlockOrderPer ? len_r[k] : ranges[b].y - ranges[b].x;
  };
  for (int b = threadIdx.x, k = 0; b < nblocks; b += kBlockOrderThreads, ++k) {
    const uint32_t len = len_of(b, k);
    atomicAdd(&s_cnt[warp][length_bucket(len)], block_items(len, split));
  }
  __syncthreads();
  // exclusive scan in (bucket, warp) order; thread t < kOrderBuckets owns bucket t
  uint32_t tot = 0;
  if (threadIdx.x < kOrderBuckets) {
    for (int w = 0; w < kBlockOrderWarps; ++w) tot += s_cnt[w][threadIdx.x];
  }
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (threadIdx.x < kOrderBuckets && lane == 31) s_part[warp] = incl;
  __syncthreads();
  if (threadIdx.x < kOrderBuckets) {
    uint32_t run = incl - tot;
    for (int w = 0; w < warp; ++w) run += s_part[w];
    for (int w = 0; w < kBlockOrderWarps; ++w) {
      const uint32_t c = s_cnt[w][threadIdx.x];
      s_cnt[w][threadIdx.x] = run;
      run += c;
    }
    if (threadIdx.x == kOrderBuckets - 1) hdr->n_items = run;
  }
  __syncthreads();
  for (int b = threadIdx.x, k = 0; b < nblocks; b += kBlockOrderThreads, ++k) {
    const uint32_t len = len_of(b, k);
    const uint32_t n = block_items(len, split);
    const uint32_t pos = atomicAdd(&s_cnt[warp][length_bucket(len)], n);
    const uint32_t code0 = n == 16u ? 16u : (n == 8u ? 8u : 0u);
    for (uint32_t j = 0; j < n; ++j) items[pos + j] = ((uint32_t)b << 5) | (code0 + j);
  }
}

cudaError_t launch_block_order(const uint2* ranges, int nblocks, uint32_t split, uint32_t* items,
                               Header* hdr, cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  block_order_kernel<<<1, kBlockOrderThreads, 0, st>>>(ranges, nblocks, split, items, hdr);
  return cudaGetLastError();
}

cudaError_t launch_bin_count(const uint32_t* sorted_ids, const SplatRec* rec,
                             const uint2* boxes_by_id, SplatRec* rec_sorted, float* g2d,
                             Header* hdr, unsigned long long* scan_status, const uint32_t* epoch,
                             uint32_t* offsets, uint2* boxes, uint32_t pair_cap, int chunked,
                             int n_cap, int grid_cap, cudaStream_t st, uint32_t* run_first,
                             uint32_t run_cap) {
  int tiles = (n_cap + kBinTile - 1) / kBinTile;
  if (tiles == 0) return cudaSuccess;
  if (tiles > grid_cap) tiles = grid_cap;
  bin_count_kernel<<<tiles, kBinThreads, 0, st>>>(sorted_ids, rec, boxes_by_id, rec_sorted,
                                                  reinterpret_cast<float4*>(g2d), hdr, scan_status,
                                                  epoch, offsets, boxes, pair_cap, chunked,
                                                  run_first, run_cap);
  return cudaGetLastError();
}

// CTAs of the emission resident at once: its runs are dealt out by a static
// grid stride, so a CTA that only starts when others finish would add a wave.
int emit_resident_ctas() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152 * 4;
  if (cache[dev] == 0) {
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bin_emit_kernel, kBinThreads, 0) != cudaSuccess ||
        occ < 1)
      occ = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
    cache[dev] = occ * sms;
  }
  return cache[dev];
}

cudaError_t launch_bin_chunk(const uint32_t* offsets, const uint2* boxes,
                             const SplatRec* rec_sorted, Header* hdr, uint32_t* epoch, uint32_t k,
                             uint32_t B,
                             uint32_t pair_cap, int mode, uint2* ranges, uint32_t* pair_keys,
                             uint32_t* pair_vals, int gw, int gh, int pair_passes, int grid_cap,
                             cudaStream_t st, uint32_t* block_done, uint32_t* done_px,
                             int reset_done, const uint32_t* run_first, uint32_t run_cap) {
  chunk_setup_kernel<<<1, 256, 0, st>>>(offsets, hdr, epoch, k, B, pair_cap, mode, ranges,
                                        gw * gh, block_done, done_px, reset_done);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int runs = (int)((pair_cap + (size_t)kEmitTask * (kBinThreads / 32) - 1) /
                   ((size_t)kEmitTask * (kBinThreads / 32)));
  if (runs > grid_cap) runs = grid_cap;
  if (runs > emit_resident_ctas()) runs = emit_resident_ctas();
  if (runs < 1) runs = 1;
  bin_emit_kernel<<<runs, kBinThreads, 0, st>>>(offsets, boxes, rec_sorted, hdr, pair_keys,
                                                pair_vals, gw, gh, pair_passes, block_done, k,
                                                run_first, run_cap);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t* keys, const Header* hdr, uint2* ranges, int nblocks,
                          int num_sms, cudaStream_t st) {
  ranges_kernel<<<num_sms * 8, 256, 0, st>>>(keys, hdr, ranges, (uint32_t)nblocks);
  return cudaGetLastError();
}

size_t bin_tiles(size_t n) { return (n + kBinTile - 1) / kBinTile; }
size_t emit_run_table(size_t pair_cap) { return pair_cap / kEmitTask + 2; }

}  // namespace gsr

// Stable LSD radix sort, one chained-scan ("Onesweep") pass per 8-bit digit.
//
// The paper sorts splats by depth with a custom Onesweep sort whose length is
// read on the device (Sec. 4.1).  Each pass here: every CTA takes the next tile
// id from an atomic counter (so all lower tiles belong to CTAs that already
// run), counts its 2048 keys per digit and publishes the counts at once, ranks
// the keys stably (warp match and per-warp digit counters) into their places
// in shared memory, looks back over lower tiles for their per-digit prefix
// (decoupled look-back; publishing before the ranking lets later tiles find
// the counts sooner) and writes the tile out.
//
// Look-back status words are 64-bit: [63:32] tag (epoch * 16 + pass, so words
// of earlier passes or views never match), [31:30] flag (1 = tile aggregate,
// 2 = inclusive prefix), [29:0] count.  Waits are bounded: after spin_limit
// polls (kSpinLimit in every pass the library runs for its callers) a CTA
// records kStatusTimeout and continues (positions it writes then stay inside
// the output; the result is wrong but nothing hangs).
#include "common.cuh"

namespace gsr {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048
constexpr int kSortWarps = kSortThreads / 32;
constexpr unsigned long long kFlagAgg = 1ull << 30;
constexpr unsigned long long kFlagPre = 2ull << 30;
constexpr unsigned long long kCount30 = (1ull << 30) - 1;
constexpr int kLookWindow = 4;   // look-back words read per round trip

__device__ __forceinline__ unsigned long long make_status(uint32_t tag, unsigned long long flag,
                                                          uint32_t count) {
  return ((unsigned long long)tag << 32) | flag | ((unsigned long long)count & kCount30);
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kSortWarps ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < kSortWarps; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kSortWarps) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  total = s_warp[kSortWarps - 1];
  const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
  __syncthreads();
  return before + x - v;
}

// One pass.  Items with index >= n are absent; with drop_sentinel, items whose
// key is 0xFFFFFFFF are absent too (culled splats).  vals_in == null means
// value = index.  hist[256] holds the global digit counts of the present items.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) onesweep_pass_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
    const uint32_t* __restrict__ n_dev, uint32_t n_static, uint32_t out_cap, int shift,
    uint32_t mask, const uint32_t* __restrict__ hist, unsigned long long* __restrict__ status,
    uint32_t* __restrict__ tile_counter, const uint32_t* __restrict__ epoch, uint32_t pass_id,
    uint32_t* __restrict__ status_word, int drop_sentinel, uint32_t spin_limit) {
  constexpr int TILE = kSortThreads * ITEMS;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_wcnt[kSortWarps][256];
  __shared__ uint32_t s_gbase[256];
  __shared__ uint32_t s_keys[TILE];
  __shared__ uint32_t s_vals[TILE];
  __shared__ uint32_t s_warp[kSortWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n = n_dev ? *n_dev : n_static;
  const uint32_t ntiles = (uint32_t)(((uint64_t)n + TILE - 1) / TILE);
  const uint32_t tag = (*epoch) * 16u + pass_id;
  // global digit bases: the exclusive scan of the pass histogram (thread d)
  uint32_t hist_total = 0;
  const uint32_t gexcl = block_excl_scan256(hist[tid], s_warp, hist_total);
  // persistent: take tiles in order until none is left; a CTA only ever waits
  // on lower tiles, which running CTAs took earlier, so the waits end
  for (;;) {
  if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
  for (int i = tid; i < kSortWarps * 256; i += kSortThreads) (&s_wcnt[0][0])[i] = 0u;
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= ntiles) break;
  const uint64_t base = (uint64_t)tile * TILE;

  uint32_t key[ITEMS], val[ITEMS];
  bool present[ITEMS];
  // every load first, at clamped indices (n >= 1 here), so that all of them
  // are in flight together; then the presence tests
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t idx = base + (uint64_t)warp * (32 * ITEMS) + k * 32 + lane;
    const uint64_t ci = idx < n ? idx : (uint64_t)(n - 1);
    key[k] = __ldcs(keys_in + ci);
    val[k] = vals_in ? __ldcs(vals_in + ci) : (uint32_t)idx;
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint64_t idx = base + (uint64_t)warp * (32 * ITEMS) + k * 32 + lane;
    present[k] = idx < n;
    if (!present[k]) key[k] = kNone;
    if (drop_sentinel && key[k] == kNone) present[k] = false;
  }
  // per-warp digit counts (order-free), so that the tile's aggregate is
  // published before the ranking: later tiles then find it sooner
#pragma unroll
  for (int k = 0; k < ITEMS; ++k)
    if (present[k]) atomicAdd(&s_wcnt[warp][(key[k] >> shift) & mask], 1u);
  __syncthreads();
  // per digit: warp-exclusive offsets and the tile total
  const uint32_t d = tid;
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const uint32_t c = s_wcnt[w][d];
    s_wcnt[w][d] = tot;
    tot += c;
  }
  unsigned long long* my = status + (uint64_t)tile * 256 + d;
  st_relaxed64(my, make_status(tag, tile == 0 ? kFlagPre : kFlagAgg, tot));
  // tile-local digit offsets; s_wcnt becomes each (warp, digit)'s first position
  uint32_t tile_valid = 0;
  const uint32_t toff = block_excl_scan256(tot, s_warp, tile_valid);
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) s_wcnt[w][d] += toff;
  __syncthreads();
  // stable rank within the warp, item by item (warp-striped order = input
  // order), which is the item's position in the tile sorted by digit
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const uint32_t dk = present[k] ? ((key[k] >> shift) & mask) : 0x100u;
    const uint32_t peers = __match_any_sync(0xffffffffu, dk);
    const int leader = __ffs(peers) - 1;
    uint32_t pre = 0;
    if (lane == leader && present[k]) {
      pre = s_wcnt[warp][dk];
      s_wcnt[warp][dk] = pre + __popc(peers);
    }
    pre = __shfl_sync(0xffffffffu, pre, leader);
    if (present[k]) {
      const uint32_t pos = pre + __popc(peers & lanemask_lt());
      s_keys[pos] = key[k];
      s_vals[pos] = val[k];
    }
    __syncwarp();
  }
  // look back for the exclusive prefix over lower tiles
  uint32_t excl = 0;
  if (tile > 0) {
    // kLookWindow predecessors per round trip: their words are loaded together,
    // then consumed nearest first until a prefix or a word not yet published
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool found = false;
    while (j >= 0 && !found) {
      unsigned long long w[kLookWindow];
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i)
        w[i] = j - i >= 0 ? ld_relaxed64(status + (uint64_t)(j - i) * 256 + d) : 0ull;
      int used = 0;
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i) {
        if (found || used < i || j - i < 0) break;
        const bool ready = (uint32_t)(w[i] >> 32) == tag && (w[i] & (3ull << 30)) != 0;
        if (!ready) break;
        excl += (uint32_t)(w[i] & kCount30);
        used = i + 1;
        found = (w[i] & (3ull << 30)) == kFlagPre;
      }
      if (used == 0) {
        if (++spins > spin_limit) {
          atomicOr(status_word, kStatusTimeout);
          break;
        }
        continue;
      }
      j -= used;
    }
    st_relaxed64(my, make_status(tag, kFlagPre, (uint32_t)min((unsigned long long)excl + tot, kCount30)));
  }
  s_gbase[d] = gexcl + excl - toff;
  __syncthreads();
  for (uint32_t i = tid; i < tile_valid; i += kSortThreads) {
    const uint32_t kk = s_keys[i];
    const uint32_t out = s_gbase[(kk >> shift) & mask] + i;
    if (out < out_cap) {
      keys_out[out] = kk;
      vals_out[out] = s_vals[i];
    }
  }
  __syncthreads();
  }
}

// Digit histograms of `bits_passes` 8-bit digits over n keys (standalone sort).
__global__ void __launch_bounds__(256) digit_hist_kernel(const uint32_t* __restrict__ keys, uint32_t n,
                                                         int passes, uint32_t* __restrict__ hist) {
  __shared__ uint32_t s_hist[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][(k >> (8 * p)) & 0xFF], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(hist + i, v);
  }
}

__global__ void bump_epoch_kernel(uint32_t* epoch) { *epoch += 1u; }
// A new epoch and n zeroed tile counters: the start of a sort.
__global__ void sort_begin_kernel(uint32_t* epoch, uint32_t* counters, int n) {
  if (threadIdx.x == 0) *epoch += 1u;
  if ((int)threadIdx.x < n) counters[threadIdx.x] = 0u;
}
__global__ void set_word_kernel(uint32_t* p, uint32_t v) { *p = v; }

cudaError_t launch_onesweep_pass(const uint32_t* keys_in, const uint32_t* vals_in,
                                 uint32_t* keys_out, uint32_t* vals_out, const uint32_t* n_dev,
                                 uint32_t n_static, uint32_t n_cap, uint32_t out_cap, int shift,
                                 uint32_t mask, const uint32_t* hist, unsigned long long* status,
                                 uint32_t* tile_counter, const uint32_t* epoch, uint32_t pass_id,
                                 uint32_t* status_word, int drop_sentinel, int grid_cap,
                                 cudaStream_t st, uint32_t spin_limit, int wide) {
  // wide: tiles of 4096 keys instead of 2048 (fewer look-back steps per key on
  // long inputs; short inputs want more tiles)
  const uint32_t tile = wide ? 2u * kSortTile : (uint32_t)kSortTile;
  uint32_t tiles = (n_cap + tile - 1) / tile;
  if (tiles == 0) return cudaSuccess;
  if (tiles > (uint32_t)grid_cap) tiles = (uint32_t)grid_cap;
  if (wide)
    onesweep_pass_kernel<2 * kSortItems><<<tiles, kSortThreads, 0, st>>>(
        keys_in, vals_in, keys_out, vals_out, n_dev, n_static, out_cap, shift, mask, hist, status,
        tile_counter, epoch, pass_id, status_word, drop_sentinel, spin_limit);
  else
    onesweep_pass_kernel<kSortItems><<<tiles, kSortThreads, 0, st>>>(
        keys_in, vals_in, keys_out, vals_out, n_dev, n_static, out_cap, shift, mask, hist, status,
        tile_counter, epoch, pass_id, status_word, drop_sentinel, spin_limit);
  return cudaGetLastError();
}

cudaError_t launch_digit_hist(const uint32_t* keys, uint32_t n, int passes, uint32_t* hist,
                              int num_sms, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > num_sms * 4) blocks = num_sms * 4;
  if (blocks < 1) blocks = 1;
  digit_hist_kernel<<<blocks, 256, 0, st>>>(keys, n, passes, hist);
  return cudaGetLastError();
}

cudaError_t launch_bump_epoch(uint32_t* epoch, cudaStream_t st) {
  bump_epoch_kernel<<<1, 1, 0, st>>>(epoch);
  return cudaGetLastError();
}

cudaError_t launch_sort_begin(uint32_t* epoch, uint32_t* counters, int n, cudaStream_t st) {
  sort_begin_kernel<<<1, 32, 0, st>>>(epoch, counters, n);
  return cudaGetLastError();
}

cudaError_t launch_set_word(uint32_t* p, uint32_t v, cudaStream_t st) {
  set_word_kernel<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

size_t sort_tiles(size_t n) { return (n + kSortTile - 1) / kSortTile; }   // the narrow tiles: an upper bound

}  // namespace gsr

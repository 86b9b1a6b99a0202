// C ABI: workspace layout, argument checks and the launch sequence of each call.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "common.cuh"

namespace gsr {

// launchers (kernels live in the other translation units)
struct CamDev;
cudaError_t launch_project_fwd(const float*, const float*, const float*, const float*, const float*,
                               int, int, const gs_camera&, int, SplatRec*, uint2*, uint32_t*,
                               Header*, uint2*, int, uint32_t*, int, cudaStream_t);
cudaError_t launch_project_bwd(const float*, const float*, const float*, const float*, const float*,
                               int, int, const gs_camera&, int, const uint32_t*, const float*,
                               const Header*, float*, float*, float*, float*, float*, int,
                               cudaStream_t, int, uint32_t*, uint32_t*);
cudaError_t launch_zero_listed(int, int, const uint32_t*, const uint32_t*, float*, float*, float*,
                               float*, float*, int, cudaStream_t);
cudaError_t launch_copy_word(const uint32_t*, uint32_t*, cudaStream_t);
cudaError_t launch_zero_left(int, int, const uint32_t*, const uint32_t*, const uint32_t*, float*,
                             float*, float*, float*, float*, int, cudaStream_t, const uint32_t*);
cudaError_t launch_zero_touched(int, int, const uint32_t*, const Header*, float*, float*, float*,
                                float*, float*, int, cudaStream_t);
cudaError_t launch_onesweep_pass(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*,
                                 const uint32_t*, uint32_t, uint32_t, uint32_t, int, uint32_t,
                                 const uint32_t*, unsigned long long*, uint32_t*, const uint32_t*,
                                 uint32_t, uint32_t*, int, int, cudaStream_t,
                                 uint32_t spin_limit = kSpinLimit, int wide = 0);
cudaError_t launch_set_word(uint32_t*, uint32_t, cudaStream_t);
int noalloc_stalled_pass(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, int32_t,
                         uint32_t, cudaStream_t);
cudaError_t launch_digit_hist(const uint32_t*, uint32_t, int, uint32_t*, int, cudaStream_t);
cudaError_t launch_bump_epoch(uint32_t*, cudaStream_t);
cudaError_t launch_sort_begin(uint32_t*, uint32_t*, int, cudaStream_t);
cudaError_t launch_bin_count(const uint32_t*, const SplatRec*, const uint2*, SplatRec*, float*,
                             Header*, unsigned long long*, const uint32_t*, uint32_t*, uint2*,
                             uint32_t, int, int, int, cudaStream_t, uint32_t*, uint32_t);
cudaError_t launch_bin_chunk(const uint32_t*, const uint2*, const SplatRec*, Header*, uint32_t*,
                             uint32_t, uint32_t, uint32_t, int, uint2*, uint32_t*, uint32_t*, int,
                             int, int, int, cudaStream_t, uint32_t*, uint32_t*, int,
                             const uint32_t*, uint32_t);
cudaError_t launch_ranges(const uint32_t*, const Header*, uint2*, int, int, cudaStream_t);
cudaError_t launch_block_order(const uint2*, int, uint32_t, uint32_t*, Header*, cudaStream_t);
cudaError_t launch_raster_fwd(const uint2*, const uint32_t*, const Header*, uint32_t*, uint32_t*,
                              const uint32_t*, const SplatRec*, int, int, int, int, float, int,
                              float*, void*, uint32_t*, uint32_t*, int, uint32_t*, uint32_t*,
                              uint32_t, int, cudaStream_t);
cudaError_t launch_raster_bwd(const uint2*, const uint32_t*, const uint32_t*, uint32_t*,
                              const Header*, uint32_t*, const uint32_t*, const SplatRec*, int, int,
                              int, int, float, int, const void*, const uint32_t*, const float*,
                              float*, int, int, int, float4*, int, int, const float*,
                              const float*, int, cudaStream_t, int order_done = 0);
cudaError_t launch_item_order(const uint32_t*, const uint32_t*, const Header*, uint32_t*,
                              cudaStream_t);
cudaError_t launch_slab_composite(const void*, int, int, int64_t, float*, float*, float*, float*,
                                  int, cudaStream_t);
cudaError_t launch_loss(const float*, const float*, int64_t, int, float*, double*, int,
                        cudaStream_t);
size_t sort_tiles(size_t n);
size_t bin_tiles(size_t n);
size_t emit_run_table(size_t pair_cap);

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define GS_CUDA(call, where)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

// Resident CTAs of a 256-thread sort/bin kernel per SM (shared memory bound).
constexpr int kPersistentPerSm = 6;

enum Slot {
  L_HDR = 0,
  L_EPOCH,
  L_STATUS,      // onesweep look-back words, shared by all passes (tags differ)
  L_SCAN,        // binning scan look-back words
  L_KEYS,        // [n] depth keys (0xFFFFFFFF = culled)
  L_KA, L_VA, L_KB, L_VB,   // [n] sort ping-pong
  L_REC,         // [n] records by splat id
  L_BOXES_ID,    // [n] uint2 16x16-block box of each splat, by splat id
  L_REC_SORTED,  // [n] records by depth rank
  L_G2D,         // [n][12] backward accumulators by depth rank
  L_OFFSETS,     // [n] first pair index of each depth rank, then the emission's run table
                 // ([pair_cap / 256 + 2] the rank holding pair m * 256), then [n] the ids
                 // whose gradient rows the last store-mode backward wrote
  L_BOXES,       // [n] uint2 block box of each depth rank
  L_CHUNK_STATE, // memory-efficiency mode: [width_cap * height_cap] float4 (g.C', T) between
                 // chunks, then [2 blocks_cap] u32: the chunk after which each block's pixels
                 // are all T-culled (0xFFFFFFFF: not yet), and this chunk's culled-pixel counts
  L_PKA, L_PVA, L_PKB, L_PVB,  // [pair_cap] pair ping-pong
  L_RANGES,      // [blocks_cap] uint2
  L_ORDER,       // [16 blocks_cap] u32 raster work items (warp footprints), longest lists first
  L_ITEM_COST,   // [16 blocks_cap] u32 cost of each item in the last forward raster
  L_BWD_ITEMS,   // [16 blocks_cap] u32 the items again, costliest first, for the backward raster
  L_END
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int64_t default_pair_cap(int64_t n_cap) {
  int64_t p = 16 * n_cap;
  if (p < (1 << 22)) p = 1 << 22;
  return p;
}

int blocks_of(int w, int h, int& gw, int& gh) {
  gw = (w + kBlock - 1) / kBlock;
  gh = (h + kBlock - 1) / kBlock;
  return gw * gh;
}

bool compute_layout(int64_t n_cap, int w_cap, int h_cap, int64_t pair_cap, int chunked,
                    uint64_t* off, size_t* total) {
  int gw, gh;
  const size_t blocks = blocks_of(w_cap, h_cap, gw, gh);
  const size_t st_tiles = std::max(sort_tiles(n_cap), sort_tiles(pair_cap)) + 1;
  size_t sz[L_END];
  sz[L_HDR] = sizeof(Header);
  sz[L_EPOCH] = 256;
  sz[L_STATUS] = st_tiles * 256 * sizeof(unsigned long long);
  sz[L_SCAN] = (bin_tiles(n_cap) + 1) * sizeof(unsigned long long);
  sz[L_KEYS] = n_cap * 4;
  sz[L_KA] = sz[L_VA] = sz[L_KB] = sz[L_VB] = n_cap * 4;
  sz[L_REC] = sz[L_REC_SORTED] = sz[L_G2D] = n_cap * sizeof(SplatRec);
  sz[L_OFFSETS] = (2 * n_cap + emit_run_table(pair_cap)) * 4;
  sz[L_BOXES_ID] = n_cap * 8;
  sz[L_BOXES] = n_cap * 8;
  sz[L_CHUNK_STATE] = chunked ? (size_t)w_cap * h_cap * 16 + blocks * 2 * 4 : 0;
  sz[L_PKA] = sz[L_PVA] = sz[L_PKB] = sz[L_PVB] = pair_cap * 4;
  sz[L_RANGES] = blocks * sizeof(uint2);
  sz[L_ORDER] = sz[L_ITEM_COST] = sz[L_BWD_ITEMS] = blocks * 16 * 4;
  size_t o = 0;
  for (int i = 0; i < L_END; ++i) {
    off[i] = o;
    o = align256(o + sz[i]);
  }
  *total = o;
  return true;
}

template <typename T>
T* at(const gs_workspace* ws, int slot) {
  return reinterpret_cast<T*>(static_cast<char*>(ws->base) + ws->layout[slot]);
}

int check_opts(const gs_raster_opts* o) {
  if (!o) return fail(GS_ERR_INVALID_ARG, "opts is null");
  if (o->state_format < 0 || o->state_format > 3) return fail(GS_ERR_INVALID_ARG, "bad state_format %d", o->state_format);
  if (o->reduce_mode < 0 || o->reduce_mode > 2) return fail(GS_ERR_INVALID_ARG, "bad reduce_mode %d", o->reduce_mode);
  if (o->reduce_mode == GS_REDUCE_FRAGMENT && o->backward_order != GS_BWD_FRONT_TO_BACK)
    return fail(GS_ERR_INVALID_ARG, "GS_REDUCE_FRAGMENT walks front to back only");
  if (o->split_threshold < 0) return fail(GS_ERR_INVALID_ARG, "bad split_threshold %d", o->split_threshold);
  if (o->reduce_threshold < 0) return fail(GS_ERR_INVALID_ARG, "bad reduce_threshold %d", o->reduce_threshold);
  if (o->backward_order < 0 || o->backward_order > 1)
    return fail(GS_ERR_INVALID_ARG, "bad backward_order %d", o->backward_order);
  if (o->chunked < 0 || o->chunked > 1) return fail(GS_ERR_INVALID_ARG, "bad chunked %d", o->chunked);
  if (o->chunked && o->backward_order != GS_BWD_FRONT_TO_BACK)
    return fail(GS_ERR_INVALID_ARG, "the memory-efficiency mode walks front to back only");
  if (o->sh_degree < 0 || o->sh_degree > kMaxShDegree) return fail(GS_ERR_INVALID_ARG, "bad sh_degree %d", o->sh_degree);
  if (!(o->t_cull >= 0.f && o->t_cull <= 1.f)) return fail(GS_ERR_INVALID_ARG, "t_cull must be in [0, 1]");
  if (o->pair_capacity < 0 || o->pair_capacity >= (1ll << 30)) return fail(GS_ERR_INVALID_ARG, "pair_capacity must be in [0, 2^30)");
  return GS_OK;
}

int check_ws(const gs_workspace* ws) {
  if (!ws || !ws->base) return fail(GS_ERR_INVALID_ARG, "workspace is null or not initialised");
  return GS_OK;
}

int check_cam(const gs_workspace* ws, const gs_camera* cam) {
  if (!cam) return fail(GS_ERR_INVALID_ARG, "camera is null");
  if (cam->width < 0 || cam->height < 0) return fail(GS_ERR_INVALID_ARG, "negative image size");
  if (cam->width > ws->width_cap || cam->height > ws->height_cap)
    return fail(GS_ERR_INVALID_ARG, "image %dx%d exceeds the workspace capacity %dx%d", cam->width,
                cam->height, ws->width_cap, ws->height_cap);
  return GS_OK;
}

int pair_passes_for(int blocks) {
  int bits = 0;
  while (bits < 32 && (1ll << bits) < blocks) ++bits;
  int p = (bits + 7) / 8;
  return p < 1 ? 1 : p;
}

}  // namespace

int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace gsr

using namespace gsr;

extern "C" {

const char* gs_last_error(void) { return g_last_error.c_str(); }

int gs_workspace_size(int32_t n_cap, int32_t width_cap, int32_t height_cap,
                      const gs_raster_opts* opts, size_t* bytes) {
  if (!bytes) return fail(GS_ERR_INVALID_ARG, "bytes is null");
  if (n_cap < 0 || width_cap < 0 || height_cap < 0) return fail(GS_ERR_INVALID_ARG, "negative capacity");
  if (n_cap >= (1 << 30)) return fail(GS_ERR_INVALID_ARG, "n_cap must be < 2^30");
  if (width_cap > 65535 * kBlock || height_cap > 65535 * kBlock)
    return fail(GS_ERR_INVALID_ARG, "image capacity too large");
  {
    int gw, gh;
    if ((int64_t)((width_cap + kBlock - 1) / kBlock) * ((height_cap + kBlock - 1) / kBlock) > (1 << 21))
      return fail(GS_ERR_INVALID_ARG, "image capacity above 2^21 pixel blocks");
    (void)gw; (void)gh;
  }
  int rc = check_opts(opts);
  if (rc) return rc;
  const int64_t pcap = opts->pair_capacity ? opts->pair_capacity : default_pair_cap(n_cap);
  if (pcap >= (1ll << 30)) return fail(GS_ERR_INVALID_ARG, "pair capacity must be < 2^30");
  uint64_t off[L_END];
  compute_layout(n_cap, width_cap, height_cap, pcap, opts->chunked, off, bytes);
  return GS_OK;
}

int gs_workspace_init(gs_workspace* ws, void* device_base, size_t bytes, int32_t n_cap,
                      int32_t width_cap, int32_t height_cap, const gs_raster_opts* opts,
                      gs_stream_t stream) {
  if (!ws) return fail(GS_ERR_INVALID_ARG, "ws is null");
  size_t need = 0;
  int rc = gs_workspace_size(n_cap, width_cap, height_cap, opts, &need);
  if (rc) return rc;
  if (!device_base) return fail(GS_ERR_INVALID_ARG, "device_base is null");
  if (reinterpret_cast<uintptr_t>(device_base) & 255)
    return fail(GS_ERR_INVALID_ARG, "device_base must be 256-byte aligned");
  if (bytes < need) return fail(GS_ERR_INVALID_ARG, "workspace has %zu bytes, needs %zu", bytes, need);
  std::memset(ws, 0, sizeof(*ws));
  ws->base = device_base;
  ws->bytes = bytes;
  ws->n_cap = n_cap;
  ws->width_cap = width_cap;
  ws->height_cap = height_cap;
  ws->pair_cap = opts->pair_capacity ? opts->pair_capacity : default_pair_cap(n_cap);
  static_assert(L_END <= 24, "layout table too small");
  size_t total = 0;
  compute_layout(n_cap, width_cap, height_cap, ws->pair_cap, opts->chunked, ws->layout, &total);
  ws->chunked = opts->chunked;
  // Header, epoch and all look-back words start at zero (a zero word never
  // carries a valid tag's flag); ordered before later work on `stream`.
  GS_CUDA(cudaMemsetAsync(device_base, 0, ws->layout[L_SCAN + 1],
                          reinterpret_cast<cudaStream_t>(stream)),
          "workspace init memset");
  return GS_OK;
}

int gs_project(gs_workspace* ws, const float* means, const float* scales, const float* quats,
               const float* opacities, const float* sh, int32_t n, const gs_camera* cam,
               const gs_raster_opts* opts, gs_stream_t stream) {
  int rc = check_ws(ws);
  if (!rc) rc = check_opts(opts);
  if (!rc) rc = check_cam(ws, cam);
  if (rc) return rc;
  if (n < 0 || n > ws->n_cap) return fail(GS_ERR_INVALID_ARG, "n = %d exceeds the workspace capacity %d", n, ws->n_cap);
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh))
    return fail(GS_ERR_INVALID_ARG, "null scene pointer");
  if (reinterpret_cast<uintptr_t>(quats) & 15) return fail(GS_ERR_INVALID_ARG, "quats must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int gw, gh;
  const int blocks = blocks_of(cam->width, cam->height, gw, gh);
  ws->n = n;
  ws->width = cam->width;
  ws->height = cam->height;
  ws->sh_degree = opts->sh_degree;
  ws->state_format = opts->state_format;
  ws->clamp01 = opts->state_format == GS_STATE_UNORM16 || opts->state_format == GS_STATE_UNORM8;
  ws->pair_passes = pair_passes_for(blocks);   // block ids 0..blocks-1
  GS_CUDA(cudaMemsetAsync(at<Header>(ws, L_HDR), 0, sizeof(Header), st), "gs_project memset");
  GS_CUDA(launch_project_fwd(means, scales, quats, opacities, sh, n, opts->sh_degree, *cam,
                             ws->clamp01, at<SplatRec>(ws, L_REC), at<uint2>(ws, L_BOXES_ID),
                             at<uint32_t>(ws, L_KEYS),
                             at<Header>(ws, L_HDR), at<uint2>(ws, L_RANGES), blocks,
                             at<uint32_t>(ws, L_EPOCH), num_sms(), st),
          "project kernel");
  return GS_OK;
}

int gs_sort(gs_workspace* ws, gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Header* hdr = at<Header>(ws, L_HDR);
  uint32_t* epoch = at<uint32_t>(ws, L_EPOCH);
  unsigned long long* status = at<unsigned long long>(ws, L_STATUS);
  const int grid_cap = num_sms() * kPersistentPerSm;
  // a sort may repeat without a new projection: fresh tile counters and look-back tags
  GS_CUDA(launch_sort_begin(epoch, &hdr->tile_counter[0], 4, st), "sort setup kernel");
  uint32_t* bufs_k[2] = {at<uint32_t>(ws, L_KA), at<uint32_t>(ws, L_KB)};
  uint32_t* bufs_v[2] = {at<uint32_t>(ws, L_VA), at<uint32_t>(ws, L_VB)};
  for (int pass = 0; pass < 4; ++pass) {
    const uint32_t* kin = pass == 0 ? at<uint32_t>(ws, L_KEYS) : bufs_k[(pass + 1) & 1];
    const uint32_t* vin = pass == 0 ? nullptr : bufs_v[(pass + 1) & 1];
    uint32_t* kout = bufs_k[pass & 1];
    uint32_t* vout = bufs_v[pass & 1];
    // the first pass reads all n keys (wide tiles from 2M on); the others only
    // the visible ones, usually far fewer (narrow tiles keep enough of them)
    GS_CUDA(launch_onesweep_pass(kin, vin, kout, vout, pass == 0 ? nullptr : &hdr->visible,
                                 (uint32_t)ws->n, (uint32_t)ws->n, (uint32_t)ws->n, 8 * pass, 0xFFu,
                                 hdr->depth_hist[pass], status, &hdr->tile_counter[pass], epoch,
                                 (uint32_t)pass, &hdr->status, pass == 0, grid_cap, st, kSpinLimit,
                                 pass == 0 && ws->n >= (1 << 21)),
            "depth sort pass");
  }
  return GS_OK;
}

static int check_bound(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts) {
  int rc = check_ws(ws);
  if (!rc) rc = check_opts(opts);
  if (!rc) rc = check_cam(ws, cam);
  if (rc) return rc;
  if (cam->width != ws->width || cam->height != ws->height)
    return fail(GS_ERR_INVALID_ARG, "camera differs from the one gs_project was given");
  if (opts->state_format != ws->state_format || opts->sh_degree != ws->sh_degree)
    return fail(GS_ERR_INVALID_ARG, "opts differ from the ones gs_project was given");
  return GS_OK;
}

namespace {

// The memory-efficiency mode's per-block arrays (after the (g.C', T) carry in
// L_CHUNK_STATE): which = 0 the chunk after which the block is done, 1 this
// chunk's culled-pixel counts; null in the other modes.
uint32_t* done_arrays(gs_workspace* ws, int which) {
  if (!ws->chunked) return nullptr;
  int gw, gh;
  const size_t blocks = blocks_of(ws->width_cap, ws->height_cap, gw, gh);
  return reinterpret_cast<uint32_t*>(at<char>(ws, L_CHUNK_STATE) +
                                     (size_t)ws->width_cap * ws->height_cap * 16) +
         (which ? blocks : 0);
}

// Binning, first pass: records into depth order, box pair counts, their scan.
// skip_capacity: the whole view's pairs may exceed the capacity (the
// memory-efficiency mode and depth slabs bin part of the view at a time).
int bin_count_stage(gs_workspace* ws, cudaStream_t st, int skip_capacity = -1) {
  Header* hdr = at<Header>(ws, L_HDR);
  const int grid_cap = num_sms() * kPersistentPerSm;
  GS_CUDA(cudaMemsetAsync(&hdr->tile_counter[8], 0, sizeof(uint32_t), st), "bin counter");
  GS_CUDA(launch_bin_count(at<uint32_t>(ws, L_VB), at<SplatRec>(ws, L_REC),
                           at<uint2>(ws, L_BOXES_ID), at<SplatRec>(ws, L_REC_SORTED),
                           at<float>(ws, L_G2D), hdr, at<unsigned long long>(ws, L_SCAN),
                           at<uint32_t>(ws, L_EPOCH), at<uint32_t>(ws, L_OFFSETS),
                           at<uint2>(ws, L_BOXES), (uint32_t)ws->pair_cap,
                           skip_capacity >= 0 ? skip_capacity : ws->chunked, ws->n, grid_cap, st,
                           at<uint32_t>(ws, L_OFFSETS) + ws->n_cap,
                           (uint32_t)emit_run_table(ws->pair_cap)),
          "bin count kernel");
  return GS_OK;
}

// Binning of chunk k (the only chunk without the memory-efficiency mode):
// emission, the pair sort by block, block ranges and raster work items.
// mode: 0 the whole view, 1 the memory-efficiency mode's chunk k of pair
// budget B, 2 depth slab k of B (chunk_setup_kernel, bin.cu).
int bin_chunk_stage(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                    uint32_t k, uint32_t B, cudaStream_t st, int mode = -1, int reset_done = 0) {
  Header* hdr = at<Header>(ws, L_HDR);
  uint32_t* epoch = at<uint32_t>(ws, L_EPOCH);
  int gw, gh;
  blocks_of(cam->width, cam->height, gw, gh);
  const int grid_cap = num_sms() * kPersistentPerSm;
  GS_CUDA(launch_bin_chunk(at<uint32_t>(ws, L_OFFSETS), at<uint2>(ws, L_BOXES),
                           at<SplatRec>(ws, L_REC_SORTED), hdr, epoch, k, B, (uint32_t)ws->pair_cap,
                           mode >= 0 ? mode : ws->chunked, at<uint2>(ws, L_RANGES),
                           at<uint32_t>(ws, L_PKA),
                           at<uint32_t>(ws, L_PVA), gw, gh, ws->pair_passes, grid_cap, st,
                           done_arrays(ws, 0), done_arrays(ws, 1), reset_done,
                           at<uint32_t>(ws, L_OFFSETS) + ws->n_cap,
                           (uint32_t)emit_run_table(ws->pair_cap)),
          "bin emit kernel");
  uint32_t* pk[2] = {at<uint32_t>(ws, L_PKA), at<uint32_t>(ws, L_PKB)};
  uint32_t* pv[2] = {at<uint32_t>(ws, L_PVA), at<uint32_t>(ws, L_PVB)};
  for (int q = 0; q < ws->pair_passes; ++q) {
    // the first pass reads every emitted pair and drops the missed ones (key
    // 0xFFFFFFFF); the others see only the live pairs
    GS_CUDA(launch_onesweep_pass(pk[q & 1], pv[q & 1], pk[(q + 1) & 1], pv[(q + 1) & 1],
                                 q == 0 ? &hdr->pairs : &hdr->live_pairs, 0u,
                                 (uint32_t)ws->pair_cap, (uint32_t)ws->pair_cap, 8 * q, 0xFFu,
                                 hdr->pair_hist[q], at<unsigned long long>(ws, L_STATUS),
                                 &hdr->tile_counter[4 + q], epoch, 4u + q, &hdr->status, q == 0,
                                 grid_cap, st, kSpinLimit, ws->pair_cap >= (1 << 22)),
            "pair sort pass");
  }
  const int fin = ws->pair_passes & 1;
  GS_CUDA(launch_ranges(pk[fin], hdr, at<uint2>(ws, L_RANGES), gw * gh, num_sms(), st),
          "ranges kernel");
  const uint32_t split = opts->split_threshold > 0 ? (uint32_t)opts->split_threshold
                                                    : (uint32_t)GS_SPLIT_THRESHOLD_DEFAULT;
  GS_CUDA(launch_block_order(at<uint2>(ws, L_RANGES), gw * gh, split, at<uint32_t>(ws, L_ORDER),
                             hdr, st),
          "block order kernel");
  return GS_OK;
}

// Chunks of the bound view in the memory-efficiency mode (synchronises `st`
// to read the view's pair count) and their pair budget B.
int count_chunks(gs_workspace* ws, const gs_camera* cam, cudaStream_t st, uint32_t* n_chunks,
                 uint32_t* B) {
  int gw, gh;
  const int64_t blocks = blocks_of(cam->width, cam->height, gw, gh);
  if (ws->pair_cap < 2 * blocks)
    return fail(GS_ERR_INVALID_ARG,
                "memory-efficiency mode needs a pair capacity of at least twice the block count (%lld)",
                (long long)(2 * blocks));
  uint32_t total = 0;
  GS_CUDA(cudaMemcpyAsync(&total, &at<Header>(ws, L_HDR)->pairs_wanted, 4, cudaMemcpyDeviceToHost,
                          st), "pair count copy");
  GS_CUDA(cudaStreamSynchronize(st), "pair count sync");
  *B = (uint32_t)(ws->pair_cap - blocks);
  *n_chunks = total == 0 ? 1u : (uint32_t)((total + (uint64_t)*B - 1) / *B);
  return GS_OK;
}

int raster_fwd_stage(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                     float* image, void* state, uint32_t* last, uint32_t* n_contrib, int resume,
                     cudaStream_t st, uint32_t chunk = 0) {
  int gw, gh;
  blocks_of(cam->width, cam->height, gw, gh);
  const int fin = ws->pair_passes & 1;
  Header* hdr = at<Header>(ws, L_HDR);
  GS_CUDA(launch_raster_fwd(at<uint2>(ws, L_RANGES), at<uint32_t>(ws, L_ORDER), hdr,
                            &hdr->raster_next[0], at<uint32_t>(ws, L_ITEM_COST),
                            at<uint32_t>(ws, fin ? L_PVB : L_PVA),
                            at<SplatRec>(ws, L_REC_SORTED), cam->width, cam->height, gw, gh,
                            opts->t_cull, opts->state_format, image, state, last, n_contrib,
                            resume, done_arrays(ws, 0), done_arrays(ws, 1), chunk, num_sms(), st),
          "raster forward kernel");
  return GS_OK;
}

int raster_bwd_stage(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                     const void* state, const uint32_t* last, const float* dL_dimage,
                     int chunk_in, int chunk_out, cudaStream_t st,
                     const float* t_front = nullptr, const float* behind = nullptr,
                     int order_done = 0) {
  int gw, gh;
  blocks_of(cam->width, cam->height, gw, gh);
  const int fin = ws->pair_passes & 1;
  Header* hdr = at<Header>(ws, L_HDR);
  GS_CUDA(launch_raster_bwd(at<uint2>(ws, L_RANGES), at<uint32_t>(ws, L_ORDER),
                            at<uint32_t>(ws, L_ITEM_COST), at<uint32_t>(ws, L_BWD_ITEMS), hdr,
                            &hdr->raster_next[1], at<uint32_t>(ws, fin ? L_PVB : L_PVA),
                            at<SplatRec>(ws, L_REC_SORTED), cam->width, cam->height, gw, gh,
                            opts->t_cull, opts->state_format, state, last, dL_dimage,
                            at<float>(ws, L_G2D), opts->reduce_mode,
                            opts->reduce_threshold > 0 ? opts->reduce_threshold
                                                       : GS_REDUCE_THRESHOLD_DEFAULT,
                            opts->backward_order, at<float4>(ws, L_CHUNK_STATE), chunk_in,
                            chunk_out, t_front, behind, num_sms(), st, order_done),
          "raster backward kernel");
  return GS_OK;
}

// gs_blend_backward; order_done: the item order was launched already.
int blend_backward_impl(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                        const void* state, const uint32_t* last, const float* dL_dimage,
                        gs_stream_t stream, int order_done) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (ws->chunked)
    return fail(GS_ERR_INVALID_ARG, "memory-efficiency mode: use gs_raster_backward");
  const size_t npix = (size_t)cam->width * cam->height;
  if (npix > 0 && (!state || !last || !dL_dimage))
    return fail(GS_ERR_INVALID_ARG, "state, last and dL_dimage are required");
  return raster_bwd_stage(ws, cam, opts, state, last, dL_dimage, 0, 0,
                          reinterpret_cast<cudaStream_t>(stream), nullptr, nullptr, order_done);
}

// The ids whose gradient rows the last store-mode backward projection wrote,
// and its state in the epoch words: [0] their count, [1] 1 while the list
// covers every non-zero gradient row (a backward projection that adds clears it).
uint32_t* live_list(gs_workspace* ws) {
  return at<uint32_t>(ws, L_OFFSETS) + ws->n_cap + emit_run_table(ws->pair_cap);
}
uint32_t* list_state(gs_workspace* ws) { return at<uint32_t>(ws, L_EPOCH) + 2; }

// The backward's item order, launched apart (gs_render_batch runs it beside the loss).
int item_order_stage(gs_workspace* ws, cudaStream_t st) {
  GS_CUDA(launch_item_order(at<uint32_t>(ws, L_ORDER), at<uint32_t>(ws, L_ITEM_COST),
                            at<Header>(ws, L_HDR), at<uint32_t>(ws, L_BWD_ITEMS), st),
          "item order kernel");
  return GS_OK;
}

}  // namespace

int gs_bin(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts, gs_stream_t stream) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (ws->chunked)
    return fail(GS_ERR_INVALID_ARG,
                "memory-efficiency mode: bin and blend through gs_raster_forward / gs_raster_backward");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rc = bin_count_stage(ws, st);
  if (rc) return rc;
  return bin_chunk_stage(ws, cam, opts, 0u, 0u, st);
}

int gs_blend_forward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                     float* image, void* state, uint32_t* last, uint32_t* n_contrib,
                     gs_stream_t stream) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (ws->chunked)
    return fail(GS_ERR_INVALID_ARG, "memory-efficiency mode: use gs_raster_forward");
  const size_t npix = (size_t)cam->width * cam->height;
  if (npix > 0 && (!state || !last)) return fail(GS_ERR_INVALID_ARG, "state and last are required");
  return raster_fwd_stage(ws, cam, opts, image, state, last, n_contrib, 0,
                          reinterpret_cast<cudaStream_t>(stream));
}

int gs_raster_forward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                      float* image, void* state, uint32_t* last, uint32_t* n_contrib,
                      gs_stream_t stream) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  const size_t npix = (size_t)cam->width * cam->height;
  if (npix > 0 && (!state || !last)) return fail(GS_ERR_INVALID_ARG, "state and last are required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!ws->chunked) {
    rc = gs_bin(ws, cam, opts, stream);
    if (rc) return rc;
    return gs_blend_forward(ws, cam, opts, image, state, last, n_contrib, stream);
  }
  // memory-efficiency mode: chunks of the depth order, front to back, each
  // pixel resuming from the state the previous chunk stored
  rc = bin_count_stage(ws, st);
  if (rc) return rc;
  uint32_t n_chunks = 0, B = 0;
  rc = count_chunks(ws, cam, st, &n_chunks, &B);
  if (rc) return rc;
  ws->n_chunks = (int32_t)n_chunks;
  for (uint32_t k = 0; k < n_chunks; ++k) {
    rc = bin_chunk_stage(ws, cam, opts, k, B, st, -1, k == 0);
    if (!rc) rc = raster_fwd_stage(ws, cam, opts, image, state, last, n_contrib, k > 0, st, k);
    if (rc) return rc;
  }
  return GS_OK;
}

int gs_blend_backward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                      const void* state, const uint32_t* last, const float* dL_dimage,
                      gs_stream_t stream) {
  return blend_backward_impl(ws, cam, opts, state, last, dL_dimage, stream, 0);
}

}  // extern "C"

namespace {
// gs_project_backward; store_grads: write the visible splats' rows (zeros where
// they have no gradient) instead of adding to them.
int project_backward_impl(gs_workspace* ws, const float* means, const float* scales,
                          const float* quats, const float* opacities, const float* sh, int32_t n,
                          const gs_camera* cam, const gs_raster_opts* opts, float* d_means,
                          float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                          gs_stream_t stream, int store_grads) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (n != ws->n) return fail(GS_ERR_INVALID_ARG, "n differs from the one gs_project was given");
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh || !d_means || !d_scales ||
                !d_quats || !d_opacities || !d_sh))
    return fail(GS_ERR_INVALID_ARG, "null parameter or gradient pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* ls = list_state(ws);
  if (store_grads) {
    // with a valid list, the rows the last store-mode view wrote are the only
    // non-zero ones: zero them, then start this view's list
    GS_CUDA(launch_zero_listed(ws->n, ws->sh_degree, live_list(ws), ls, d_means, d_scales, d_quats,
                               d_opacities, d_sh, num_sms(), st),
            "listed-rows zeroing kernel");
    GS_CUDA(cudaMemsetAsync(ls, 0, sizeof(uint32_t), st), "list count reset");
  }
  GS_CUDA(launch_project_bwd(means, scales, quats, opacities, sh, ws->n, ws->sh_degree, *cam,
                             ws->clamp01, at<uint32_t>(ws, L_VB), at<float>(ws, L_G2D),
                             at<Header>(ws, L_HDR), d_means, d_scales, d_quats, d_opacities, d_sh,
                             num_sms(), st, store_grads, live_list(ws), ls),
          "projection backward kernel");
  // store: the list now holds every row this view wrote (an adding backward
  // marks it invalid itself)
  if (store_grads) GS_CUDA(launch_set_word(ls + 1, 1u, st), "list state");
  return GS_OK;
}
}  // namespace

extern "C" {

int gs_project_backward(gs_workspace* ws, const float* means, const float* scales,
                        const float* quats, const float* opacities, const float* sh, int32_t n,
                        const gs_camera* cam, const gs_raster_opts* opts, float* d_means,
                        float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                        gs_stream_t stream) {
  return project_backward_impl(ws, means, scales, quats, opacities, sh, n, cam, opts, d_means,
                               d_scales, d_quats, d_opacities, d_sh, stream, 0);
}

int gs_zero_touched_gradients(gs_workspace* ws, int32_t n, float* d_means, float* d_scales,
                              float* d_quats, float* d_opacities, float* d_sh,
                              gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  if (n != ws->n) return fail(GS_ERR_INVALID_ARG, "n differs from the one gs_project was given");
  if (n > 0 && (!d_means || !d_scales || !d_quats || !d_opacities || !d_sh))
    return fail(GS_ERR_INVALID_ARG, "null gradient pointer");
  GS_CUDA(launch_zero_touched(ws->n, ws->sh_degree, at<uint32_t>(ws, L_VB), at<Header>(ws, L_HDR),
                              d_means, d_scales, d_quats, d_opacities, d_sh, num_sms(),
                              reinterpret_cast<cudaStream_t>(stream)),
          "gradient zeroing kernel");
  return GS_OK;
}

}  // extern "C"

namespace {
// A second stream and two events per workspace, created on first use:
// gs_render_batch runs the backward's item order on it beside the loss (a
// fork and join inside its CUDA graph).  Freed by gs_graph_release.
struct ForkRes {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_fork_mu;
std::unordered_map<const gs_workspace*, ForkRes> g_forks;

void release_fork(ForkRes& f) {
  if (f.fork) cudaEventDestroy(f.fork);
  if (f.join) cudaEventDestroy(f.join);
  if (f.side) cudaStreamDestroy(f.side);
  f = ForkRes{};
}

// The workspace's fork resources, or null (then the caller stays on one stream).
const ForkRes* fork_res(const gs_workspace* ws) {
  std::lock_guard<std::mutex> lock(g_fork_mu);
  ForkRes& f = g_forks[ws];
  if (!f.side) {
    if (cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release_fork(f);
      g_forks.erase(ws);
      return nullptr;
    }
  }
  return &f;
}

int raster_backward_impl(gs_workspace* ws, const float* means, const float* scales,
                         const float* quats, const float* opacities, const float* sh, int32_t n,
                         const gs_camera* cam, const gs_raster_opts* opts, const void* state,
                         const uint32_t* last, const float* dL_dimage, float* d_means,
                         float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                         gs_stream_t stream, int store_grads, int order_done = 0) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (n != ws->n) return fail(GS_ERR_INVALID_ARG, "n differs from the one gs_project was given");
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh || !d_means || !d_scales ||
                !d_quats || !d_opacities || !d_sh))
    return fail(GS_ERR_INVALID_ARG, "null parameter or gradient pointer");
  if (!ws->chunked) {
    rc = blend_backward_impl(ws, cam, opts, state, last, dL_dimage, stream, order_done);
  } else {
    // memory-efficiency mode: the chunks again, front to back, (C', T) carried
    // between them; the pair buffers hold one chunk, so each is binned anew
    const size_t npix = (size_t)cam->width * cam->height;
    if (npix > 0 && (!state || !last || !dL_dimage))
      return fail(GS_ERR_INVALID_ARG, "state, last and dL_dimage are required");
    const uint32_t n_chunks = (uint32_t)ws->n_chunks;
    if (n_chunks == 0) return fail(GS_ERR_INVALID_ARG, "gs_raster_forward must run first");
    int gw, gh;
    const uint32_t B = (uint32_t)(ws->pair_cap - blocks_of(cam->width, cam->height, gw, gh));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (uint32_t k = 0; k < n_chunks && !rc; ++k) {
      rc = bin_chunk_stage(ws, cam, opts, k, B, st);
      if (!rc) rc = raster_bwd_stage(ws, cam, opts, state, last, dL_dimage, k > 0, k + 1 < n_chunks, st);
    }
  }
  if (rc) return rc;
  return project_backward_impl(ws, means, scales, quats, opacities, sh, n, cam, opts, d_means,
                               d_scales, d_quats, d_opacities, d_sh, stream, store_grads);
}
}  // namespace

extern "C" {

int gs_raster_backward(gs_workspace* ws, const float* means, const float* scales,
                       const float* quats, const float* opacities, const float* sh, int32_t n,
                       const gs_camera* cam, const gs_raster_opts* opts, const void* state,
                       const uint32_t* last, const float* dL_dimage, float* d_means,
                       float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                       gs_stream_t stream) {
  return raster_backward_impl(ws, means, scales, quats, opacities, sh, n, cam, opts, state, last,
                              dL_dimage, d_means, d_scales, d_quats, d_opacities, d_sh, stream, 0);
}

int gs_raster_forward_slab(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                           int32_t slab, int32_t n_slabs, float* image, void* state,
                           uint32_t* last, uint32_t* n_contrib, gs_stream_t stream) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (ws->chunked) return fail(GS_ERR_INVALID_ARG, "depth slabs do not combine with the memory-efficiency mode");
  if (n_slabs < 1 || slab < 0 || slab >= n_slabs)
    return fail(GS_ERR_INVALID_ARG, "slab %d of %d is out of range", slab, n_slabs);
  const size_t npix = (size_t)cam->width * cam->height;
  if (npix > 0 && (!state || !last)) return fail(GS_ERR_INVALID_ARG, "state and last are required");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rc = bin_count_stage(ws, st, 1);
  if (!rc) rc = bin_chunk_stage(ws, cam, opts, (uint32_t)slab, (uint32_t)n_slabs, st, 2);
  if (!rc) rc = raster_fwd_stage(ws, cam, opts, image, state, last, n_contrib, 0, st);
  return rc;
}

int gs_raster_backward_slab(gs_workspace* ws, const float* means, const float* scales,
                            const float* quats, const float* opacities, const float* sh,
                            int32_t n, const gs_camera* cam, const gs_raster_opts* opts,
                            int32_t slab, int32_t n_slabs, const void* state, const uint32_t* last,
                            const float* t_front, const float* behind, const float* dL_dimage,
                            float* d_means, float* d_scales, float* d_quats, float* d_opacities,
                            float* d_sh, gs_stream_t stream) {
  int rc = check_bound(ws, cam, opts);
  if (rc) return rc;
  if (ws->chunked) return fail(GS_ERR_INVALID_ARG, "depth slabs do not combine with the memory-efficiency mode");
  if (n_slabs < 1 || slab < 0 || slab >= n_slabs)
    return fail(GS_ERR_INVALID_ARG, "slab %d of %d is out of range", slab, n_slabs);
  if (n != ws->n) return fail(GS_ERR_INVALID_ARG, "n differs from the one gs_project was given");
  if (n > 0 && (!means || !scales || !quats || !opacities || !sh || !d_means || !d_scales ||
                !d_quats || !d_opacities || !d_sh))
    return fail(GS_ERR_INVALID_ARG, "null parameter or gradient pointer");
  const size_t npix = (size_t)cam->width * cam->height;
  if (npix > 0 && (!state || !last || !dL_dimage))
    return fail(GS_ERR_INVALID_ARG, "state, last and dL_dimage are required");
  rc = raster_bwd_stage(ws, cam, opts, state, last, dL_dimage, 0, 0,
                        reinterpret_cast<cudaStream_t>(stream), t_front, behind);
  if (rc) return rc;
  return gs_project_backward(ws, means, scales, quats, opacities, sh, n, cam, opts, d_means,
                             d_scales, d_quats, d_opacities, d_sh, stream);
}

int gs_slab_composite(const void* states, int32_t state_format, int32_t n_slabs, int64_t npix,
                      float* image, float* trans, float* t_front, float* behind,
                      gs_stream_t stream) {
  if (state_format < 0 || state_format > 3) return fail(GS_ERR_INVALID_ARG, "bad state_format %d", state_format);
  if (n_slabs < 1) return fail(GS_ERR_INVALID_ARG, "n_slabs must be >= 1");
  if (npix < 0) return fail(GS_ERR_INVALID_ARG, "negative npix");
  if (npix > 0 && !states) return fail(GS_ERR_INVALID_ARG, "states is null");
  GS_CUDA(launch_slab_composite(states, state_format, n_slabs, npix, image, trans, t_front, behind,
                                num_sms(), reinterpret_cast<cudaStream_t>(stream)),
          "slab composite kernel");
  return GS_OK;
}

int gs_loss(const float* image, const float* target, int64_t n_values, int32_t kind,
            float* dL_dimage, double* loss, gs_stream_t stream) {
  if (kind != GS_LOSS_L1 && kind != GS_LOSS_L2) return fail(GS_ERR_INVALID_ARG, "bad loss kind %d", kind);
  if (n_values < 0) return fail(GS_ERR_INVALID_ARG, "negative n_values");
  if (!loss || (n_values > 0 && (!image || !target)))
    return fail(GS_ERR_INVALID_ARG, "null pointer");
  GS_CUDA(launch_loss(image, target, n_values, kind, dL_dimage, loss, num_sms(),
                      reinterpret_cast<cudaStream_t>(stream)),
          "loss kernel");
  return GS_OK;
}

int gs_render_batch(const gs_request* reqs, int32_t n, gs_workspace* ws, gs_stream_t stream) {
  if (n < 0 || (n > 0 && !reqs)) return fail(GS_ERR_INVALID_ARG, "bad request list");
  for (int i = 0; i < n; ++i) {
    const gs_request& q = reqs[i];
    if (q.opts.sh_degree != q.scene.sh_degree)
      return fail(GS_ERR_INVALID_ARG, "request %d: opts.sh_degree differs from the scene's", i);
    int rc = GS_OK;
    if (q.zero_touched < 0 || q.zero_touched > 2)
      return fail(GS_ERR_INVALID_ARG, "request %d: bad zero_touched %d", i, q.zero_touched);
    const bool fb = q.mode == GS_MODE_FORWARD_BACKWARD;
    const bool store = fb && q.zero_touched == 2;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // (a workspace that never projected has no previous view: nothing to zero)
    if (fb && q.zero_touched == 1 && ws->n > 0)
      rc = gs_zero_touched_gradients(ws, q.scene.n, q.d_means, q.d_scales, q.d_quats,
                                     q.d_opacities, q.d_sh, stream);
    if (!rc && store) {   // the previous view's visible count survives the projection here
      if (q.scene.n > 0 && (!q.d_means || !q.d_scales || !q.d_quats || !q.d_opacities || !q.d_sh))
        return fail(GS_ERR_INVALID_ARG, "request %d: null gradient pointer", i);
      GS_CUDA(launch_copy_word(&at<Header>(ws, L_HDR)->visible, at<uint32_t>(ws, L_EPOCH) + 1, st),
              "visible count copy");
    }
    if (!rc)
      rc = gs_project(ws, q.scene.means, q.scene.scales, q.scene.quats, q.scene.opacities,
                      q.scene.sh, q.scene.n, &q.camera, &q.opts, stream);
    if (!rc && store)   // rows of the splats that left the view (before the sort replaces the order)
      GS_CUDA(launch_zero_left(q.scene.n, q.scene.sh_degree, at<uint32_t>(ws, L_VB),
                               at<uint32_t>(ws, L_EPOCH) + 1, at<uint32_t>(ws, L_KEYS), q.d_means,
                               q.d_scales, q.d_quats, q.d_opacities, q.d_sh, num_sms(), st, list_state(ws)),
              "gradient zeroing kernel");
    if (!rc) rc = gs_sort(ws, stream);
    if (!rc) rc = gs_raster_forward(ws, &q.camera, &q.opts, q.image, q.state, q.last, q.n_contrib, stream);
    if (!rc && q.mode == GS_MODE_FORWARD_BACKWARD) {
      const int64_t nv = (int64_t)q.camera.width * q.camera.height * 3;
      // the backward's item order needs only the forward: it runs beside the loss
      const ForkRes* f = (q.loss_kind != GS_LOSS_NONE && !ws->chunked) ? fork_res(ws) : nullptr;
      if (f) {
        GS_CUDA(cudaEventRecord(f->fork, st), "fork event");
        GS_CUDA(cudaStreamWaitEvent(f->side, f->fork, 0), "fork wait");
        rc = item_order_stage(ws, f->side);
        if (rc) return rc;
        GS_CUDA(cudaEventRecord(f->join, f->side), "join event");
      }
      if (q.loss_kind != GS_LOSS_NONE) {
        if (!q.image) return fail(GS_ERR_INVALID_ARG, "request %d: a loss needs the image", i);
        rc = gs_loss(q.image, q.target, nv, q.loss_kind, q.dL_dimage, q.loss, stream);
      }
      if (f) GS_CUDA(cudaStreamWaitEvent(st, f->join, 0), "join wait");
      if (!rc)
        rc = raster_backward_impl(ws, q.scene.means, q.scene.scales, q.scene.quats,
                                  q.scene.opacities, q.scene.sh, q.scene.n, &q.camera, &q.opts,
                                  q.state, q.last, q.dL_dimage, q.d_means, q.d_scales, q.d_quats,
                                  q.d_opacities, q.d_sh, stream, store, f != nullptr);
      if (!rc && q.loss_host && q.loss_kind != GS_LOSS_NONE)
        GS_CUDA(cudaMemcpyAsync(q.loss_host, q.loss, sizeof(double), cudaMemcpyDeviceToHost,
                                reinterpret_cast<cudaStream_t>(stream)),
                "loss copy to the host");
    } else if (!rc && q.mode != GS_MODE_FORWARD) {
      return fail(GS_ERR_INVALID_ARG, "request %d: bad mode %d", i, q.mode);
    }
    if (rc) return rc;
  }
  return GS_OK;
}

namespace {
// Executable graphs of gs_render_batch_graph, one per workspace.
std::mutex g_graph_mu;
std::unordered_map<const gs_workspace*, cudaGraphExec_t> g_graphs;
}  // namespace

int gs_render_batch_graph(const gs_request* reqs, int32_t n, gs_workspace* ws,
                          gs_stream_t stream) {
  if (n < 0 || (n > 0 && !reqs)) return fail(GS_ERR_INVALID_ARG, "bad request list");
  int rc = check_ws(ws);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bool direct = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
  for (int i = 0; i < n && !direct; ++i) direct = reqs[i].opts.chunked != 0;
  if (!direct) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GS_CUDA(cudaStreamIsCapturing(st, &cs), "capture status");
    direct = cs != cudaStreamCaptureStatusNone;
  }
  if (!direct) {
    // a workspace's first call runs directly: it sets up every launch's
    // one-time host state (occupancy queries) outside any capture
    std::lock_guard<std::mutex> lock(g_graph_mu);
    if (g_graphs.find(ws) == g_graphs.end()) {
      g_graphs[ws] = nullptr;
      direct = true;
    }
  }
  if (direct) return gs_render_batch(reqs, n, ws, stream);
  // the second stream of the item-order fork is created outside the capture
  for (int i = 0; i < n; ++i)
    if (reqs[i].mode == GS_MODE_FORWARD_BACKWARD && reqs[i].loss_kind != GS_LOSS_NONE) {
      fork_res(ws);
      break;
    }
  GS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
  rc = gs_render_batch(reqs, n, ws, stream);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (rc || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (rc) return rc;
    return fail(GS_ERR_CUDA, "end capture: %s", cudaGetErrorString(ce));
  }
  std::lock_guard<std::mutex> lock(g_graph_mu);
  cudaGraphExec_t& exec = g_graphs[ws];
  if (exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();   // a failed update is not an error: rebuild
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
  }
  cudaError_t e = cudaSuccess;
  if (!exec) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    exec = nullptr;
    return fail(GS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  GS_CUDA(cudaGraphLaunch(exec, st), "graph launch");
  return GS_OK;
}

int gs_graph_release(gs_workspace* ws) {
  {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    auto it = g_graphs.find(ws);
    if (it != g_graphs.end()) {
      if (it->second) cudaGraphExecDestroy(it->second);
      g_graphs.erase(it);
    }
  }
  std::lock_guard<std::mutex> lock(g_fork_mu);
  auto f = g_forks.find(ws);
  if (f != g_forks.end()) {
    release_fork(f->second);
    g_forks.erase(f);
  }
  return GS_OK;
}

int gs_workspace_sort_bytes(const gs_workspace* ws, size_t* depth_sort, size_t* pair_sort) {
  if (!ws || !ws->base) return fail(GS_ERR_INVALID_ARG, "workspace is null or not initialised");
  if (!depth_sort || !pair_sort) return fail(GS_ERR_INVALID_ARG, "null output");
  auto span = [&](int first, int last_excl) { return (size_t)(ws->layout[last_excl] - ws->layout[first]); };
  // the look-back words serve the depth and the pair passes alike: counted with the depth sort
  *depth_sort = span(L_STATUS, L_STATUS + 1) + span(L_KEYS, L_VB + 1);
  *pair_sort = span(L_PKA, L_PVB + 1);
  return GS_OK;
}

int gs_check_status(gs_workspace* ws, gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t status = 0;
  GS_CUDA(cudaMemcpyAsync(&status, &at<Header>(ws, L_HDR)->status, 4, cudaMemcpyDeviceToHost, st),
          "status copy");
  GS_CUDA(cudaStreamSynchronize(st), "status sync");
  if (status & kStatusTimeout) return fail(GS_ERR_TIMEOUT, "a device-side look-back wait gave up");
  if (status & kStatusCapacity) {
    uint32_t want = 0;
    cudaMemcpy(&want, &at<Header>(ws, L_HDR)->pairs_wanted, 4, cudaMemcpyDeviceToHost);
    return fail(GS_ERR_CAPACITY, "%u (splat, block) pairs needed, capacity %lld", want,
                (long long)ws->pair_cap);
  }
  return GS_OK;
}

int gs_read_counters(gs_workspace* ws, int64_t* out, gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  if (!out) return fail(GS_ERR_INVALID_ARG, "out is null");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t h[5] = {0, 0, 0, 0, 0};   // status, visible, pairs, pairs_wanted, live_pairs
  GS_CUDA(cudaMemcpyAsync(h, at<Header>(ws, L_HDR), 20, cudaMemcpyDeviceToHost, st), "counter copy");
  GS_CUDA(cudaStreamSynchronize(st), "counter sync");
  int gw, gh;
  out[0] = h[1];
  out[1] = h[2];
  out[2] = h[0];
  out[3] = blocks_of(ws->width, ws->height, gw, gh);
  out[4] = h[3];
  out[5] = h[4];
  return GS_OK;
}

int gs_copy_array(gs_workspace* ws, int32_t which, void* dst, size_t bytes, gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  if (!dst && bytes) return fail(GS_ERR_INVALID_ARG, "dst is null");
  const int fin = ws->pair_passes & 1;
  int slot;
  size_t cap;
  int gw, gh;
  switch (which) {
    case GS_ARRAY_SORTED_IDS: slot = L_VB; cap = (size_t)ws->n_cap * 4; break;
    case GS_ARRAY_DEPTH_KEYS: slot = L_KEYS; cap = (size_t)ws->n_cap * 4; break;
    case GS_ARRAY_RECORDS: slot = L_REC; cap = (size_t)ws->n_cap * sizeof(SplatRec); break;
    case GS_ARRAY_PAIR_BLOCKS: slot = fin ? L_PKB : L_PKA; cap = (size_t)ws->pair_cap * 4; break;
    case GS_ARRAY_PAIR_RANKS: slot = fin ? L_PVB : L_PVA; cap = (size_t)ws->pair_cap * 4; break;
    case GS_ARRAY_RANGES: slot = L_RANGES; cap = (size_t)blocks_of(ws->width_cap, ws->height_cap, gw, gh) * 8; break;
    case GS_ARRAY_GRAD2D: slot = L_G2D; cap = (size_t)ws->n_cap * 48; break;
    case GS_ARRAY_BOXES: slot = L_BOXES; cap = (size_t)ws->n_cap * 8; break;
    default: return fail(GS_ERR_INVALID_ARG, "unknown array %d", which);
  }
  if (bytes > cap) return fail(GS_ERR_INVALID_ARG, "asked for %zu bytes, array holds %zu", bytes, cap);
  GS_CUDA(cudaMemcpyAsync(dst, at<char>(ws, slot), bytes, cudaMemcpyDeviceToDevice,
                          reinterpret_cast<cudaStream_t>(stream)),
          "array copy");
  return GS_OK;
}

int gs_sort_pairs(gs_workspace* ws, const uint32_t* keys_in, const uint32_t* vals_in,
                  uint32_t* keys_out, uint32_t* vals_out, int32_t n, int32_t key_bits,
                  gs_stream_t stream) {
  int rc = check_ws(ws);
  if (rc) return rc;
  if (n < 0 || n > ws->n_cap) return fail(GS_ERR_INVALID_ARG, "n = %d exceeds the capacity %d", n, ws->n_cap);
  if (key_bits < 1 || key_bits > 32) return fail(GS_ERR_INVALID_ARG, "key_bits must be in [1, 32]");
  if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out)) return fail(GS_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Header* hdr = at<Header>(ws, L_HDR);
  uint32_t* epoch = at<uint32_t>(ws, L_EPOCH);
  const int passes = (key_bits + 7) / 8;
  GS_CUDA(cudaMemsetAsync(hdr, 0, sizeof(Header), st), "sort memset");
  GS_CUDA(launch_bump_epoch(epoch, st), "epoch kernel");
  GS_CUDA(launch_digit_hist(keys_in, (uint32_t)n, passes, &hdr->depth_hist[0][0], num_sms(), st), "histogram kernel");
  uint32_t* bk[2] = {at<uint32_t>(ws, L_KA), at<uint32_t>(ws, L_KB)};
  uint32_t* bv[2] = {at<uint32_t>(ws, L_VA), at<uint32_t>(ws, L_VB)};
  const int grid_cap = num_sms() * kPersistentPerSm;
  for (int p = 0; p < passes; ++p) {
    const uint32_t* kin = p == 0 ? keys_in : bk[(p + 1) & 1];
    const uint32_t* vin = p == 0 ? vals_in : bv[(p + 1) & 1];
    uint32_t* kout = p == passes - 1 ? keys_out : bk[p & 1];
    uint32_t* vout = p == passes - 1 ? vals_out : bv[p & 1];
    const uint32_t mask = 0xFFu;
    GS_CUDA(launch_onesweep_pass(kin, vin, kout, vout, nullptr, (uint32_t)n, (uint32_t)n, (uint32_t)n,
                                 8 * p, mask, hdr->depth_hist[p], at<unsigned long long>(ws, L_STATUS),
                                 &hdr->tile_counter[9 + p], epoch, 8u + p, &hdr->status, 0,
                                 grid_cap, st, kSpinLimit, n >= (1 << 22)),
            "sort pass");
  }
  return GS_OK;
}

int gs_test_stalled_sort(gs_workspace* ws, const uint32_t* keys_in, const uint32_t* vals_in,
                         uint32_t* keys_out, uint32_t* vals_out, int32_t n, uint32_t spin_limit,
                         gs_stream_t stream) {
  if (spin_limit < 1 || spin_limit > kSpinLimit)
    return fail(GS_ERR_INVALID_ARG, "spin_limit must be in [1, %u]", kSpinLimit);
  if (!keys_in || !vals_in || !keys_out || !vals_out) return fail(GS_ERR_INVALID_ARG, "null pointer");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (!ws) return noalloc_stalled_pass(keys_in, vals_in, keys_out, vals_out, n, spin_limit, st);
  int rc = check_ws(ws);
  if (rc) return rc;
  if (n <= 2048) return fail(GS_ERR_INVALID_ARG, "n must span at least two sort tiles (> 2048)");
  if (n > ws->n_cap) return fail(GS_ERR_INVALID_ARG, "n = %d exceeds the capacity %d", n, ws->n_cap);
  Header* hdr = at<Header>(ws, L_HDR);
  uint32_t* epoch = at<uint32_t>(ws, L_EPOCH);
  GS_CUDA(cudaMemsetAsync(hdr, 0, sizeof(Header), st), "sort memset");
  GS_CUDA(launch_bump_epoch(epoch, st), "epoch kernel");
  GS_CUDA(launch_digit_hist(keys_in, (uint32_t)n, 1, &hdr->depth_hist[0][0], num_sms(), st), "histogram kernel");
  // tile 0 withheld: CTAs take tiles from 1 on, so no CTA publishes tile 0
  GS_CUDA(launch_set_word(&hdr->tile_counter[9], 1u, st), "tile counter");
  GS_CUDA(launch_onesweep_pass(keys_in, vals_in, keys_out, vals_out, nullptr, (uint32_t)n,
                               (uint32_t)n, (uint32_t)n, 0, 0xFFu, hdr->depth_hist[0],
                               at<unsigned long long>(ws, L_STATUS), &hdr->tile_counter[9], epoch,
                               8u, &hdr->status, 0, num_sms() * kPersistentPerSm, st, spin_limit),
          "stalled sort pass");
  return GS_OK;
}

}  // extern "C"

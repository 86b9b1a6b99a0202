// Allocation-free variant of the standalone pair sort.
//
// Its scratch (header with tile counters and digit histograms, the look-back
// status words, an epoch word and the ping-pong key/value buffers) lives in
// one file-scope device array of fixed size instead of a caller-provided
// workspace, so the call needs no device memory beyond its inputs and outputs.
// Every GPU that loads the library holds the array until the process exits.
#include <mutex>

#include "common.cuh"

namespace gsr {

cudaError_t launch_onesweep_pass(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*,
                                 const uint32_t*, uint32_t, uint32_t, uint32_t, int, uint32_t,
                                 const uint32_t*, unsigned long long*, uint32_t*, const uint32_t*,
                                 uint32_t, uint32_t*, int, int, cudaStream_t,
                                 uint32_t spin_limit = kSpinLimit, int wide = 0);
cudaError_t launch_set_word(uint32_t*, uint32_t, cudaStream_t);
cudaError_t launch_digit_hist(const uint32_t*, uint32_t, int, uint32_t*, int, cudaStream_t);
cudaError_t launch_bump_epoch(uint32_t*, cudaStream_t);
size_t sort_tiles(size_t n);
int record_error(int code, const char* msg);  // sets gs_last_error() (api.cu)

namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Layout of the static scratch (byte offsets).
constexpr size_t kOffHeader = 0;
constexpr size_t kOffEpoch = align_up(kOffHeader + sizeof(Header));
constexpr size_t kOffStatus = kOffEpoch + kAlign;
constexpr int kSortTileSize = 2048;   // keys per onesweep tile (sort.cu)
constexpr size_t kMaxTiles = (GS_SORT_NOALLOC_MAX_PAIRS + kSortTileSize - 1) / kSortTileSize;
constexpr size_t kOffKeysA = align_up(kOffStatus + kMaxTiles * 256 * sizeof(unsigned long long));
constexpr size_t kBuf = align_up((size_t)GS_SORT_NOALLOC_MAX_PAIRS * 4);
constexpr size_t kOffValsA = kOffKeysA + kBuf;
constexpr size_t kOffKeysB = kOffValsA + kBuf;
constexpr size_t kOffValsB = kOffKeysB + kBuf;
constexpr size_t kScratchBytes = kOffValsB + kBuf;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[64] = {nullptr};

int noalloc_fail(int code, const char* msg) { return record_error(code, msg); }

// Device address of the array on the current device.  It is looked up on every
// call (a cheap query): after cudaDeviceReset the next context may place the
// array elsewhere.  Whenever the address differs from the one this device had
// (the first call on the device, or a new context at a new address), the array
// is zeroed on `st` ahead of the call's kernels, since the look-back words and
// the epoch must start at zero.  A new context that reuses the old address
// needs no zeroing: loading the module into it zero-fills the array.
cudaError_t scratch_for_current_device(cudaStream_t st, unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_sort_scratch);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev] != p) {
    e = cudaMemsetAsync(p, 0, kScratchBytes, st);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// GS_OK when `ptr` is device memory of the current device (or memory every
// device can reach), else GS_ERR_INVALID_ARG with a message.
int check_on_current_device(const void* ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, "cudaGetDevice failed");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(GS_ERR_INVALID_ARG, "keys_in is not a CUDA pointer");
  }
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
    return noalloc_fail(GS_ERR_INVALID_ARG,
                        "keys_in lives on another device than the current one; make that device current");
  if (attr.type == cudaMemoryTypeUnregistered || attr.type == cudaMemoryTypeHost)
    return noalloc_fail(GS_ERR_INVALID_ARG, "keys_in is host memory; pass device memory");
  return GS_OK;
}

struct Scratch {
  Header* hdr;
  uint32_t* epoch;
  unsigned long long* status;
  uint32_t* bk[2];
  uint32_t* bv[2];
};

Scratch carve(unsigned char* base) {
  Scratch s;
  s.hdr = reinterpret_cast<Header*>(base + kOffHeader);
  s.epoch = reinterpret_cast<uint32_t*>(base + kOffEpoch);
  s.status = reinterpret_cast<unsigned long long*>(base + kOffStatus);
  s.bk[0] = reinterpret_cast<uint32_t*>(base + kOffKeysA);
  s.bk[1] = reinterpret_cast<uint32_t*>(base + kOffKeysB);
  s.bv[0] = reinterpret_cast<uint32_t*>(base + kOffValsA);
  s.bv[1] = reinterpret_cast<uint32_t*>(base + kOffValsB);
  return s;
}

int current_sms() {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

// The first pass of the allocation-free sort with tile 0 withheld (the
// bounded-wait self-test, gs_test_stalled_sort with no workspace).
int noalloc_stalled_pass(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                         uint32_t* vals_out, int32_t n, uint32_t spin_limit, cudaStream_t st) {
  if (n <= kSortTileSize || n > GS_SORT_NOALLOC_MAX_PAIRS)
    return noalloc_fail(GS_ERR_INVALID_ARG, "n must span at least two tiles and fit the array");
  unsigned char* base = nullptr;
  cudaError_t e = scratch_for_current_device(st, &base);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  Scratch s = carve(base);
  const int sms = current_sms();
  e = cudaMemsetAsync(s.hdr, 0, sizeof(Header), st);
  if (e == cudaSuccess) e = launch_bump_epoch(s.epoch, st);
  if (e == cudaSuccess) e = launch_digit_hist(keys_in, (uint32_t)n, 1, &s.hdr->depth_hist[0][0], sms, st);
  if (e == cudaSuccess) e = launch_set_word(&s.hdr->tile_counter[9], 1u, st);
  if (e == cudaSuccess)
    e = launch_onesweep_pass(keys_in, vals_in, keys_out, vals_out, nullptr, (uint32_t)n,
                             (uint32_t)n, (uint32_t)n, 0, 0xFFu, s.hdr->depth_hist[0], s.status,
                             &s.hdr->tile_counter[9], s.epoch, 8u, &s.hdr->status, 0, sms * 6, st,
                             spin_limit);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

}  // namespace gsr

using namespace gsr;

extern "C" int gs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in,
                                     uint32_t* keys_out, uint32_t* vals_out, int32_t n,
                                     int32_t key_bits, gs_stream_t stream) {
  if (n < 0) return noalloc_fail(GS_ERR_INVALID_ARG, "n must be >= 0");
  if (n > GS_SORT_NOALLOC_MAX_PAIRS)
    return noalloc_fail(GS_ERR_INVALID_ARG,
                        "n exceeds GS_SORT_NOALLOC_MAX_PAIRS (262144); use gs_sort_pairs with a workspace");
  if (key_bits < 1 || key_bits > 32) return noalloc_fail(GS_ERR_INVALID_ARG, "key_bits must be in [1, 32]");
  if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out))
    return noalloc_fail(GS_ERR_INVALID_ARG, "null pointer");
  if (n > 0) {
    const int rc = check_on_current_device(keys_in);
    if (rc) return rc;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = scratch_for_current_device(st, &base);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  Scratch s = carve(base);
  // the array keeps the previous call's contents: counters, histograms and the
  // status word restart at zero
  e = cudaMemsetAsync(s.hdr, 0, sizeof(Header), st);
  if (e == cudaSuccess) e = launch_bump_epoch(s.epoch, st);
  const int passes = (key_bits + 7) / 8;
  const int sms = current_sms();
  if (e == cudaSuccess) e = launch_digit_hist(keys_in, (uint32_t)n, passes, &s.hdr->depth_hist[0][0], sms, st);
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    const uint32_t* kin = p == 0 ? keys_in : s.bk[(p + 1) & 1];
    const uint32_t* vin = p == 0 ? vals_in : s.bv[(p + 1) & 1];
    uint32_t* kout = p == passes - 1 ? keys_out : s.bk[p & 1];
    uint32_t* vout = p == passes - 1 ? vals_out : s.bv[p & 1];
    e = launch_onesweep_pass(kin, vin, kout, vout, nullptr, (uint32_t)n, (uint32_t)n, (uint32_t)n,
                             8 * p, 0xFFu, s.hdr->depth_hist[p], s.status, &s.hdr->tile_counter[9 + p],
                             s.epoch, 8u + p, &s.hdr->status, 0, sms * 6, st);
  }
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

extern "C" int gs_sort_pairs_noalloc_status(gs_stream_t stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return noalloc_fail(GS_ERR_CUDA, "device index out of range");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    base = g_scratch_ptr[dev];
  }
  if (!base) {   // no call on this device yet: nothing to report
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
    return GS_OK;
  }
  uint32_t status = 0;
  e = cudaMemcpyAsync(&status, &carve(base).hdr->status, sizeof(status), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  if (status & kStatusTimeout)
    return noalloc_fail(GS_ERR_TIMEOUT, "a device-side look-back wait of the allocation-free sort gave up");
  return GS_OK;
}

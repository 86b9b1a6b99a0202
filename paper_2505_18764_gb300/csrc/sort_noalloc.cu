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
                                 uint32_t, uint32_t*, int, int, cudaStream_t);
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
constexpr size_t kMaxTiles = (GS_SORT_NOALLOC_MAX_PAIRS + 2047) / 2048;
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

// Device address of the array on the current device; the first call on a
// device looks it up and zeroes the array (look-back words and the epoch must
// start at zero) on `st`, ahead of that call's kernels.
cudaError_t scratch_for_current_device(cudaStream_t st, unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p, 0, kScratchBytes, st);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  cudaError_t e = scratch_for_current_device(st, &base);
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  Header* hdr = reinterpret_cast<Header*>(base + kOffHeader);
  uint32_t* epoch = reinterpret_cast<uint32_t*>(base + kOffEpoch);
  unsigned long long* status = reinterpret_cast<unsigned long long*>(base + kOffStatus);
  uint32_t* bk[2] = {reinterpret_cast<uint32_t*>(base + kOffKeysA), reinterpret_cast<uint32_t*>(base + kOffKeysB)};
  uint32_t* bv[2] = {reinterpret_cast<uint32_t*>(base + kOffValsA), reinterpret_cast<uint32_t*>(base + kOffValsB)};
  // the array keeps the previous call's contents: counters and histograms restart at zero
  e = cudaMemsetAsync(hdr, 0, sizeof(Header), st);
  if (e == cudaSuccess) e = launch_bump_epoch(epoch, st);
  const int passes = (key_bits + 7) / 8;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = launch_digit_hist(keys_in, (uint32_t)n, passes, &hdr->depth_hist[0][0], sms, st);
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    const uint32_t* kin = p == 0 ? keys_in : bk[(p + 1) & 1];
    const uint32_t* vin = p == 0 ? vals_in : bv[(p + 1) & 1];
    uint32_t* kout = p == passes - 1 ? keys_out : bk[p & 1];
    uint32_t* vout = p == passes - 1 ? vals_out : bv[p & 1];
    e = launch_onesweep_pass(kin, vin, kout, vout, nullptr, (uint32_t)n, (uint32_t)n, (uint32_t)n,
                             8 * p, 0xFFu, hdr->depth_hist[p], status, &hdr->tile_counter[9 + p],
                             epoch, 8u + p, &hdr->status, 0, sms * 6, st);
  }
  if (e != cudaSuccess) return noalloc_fail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

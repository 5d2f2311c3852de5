// wg_noalloc.cu -- wg_sort_keys_noalloc: the radix sort of wg_sort_keys for
// callers that cannot allocate device memory.
//
// Some callers run where cudaMalloc (or any allocator, PyTorch's included) is
// off limits: code inside another framework's memory arena, a plug-in that must
// not grow the process's device footprint, or a real-time path that must not
// block on the driver's allocator.  This entry point takes the caller's key
// buffer and a stream and nothing else: everything the sort needs besides the
// keys -- the stage records, the digit histograms, the decoupled-lookback words
// and the ping-pong key buffer -- lives in one file-scope static device array,
// g_sort_scratch, of a fixed size.  Every GPU that loads the library holds that
// array until the process exits.
//
// Because every call shares the array, two calls whose work overlaps on the GPU
// (different streams, or different host threads, with no ordering between
// them) race and corrupt each other's results; calls on one stream, or
// otherwise ordered, are safe.  The array keeps the previous call's contents, so
// each call first clears the parts that must start at zero (histograms and
// lookback words).
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture on the device.
//
// A radix pass whose bounded lookback wait gives up marks the control block in
// the scratch (the later passes of that call then return at once, so the keys
// are left unspecified).  The call has already returned by then, so the mark is
// kept: each call's set-up kernel folds the previous control block's error
// into a sticky word before clearing it, and a call with n = 0 synchronises the
// stream, reads and clears that word and returns WG_E_DEVICE_TIMEOUT if any
// call since the last such check gave up.
#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/wg.h"
#include "wg_device.cuh"
#include "wg_launch.h"

namespace wg {

namespace {

constexpr size_t kNoAllocMaxKeys = WG_NOALLOC_MAX_KEYS;
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t b) { return (b + kAlign - 1) / kAlign * kAlign; }

// Scratch layout: stage records (the histogram's, then one per pass, in a
// region of fixed size) | Seg | Ctl | sticky error word |
// hist u64[kMaxPasses*kRadix] | status u64[(tiles+1)*kRadix] |
// ping-pong keys (8-byte keys, kNoAllocMaxKeys)
constexpr size_t kTiles = (kNoAllocMaxKeys + kTileC - 1) / kTileC;
constexpr size_t kOffStage = 0;
constexpr size_t kStageBytes = 2816;
static_assert(sizeof(Stage) * (1 + kMaxPasses) <= kStageBytes, "stage records fit their region");
constexpr size_t kOffSeg = align_up(kOffStage + kStageBytes);
constexpr size_t kOffCtl = align_up(kOffSeg + sizeof(Seg));
constexpr size_t kOffSticky = align_up(kOffCtl + sizeof(Ctl));
constexpr size_t kOffHist = align_up(kOffSticky + sizeof(uint32_t));
constexpr size_t kOffStatus = align_up(kOffHist + sizeof(unsigned long long) * kMaxPasses * kRadix);
constexpr size_t kOffKeys = align_up(kOffStatus + sizeof(unsigned long long) * (kTiles + 1) * kRadix);
constexpr size_t kScratchBytes = align_up(kOffKeys + sizeof(unsigned long long) * kNoAllocMaxKeys);
static_assert(kScratchBytes == WG_NOALLOC_SCRATCH_BYTES, "the header states the scratch size");

}  // namespace

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices];  // device address of g_sort_scratch, per device

// Writes the stage records of one sort into the scratch and clears the
// histograms and lookback words: everything the sort reads before it writes.
__global__ void k_noalloc_setup(unsigned char* base, void* keys, unsigned long long n,
                                uint32_t passes, uint32_t dbits, uint32_t ntiles) {
  const size_t nzero_h = (size_t)kMaxPasses * kRadix;
  const size_t nzero_s = (size_t)(ntiles + 1) * kRadix;
  unsigned long long* hist = (unsigned long long*)(base + kOffHist);
  unsigned long long* status = (unsigned long long*)(base + kOffStatus);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nzero_h + nzero_s;
       i += (size_t)gridDim.x * blockDim.x) {
    if (i < nzero_h) hist[i] = 0;
    else status[i - nzero_h] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Stage* st = (Stage*)(base + kOffStage);
    Seg* sg = (Seg*)(base + kOffSeg);
    Ctl* ctl = (Ctl*)(base + kOffCtl);
    *(uint32_t*)(base + kOffSticky) |= ctl->error;  // kept until a call with n = 0 reads it
    *ctl = Ctl{};
    Seg s{};
    s.n = n; s.ntiles = ntiles;
    *sg = s;
    Stage h{};
    h.segs = sg; h.ctl = ctl; h.status = status; h.hist = hist;
    h.nseg = 1; h.ntiles = ntiles; h.in = keys; h.passes = passes; h.dbits = dbits;
    st[0] = h;
    void* buf[2] = {keys, base + kOffKeys};
    for (uint32_t p = 0; p < passes; ++p) {
      Stage x = h;
      x.in = buf[p & 1]; x.out = buf[(p + 1) & 1];
      // a distinct epoch per pass; the words were just cleared to epoch 0
      x.shift = p * dbits; x.pass = p; x.epoch = 1 + p;
      st[1 + p] = x;
    }
  }
}

int scratch_of(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return set_error(WG_E_INVAL, "device index out of range");
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p)
      return set_error(WG_E_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return WG_OK;
}

// n = 0: did a call since the last check give up a device wait?  Reads the
// sticky word and the last call's control block after the stream's earlier
// work, then clears both.
int noalloc_check(cudaStream_t s, int dev) {
  unsigned char* base = nullptr;
  int rc = scratch_of(dev, &base);
  if (rc != WG_OK) return rc;
  uint32_t sticky = 0, err = 0;
  cudaError_t e = cudaMemcpyAsync(&sticky, base + kOffSticky, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&err, base + kOffCtl + offsetof(Ctl, error), 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && (sticky || err)) {
    e = cudaMemsetAsync(base + kOffSticky, 0, 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffCtl, 0, sizeof(Ctl), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  if (sticky || err) return set_error(WG_E_DEVICE_TIMEOUT, "an earlier allocation-free sort gave up a device wait");
  return WG_OK;
}

template <typename K>
int sort_noalloc(K* keys, size_t n, uint32_t bits, cudaStream_t s, int dev) {
  unsigned char* base = nullptr;
  int rc = scratch_of(dev, &base);
  if (rc != WG_OK) return rc;
  if (n <= 1) return WG_OK;
  const uint32_t passes = (bits + 7) / 8, dbits = (bits + passes - 1) / passes;
  const uint32_t ntiles = (uint32_t)((n + kTileC - 1) / kTileC);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_noalloc_setup<<<64, 256, 0, s>>>(base, keys, n, passes, dbits, ntiles);
  Stage* st = (Stage*)(base + kOffStage);
  launch_sort_hist<K>(st, sms * std::max(1, occupancy_sort<K>(0)), s);
  for (uint32_t p = 0; p < passes; ++p)
    launch_sort_pass<K>(st + 1 + p, sms * std::max(1, occupancy_sort<K>(1)), s, dbits);
  if (passes & 1) {
    const cudaError_t e = cudaMemcpyAsync(keys, base + kOffKeys, n * sizeof(K),
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  return WG_OK;
}

}  // namespace

// Self-test of the bounded wait in the allocation-free sort's control block:
// the scan stages' lookback wait on a status word of the scratch that nothing
// publishes.  The wait gives up, records DEV_TIMEOUT in the scratch's control
// block and returns; the next check (a call with n = 0) reports it.
int noalloc_selftest_wait(cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  unsigned char* base = nullptr;
  const int rc = scratch_of(dev, &base);
  if (rc != WG_OK) return rc;
  unsigned long long* status = (unsigned long long*)(base + kOffStatus);
  e = cudaMemsetAsync(status, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffCtl, 0, sizeof(Ctl), s);
  if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  launch_selftest_wait(status, (Ctl*)(base + kOffCtl), (unsigned long long*)(base + kOffHist), s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? WG_OK : set_error(WG_E_CUDA, cudaGetErrorString(e));
}

}  // namespace wg

extern "C" int wg_sort_keys_noalloc(void* d_keys, size_t n, int key_bytes, uint32_t bits,
                                    void* cuda_stream) {
  using namespace wg;
  if ((n && !d_keys) || (key_bytes != 4 && key_bytes != 8) || bits == 0 ||
      bits > 8u * (uint32_t)key_bytes)
    return set_error(WG_E_INVAL, "bad argument");
  if (n == 0) {
    int dev = 0;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
    return noalloc_check((cudaStream_t)cuda_stream, dev);
  }
  if (n > kNoAllocMaxKeys)
    return set_error(WG_E_CAPACITY, ("wg_sort_keys_noalloc sorts at most " +
                                     std::to_string(kNoAllocMaxKeys) + " keys, got " +
                                     std::to_string(n)).c_str());
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(WG_E_CUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  return key_bytes == 4 ? sort_noalloc<uint32_t>((uint32_t*)d_keys, n, bits, s, dev)
                        : sort_noalloc<unsigned long long>((unsigned long long*)d_keys, n, bits, s, dev);
}

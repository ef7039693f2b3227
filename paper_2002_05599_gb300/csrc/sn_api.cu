// C ABI of libsmallsort.so (declared in include/smallsort.h): argument
// checks, per-device state, stream-ordered scratch and the device status word.
#include <atomic>
#include <cstdint>
#include <mutex>

#include "smallsort.h"
#include "smallsort_testing.h"
#include "sn_common.cuh"
#include "sn_internal.h"
#include "sn_seg_scratch.h"

namespace sn {

// Per-device control block: the status word OR-ed by kernels (kStatusRange,
// kStatusTimeout, ...), the test flags and the limit of every bounded wait.
__device__ DevCtl g_ctl = {0u, 0u, kDefaultWaitLimitNs};

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_init_mu;
DeviceInfo g_info[kMaxDevices];
std::atomic<bool> g_ready[kMaxDevices];

int init_device(int dev, DeviceInfo* out) {
  DeviceInfo d;
  d.device = dev;
  if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SN_ECUDA;
  if (cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return SN_ECUDA;
  if (cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return SN_ECUDA;
  if (d.cc_major != 10 || d.cc_minor != 3) return SN_EUNSUPPORTED;  // built for sm_103a only
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_ctl) != cudaSuccess) return SN_EUNSUPPORTED;
  d.status = &static_cast<DevCtl*>(p)->status;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&d.pool, &props) != cudaSuccess) return SN_ECUDA;
  uint64_t keep = ~0ull;  // keep freed scratch in the pool between calls
  cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep);
  *out = d;
  return SN_OK;
}

cudaError_t clear_status(const DeviceInfo& d, cudaStream_t s) {
  return cudaMemsetAsync(d.status, 0, sizeof(unsigned), s);
}

}  // namespace

const DeviceInfo* device_info(int* err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *err = SN_ECUDA;
    return nullptr;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *err = SN_EUNSUPPORTED;
    return nullptr;
  }
  if (!g_ready[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_init_mu);
    if (!g_ready[dev].load(std::memory_order_relaxed)) {
      const int rc = init_device(dev, &g_info[dev]);
      if (rc != SN_OK) {
        *err = rc;
        return nullptr;
      }
      g_ready[dev].store(true, std::memory_order_release);
    }
  }
  *err = SN_OK;
  return &g_info[dev];
}

int status_from_word(unsigned word) {
  if (word & kStatusRange) return SN_ERANGE;
  if (word & kStatusTimeout) return SN_ETIMEOUT;
  if (word & (kStatusInternal | kCheckStageMoved | kCheckCopyArgs | kCheckSegment)) return SN_ECUDA;
  return SN_OK;
}

}  // namespace sn

namespace {

template <class K>
int fixed_entry(K* keys, int n, uint64_t count, int family, sn_stream_t stream,
                cudaError_t (*launch)(K*, int, uint64_t, int, cudaStream_t, const sn::DeviceInfo&)) {
  if (n < 2 || n > 16) return SN_EINVAL;
  if (family != SN_NETWORK_BEST && family != SN_NETWORK_BOSE_NELSON) return SN_EINVAL;
  if (count == 0) return SN_OK;
  if (keys == nullptr) return SN_EINVAL;
  if (count > (1ull << 62) / static_cast<uint64_t>(n)) return SN_ERANGE;
  if (reinterpret_cast<uintptr_t>(keys) % (sizeof(K) < 8 ? sizeof(K) : 8) != 0) return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  return launch(keys, n, count, family, reinterpret_cast<cudaStream_t>(stream), *d) == cudaSuccess ? SN_OK
                                                                                                  : SN_ECUDA;
}

template <class K>
int segments_entry(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream,
                   sn::SegMode mode,
                   cudaError_t (*launch)(K*, uint32_t*, const uint32_t*, uint64_t, sn::SegMode, void*, size_t,
                                         const sn::SegTuning&, cudaStream_t, const sn::DeviceInfo&)) {
  if (nseg == 0) return SN_OK;
  if (keys == nullptr || offsets == nullptr) return SN_EINVAL;
  if (nseg >= (1ull << 32)) return SN_ERANGE;  // segment indices are 32-bit
  if (reinterpret_cast<uintptr_t>(keys) % sizeof(K) != 0 || reinterpret_cast<uintptr_t>(offsets) % 4 != 0 ||
      reinterpret_cast<uintptr_t>(vals) % 4 != 0)
    return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const sn::SegTuning tun = sn::current_tuning(d->device, static_cast<int>(sizeof(K)), vals != nullptr);
  const size_t bytes = sn::segments_scratch_bytes(nseg, tun);
  void* scratch = nullptr;
  // Under stream capture the scratch comes from the device's default pool, so
  // that the graph records an allocation node it owns; otherwise from the
  // library's pool, which keeps freed scratch for the next call.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return SN_ECUDA;
  }
  const cudaError_t ae = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(&scratch, bytes, s)
                                                              : cudaMallocFromPoolAsync(&scratch, bytes, d->pool, s);
  if (ae != cudaSuccess) {
    cudaGetLastError();
    return SN_ENOMEM;
  }
  const cudaError_t e = launch(keys, vals, offsets, nseg, mode, scratch, bytes, tun, s, *d);
  cudaFreeAsync(scratch, s);
  return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

template <class K>
int large_entry(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream,
                cudaError_t (*launch)(K*, uint32_t*, const uint32_t*, const uint32_t*, uint64_t, void*,
                                      cudaStream_t, const sn::DeviceInfo&)) {
  if (nseg == 0) return SN_OK;
  if (keys == nullptr || offsets == nullptr) return SN_EINVAL;
  if (nseg >= (1ull << 32)) return SN_ERANGE;
  if (reinterpret_cast<uintptr_t>(keys) % sizeof(K) != 0 || reinterpret_cast<uintptr_t>(offsets) % 4 != 0 ||
      reinterpret_cast<uintptr_t>(vals) % 4 != 0)
    return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return SN_ECUDA;
  }
  const cudaError_t ae = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(&scratch, 256, s)
                                                              : cudaMallocFromPoolAsync(&scratch, 256, d->pool, s);
  if (ae != cudaSuccess) {
    cudaGetLastError();
    return SN_ENOMEM;
  }
  const cudaError_t e = launch(keys, vals, offsets, offsets + 1, nseg, scratch, s, *d);
  cudaFreeAsync(scratch, s);
  return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

}  // namespace

namespace sn {

size_t segments_scratch_bytes(uint64_t nseg, const SegTuning& t) {
  // the window kernel (tile_mode 2) needs only the validation word
  return t.tile_mode == 2 ? 256 : seg::ScratchLayout(nseg, static_cast<uint32_t>(t.tile_units)).total;
}

}  // namespace sn

extern "C" {

int sn_sort_fixed(uint32_t* keys, int n, uint64_t count, sn_stream_t stream) {
  return fixed_entry<uint32_t>(keys, n, count, SN_NETWORK_BEST, stream, sn::launch_fixed_u32);
}

int sn_sort_fixed_u64(uint64_t* keys, int n, uint64_t count, sn_stream_t stream) {
  return fixed_entry<uint64_t>(keys, n, count, SN_NETWORK_BEST, stream, sn::launch_fixed_u64);
}

int sn_sort_fixed_family(uint32_t* keys, int n, uint64_t count, int family, sn_stream_t stream) {
  return fixed_entry<uint32_t>(keys, n, count, family, stream, sn::launch_fixed_u32);
}

int sn_sort_fixed_items(sn_item64* items, int n, uint64_t count, int family, sn_stream_t stream) {
  return fixed_entry<sn_item64>(items, n, count, family, stream, sn::launch_fixed_items);
}

int sn_sort_fixed_f32(float* keys, int n, uint64_t count, sn_stream_t stream) {
  return fixed_entry<float>(keys, n, count, SN_NETWORK_BEST, stream, sn::launch_fixed_f32);
}

int sn_sort_fixed_f64(double* keys, int n, uint64_t count, sn_stream_t stream) {
  return fixed_entry<double>(keys, n, count, SN_NETWORK_BEST, stream, sn::launch_fixed_f64);
}

int sn_sort_segments(uint32_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream) {
  return segments_entry<uint32_t>(keys, vals, offsets, nseg, stream, sn::SegMode::kNetworkWarpRss,
                                  sn::launch_segments_u32);
}

int sn_sort_segments_u64(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                         sn_stream_t stream) {
  return segments_entry<uint64_t>(keys, vals, offsets, nseg, stream, sn::SegMode::kNetworkWarpRss,
                                  sn::launch_segments_u64);
}

int sn_sort_segments_f32(float* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream) {
  return segments_entry<float>(keys, vals, offsets, nseg, stream, sn::SegMode::kNetworkWarpRss,
                               sn::launch_segments_f32);
}

int sn_sort_segments_f64(double* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream) {
  return segments_entry<double>(keys, vals, offsets, nseg, stream, sn::SegMode::kNetworkWarpRss,
                                sn::launch_segments_f64);
}

int sn_sort_segments_large(uint32_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                           sn_stream_t stream) {
  return large_entry<uint32_t>(keys, vals, offsets, nseg, stream, sn::launch_large_u32);
}

int sn_sort_segments_large_u64(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                               sn_stream_t stream) {
  return large_entry<uint64_t>(keys, vals, offsets, nseg, stream, sn::launch_large_u64);
}

int sn_sort_large(uint32_t* keys, uint64_t n, sn_stream_t stream) {
  if (n <= 1) return SN_OK;
  if (keys == nullptr) return SN_EINVAL;
  if (n >= (1ull << 32)) return SN_ERANGE;
  if (reinterpret_cast<uintptr_t>(keys) % 4 != 0) return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const cudaError_t e = sn::sort_large_u32(keys, n, reinterpret_cast<cudaStream_t>(stream), *d);
  if (e == cudaErrorMemoryAllocation) return SN_ENOMEM;
  return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

int rss_sort_segments(uint32_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, sn_stream_t stream) {
  return segments_entry<uint32_t>(keys, vals, offsets, nseg, stream, sn::SegMode::kRssOnly,
                                  sn::launch_segments_u32);
}

int rss_sort_segments_u64(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                          sn_stream_t stream) {
  return segments_entry<uint64_t>(keys, vals, offsets, nseg, stream, sn::SegMode::kRssOnly,
                                  sn::launch_segments_u64);
}

namespace {
std::atomic<unsigned> g_last_word{0};
}

// Raw device status word seen by the latest sn_check (diagnostics; not part
// of the public interface).
unsigned sn_debug_status_word(void) { return g_last_word.load(); }

namespace {
int status_of_word(unsigned word) { return sn::status_from_word(word); }
}  // namespace

int sn_check(sn_stream_t stream) {
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return SN_ECUDA;
  unsigned word = 0;
  if (cudaMemcpyAsync(&word, d->status, sizeof(word), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SN_ECUDA;
  if (sn::clear_status(*d, s) != cudaSuccess) return SN_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SN_ECUDA;
  g_last_word.store(word);
  return status_of_word(word);
}

int sn_get_last_cuda_error(void) {
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  // every stream of the device: errors of earlier asynchronous calls surface here
  if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) return SN_ECUDA;
  unsigned word = 0;
  if (cudaMemcpy(&word, d->status, sizeof(word), cudaMemcpyDeviceToHost) != cudaSuccess) return SN_ECUDA;
  if (cudaMemset(d->status, 0, sizeof(word)) != cudaSuccess) return SN_ECUDA;
  g_last_word.store(word);
  return status_of_word(word);
}

int sn_set_wait_limit(uint64_t ns) {
  if (ns < 1000ull || ns > 60000000000ull) return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const unsigned long long v = ns;
  sn::DevCtl* ctl = reinterpret_cast<sn::DevCtl*>(d->status);
  return cudaMemcpy(&ctl->wait_limit_ns, &v, sizeof(v), cudaMemcpyHostToDevice) == cudaSuccess ? SN_OK : SN_ECUDA;
}

int sn_test_set_flags(unsigned flags) {
  if (flags & ~(sn::kTestSkipFixedCopy | sn::kTestSkipTileCopy | sn::kTestSkipRssCopy)) return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  sn::DevCtl* ctl = reinterpret_cast<sn::DevCtl*>(d->status);
  return cudaMemcpy(&ctl->test_flags, &flags, sizeof(flags), cudaMemcpyHostToDevice) == cudaSuccess ? SN_OK
                                                                                                   : SN_ECUDA;
}

const char* sn_status_string(int status) {
  switch (status) {
    case SN_OK: return "ok";
    case SN_EINVAL: return "invalid argument";
    case SN_ERANGE: return "size or offsets out of range";
    case SN_ENOMEM: return "device scratch allocation failed";
    case SN_ECUDA: return "CUDA error";
    case SN_ETIMEOUT: return "bounded device wait timed out";
    case SN_EUNSUPPORTED: return "device not supported (needs sm_103)";
    default: return "unknown status";
  }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Segmented sort without any allocation (sn_sort_segments_u64_noalloc).
//
// Some callers cannot allocate device memory at the moment they sort: code
// running on a fixed device-memory budget that was reserved up front, hosts
// whose allocator must not be entered from the sorting thread (a real-time
// loop, a callback that holds the allocator's lock), or frameworks that only
// hand out the buffers they manage.  This entry point serves them: its
// scratch is the file-scope array below, which every GPU that loads the
// library keeps until the process exits, so the call itself allocates
// nothing.  The kernels are the ones sn_sort_segments_u64 runs.
// ---------------------------------------------------------------------------

#include "sn_window.cuh"

namespace sn {
namespace {

constexpr uint64_t kNoAllocMaxSegments = SN_NOALLOC_MAX_SEGMENTS;
constexpr uint32_t kNoAllocTileUnits = 2048;
constexpr size_t kNoAllocScratchBytes = seg::ScratchLayout(kNoAllocMaxSegments, kNoAllocTileUnits).total;

// Shared by every call on a device; holds the last call's plan and bins.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  DeviceInfo info;
  void* scratch = nullptr;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[kMaxDevices];
std::atomic<bool> g_noalloc_ready[kMaxDevices];

// Once per device, with that device current: device facts and the device
// addresses of the scratch array and the status word (host code cannot use
// the arrays' names as device addresses).
int noalloc_setup(int dev, NoAllocDevice* out) {
  NoAllocDevice nd;
  nd.info.device = dev;
  if (cudaDeviceGetAttribute(&nd.info.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SN_ECUDA;
  if (cudaDeviceGetAttribute(&nd.info.cc_major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess)
    return SN_ECUDA;
  if (cudaDeviceGetAttribute(&nd.info.cc_minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
    return SN_ECUDA;
  if (nd.info.cc_major != 10 || nd.info.cc_minor != 3) return SN_EUNSUPPORTED;
  void* status = nullptr;
  if (cudaGetSymbolAddress(&status, g_ctl) != cudaSuccess) return SN_EUNSUPPORTED;
  nd.info.status = &static_cast<DevCtl*>(status)->status;
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess) return SN_EUNSUPPORTED;
  nd.scratch = scratch;
  *out = nd;
  return SN_OK;
}

}  // namespace
}  // namespace sn

extern "C" int sn_sort_segments_u64_noalloc(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                                            sn_stream_t stream) {
  if (nseg == 0) return SN_OK;
  if (keys == nullptr || offsets == nullptr) return SN_EINVAL;
  if (nseg > sn::kNoAllocMaxSegments) return SN_ERANGE;
  if (reinterpret_cast<uintptr_t>(keys) % 8 != 0 || reinterpret_cast<uintptr_t>(offsets) % 4 != 0 ||
      reinterpret_cast<uintptr_t>(vals) % 4 != 0)
    return SN_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SN_ECUDA;
  if (dev < 0 || dev >= sn::kMaxDevices) return SN_EUNSUPPORTED;
  if (!sn::g_noalloc_ready[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(sn::g_noalloc_mu);
    if (!sn::g_noalloc_ready[dev].load(std::memory_order_relaxed)) {
      const int rc = sn::noalloc_setup(dev, &sn::g_noalloc[dev]);
      if (rc != SN_OK) return rc;
      sn::g_noalloc_ready[dev].store(true, std::memory_order_release);
    }
  }
  const sn::NoAllocDevice& nd = sn::g_noalloc[dev];
  sn::SegTuning tun;
  tun.tile_units = static_cast<int>(sn::kNoAllocTileUnits);
  const cudaError_t e = sn::seg::launch_segments<uint64_t>(keys, vals, offsets, nseg, sn::SegMode::kNetworkWarpRss,
                                                           nd.scratch, sn::kNoAllocScratchBytes, tun,
                                                           reinterpret_cast<cudaStream_t>(stream), nd.info);
  return e == cudaSuccess ? SN_OK : SN_ECUDA;
}

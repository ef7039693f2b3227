// Internal host-side interface between the C ABI (sn_api.cu) and the kernel
// translation units.  Not installed; the public interface is smallsort.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "smallsort.h"

namespace sn {

struct DeviceInfo {
  int device = -1;
  int sm_count = 0;
  int cc_major = 0, cc_minor = 0;
  unsigned* status = nullptr;  // device address of the status word
  cudaMemPool_t pool = nullptr;
};

// Per-device facts, initialised once per device (thread-safe).
const DeviceInfo* device_info(int* err);

// Size of the per-device control block whose first word `DeviceInfo::status`
// points at (status word, test flags, wait limit: sn_common.cuh DevCtl).
constexpr size_t kDevCtlBytes = 16;

// The status code a device status word maps to (SN_OK if no bit is set).
int status_from_word(unsigned word);

// Fixed-size arrays (sn_fixed_*.cu; kernels in sn_fixed.cuh).  `family` is
// SN_NETWORK_BEST or SN_NETWORK_BOSE_NELSON (u64 keys: best only).  Return a
// cudaError_t.
cudaError_t launch_fixed_u32(uint32_t* keys, int n, uint64_t count, int family, cudaStream_t s,
                             const DeviceInfo& d);
cudaError_t launch_fixed_u64(uint64_t* keys, int n, uint64_t count, int family, cudaStream_t s,
                             const DeviceInfo& d);
cudaError_t launch_fixed_items(sn_item64* items, int n, uint64_t count, int family, cudaStream_t s,
                               const DeviceInfo& d);
cudaError_t launch_fixed_f32(float* keys, int n, uint64_t count, int family, cudaStream_t s, const DeviceInfo& d);
cudaError_t launch_fixed_f64(double* keys, int n, uint64_t count, int family, cudaStream_t s, const DeviceInfo& d);

// Segments (sn_segments.cu).
enum class SegMode : int { kNetworkWarpRss = 0, kRssOnly = 1 };

struct SegTuning {
  int tile_units = 4096;       // segments + elements per tile (512..16384)
  uint32_t net_classes = 0x1F;  // bits 0..3: padded classes 2, 4, 8, 12 channels (16 always);
                                // bit 4: 64-channel warp network for 33..64 items
  int rss_two_min = 160;       // RSS segments longer than this take a 64-item sample, else 32 (16..256)
  int tile_stages = 2;         // staging depth of the tile kernel (2..4)
  int tile_mode = 0;           // 0: task-ring tile kernel, 1: synchronous tile kernel
};

// Parameters installed for (device, key bytes, payload) (sn_tune.cu); the
// defaults until sn_tuning_set / sn_tune_segments / sn_tuning_load.
SegTuning current_tuning(int device, int key_bytes, bool vals);
bool tuning_valid(const SegTuning& t);

// Whether the tile kernel's staging (tile_units, tile_stages) fits in shared
// memory for this key type, payload kind and tile_mode (sn_segments_*.cu).
bool tile_fits_u32(bool vals, int tile_units, int stages, int mode);
bool tile_fits_u64(bool vals, int tile_units, int stages, int mode);
inline bool tile_fits(int key_bytes, bool vals, int tile_units, int stages, int mode) {
  return key_bytes == 8 ? tile_fits_u64(vals, tile_units, stages, mode)
                        : tile_fits_u32(vals, tile_units, stages, mode);
}

// Device scratch needed for a segmented call with nseg segments.
size_t segments_scratch_bytes(uint64_t nseg, const SegTuning& t);

cudaError_t launch_segments_u32(uint32_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                                SegMode mode, void* scratch, size_t scratch_bytes, const SegTuning& t,
                                cudaStream_t s, const DeviceInfo& d);
cudaError_t launch_segments_u64(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                                SegMode mode, void* scratch, size_t scratch_bytes, const SegTuning& t,
                                cudaStream_t s, const DeviceInfo& d);
// Segments of up to SN_MAX_SEGMENT_LARGE items, one CTA per segment
// (sn_large.cu): segment s is keys[starts[s] .. ends[s]) (CSR offsets: ends =
// offsets + 1); `scratch` holds one device word (the validation flag).
cudaError_t launch_large_u32(uint32_t* keys, uint32_t* vals, const uint32_t* starts, const uint32_t* ends,
                             uint64_t nseg, void* scratch, cudaStream_t s, const DeviceInfo& d);
cudaError_t launch_large_u64(uint64_t* keys, uint32_t* vals, const uint32_t* starts, const uint32_t* ends,
                             uint64_t nseg, void* scratch, cudaStream_t s, const DeviceInfo& d);

// One large array of u32 keys, sample-sort partition + segmented base case
// (sn_large_sort.cu); returns after the sort (it reads counts back).
cudaError_t sort_large_u32(uint32_t* keys, uint64_t n, cudaStream_t s, const DeviceInfo& d);

// f32 / f64 keys, ordered by IEEE-754 totalOrder (sn_segments_f32.cu / _f64.cu).
cudaError_t launch_segments_f32(float* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, SegMode mode,
                                void* scratch, size_t scratch_bytes, const SegTuning& t, cudaStream_t s,
                                const DeviceInfo& d);
cudaError_t launch_segments_f64(double* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, SegMode mode,
                                void* scratch, size_t scratch_bytes, const SegTuning& t, cudaStream_t s,
                                const DeviceInfo& d);

}  // namespace sn

// Segmented sorting, uint32_t keys: instantiation unit (kernels in sn_segments.cuh).
#include "sn_segments.cuh"

namespace sn {

cudaError_t launch_segments_u32(uint32_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                                SegMode mode, void* scratch, size_t scratch_bytes, const SegTuning& t,
                                cudaStream_t s, const DeviceInfo& d) {
  return seg::launch_segments<uint32_t>(keys, vals, offsets, nseg, mode, scratch, scratch_bytes, t, s, d);
}

int max_tile_units_u32(bool vals) {
  return vals ? seg::max_tile_units_for<uint32_t, true>() : seg::max_tile_units_for<uint32_t, false>();
}

}  // namespace sn

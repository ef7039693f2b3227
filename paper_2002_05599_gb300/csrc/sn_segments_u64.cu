// Segmented sorting, uint64_t keys: instantiation unit (kernels in sn_segments.cuh).
#include "sn_window.cuh"

namespace sn {

cudaError_t launch_segments_u64(uint64_t* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg,
                                SegMode mode, void* scratch, size_t scratch_bytes, const SegTuning& t,
                                cudaStream_t s, const DeviceInfo& d) {
  return seg::launch_segments<uint64_t>(keys, vals, offsets, nseg, mode, scratch, scratch_bytes, t, s, d);
}

bool tile_fits_u64(bool vals, int tile_units, int stages, int mode) {
  return vals ? seg::seg_fits<uint64_t, true>(tile_units, stages, mode)
              : seg::seg_fits<uint64_t, false>(tile_units, stages, mode);
}

}  // namespace sn

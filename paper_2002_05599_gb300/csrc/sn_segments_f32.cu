// Segmented sorting, f32 keys (IEEE-754 totalOrder through the order-preserving
// code of key_enc): instantiation unit (kernels in sn_segments.cuh).
#include "sn_window.cuh"

namespace sn {

cudaError_t launch_segments_f32(float* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, SegMode mode,
                                void* scratch, size_t scratch_bytes, const SegTuning& t, cudaStream_t s,
                                const DeviceInfo& d) {
  return seg::launch_segments<uint32_t, true>(reinterpret_cast<uint32_t*>(keys), vals, offsets, nseg, mode, scratch,
                                            scratch_bytes, t, s, d);
}

}  // namespace sn

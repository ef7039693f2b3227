// Fixed-size arrays of f32 / f64 keys (IEEE-754 totalOrder): instantiation
// unit (kernels in sn_fixed.cuh), best known networks.
#include "sn_fixed.cuh"

namespace sn {

cudaError_t launch_fixed_f32(float* keys, int n, uint64_t count, int /*family*/, cudaStream_t s,
                             const DeviceInfo& d) {
  return launch_fixed<FloatBits<uint32_t>, BestNets>(reinterpret_cast<FloatBits<uint32_t>*>(keys), n, count, s, d);
}

cudaError_t launch_fixed_f64(double* keys, int n, uint64_t count, int /*family*/, cudaStream_t s,
                             const DeviceInfo& d) {
  return launch_fixed<FloatBits<uint64_t>, BestNets>(reinterpret_cast<FloatBits<uint64_t>*>(keys), n, count, s, d);
}

}  // namespace sn

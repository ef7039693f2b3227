// Fixed-size arrays of u64 keys: instantiation unit (kernels in sn_fixed.cuh),
// best known networks.
#include "sn_fixed.cuh"

namespace sn {

cudaError_t launch_fixed_u64(uint64_t* keys, int n, uint64_t count, int /*family*/, cudaStream_t s,
                             const DeviceInfo& d) {
  return launch_fixed<uint64_t, BestNets>(keys, n, count, s, d);
}

}  // namespace sn

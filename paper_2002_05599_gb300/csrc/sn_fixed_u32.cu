// Fixed-size arrays of u32 keys: instantiation unit (kernels in sn_fixed.cuh),
// both network families.
#include "sn_fixed.cuh"

namespace sn {

cudaError_t launch_fixed_u32(uint32_t* keys, int n, uint64_t count, int family, cudaStream_t s,
                             const DeviceInfo& d) {
  if (family == SN_NETWORK_BOSE_NELSON) return launch_fixed<uint32_t, BoseNelsonNets>(keys, n, count, s, d);
  return launch_fixed<uint32_t, BestNets>(keys, n, count, s, d);
}

}  // namespace sn

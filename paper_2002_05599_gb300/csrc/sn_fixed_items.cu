// Fixed-size arrays of 16-byte items (u64 key + u64 reference): instantiation
// unit (kernels in sn_fixed.cuh), both network families.
#include "sn_fixed.cuh"

namespace sn {

cudaError_t launch_fixed_items(sn_item64* items, int n, uint64_t count, int family, cudaStream_t s,
                               const DeviceInfo& d) {
  Pair* p = reinterpret_cast<Pair*>(items);
  if (family == SN_NETWORK_BOSE_NELSON) return launch_fixed<Pair, BoseNelsonNets>(p, n, count, s, d);
  return launch_fixed<Pair, BestNets>(p, n, count, s, d);
}

}  // namespace sn

// Segments of up to 4096 items (include/smallsort.h: sn_sort_segments_large).
//
// The paper stops at 256 items and names merging networks as the way beyond
// (Sec. 5).  Here one CTA takes one segment at a time: its items, as
// (key, position) pairs, are loaded into shared memory, padded with +inf to
// the next power of two P, sorted by the ascending bitonic sorting network on
// P channels (log2 P (log2 P + 1) / 2 steps; each step's P/2 comparators are
// spread over the CTA's threads), and written back with the payload gathered
// by position.  A validation pass runs first: a segment longer than 4096 or
// decreasing offsets leave every key untouched and set the range bit of the
// status word.
#include <algorithm>
#include <atomic>

#include "smallsort.h"
#include "sn_common.cuh"
#include "sn_internal.h"

namespace sn {
namespace {

constexpr int kLargeThreads = 256;
constexpr uint32_t kLargeMax = SN_MAX_SEGMENT_LARGE;

// Segment s is keys[starts[s] .. ends[s]); for CSR offsets, ends = offsets + 1.
__global__ void __launch_bounds__(256)
    large_check_kernel(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ ends, uint64_t nseg,
                       unsigned* bad, unsigned* status) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool ok = true;
  for (uint64_t s = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < nseg; s += stride) {
    const uint32_t a = starts[s], b = ends[s];
    if (b < a || b - a > kLargeMax) ok = false;
  }
  if (__any_sync(0xFFFFFFFFu, !ok) && (threadIdx.x & 31) == 0) {
    atomicOr(bad, 1u);
    atomicOr(status, kStatusRange);
  }
}

// Shared-memory items of one segment: (key, position) with the position in a
// separate array for 8-byte keys.
template <class K> struct LargeMem;
template <> struct LargeMem<uint32_t> {
  static constexpr size_t kItemBytes = 8;
  uint64_t* it;
  __device__ explicit LargeMem(unsigned char* p) : it(reinterpret_cast<uint64_t*>(p)) {}
  __device__ __forceinline__ uint64_t get(int i) const { return it[i]; }
  __device__ __forceinline__ void set(int i, uint64_t v) const { it[i] = v; }
};
template <> struct LargeMem<uint64_t> {
  static constexpr size_t kItemBytes = 12;
  uint64_t* key;
  uint32_t* idx;
  __device__ explicit LargeMem(unsigned char* p)
      : key(reinterpret_cast<uint64_t*>(p)), idx(reinterpret_cast<uint32_t*>(p + 8 * kLargeMax)) {}
  __device__ __forceinline__ Item64 get(int i) const { return Item64{key[i], idx[i]}; }
  __device__ __forceinline__ void set(int i, const Item64& v) const {
    key[i] = v.key;
    idx[i] = v.idx;
  }
};

template <class K, bool kVals>
constexpr size_t large_smem() {
  return LargeMem<K>::kItemBytes * kLargeMax + (kVals ? 4 * kLargeMax : 0);
}

template <class K, bool kVals, bool kF>
__global__ void __launch_bounds__(kLargeThreads)
    large_sort_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ starts,
                      const uint32_t* __restrict__ ends, uint64_t nseg, const unsigned* bad) {
  using IO = ItemOf<K>;
  extern __shared__ __align__(16) unsigned char smem[];
  if (*bad) return;
  const LargeMem<K> m(smem);
  uint32_t* vs = reinterpret_cast<uint32_t*>(smem + LargeMem<K>::kItemBytes * kLargeMax);
  const int tid = threadIdx.x;
  for (uint64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
    const uint32_t e0 = starts[s];
    const int L = static_cast<int>(ends[s] - e0);
    if (L <= 1) continue;
    int P = 2;
    while (P < L) P <<= 1;
    for (int i = tid; i < P; i += kLargeThreads)
      m.set(i, i < L ? IO::make(key_enc<K, kF>(keys[e0 + i]), static_cast<uint32_t>(i)) : IO::sentinel(i));
    if constexpr (kVals)
      for (int i = tid; i < L; i += kLargeThreads) vs[i] = vals[e0 + i];
    __syncthreads();
    // ascending bitonic sorter: merges of size k = 2, 4, ..., P; the first step
    // of each merge compares mirrored slots (mask k - 1), the rest are
    // half-cleaners (mask k/4, ..., 1); the lower slot keeps the smaller item
    for (int k = 2; k <= P; k <<= 1) {
      for (int mask = k - 1; mask > 0; mask = (mask == k - 1) ? (k >> 2) : (mask >> 1)) {
        for (int c = tid; c < (P >> 1); c += kLargeThreads) {
          const int i = bitonic_slot(c, mask);
          const int j = i ^ mask;
          const auto a = m.get(i);
          const auto b = m.get(j);
          if (item_less(b, a)) {
            m.set(i, b);
            m.set(j, a);
          }
        }
        __syncthreads();
        if (mask == 1) break;
      }
    }
    for (int i = tid; i < L; i += kLargeThreads) {
      const auto y = m.get(i);
      keys[e0 + i] = key_dec<K, kF>(IO::key(y));
      if constexpr (kVals) vals[e0 + i] = vs[IO::idx(y)];
    }
    __syncthreads();  // the next segment overwrites shared memory
  }
}

template <class K, bool kVals, bool kF>
cudaError_t launch_large_t(K* keys, uint32_t* vals, const uint32_t* starts, const uint32_t* ends, uint64_t nseg,
                           void* scratch, cudaStream_t s, const DeviceInfo& d) {
  unsigned* bad = static_cast<unsigned*>(scratch);
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const unsigned g1 =
      static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>((nseg + 255) / 256, 8ull * d.sm_count)));
  large_check_kernel<<<g1, 256, 0, s>>>(starts, ends, nseg, bad, d.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  constexpr int kSmem = static_cast<int>(large_smem<K, kVals>());
  static std::atomic<int> occ[64];
  int per_sm = d.device >= 0 && d.device < 64 ? occ[d.device].load(std::memory_order_relaxed) : 0;
  if (per_sm == 0) {
    auto kern = large_sort_kernel<K, kVals, kF>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLargeThreads, kSmem)) != cudaSuccess)
      return e;
    per_sm = std::max(per_sm, 1);
    if (d.device >= 0 && d.device < 64) occ[d.device].store(per_sm, std::memory_order_relaxed);
  }
  const unsigned g2 = static_cast<unsigned>(
      std::max<uint64_t>(1, std::min<uint64_t>(nseg, static_cast<uint64_t>(d.sm_count) * per_sm)));
  large_sort_kernel<K, kVals, kF><<<g2, kLargeThreads, kSmem, s>>>(keys, vals, starts, ends, nseg, bad);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_large_u32(uint32_t* keys, uint32_t* vals, const uint32_t* starts, const uint32_t* ends,
                             uint64_t nseg, void* scratch, cudaStream_t s, const DeviceInfo& d) {
  return vals ? launch_large_t<uint32_t, true, false>(keys, vals, starts, ends, nseg, scratch, s, d)
              : launch_large_t<uint32_t, false, false>(keys, vals, starts, ends, nseg, scratch, s, d);
}

cudaError_t launch_large_u64(uint64_t* keys, uint32_t* vals, const uint32_t* starts, const uint32_t* ends,
                             uint64_t nseg, void* scratch, cudaStream_t s, const DeviceInfo& d) {
  return vals ? launch_large_t<uint64_t, true, false>(keys, vals, starts, ends, nseg, scratch, s, d)
              : launch_large_t<uint64_t, false, false>(keys, vals, starts, ends, nseg, scratch, s, d);
}

}  // namespace sn

// Fixed-size arrays: `count` contiguous arrays of N elements (the ArrayInRow
// layout of Sec. 4.1 / 4.3), each sorted by an N-channel network of Sec. 2
// (the best known networks or Bose and Nelson's construction), one array per
// thread, all in registers.  Elements are u32 or u64 keys, or the paper's
// 16-byte items (u64 key + u64 reference, Sec. 4.1) ordered by (key, position
// in the array) with the reference carried along.
//
// Included by the instantiation units sn_fixed_u32.cu, sn_fixed_u64.cu and
// sn_fixed_items.cu (internal linkage: each unit has its own copy).
//
// Data movement is HBM-bound by design (8 bytes moved per u32 key against at
// most 3.75 compare-exchanges per key), so the kernel is built around the copy:
//   * persistent CTAs walk tiles of ~16 KB with a 4-stage ring of 1-D bulk
//     copies (cp.async.bulk global->shared, completion on an mbarrier) and
//     write each sorted tile back with a bulk copy shared->global;
//   * each thread reads its array from shared memory with the widest vector
//     access the array size allows.  When the array stride would make lanes of
//     one shared-memory wavefront hit the same banks (N = 8, 16 for u32), each
//     lane starts at a different chunk of its array (a rotation by lane) and
//     the rotation is undone in registers with selects, so every wavefront is
//     conflict-free;
//   * the ragged tail (fewer arrays than one tile) and keys that are not
//     16-byte aligned use plain global loads and stores.
#pragma once

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "smallsort.h"
#include "sn_common.cuh"
#include "sn_internal.h"

namespace sn {
namespace {

// Network families (SN_NETWORK_BEST, SN_NETWORK_BOSE_NELSON).
struct BestNets {
  template <int N> using type = Net<N>;
};
struct BoseNelsonNets {
  template <int N> using type = NetBN<N>;
};

// IEEE-754 keys held as their bit patterns; sorted through the
// order-preserving code of key_enc (totalOrder).
template <class K>
struct FloatBits {
  K bits;
};
template <class E>
struct KeyOf {
  using type = E;
  static constexpr bool kF = false;
};
template <class K>
struct KeyOf<FloatBits<K>> {
  using type = K;
  static constexpr bool kF = true;
};

// 16-byte item of the paper's experiments, same layout as sn_item64.
struct Pair {
  uint64_t key, ref;
};
static_assert(sizeof(Pair) == 16 && sizeof(sn_item64) == 16, "item layout");

constexpr int kFixedThreads = 256;
constexpr int kFixedStages = 4;
constexpr int kFixedSmemCap = 200 * 1024;  // dynamic shared memory for the staging ring
constexpr int kTileTarget = 16384;

constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

template <int N, class E>
struct FixedCfg {
  static constexpr int kElem = sizeof(E);
  static constexpr int kArrayBytes = N * kElem;
  static constexpr int kApt =
      kTileTarget / (kFixedThreads * kArrayBytes) > 0 ? kTileTarget / (kFixedThreads * kArrayBytes) : 1;
  static constexpr int kTileArrays = kFixedThreads * kApt;
  static constexpr int kTileBytes = kTileArrays * kArrayBytes;
  // widest shared-memory access that divides the array
  static constexpr int kVec = (kArrayBytes % 16 == 0) ? 16 : (kArrayBytes % 8 == 0) ? 8 : 4;
  static constexpr int kChunks = kArrayBytes / kVec;
  static constexpr int kWordsPerChunk = kVec / 4;
  static constexpr int kWords = kArrayBytes / 4;
  static constexpr int kPhase = 128 / kVec;                  // lanes served per wavefront
  static constexpr int kConflict = cgcd(kChunks, kPhase);    // lanes per bank group, unrotated
  // staging ring depth: 4 tiles, fewer when large tiles would not fit
  static constexpr int kStages = (kFixedSmemCap / kTileBytes) < kFixedStages ? (kFixedSmemCap / kTileBytes)
                                                                            : kFixedStages;
  static_assert(kStages >= 2, "at least two tiles in flight");
  static_assert(kTileBytes % 16 == 0, "bulk copies need multiples of 16 bytes");
};

template <int V>
__device__ __forceinline__ void ld_chunk(const unsigned char* p, uint32_t* w) {
  if constexpr (V == 16) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (V == 8) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x; w[1] = v.y;
  } else {
    w[0] = *reinterpret_cast<const uint32_t*>(p);
  }
}

template <int V>
__device__ __forceinline__ void st_chunk(unsigned char* p, const uint32_t* w) {
  if constexpr (V == 16) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
  } else if constexpr (V == 8) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
  } else {
    *reinterpret_cast<uint32_t*>(p) = w[0];
  }
}

// Rotate the M chunks (W words each) of x by r in [0, G), one power of two at
// a time with selects.  Forward: out[c] = in[(c - r) mod M]; backward:
// out[c] = in[(c + r) mod M].
template <int M, int W, int G, bool kForward>
__device__ __forceinline__ void rotate_chunks(uint32_t* x, int r) {
#pragma unroll
  for (int b = 0; (1 << b) < G; ++b) {
    const bool on = (r >> b) & 1;
    const int s = 1 << b;
    uint32_t y[M * W];
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int src = kForward ? (c - s + M) % M : (c + s) % M;
#pragma unroll
      for (int w = 0; w < W; ++w) y[c * W + w] = on ? x[src * W + w] : x[c * W + w];
    }
#pragma unroll
    for (int i = 0; i < M * W; ++i) x[i] = y[i];
  }
}

template <class K, int N>
__device__ __forceinline__ void words_to_keys(const uint32_t* w, K* k) {
  if constexpr (sizeof(K) == 4) {
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = w[i];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = static_cast<uint64_t>(w[2 * i]) | (static_cast<uint64_t>(w[2 * i + 1]) << 32);
  }
}

template <class K, int N>
__device__ __forceinline__ void keys_to_words(const K* k, uint32_t* w) {
  if constexpr (sizeof(K) == 4) {
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = k[i];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      w[2 * i] = static_cast<uint32_t>(k[i]);
      w[2 * i + 1] = static_cast<uint32_t>(k[i] >> 32);
    }
  }
}

// Network on the words of one array (words as loaded: element i at words
// [i * kElem / 4, (i + 1) * kElem / 4)).  `src` is the array's location (shared
// or global memory) for items, whose references are gathered from it by
// original position after the network has ordered (key, position).
template <int N, class E, class Fam>
__device__ __forceinline__ void sort_words(uint32_t* w, const E* src) {
  using NetT = typename Fam::template type<N>;
  if constexpr (std::is_same<E, Pair>::value) {
    Item64 it[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
      it[i] = Item64{static_cast<uint64_t>(w[4 * i]) | (static_cast<uint64_t>(w[4 * i + 1]) << 32),
                     static_cast<uint32_t>(i)};
    NetT::run(it);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const uint64_t ref = src[it[q].idx].ref;
      w[4 * q] = static_cast<uint32_t>(it[q].key);
      w[4 * q + 1] = static_cast<uint32_t>(it[q].key >> 32);
      w[4 * q + 2] = static_cast<uint32_t>(ref);
      w[4 * q + 3] = static_cast<uint32_t>(ref >> 32);
    }
  } else {
    using KT = typename KeyOf<E>::type;
    constexpr bool kF = KeyOf<E>::kF;
    KT k[N];
    words_to_keys<KT, N>(w, k);
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = key_enc<KT, kF>(k[i]);
    NetT::run(k);
#pragma unroll
    for (int i = 0; i < N; ++i) k[i] = key_dec<KT, kF>(k[i]);
    keys_to_words<KT, N>(k, w);
  }
}

// Sort the array at `arr` (shared memory) in place.
template <int N, class E, class Fam>
__device__ __forceinline__ void sort_array_smem(unsigned char* arr, int lane) {
  using C = FixedCfg<N, E>;
  uint32_t w[C::kWords];
  const int r = (C::kConflict > 1) ? ((lane % C::kPhase) / (C::kPhase / C::kConflict)) : 0;
#pragma unroll
  for (int j = 0; j < C::kChunks; ++j) {
    const int c = (C::kConflict > 1) ? (j + r) % C::kChunks : j;
    ld_chunk<C::kVec>(arr + c * C::kVec, &w[j * C::kWordsPerChunk]);
  }
  if constexpr (C::kConflict > 1) rotate_chunks<C::kChunks, C::kWordsPerChunk, C::kConflict, true>(w, r);
  sort_words<N, E, Fam>(w, reinterpret_cast<const E*>(arr));
  if constexpr (C::kConflict > 1) rotate_chunks<C::kChunks, C::kWordsPerChunk, C::kConflict, false>(w, r);
#pragma unroll
  for (int j = 0; j < C::kChunks; ++j) {
    const int c = (C::kConflict > 1) ? (j + r) % C::kChunks : j;
    st_chunk<C::kVec>(arr + c * C::kVec, &w[j * C::kWordsPerChunk]);
  }
}

// Sort one array straight from global memory (tail and unaligned path).
template <int N, class E, class Fam>
__device__ __forceinline__ void sort_array_global(E* p) {
  using C = FixedCfg<N, E>;
  uint32_t w[C::kWords];
  const uint32_t* pw = reinterpret_cast<const uint32_t*>(p);
#pragma unroll
  for (int i = 0; i < C::kWords; ++i) w[i] = pw[i];
  sort_words<N, E, Fam>(w, p);
  uint32_t* qw = reinterpret_cast<uint32_t*>(p);
#pragma unroll
  for (int i = 0; i < C::kWords; ++i) qw[i] = w[i];
}

template <int N, class K, class Fam>
__global__ void __launch_bounds__(kFixedThreads)
    fixed_tma_kernel(K* __restrict__ keys, uint64_t count, unsigned* status) {
  using C = FixedCfg<N, K>;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int kStages = C::kStages;
  __shared__ __align__(8) uint64_t full[kStages];

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const uint64_t ntiles = count / C::kTileArrays;
  const uint64_t my = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  unsigned char* gbase = reinterpret_cast<unsigned char*>(keys);
  auto tile_ptr = [&](uint64_t i) {
    return gbase + (static_cast<uint64_t>(blockIdx.x) + i * gridDim.x) * static_cast<uint64_t>(C::kTileBytes);
  };

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool skip_copy = tid == 0 && (test_flags(status) & kTestSkipFixedCopy);
  if (tid == 0) {
    for (uint64_t s = 0; s < kStages && s < my; ++s) {
      mbar_arrive_expect_tx(&full[s], C::kTileBytes);
      if (!skip_copy) bulk_g2s(smem + s * C::kTileBytes, tile_ptr(s), C::kTileBytes, &full[s]);
    }
  }

  bool failed = false;
  uint64_t i = 0;
  for (; i < my; ++i) {
    const int s = static_cast<int>(i % kStages);
    const bool ok = mbar_wait(&full[s], static_cast<uint32_t>(i / kStages) & 1u, status);
    if (ok) {
      unsigned char* buf = smem + s * C::kTileBytes;
#pragma unroll
      for (int q = 0; q < C::kApt; ++q)
        sort_array_smem<N, K, Fam>(buf + (q * kFixedThreads + tid) * C::kArrayBytes, lane);
      fence_proxy_async_smem();
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (tid == 0) {
      bulk_s2g(tile_ptr(i), smem + s * C::kTileBytes, C::kTileBytes);
      bulk_commit();
      if (i >= 1 && i - 1 + kStages < my) {
        const int ps = static_cast<int>((i - 1) % kStages);
        bulk_wait_read<1>();  // the store of tile i-1 has read its buffer
        mbar_arrive_expect_tx(&full[ps], C::kTileBytes);
        if (!skip_copy) bulk_g2s(smem + ps * C::kTileBytes, tile_ptr(i - 1 + kStages), C::kTileBytes, &full[ps]);
      }
    }
  }

  // Ragged tail: the arrays after the last full tile, from global memory.
  if (!failed && blockIdx.x == gridDim.x - 1) {
    for (uint64_t a = ntiles * C::kTileArrays + tid; a < count; a += kFixedThreads)
      sort_array_global<N, K, Fam>(keys + a * N);
  }

  if (tid == 0) {
    bulk_wait_all<0>();
    if (failed) {
      atomicOr(status, kStatusTimeout);
      // let the loads that were issued but never consumed land before exit
      const uint64_t issued_end = min(my, max(static_cast<uint64_t>(kStages), i + kStages - 1));
      for (uint64_t t = i; t < issued_end; ++t)
        (void)mbar_wait(&full[t % kStages], static_cast<uint32_t>(t / kStages) & 1u, status);
    }
  }
}

template <int N, class K, class Fam>
__global__ void __launch_bounds__(256) fixed_direct_kernel(K* __restrict__ keys, uint64_t count) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t a = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; a < count; a += stride)
    sort_array_global<N, K, Fam>(keys + a * N);
}

constexpr int kMaxDevices = 64;

template <int N, class K, class Fam>
cudaError_t launch_n(K* keys, uint64_t count, cudaStream_t stream, const DeviceInfo& d) {
  using C = FixedCfg<N, K>;
  if ((reinterpret_cast<uintptr_t>(keys) & 15u) != 0) {
    const uint64_t want = (count + 255) / 256;
    const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(want, 8ull * d.sm_count)));
    fixed_direct_kernel<N, K, Fam><<<grid, 256, 0, stream>>>(keys, count);
    return cudaGetLastError();
  }
  constexpr int kSmem = C::kStages * C::kTileBytes;
  // blocks per SM, cached per device (0 = not yet known)
  static std::atomic<int> occ[kMaxDevices];
  int per_sm = d.device < kMaxDevices ? occ[d.device].load(std::memory_order_relaxed) : 0;
  if (per_sm == 0) {
    cudaError_t e =
        cudaFuncSetAttribute(fixed_tma_kernel<N, K, Fam>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fixed_tma_kernel<N, K, Fam>, kFixedThreads, kSmem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    if (d.device < kMaxDevices) occ[d.device].store(per_sm, std::memory_order_relaxed);
  }
  const uint64_t ntiles = count / C::kTileArrays;
  const uint64_t cap = static_cast<uint64_t>(d.sm_count) * per_sm;
  const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min(ntiles, cap)));
  fixed_tma_kernel<N, K, Fam><<<grid, kFixedThreads, kSmem, stream>>>(keys, count, d.status);
  return cudaGetLastError();
}

template <class K, class Fam>
cudaError_t launch_fixed(K* keys, int n, uint64_t count, cudaStream_t s, const DeviceInfo& d) {
  switch (n) {
    case 2: return launch_n<2, K, Fam>(keys, count, s, d);
    case 3: return launch_n<3, K, Fam>(keys, count, s, d);
    case 4: return launch_n<4, K, Fam>(keys, count, s, d);
    case 5: return launch_n<5, K, Fam>(keys, count, s, d);
    case 6: return launch_n<6, K, Fam>(keys, count, s, d);
    case 7: return launch_n<7, K, Fam>(keys, count, s, d);
    case 8: return launch_n<8, K, Fam>(keys, count, s, d);
    case 9: return launch_n<9, K, Fam>(keys, count, s, d);
    case 10: return launch_n<10, K, Fam>(keys, count, s, d);
    case 11: return launch_n<11, K, Fam>(keys, count, s, d);
    case 12: return launch_n<12, K, Fam>(keys, count, s, d);
    case 13: return launch_n<13, K, Fam>(keys, count, s, d);
    case 14: return launch_n<14, K, Fam>(keys, count, s, d);
    case 15: return launch_n<15, K, Fam>(keys, count, s, d);
    case 16: return launch_n<16, K, Fam>(keys, count, s, d);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace sn

// Segmented sorting: CSR segments of 0..256 items, keys (u32 / u64) with an
// optional u32 payload, in one persistent launch.
//
// Plan (seg_plan_kernel): the batch is cut into tiles.  Segment s gets the
// position u_s = s + (offsets[s] - offsets[0]) and belongs to tile u_s / E,
// so a tile holds at most E segments and at most E + 256 items.  The kernel
// validates every segment and records the first segment of each tile.
//
// Sort (seg_sort_kernel, one CTA per SM): one producer warp moves whole tiles
// (offsets, keys, payload) into shared memory with 1-D bulk copies on a
// two-stage mbarrier ring.  Sixteen consumer warps bin the tile's segments by
// length -- the paper's suggestion (Sec. 5) of bucketing base cases by size and
// solving batches of identical size -- and take work items from a shared
// counter, largest first:
//   * 33..256 items (17..256 in RSS-only mode): Register Sample Sort by one
//     warp (Sec. 3): a sample of 2k items sorted by a network, k-1 splitters
//     taken equidistant, every item classified by the branch-free descent
//     j <- 2j + [t_j < e] over the splitter tree (Algorithm 1 generalised), a
//     stable counting scatter in shared memory, and one network per bucket;
//   * 17..32 items: the 32-lane warp network, one item per lane;
//   * 2..16 items: 32 segments of one size class at a time, one per lane, each
//     sorted in registers by the class's network (2, 4, 8, 12 or 16 channels,
//     shorter segments padded with +inf).
// Few distinct networks keep the instruction working set small: with one
// network per n, warps running different n thrashed the instruction cache
// (the GPU analogue of the L1i misses the paper measured in Sec. 4.4 / 4.6).
// With a payload, items are (key, position) pairs so ties keep input order and
// the payload is gathered by position at the end.  Sorted tiles go back with
// bulk stores; the partial 16-byte granules at a tile's two ends, which it
// shares with its neighbours, are written with plain stores.
#pragma once

#include <algorithm>
#include <atomic>

#include "sn_common.cuh"
#include "sn_internal.h"

namespace sn {
namespace seg {
namespace {  // internal linkage: each instantiation unit gets its own copy

constexpr int kConsumerWarps = 16;
constexpr int kConsumers = kConsumerWarps * 32;
constexpr int kThreads = kConsumers + 32;  // + one producer warp
constexpr int kStages = 2;
constexpr int kMaxSeg = 256;
constexpr uint32_t kDone = 0xFFFFFFFFu;
constexpr int kConsumerBar = 1;  // named barrier id for the consumer warps
constexpr int kRssMaxBuckets = 64;

// Size classes of a tile, in the order their work items are handed out.
enum Cls : int {
  kRss64 = 0, kRss32, kRss16, kRss8,  // Register Sample Sort with k buckets
  kWarp,                              // 17..32 items, warp network
  kNet16, kNet12, kNet8, kNet4, kNet2,
  kNumCls,
  kSkip = kNumCls                     // 0 or 1 item
};

__device__ __forceinline__ int seg_class(uint32_t len, bool rss_only) {
  if (len <= 1) return kSkip;
  if (len == 2) return kNet2;
  if (len <= 4) return kNet4;
  if (len <= 8) return kNet8;
  if (len <= 12) return kNet12;
  if (len <= 16) return kNet16;
  if (len <= 32) return rss_only ? kRss8 : kWarp;
  if (len <= 64) return kRss16;
  if (len <= 128) return kRss32;
  return kRss64;
}

__device__ __forceinline__ bool cls_is_net(int c) { return c >= kNet16; }

struct Plan {
  unsigned bad;        // offsets failed validation
  unsigned next_tile;  // dynamic tile counter
  unsigned ntiles;
  unsigned pad;
};

struct TileMeta {
  uint32_t tile;
  uint32_t s0, s1;        // segments [s0, s1)
  uint32_t e0, e1;        // items [e0, e1)
  uint32_t off_shift;     // index of offsets[s0] in the staged offsets
  uint32_t key_shift;     // index of keys[e0] in the staged keys
  uint32_t val_shift;     // index of vals[e0] in the staged payload
};

// ------------------------------------------------------------ layout -------

template <class K, bool kVals>
struct Layout {
  uint32_t E;
  uint32_t off_cap, key_cap, val_cap;  // staged elements per stage
  size_t off_at, key_at, val_at, stage_bytes;
  size_t list_at, rss_at, total;

  __host__ __device__ explicit Layout(uint32_t tile_units) : E(tile_units) {
    off_cap = E + 1 + 8;
    key_cap = E + kMaxSeg + 2 * (16 / sizeof(K));
    val_cap = kVals ? E + kMaxSeg + 8 : 0;
    off_at = 0;
    key_at = align16(off_at + off_cap * 4);
    val_at = align16(key_at + static_cast<size_t>(key_cap) * sizeof(K));
    stage_bytes = align128(val_at + val_cap * 4);
    list_at = kStages * stage_bytes;
    rss_at = align128(list_at + static_cast<size_t>(E) * 2);
    total = rss_at + kConsumerWarps * rss_bytes();
  }
  __host__ __device__ static size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }
  __host__ __device__ static size_t align128(size_t x) { return (x + 127) & ~static_cast<size_t>(127); }
  // per-warp Register Sample Sort scratch: 256 items + 64 bucket counters
  __host__ __device__ static size_t rss_bytes() {
    return sizeof(K) == 4 ? 256 * 8 + kRssMaxBuckets * 4 : 256 * 8 + 256 * 2 + kRssMaxBuckets * 4;
  }
};

// Per-warp RSS scratch.  The item buffer also holds the sorted sample (slots
// 0..S-1) and then the splitter tree (slots S..S+k-1) before the scatter
// overwrites it: classification finishes before the first scatter store.
template <class K> struct RssMem;
template <> struct RssMem<uint32_t> {
  uint64_t* buf;  // 256 packed items
  uint32_t* cnt;  // 64 bucket counters
  __device__ __forceinline__ explicit RssMem(unsigned char* p)
      : buf(reinterpret_cast<uint64_t*>(p)), cnt(reinterpret_cast<uint32_t*>(p + 256 * 8)) {}
  __device__ __forceinline__ uint64_t get(int i) const { return buf[i]; }
  __device__ __forceinline__ void set(int i, uint64_t v) const { buf[i] = v; }
};
template <> struct RssMem<uint64_t> {
  uint64_t* key;  // 256
  uint16_t* idx;  // 256
  uint32_t* cnt;  // 64
  __device__ __forceinline__ explicit RssMem(unsigned char* p)
      : key(reinterpret_cast<uint64_t*>(p)), idx(reinterpret_cast<uint16_t*>(p + 256 * 8)),
        cnt(reinterpret_cast<uint32_t*>(p + 256 * 10)) {}
  __device__ __forceinline__ Item64 get(int i) const { return Item64{key[i], idx[i]}; }
  __device__ __forceinline__ void set(int i, const Item64& v) const {
    key[i] = v.key;
    idx[i] = static_cast<uint16_t>(v.idx);
  }
};

// ---------------------------------------------------------------- plan -----

__global__ void __launch_bounds__(256)
    seg_plan_kernel(const uint32_t* __restrict__ offsets, uint64_t nseg, uint32_t E, Plan* plan,
                    uint32_t* __restrict__ tile_first, uint64_t tile_cap, unsigned* status) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint32_t base = offsets[0];
  bool bad = false;
  for (uint64_t s = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < nseg; s += stride) {
    const uint32_t o = offsets[s];
    const uint32_t o1 = offsets[s + 1];
    if (o1 < o || o1 - o > kMaxSeg || o < base) bad = true;
    const uint64_t u = s + static_cast<uint64_t>(o - base);
    const uint64_t t = u / E;
    uint64_t tp = ~0ull;
    if (s > 0) {
      const uint32_t op = offsets[s - 1];
      tp = ((s - 1) + static_cast<uint64_t>(op - base)) / E;
    }
    if (t != tp && t < tile_cap) tile_first[t] = static_cast<uint32_t>(s);
    if (s == nseg - 1) {
      if (t + 1 < tile_cap) {
        tile_first[t + 1] = static_cast<uint32_t>(nseg);
        plan->ntiles = static_cast<unsigned>(t + 1);
      } else {
        bad = true;
      }
    }
  }
  if (bad) {
    atomicOr(&plan->bad, 1u);
    atomicOr(status, kStatusRange);
  }
}

// ------------------------------------------------------ per-lane networks --

// Segment of L <= N items at kbuf[p..p+L), padded with +inf to N channels
// (payload at vbuf[pv..pv+L)).
template <int N, class K, bool kVals>
__device__ __forceinline__ void net_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L) {
  if constexpr (kVals) {
    using IO = ItemOf<K>;
    typename IO::T it[N];
#pragma unroll
    for (int q = 0; q < N; ++q) it[q] = q < L ? IO::make(kbuf[p + q], q) : IO::sentinel(q);
    Net<N>::run(it);
    uint32_t v[N];
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < L) v[q] = vbuf[pv + IO::idx(it[q])];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      if (q < L) {
        kbuf[p + q] = IO::key(it[q]);
        vbuf[pv + q] = v[q];
      }
    }
  } else {
    K k[N];
#pragma unroll
    for (int q = 0; q < N; ++q) k[q] = q < L ? kbuf[p + q] : static_cast<K>(~static_cast<K>(0));
    Net<N>::run(k);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < L) kbuf[p + q] = k[q];
  }
}

// ------------------------------------------------------- warp network ------

template <class K, bool kVals>
__device__ __forceinline__ void warp_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L, int lane) {
  if constexpr (kVals) {
    using IO = ItemOf<K>;
    typename IO::T x = lane < L ? IO::make(kbuf[p + lane], lane) : IO::sentinel(lane);
    warp_network32(x, lane);
    uint32_t v = 0;
    if (lane < L) v = vbuf[pv + IO::idx(x)];
    __syncwarp();
    if (lane < L) {
      kbuf[p + lane] = IO::key(x);
      vbuf[pv + lane] = v;
    }
  } else {
    K x = lane < L ? kbuf[p + lane] : static_cast<K>(~static_cast<K>(0));
    warp_network32(x, lane);
    __syncwarp();
    if (lane < L) kbuf[p + lane] = x;
  }
}

// --------------------------------------------------- Register Sample Sort --

// Bucket of c (<= N) items at rm[st..st+c), padded to N with +inf.
template <int N, class K, bool kVals>
__device__ __forceinline__ void bucket_network(const RssMem<K>& rm, int st, int c) {
  using IO = ItemOf<K>;
  if constexpr (kVals) {
    typename IO::T it[N];
#pragma unroll
    for (int q = 0; q < N; ++q) it[q] = q < c ? rm.get(st + q) : IO::sentinel(q);
    Net<N>::run(it);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < c) rm.set(st + q, it[q]);
  } else {
    // keys only: equal keys are interchangeable, so the network orders keys
    // alone (the stored position is not needed after classification)
    K k[N];
#pragma unroll
    for (int q = 0; q < N; ++q) k[q] = q < c ? IO::key(rm.get(st + q)) : static_cast<K>(~static_cast<K>(0));
    Net<N>::run(k);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < c) rm.set(st + q, IO::make(k[q], 0));
  }
}

template <class K, bool kVals>
__device__ __forceinline__ void bucket_network_class(int m, const RssMem<K>& rm, int st, int c) {
  if (m <= 4)
    bucket_network<4, K, kVals>(rm, st, c);
  else if (m <= 8)
    bucket_network<8, K, kVals>(rm, st, c);
  else if (m <= 12)
    bucket_network<12, K, kVals>(rm, st, c);
  else
    bucket_network<16, K, kVals>(rm, st, c);
}

// Comparator `c` of the step with XOR mask `mask` of the ascending bitonic
// sorter (mask = k-1 for the mirrored first step of a merge of size k, else a
// power of two): returns the lower slot; the partner is slot ^ mask.
__device__ __forceinline__ int bitonic_slot(int c, int mask) {
  const int h = (mask & (mask + 1)) == 0 ? (mask + 1) >> 1 : mask;  // highest bit of the pair distance
  const int b = __ffs(h) - 1;
  return ((c >> b) << (b + 1)) | (c & (h - 1));
}

// Warp-cooperative ascending bitonic sort of n <= 256 stored items at
// rm[st..st+n), padded virtually to the next power of two with +inf:
// comparators that reach past n are skipped.
template <class K, bool kByKey>
__device__ __forceinline__ void warp_bitonic_smem(const RssMem<K>& rm, int st, int n, int lane) {
  using IO = ItemOf<K>;
  int P = 1;
  while (P < n) P <<= 1;
  for (int k = 2; k <= P; k <<= 1) {
    for (int mask = k - 1; mask > 0; mask = (mask == k - 1) ? (k >> 2) : (mask >> 1)) {
      for (int c = lane; c < (P >> 1); c += 32) {
        const int i = bitonic_slot(c, mask);
        const int j = i ^ mask;
        if (j < n) {
          const auto a = rm.get(st + i);
          const auto b = rm.get(st + j);
          const bool swap = kByKey ? (IO::key(b) < IO::key(a)) : item_less(b, a);
          if (swap) {
            rm.set(st + i, b);
            rm.set(st + j, a);
          }
        }
      }
      __syncwarp();
      if (mask == 1) break;
    }
  }
}

template <class K, bool kVals>
__device__ __forceinline__ void rss_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L, const RssMem<K>& rm,
                                            int lane) {
  using IO = ItemOf<K>;
  using It = typename IO::T;
  const unsigned kFull = 0xFFFFFFFFu;

  // k buckets with at most L/4 expected items each (k in 8..64), sample of 2k
  int B = 8;
  while (B * 4 < L) B <<= 1;
  const int logB = __ffs(B) - 1;
  const int S = 2 * B;

  // 1. equidistant sample (this library's reading of "a sample subset"),
  //    sorted by a bitonic network; kept in slots 0..S-1
  for (int q = lane; q < S; q += 32) {
    const int pos = ((2 * q + 1) * L) / (2 * S);
    rm.set(q, IO::make(kbuf[p + pos], pos));
  }
  __syncwarp();
  warp_bitonic_smem<K, false>(rm, 0, S, lane);

  // 2. splitters s_j = S_{2j} (1-based), heap-ordered tree in slots S+1..S+k-1
  for (int node = lane; node < B; node += 32) {
    if (node >= 1) {
      const int d = 31 - __clz(node);
      const int pos = node - (1 << d);
      const int rank = (2 * pos + 1) * (B >> (d + 1));
      rm.set(S + node, rm.get(2 * rank - 1));
    }
  }
  for (int b = lane; b < B; b += 32) rm.cnt[b] = 0;
  __syncwarp();

  // 3. classify (j <- 2j + [t_j < e]) and rank items stably within buckets
  const int rounds = (L + 31) >> 5;
  uint32_t packed[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    packed[r] = 0;
    if (r < rounds) {
      const int e = (r << 5) + lane;
      const bool valid = e < L;
      const It x = valid ? IO::make(kbuf[p + e], e) : IO::sentinel(0);
      int j = 1;
      for (int lv = 0; lv < logB; ++lv) j = 2 * j + (item_less(rm.get(S + j), x) ? 1 : 0);
      const int b = j - B;
      unsigned peers = __ballot_sync(kFull, valid);
      for (int bit = 0; bit < logB; ++bit) {
        const unsigned m = __ballot_sync(kFull, (b >> bit) & 1);
        peers &= ((b >> bit) & 1) ? m : ~m;
      }
      const unsigned before = valid ? rm.cnt[b] : 0;
      __syncwarp();
      const unsigned below = __popc(peers & ((1u << lane) - 1u));
      if (valid && below == 0) rm.cnt[b] = before + __popc(peers);
      __syncwarp();
      packed[r] = (static_cast<uint32_t>(b) << 16) | (before + below);
    }
  }

  // 4. bucket starts: exclusive scan over the k counters, lane l owns buckets
  //    l and l + 32
  const uint32_t c0 = lane < B ? rm.cnt[lane] : 0;
  const uint32_t c1 = lane + 32 < B ? rm.cnt[lane + 32] : 0;
  uint32_t incl = c0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t start0 = incl - c0;
  const uint32_t total0 = __shfl_sync(kFull, incl, 31);
  uint32_t incl1 = c1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl1, d);
    if (lane >= d) incl1 += y;
  }
  const uint32_t start1 = total0 + incl1 - c1;
  __syncwarp();

  // 5. stable scatter into the item buffer (overwrites sample and tree)
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (r < rounds) {
      const int e = (r << 5) + lane;
      const int b = static_cast<int>(packed[r] >> 16);
      const uint32_t s_lo = __shfl_sync(kFull, start0, b & 31);
      const uint32_t s_hi = __shfl_sync(kFull, start1, b & 31);
      const uint32_t st = b < 32 ? s_lo : s_hi;
      if (e < L) rm.set(static_cast<int>(st + (packed[r] & 0xFFFFu)), IO::make(kbuf[p + e], e));
    }
  }
  __syncwarp();

  // 6. finish every bucket with a network: every lane pads its buckets to the
  //    warp's largest bucket (network of 4, 8, 12 or 16 channels); buckets
  //    above 16 items (rare) are sorted afterwards by the whole warp
  const uint32_t maxc = __reduce_max_sync(kFull, max(c0, c1));
  const int m = static_cast<int>(maxc < 16 ? maxc : 16);
  if (m >= 2) {
    if (lane < B && c0 <= 16) bucket_network_class<K, kVals>(m, rm, static_cast<int>(start0), static_cast<int>(c0));
    if (lane + 32 < B && c1 <= 16)
      bucket_network_class<K, kVals>(m, rm, static_cast<int>(start1), static_cast<int>(c1));
  }
  __syncwarp();
  if (maxc > 16) {
    for (int half = 0; half < 2; ++half) {
      const uint32_t c = half ? c1 : c0;
      const uint32_t st0 = half ? start1 : start0;
      unsigned big = __ballot_sync(kFull, lane + 32 * half < B && c > 16);
      while (big) {
        const int b = __ffs(big) - 1;
        big &= big - 1;
        const int st = static_cast<int>(__shfl_sync(kFull, st0, b));
        const int cb = static_cast<int>(__shfl_sync(kFull, c, b));
        warp_bitonic_smem<K, !kVals>(rm, st, cb, lane);
      }
    }
  }
  __syncwarp();

  // 7. write back (payload gathered by original position)
  if constexpr (kVals) {
    uint32_t vv[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) {
        const It y = rm.get(e);
        kbuf[p + e] = IO::key(y);
        vv[r] = vbuf[pv + IO::idx(y)];
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) vbuf[pv + e] = vv[r];
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) kbuf[p + e] = IO::key(rm.get(e));
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------ main kernel --

__device__ __forceinline__ bool consumers_or(bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(pred ? 1u : 0u), "n"(kConsumerBar), "n"(kConsumers)
      : "memory");
  return out != 0;
}

template <class K, bool kVals, bool kRssOnly>
__global__ void __launch_bounds__(kThreads, 1)
    seg_sort_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ offsets,
                    const Plan* plan_c, Plan* plan, const uint32_t* __restrict__ tile_first, uint32_t E,
                    unsigned* status) {
  using L_ = Layout<K, kVals>;
  const L_ lay(E);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ TileMeta meta[kStages];
  __shared__ uint32_t cls_cnt[kNumCls], cls_base[kNumCls], cls_cur[kNumCls];
  __shared__ uint32_t task_base[kNumCls + 1];
  __shared__ uint32_t task_ctr;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    fence_mbar_init();
  }
  if (tid < kNumCls) cls_cnt[tid] = 0;
  if (tid == 0) task_ctr = 0;
  __syncthreads();

  // ------------------------------------------------------------ producer --
  if (warp == kConsumerWarps) {
    if (lane == 0) {
      const uint32_t ntiles = plan_c->bad ? 0u : plan_c->ntiles;
      const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
      const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);
      const uintptr_t ob = reinterpret_cast<uintptr_t>(offsets);
      for (uint32_t k = 0;; ++k) {
        const int s = k & 1;
        if (k >= kStages && !mbar_wait(&empty[s], ((k >> 1) - 1) & 1u)) {
          atomicOr(status, kStatusTimeout);
          break;
        }
        const uint32_t t = atomicAdd(&plan->next_tile, 1u);
        TileMeta& m = meta[s];
        if (t >= ntiles) {
          m.tile = kDone;
          mbar_arrive(&full[s]);
          break;
        }
        const uint32_t s0 = tile_first[t], s1 = tile_first[t + 1];
        const uint32_t e0 = offsets[s0], e1 = offsets[s1];
        unsigned char* stage = smem + s * lay.stage_bytes;
        // granule-rounded source ranges (a 16-byte granule never crosses a
        // page, so reading its unused part cannot fault; it is discarded)
        const uintptr_t oa = (ob + 4ull * s0) & ~uintptr_t(15);
        const uintptr_t oz = (ob + 4ull * (s1 + 1) + 15) & ~uintptr_t(15);
        const uintptr_t ka = (kb + sizeof(K) * e0) & ~uintptr_t(15);
        const uintptr_t kz = (kb + sizeof(K) * e1 + 15) & ~uintptr_t(15);
        uint32_t bytes = static_cast<uint32_t>(oz - oa);
        m.tile = t;
        m.s0 = s0;
        m.s1 = s1;
        m.e0 = e0;
        m.e1 = e1;
        m.off_shift = static_cast<uint32_t>((ob + 4ull * s0 - oa) / 4);
        m.key_shift = static_cast<uint32_t>((kb + sizeof(K) * e0 - ka) / sizeof(K));
        const bool has_items = e1 > e0;
        if (has_items) bytes += static_cast<uint32_t>(kz - ka);
        uintptr_t va = 0, vz = 0;
        if constexpr (kVals) {
          va = (vb + 4ull * e0) & ~uintptr_t(15);
          vz = (vb + 4ull * e1 + 15) & ~uintptr_t(15);
          m.val_shift = static_cast<uint32_t>((vb + 4ull * e0 - va) / 4);
          if (has_items) bytes += static_cast<uint32_t>(vz - va);
        } else {
          m.val_shift = 0;
        }
        mbar_arrive_expect_tx(&full[s], bytes);
        bulk_g2s(stage + lay.off_at, reinterpret_cast<const void*>(oa), static_cast<uint32_t>(oz - oa), &full[s]);
        if (has_items) {
          bulk_g2s(stage + lay.key_at, reinterpret_cast<const void*>(ka), static_cast<uint32_t>(kz - ka), &full[s]);
          if constexpr (kVals)
            bulk_g2s(stage + lay.val_at, reinterpret_cast<const void*>(va), static_cast<uint32_t>(vz - va),
                     &full[s]);
        }
      }
    }
    return;
  }

  // ----------------------------------------------------------- consumers --
  uint16_t* seg_list = reinterpret_cast<uint16_t*>(smem + lay.list_at);
  const RssMem<K> rm(smem + lay.rss_at + warp * L_::rss_bytes());
  const unsigned kFull = 0xFFFFFFFFu;

  for (uint32_t k = 0;; ++k) {
    const int s = k & 1;
    const bool ok = mbar_wait(&full[s], (k >> 1) & 1u);
    if (consumers_or(!ok)) {
      if (tid == 0) atomicOr(status, kStatusTimeout);
      break;
    }
    const TileMeta m = meta[s];
    if (m.tile == kDone) break;

    unsigned char* stage = smem + s * lay.stage_bytes;
    const uint32_t* obuf = reinterpret_cast<const uint32_t*>(stage + lay.off_at) + m.off_shift;
    K* kbuf = reinterpret_cast<K*>(stage + lay.key_at);
    uint32_t* vbuf = reinterpret_cast<uint32_t*>(stage + lay.val_at);
    const int ns = static_cast<int>(m.s1 - m.s0);
    const int nrounds = (ns + kConsumers - 1) / kConsumers;

    // --- bin the tile's segments by size class (warp-aggregated counts)
    for (int r = 0; r < nrounds; ++r) {
      const int i = r * kConsumers + tid;
      const int c = i < ns ? seg_class(obuf[i + 1] - obuf[i], kRssOnly) : kSkip;
#pragma unroll
      for (int q = 0; q < kNumCls; ++q) {
        const unsigned mask = __ballot_sync(kFull, c == q);
        if (mask && lane == __ffs(mask) - 1) atomicAdd(&cls_cnt[q], __popc(mask));
      }
    }
    named_bar_sync(kConsumerBar, kConsumers);
    if (tid == 0) {
      uint32_t at = 0, tasks = 0;
      for (int q = 0; q < kNumCls; ++q) {
        cls_base[q] = at;
        cls_cur[q] = at;
        at += cls_cnt[q];
        task_base[q] = tasks;
        tasks += cls_is_net(q) ? (cls_cnt[q] + 31) / 32 : cls_cnt[q];
      }
      task_base[kNumCls] = tasks;
    }
    named_bar_sync(kConsumerBar, kConsumers);
    for (int r = 0; r < nrounds; ++r) {
      const int i = r * kConsumers + tid;
      const int c = i < ns ? seg_class(obuf[i + 1] - obuf[i], kRssOnly) : kSkip;
#pragma unroll
      for (int q = 0; q < kNumCls; ++q) {
        const unsigned mask = __ballot_sync(kFull, c == q);
        if (mask) {
          uint32_t at = 0;
          if (lane == __ffs(mask) - 1) at = atomicAdd(&cls_cur[q], __popc(mask));
          at = __shfl_sync(kFull, at, __ffs(mask) - 1);
          if (c == q) seg_list[at + __popc(mask & ((1u << lane) - 1u))] = static_cast<uint16_t>(i);
        }
      }
    }
    named_bar_sync(kConsumerBar, kConsumers);

    // --- work items, largest classes first
    const uint32_t ntasks = task_base[kNumCls];
    const uint32_t e0 = m.e0;
    for (;;) {
      uint32_t task = 0;
      if (lane == 0) task = atomicAdd(&task_ctr, 1u);
      task = __shfl_sync(kFull, task, 0);
      if (task >= ntasks) break;
      int q = 0;
      while (task >= task_base[q + 1]) ++q;
      const uint32_t j = task - task_base[q];
      if (!cls_is_net(q)) {
        const int i = seg_list[cls_base[q] + j];
        const uint32_t o = obuf[i];
        const int L = static_cast<int>(obuf[i + 1] - o);
        const int p = static_cast<int>(o - e0 + m.key_shift);
        const int pv = static_cast<int>(o - e0 + m.val_shift);
        if (q == kWarp)
          warp_segment<K, kVals>(kbuf, vbuf, p, pv, L, lane);
        else
          rss_segment<K, kVals>(kbuf, vbuf, p, pv, L, rm, lane);
      } else {
        const uint32_t slot = j * 32 + lane;
        if (slot < cls_cnt[q]) {
          const int i = seg_list[cls_base[q] + slot];
          const uint32_t o = obuf[i];
          const int L = static_cast<int>(obuf[i + 1] - o);
          const int p = static_cast<int>(o - e0 + m.key_shift);
          const int pv = static_cast<int>(o - e0 + m.val_shift);
          switch (q) {
            case kNet16: net_segment<16, K, kVals>(kbuf, vbuf, p, pv, L); break;
            case kNet12: net_segment<12, K, kVals>(kbuf, vbuf, p, pv, L); break;
            case kNet8: net_segment<8, K, kVals>(kbuf, vbuf, p, pv, L); break;
            case kNet4: net_segment<4, K, kVals>(kbuf, vbuf, p, pv, L); break;
            default: net_segment<2, K, kVals>(kbuf, vbuf, p, pv, L); break;
          }
        }
      }
    }

    // --- store the tile; reset the counters for the next one
    fence_proxy_async_smem();
    named_bar_sync(kConsumerBar, kConsumers);
    if (tid < kNumCls) cls_cnt[tid] = 0;
    if (tid == 32) task_ctr = 0;
    if (m.e1 > m.e0) {
      const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
      const uintptr_t a = kb + sizeof(K) * m.e0, z = kb + sizeof(K) * m.e1;
      const uintptr_t ia = (a + 15) & ~uintptr_t(15), iz = z & ~uintptr_t(15);
      uintptr_t va = 0, vz = 0, via = 0, viz = 0;
      if constexpr (kVals) {
        const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);
        va = vb + 4ull * m.e0;
        vz = vb + 4ull * m.e1;
        via = (va + 15) & ~uintptr_t(15);
        viz = vz & ~uintptr_t(15);
      }
      if (tid == 0) {
        if (ia < iz)
          bulk_s2g(reinterpret_cast<void*>(ia), kbuf + m.key_shift + (ia - a) / sizeof(K),
                   static_cast<uint32_t>(iz - ia));
        if constexpr (kVals) {
          if (via < viz)
            bulk_s2g(reinterpret_cast<void*>(via), vbuf + m.val_shift + (via - va) / 4,
                     static_cast<uint32_t>(viz - via));
        }
        bulk_commit();
      }
      // partial granules at both ends: plain stores
      if (warp == 1) {
        const uint32_t n_items = m.e1 - m.e0;
        const uint32_t head = ia < iz ? static_cast<uint32_t>((ia - a) / sizeof(K)) : n_items;
        const uint32_t tail_from = ia < iz ? static_cast<uint32_t>((iz - a) / sizeof(K)) : n_items;
        for (uint32_t e = lane; e < head; e += 32) keys[m.e0 + e] = kbuf[m.key_shift + e];
        for (uint32_t e = tail_from + lane; e < n_items; e += 32) keys[m.e0 + e] = kbuf[m.key_shift + e];
        if constexpr (kVals) {
          const uint32_t vhead = via < viz ? static_cast<uint32_t>((via - va) / 4) : n_items;
          const uint32_t vtail = via < viz ? static_cast<uint32_t>((viz - va) / 4) : n_items;
          for (uint32_t e = lane; e < vhead; e += 32) vals[m.e0 + e] = vbuf[m.val_shift + e];
          for (uint32_t e = vtail + lane; e < n_items; e += 32) vals[m.e0 + e] = vbuf[m.val_shift + e];
        }
      }
      if (tid == 0) bulk_wait_read<0>();
    }
    named_bar_sync(kConsumerBar, kConsumers);
    if (tid == 0) mbar_arrive(&empty[s]);
  }
  if (tid == 0) bulk_wait_all<0>();
}

// ------------------------------------------------------------ host side ----

inline uint64_t tile_capacity(uint64_t nseg, uint32_t E) {
  // tiles for valid offsets: u_{nseg-1} <= 257 (nseg - 1); one extra entry
  return (257ull * (nseg - 1)) / E + 2;
}

template <class K, bool kVals, bool kRssOnly>
cudaError_t launch_sort(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, void* scratch,
                        const SegTuning& tun, cudaStream_t stream, const DeviceInfo& d) {
  const uint32_t E = static_cast<uint32_t>(tun.tile_units);
  Plan* plan = reinterpret_cast<Plan*>(scratch);
  uint32_t* tile_first = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(scratch) + 256);
  const uint64_t cap = tile_capacity(nseg, E);

  cudaError_t e = cudaMemsetAsync(plan, 0, sizeof(Plan), stream);
  if (e != cudaSuccess) return e;
  const uint64_t want = (nseg + 255) / 256;
  const unsigned g1 = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(want, 16ull * d.sm_count)));
  seg_plan_kernel<<<g1, 256, 0, stream>>>(offsets, nseg, E, plan, tile_first, cap, d.status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  const Layout<K, kVals> lay(E);
  const int smem_bytes = static_cast<int>(lay.total);
  auto kern = seg_sort_kernel<K, kVals, kRssOnly>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem_bytes);
  if (e != cudaSuccess) return e;
  per_sm = std::max(per_sm, 1);
  const uint64_t max_tiles = cap - 1;
  const unsigned g2 = static_cast<unsigned>(
      std::max<uint64_t>(1, std::min<uint64_t>(max_tiles, static_cast<uint64_t>(d.sm_count) * per_sm)));
  kern<<<g2, kThreads, smem_bytes, stream>>>(keys, vals, offsets, plan, plan, tile_first, E, d.status);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_segments(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, SegMode mode,
                            void* scratch, size_t scratch_bytes, const SegTuning& t, cudaStream_t s,
                            const DeviceInfo& d) {
  if (scratch_bytes < segments_scratch_bytes(nseg, t)) return cudaErrorInvalidValue;
  if (t.tile_units < 512 || t.tile_units > 8192) return cudaErrorInvalidValue;
  const bool rss = mode == SegMode::kRssOnly;
  if (vals) {
    return rss ? launch_sort<K, true, true>(keys, vals, offsets, nseg, scratch, t, s, d)
               : launch_sort<K, true, false>(keys, vals, offsets, nseg, scratch, t, s, d);
  }
  return rss ? launch_sort<K, false, true>(keys, vals, offsets, nseg, scratch, t, s, d)
             : launch_sort<K, false, false>(keys, vals, offsets, nseg, scratch, t, s, d);
}

}  // namespace
}  // namespace seg
}  // namespace sn

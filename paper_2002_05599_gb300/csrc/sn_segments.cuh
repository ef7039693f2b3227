// Segmented sorting: CSR segments of 0..256 items, keys (u32 / u64) with an
// optional u32 payload.  Four stream-ordered launches:
//
// 1. seg_plan_kernel -- cuts the batch into tiles.  Segment s gets the
//    position u_s = s + (offsets[s] - offsets[0]) and belongs to tile u_s / E,
//    so a tile holds at most E segments and at most E + 256 items.  Every
//    segment is validated here, and classified by length (one class byte per
//    segment); bad offsets stop the call before any data is touched.
// 2. seg_bin_kernel -- bins every tile's segments by class: the paper's
//    suggestion (Sec. 5) of bucketing base cases by size so that batches of
//    identical size are solved together.  Each tile gets class counts and an
//    index list grouped by class; segments for Register Sample Sort (33+
//    items, 17+ in RSS-only mode) come last in the list.
// 3. seg_tile_kernel -- persistent, tiles assigned round-robin (no shared
//    counter); a producer warp reads the metadata of 32 tiles at a time,
//    skips tiles with nothing to do and stages the others
//    (offsets, keys, payload, bins) in shared memory with 1-D bulk copies on
//    a ring of 2..4 mbarrier stages, fifteen consumer warps take work items:
//      * 2..16 items: 32 segments per item, one per lane, each sorted in
//        registers by the network of Sec. 2 for its class (2, 4, 8, 12 or 16
//        channels, shorter segments padded with +inf);
//      * 17..32 items: 16 segments per item, two lanes per segment: each
//        lane sorts 16 items with the 16-channel network, then the lane pair
//        merges through shuffles (mirrored exchange + in-register half
//        cleaners), i.e. a 32-item bitonic merge across two lanes.
//    Sorted tiles return through bulk stores; the partial 16-byte granules at
//    a tile's ends, shared with its neighbours, are written with plain stores.
// 4. seg_rss_kernel -- persistent independent warps, tiles assigned
//    round-robin to warps; each warp lists the RSS entries of its tiles,
//    stages segments with bulk copies two ahead of the one it sorts, and sorts
//    each by Register Sample Sort (Sec. 3): a sample of a*k items sorted by a
//    network, k-1 splitters taken equidistant, the branch-free descent
//    j <- 2j + [t_j < e] over the splitter tree (Algorithm 1 generalised), a
//    counting scatter, and a network per bucket; results go straight to
//    global memory.  Segments of 33..64 items may take a 64-channel warp
//    network instead (a launch parameter; never in the RSS-only calls).
// With a payload, items are (key, position) pairs so ties keep input order and
// the payload is gathered by position at the end.  Few distinct network sizes
// keep the instruction working set small: with one network per n, warps
// running different n thrashed the instruction cache (the GPU analogue of the
// L1i misses the paper measured in Sec. 4.4 / 4.6).
#pragma once

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "sn_common.cuh"
#include "sn_internal.h"
#include "sn_seg_scratch.h"

namespace sn {
namespace seg {
namespace {  // internal linkage: each instantiation unit gets its own copy

constexpr int kTileWarps = 15;
constexpr int kTileConsumers = kTileWarps * 32;
constexpr int kTileThreads = kTileConsumers + 32;  // + one producer warp
constexpr int kMaxStages = 4;  // tile-kernel staging depth: 2..4 stages (a launch parameter)
constexpr int kRssWarps = 8;
constexpr int kRssThreads = kRssWarps * 32;
constexpr int kMaxSeg = 256;
constexpr uint32_t kDone = 0xFFFFFFFFu;
constexpr int kRssMaxBuckets = 32;  // one bucket per lane
constexpr unsigned kFull = 0xFFFFFFFFu;

// Classes handled by the tile kernel, in list and hand-out order.
enum TileCls : int { kPair = 0, kNet16, kNet12, kNet8, kNet4, kNet2, kNumTileCls };
constexpr int kRssCls = kNumTileCls;
constexpr int kSkipCls = kNumTileCls + 1;

// Bit q of `net_mask` enables the padded network class 2, 4, 8, 12 (q = 0..3);
// a segment of 2..16 items takes the smallest enabled class that holds it,
// 16 channels if none does.
__device__ __forceinline__ int seg_class(uint32_t len, bool rss_only, uint32_t net_mask) {
  if (len <= 1) return kSkipCls;
  if (len == 2 && (net_mask & 1u)) return kNet2;
  if (len <= 4 && (net_mask & 2u)) return kNet4;
  if (len <= 8 && (net_mask & 4u)) return kNet8;
  if (len <= 12 && (net_mask & 8u)) return kNet12;
  if (len <= 16) return kNet16;
  if (len <= 32 && !rss_only) return kPair;
  return kRssCls;
}

struct TileMeta {
  uint32_t tile;
  uint32_t s0, s1;        // segments [s0, s1)
  uint32_t e0, e1;        // items [e0, e1)
  uint32_t off_shift;     // index of offsets[s0] in the staged offsets
  uint32_t key_shift;     // index of keys[e0] in the staged keys
  uint32_t val_shift;     // index of vals[e0] in the staged payload
  uint32_t ord_shift;     // index of order[s0] in the staged bins
  // ring tile kernel: byte offsets of the packed regions in the stage (the
  // offsets start at 0) and the staged key / payload capacities in elements
  uint32_t ord_at, cnt_at, key_at, val_at;
  uint32_t key_cap, val_cap;
};

// ------------------------------------------------------ staging layouts ----

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }
__host__ __device__ inline size_t align128(size_t x) { return (x + 127) & ~static_cast<size_t>(127); }

template <class K, bool kVals>
struct TileLayout {
  size_t off_at, key_at, val_at, ord_at, cnt_at, stage_bytes;
  __host__ __device__ size_t total(int stages) const { return stages * stage_bytes; }
  __host__ __device__ explicit TileLayout(uint32_t E) {
    off_at = 0;
    key_at = align16(off_at + (E + 1 + 8) * 4);
    val_at = align16(key_at + static_cast<size_t>(E + kMaxSeg + 2 * (16 / sizeof(K))) * sizeof(K));
    ord_at = align16(val_at + (kVals ? (E + kMaxSeg + 8) * 4 : 0));
    cnt_at = align16(ord_at + (E + 16) * 2);
    stage_bytes = align128(cnt_at + 16);
  }
};

// Ring tile kernel staging: a staged tile's regions (offsets, bins, class
// counts, keys, payload) are packed one after the other, each sized by the
// tile itself (TileMeta records where they start).  A tile of ns segments and
// `items` items has ns + items <= E + 256, so a stage of
// max(6, key + payload bytes) bytes per unit of E + 256, plus the granule
// rounding of each copy, holds any tile: about two thirds of the fixed
// layout's stage for 8-byte keys with payload.
template <class K, bool kVals>
struct RingLayout {
  static constexpr size_t kPerItem = sizeof(K) + (kVals ? 4 : 0);
  static constexpr size_t kPerUnit = kPerItem > 6 ? kPerItem : 6;
  size_t stage_bytes;
  __host__ __device__ size_t total(int stages) const { return stages * stage_bytes; }
  __host__ __device__ explicit RingLayout(uint32_t E) {
    stage_bytes = align128(kPerUnit * (static_cast<size_t>(E) + kMaxSeg) + 256);
  }
};

// Items of the RSS buckets: (key, position) pairs when a payload must follow
// its key, bare keys otherwise (equal keys are then interchangeable).
template <class K>
struct KeyOnly {
  using T = K;
  static __device__ __forceinline__ K make(K key, uint32_t) { return key; }
  static __device__ __forceinline__ K key(K it) { return it; }
  static __device__ __forceinline__ uint32_t idx(K) { return 0; }
  static __device__ __forceinline__ K sentinel(uint32_t) { return static_cast<K>(~static_cast<K>(0)); }
};
template <class K, bool kVals>
using RssIO = typename std::conditional<kVals, ItemOf<K>, KeyOnly<K>>::type;

// Per-warp Register Sample Sort scratch: 256 bucket items + 32 bucket counters.
template <class K, bool kVals> struct RssMem;
template <class K> struct RssMem<K, false> {
  static constexpr size_t kBytes = 256 * sizeof(K) + kRssMaxBuckets * 4;
  K* key;
  uint32_t* cnt;
  __device__ __forceinline__ explicit RssMem(unsigned char* p)
      : key(reinterpret_cast<K*>(p)), cnt(reinterpret_cast<uint32_t*>(p + 256 * sizeof(K))) {}
  __device__ __forceinline__ K get(int i) const { return key[i]; }
  __device__ __forceinline__ void set(int i, K v) const { key[i] = v; }
};
template <> struct RssMem<uint32_t, true> {
  static constexpr size_t kBytes = 256 * 8 + kRssMaxBuckets * 4;
  uint64_t* buf;  // packed (key, position) items
  uint32_t* cnt;
  __device__ __forceinline__ explicit RssMem(unsigned char* p)
      : buf(reinterpret_cast<uint64_t*>(p)), cnt(reinterpret_cast<uint32_t*>(p + 256 * 8)) {}
  __device__ __forceinline__ uint64_t get(int i) const { return buf[i]; }
  __device__ __forceinline__ void set(int i, uint64_t v) const { buf[i] = v; }
  // slot i as a parking place for a payload word (in-place write-back)
  __device__ __forceinline__ void stash(int i, uint32_t v) const { buf[i] = v; }
  __device__ __forceinline__ uint32_t unstash(int i) const { return static_cast<uint32_t>(buf[i]); }
};
template <> struct RssMem<uint64_t, true> {
  static constexpr size_t kBytes = 256 * 8 + 256 * 2 + kRssMaxBuckets * 4;
  uint64_t* key;
  uint16_t* idx;
  uint32_t* cnt;
  __device__ __forceinline__ explicit RssMem(unsigned char* p)
      : key(reinterpret_cast<uint64_t*>(p)), idx(reinterpret_cast<uint16_t*>(p + 256 * 8)),
        cnt(reinterpret_cast<uint32_t*>(p + 256 * 10)) {}
  __device__ __forceinline__ Item64 get(int i) const { return Item64{key[i], idx[i]}; }
  __device__ __forceinline__ void set(int i, const Item64& v) const {
    key[i] = v.key;
    idx[i] = static_cast<uint16_t>(v.idx);
  }
  __device__ __forceinline__ void stash(int i, uint32_t v) const { key[i] = v; }
  __device__ __forceinline__ uint32_t unstash(int i) const { return static_cast<uint32_t>(key[i]); }
};

// Per-warp region of the RSS kernel: kRssBufs staging buffers (keys, payload)
// with one mbarrier each, the RSS scratch.
constexpr int kRssBufs = 3;
template <class K, bool kVals>
struct RssWarpLayout {
  static constexpr size_t kKeyCap = (kMaxSeg + 2 * (16 / sizeof(K))) * sizeof(K);
  static constexpr size_t kValCap = kVals ? (kMaxSeg + 8) * 4 : 0;
  static constexpr size_t kBar = 0;
  static constexpr size_t kKeys = 32;
  static constexpr size_t kVals_ = kKeys + kRssBufs * kKeyCap;
  static constexpr size_t kScratch = (kVals_ + kRssBufs * kValCap + 15) & ~static_cast<size_t>(15);
  static constexpr size_t kBytes = (kScratch + RssMem<K, kVals>::kBytes + 127) & ~static_cast<size_t>(127);
};

// ---------------------------------------------------------------- plan -----

// Position p = s + a of segment s, a = (address of offsets / 4) mod 4: the
// offsets are read in aligned 16-byte groups, group g holding the offsets of
// positions 4g .. 4g + 3, and the segment classes are written one byte per
// position, a 4-byte word per group.  A group's 16 bytes never leave the
// 16-byte granule of an offset that exists, so reading the unused part of the
// first and last groups cannot fault.
__device__ __forceinline__ int plan_shift(const uint32_t* offsets) {
  return static_cast<int>((reinterpret_cast<uintptr_t>(offsets) & 15) / 4);
}

// Tile of position u (u < 2^33: a segment index plus an item offset) for
// tiles of E = m 2^k units, m odd: u >> k for m = 1; for m = 3 (E = 3072,
// 6144, 12288; k >= 8, so u >> k fits 32 bits) a multiply-high by the
// rounded-up 2^33 / 3, exact for every 32-bit dividend (division by an
// invariant integer through multiplication, Granlund and Montgomery); else
// u / E.
struct TileDiv {
  int k;
  uint32_t m, E;
  __device__ __forceinline__ uint32_t operator()(uint64_t u) const {
    if (m == 1) return static_cast<uint32_t>(u >> k);
    if (m == 3) return __umulhi(static_cast<uint32_t>(u >> k), 0xAAAAAAABu) >> 1;
    return static_cast<uint32_t>(u / E);
  }
};

constexpr int kPlanU = 4;

// One thread per group (grid-stride over whole warps): validates every
// segment, records the first segment of every tile, and writes each
// segment's class byte (seg_class of its length; kSkipCls past the batch).
// Groups whose four segments all exist and precede the last one take a
// 32-bit path; the others (the batch's two ends) the general one.
__global__ void __launch_bounds__(256)
    seg_plan_kernel(const uint32_t* __restrict__ offsets, uint64_t nseg, TileDiv tile_of, Plan* plan,
                    uint32_t* __restrict__ tile_first, uint64_t tile_cap, uint32_t* __restrict__ cls, bool rss_only,
                    uint32_t net_mask, unsigned* status) {
  __shared__ uint8_t cls_of[34];
  if (threadIdx.x < 34) cls_of[threadIdx.x] = static_cast<uint8_t>(seg_class(threadIdx.x, rss_only, net_mask));
  __syncthreads();
  const int a = plan_shift(offsets);
  const uint4* ov = reinterpret_cast<const uint4*>(offsets - a);
  const uint32_t base = offsets[0];
  const int lane = threadIdx.x & 31;
  // groups covering offsets[0 .. nseg]
  const uint64_t ngroups = (nseg + static_cast<uint64_t>(a)) / 4 + 1;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  // kPlanU runs of 32 groups per warp and step (run u: groups g0 + 32 u +
  // lane), their loads issued together
  for (uint64_t gw = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31u)) * kPlanU;
       gw < ngroups; gw += stride * kPlanU) {
    uint4 vv[kPlanU];
#pragma unroll
    for (int u = 0; u < kPlanU; ++u) {
      const uint64_t g = gw + 32 * u + lane;
      vv[u] = g < ngroups ? ov[g] : make_uint4(0u, 0u, 0u, 0u);
    }
    // the offsets just before and just after the step's groups
    const int64_t lo_i = static_cast<int64_t>(4 * gw) - a - 1;
    const int64_t hi_i = static_cast<int64_t>(4 * (gw + 32 * kPlanU)) - a;
    const uint32_t edge_lo = lo_i >= 0 ? offsets[lo_i] : 0u;
    const uint32_t edge_hi = hi_i <= static_cast<int64_t>(nseg) ? offsets[hi_i] : 0u;
#pragma unroll
    for (int u = 0; u < kPlanU; ++u) {
    const uint64_t g = gw + 32 * u + lane;
    const bool in = g < ngroups;
    const uint4 v = vv[u];
    // the offset after the group's last position and the one before its first
    // (across runs from the neighbouring run, across steps from the edges)
    uint32_t nx = __shfl_down_sync(kFull, v.x, 1);
    uint32_t pw = __shfl_up_sync(kFull, v.w, 1);
    const uint32_t nx31 = u + 1 < kPlanU ? __shfl_sync(kFull, vv[u + 1 < kPlanU ? u + 1 : u].x, 0) : edge_hi;
    const uint32_t pw0 = u > 0 ? __shfl_sync(kFull, vv[u > 0 ? u - 1 : 0].w, 31) : edge_lo;
    if (lane == 31) nx = nx31;
    if (lane == 0) pw = pw0;
    const int64_t first = static_cast<int64_t>(4 * g) - a;  // segment of position 4g
    const uint32_t o[6] = {pw, v.x, v.y, v.z, v.w, nx};
    uint32_t word = 0;
    if (in && first >= 1 && first + 5 <= static_cast<int64_t>(nseg)) {
      const uint64_t f = static_cast<uint64_t>(first);
      uint32_t tp = tile_of(f - 1 + (pw - base));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t o0 = o[k + 1], o1 = o[k + 2];
        const uint32_t len = o1 - o0;
        bad |= o1 < o0 || len > kMaxSeg || o0 < base;
        word |= static_cast<uint32_t>(cls_of[min(len, 33u)]) << (8 * k);
        const uint32_t t = tile_of(f + k + (o0 - base));
        if (t != tp && t < tile_cap) tile_first[t] = static_cast<uint32_t>(f + k);
        tp = t;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t sk = first + k;
        uint32_t c = kSkipCls;
        if (in && sk >= 0 && sk < static_cast<int64_t>(nseg)) {
          const uint64_t sq = static_cast<uint64_t>(sk);
          const uint32_t o0 = o[k + 1], o1 = o[k + 2], op = o[k];
          const uint32_t len = o1 - o0;
          if (o1 < o0 || len > kMaxSeg || o0 < base) bad = true;
          c = cls_of[len < 33u ? len : 33u];
          const uint64_t t = tile_of(sq + static_cast<uint64_t>(o0 - base));
          const uint64_t tp = sq > 0 ? tile_of((sq - 1) + static_cast<uint64_t>(op - base)) : ~0ull;
          if (t != tp && t < tile_cap) tile_first[t] = static_cast<uint32_t>(sq);
          if (sq == nseg - 1) {
            if (t + 1 < tile_cap) {
              tile_first[t + 1] = static_cast<uint32_t>(nseg);
              plan->ntiles = static_cast<unsigned>(t + 1);
            } else {
              bad = true;
            }
          }
        }
        word |= c << (8 * k);
      }
    }
    if (in) cls[g] = word;
    }
  }
  if (bad) {
    atomicOr(&plan->bad, 1u);
    atomicOr(status, kStatusRange);
  }
}

// ----------------------------------------------------------------- bin -----

// One warp per tile (grid-stride over warps), reading the class bytes of the
// tile's segments, four per lane (one word) and 128 per warp step:
// counts[8t + c] for the tile classes c and counts[8t + 6] for Register
// Sample Sort, and the tile-local indices of its segments grouped by class
// (classes in hand-out order, RSS last; any order inside a class) in
// order[s0 .. s1).  Each class has a one-byte field of a 64-bit word; a
// lane's four bytes give its fields, and a warp-wide add per half word sums
// a step.  Placing: an inclusive warp scan of the lanes' field words gives
// every lane, per class, the entries of the lanes before it; a segment's
// place is its class's running start (per-warp shared memory) plus that plus
// its rank among the lane's own bytes.  (Fields never carry: a step adds at
// most 128 to one.)
constexpr int kBinWarps = 8;
constexpr int kBinU = 4;  // warp steps whose loads are issued together
__global__ void __launch_bounds__(kBinWarps * 32)
    seg_bin_kernel(const uint32_t* __restrict__ cls, const uint32_t* __restrict__ offsets, const Plan* plan,
                   const uint32_t* __restrict__ tile_first, uint16_t* __restrict__ counts,
                   uint16_t* __restrict__ order) {
  constexpr int kCls = kNumTileCls + 1;  // tile classes + RSS; kSkipCls (= kCls) is not listed
  static_assert(kSkipCls == 7, "eight class fields");
  __shared__ uint32_t cur_s[kBinWarps][8];
  const int lane = threadIdx.x & 31;
  uint32_t* cur = cur_s[threadIdx.x >> 5];
  const unsigned ntiles = plan->bad ? 0u : plan->ntiles;
  const unsigned W = gridDim.x * kBinWarps;
  const uint32_t a = static_cast<uint32_t>(plan_shift(offsets));
  // a word's four class bytes, those outside positions [p0, p1) set to kSkipCls
  auto load = [&](uint32_t wi, uint32_t p0, uint32_t p1, uint32_t w1) -> uint32_t {
    uint32_t w = wi < w1 ? cls[wi] : 0x07070707u;
    if (4 * wi < p0 || 4 * wi + 4 > p1) {  // the tile's first or last word
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t p = 4 * wi + k;
        if (p < p0 || p >= p1) w |= 7u << (8 * k);
      }
    }
    return w;
  };
  // one-byte class fields: fld[c] = 1 << 8c
  __shared__ uint64_t fld[8];
  if (threadIdx.x < 8) fld[threadIdx.x] = 1ull << (8 * threadIdx.x);
  __syncthreads();
  auto fields = [&](uint32_t w) -> uint64_t {
    uint64_t f = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) f += fld[(w >> (8 * k)) & 7u];
    return f;
  };
  for (unsigned t = blockIdx.x * kBinWarps + (threadIdx.x >> 5); t < ntiles; t += W) {
    const uint32_t s0 = tile_first[t], s1 = tile_first[t + 1];
    const uint32_t p0 = s0 + a, p1 = s1 + a;
    const uint32_t w0 = p0 / 4, w1 = (p1 + 3) / 4;
    uint32_t tot[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (uint32_t wb = w0; wb < w1; wb += 32 * kBinU) {
      uint32_t ws[kBinU];  // kBinU steps' loads in flight together
#pragma unroll
      for (int u = 0; u < kBinU; ++u) ws[u] = load(wb + 32 * u + lane, p0, p1, w1);
#pragma unroll
      for (int u = 0; u < kBinU; ++u) {
        if (wb + 32 * u >= w1) break;  // warp-uniform
        const uint64_t f = fields(ws[u]);
        const uint32_t lo = __reduce_add_sync(kFull, static_cast<uint32_t>(f));
        const uint32_t hi = __reduce_add_sync(kFull, static_cast<uint32_t>(f >> 32));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          tot[q] += __byte_perm(lo, 0u, 0x4440 + q);
          tot[4 + q] += __byte_perm(hi, 0u, 0x4440 + q);
        }
      }
    }
    uint32_t at = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (lane == q) {
        cur[q] = at;
        counts[8ull * t + q] = static_cast<uint16_t>(q < kCls ? tot[q] : 0u);
      }
      at += tot[q];
    }
    __syncwarp();
    for (uint32_t wb0 = w0; wb0 < w1; wb0 += 32 * kBinU) {
      uint32_t ws[kBinU];
#pragma unroll
      for (int u = 0; u < kBinU; ++u) ws[u] = load(wb0 + 32 * u + lane, p0, p1, w1);
#pragma unroll
      for (int u = 0; u < kBinU; ++u) {
      if (wb0 + 32 * u >= w1) break;  // warp-uniform
      const uint32_t wi = wb0 + 32 * u + lane;
      const uint32_t w = ws[u];
      const uint64_t f = fields(w);
      uint32_t slo = static_cast<uint32_t>(f), shi = static_cast<uint32_t>(f >> 32);
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t ylo = __shfl_up_sync(kFull, slo, d), yhi = __shfl_up_sync(kFull, shi, d);
        if (lane >= d) {
          slo += ylo;
          shi += yhi;
        }
      }
      const uint32_t tlo = __shfl_sync(kFull, slo, 31), thi = __shfl_sync(kFull, shi, 31);
      // entries before a byte: its class's field of the lanes below, plus
      // the lane's own earlier bytes of that class
      const uint64_t ex = ((static_cast<uint64_t>(shi) << 32) | slo) - f;
      const uint32_t elo = static_cast<uint32_t>(ex), ehi = static_cast<uint32_t>(ex >> 32);
      uint32_t c[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) c[k] = (w >> (8 * k)) & 7u;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        uint32_t rank = __byte_perm(elo, ehi, c[k]) & 0xFFu;
#pragma unroll
        for (int k2 = 0; k2 < k; ++k2) rank += c[k2] == c[k] ? 1u : 0u;
        if (c[k] < static_cast<uint32_t>(kCls))
          order[s0 + cur[c[k]] + rank] = static_cast<uint16_t>(4 * wi + k - p0);
      }
      __syncwarp();
      if (lane < 8) cur[lane] += ((lane < 4 ? tlo : thi) >> ((lane & 3) * 8)) & 0xFFu;
      __syncwarp();
      }
    }
  }
}

// ----------------------------------------------- slot-composite networks --
//
// With a payload the networks run on 32-bit composites instead of (key,
// position) items: item q of a segment becomes c_q = w_q << B | q, B the bits
// of a slot number and w_q a (32 - B)-bit window of its order-encoded key.
// The window ends at the highest bit in which the segment's keys differ (all
// keys agree above it), so two composites compare like their keys whenever
// their windows differ, and like their positions when the window holds every
// differing bit and the keys are equal: the composite order is then exactly
// the (key, position) order, at one 32-bit min/max per side of a
// compare-exchange (Sec. 2.1's comparator on a derived key).  Only when the
// differing bits are wider than the window can two different keys share a
// window; a check of adjacent composites finds that, and the segment is then
// sorted again, exactly, by a stable insertion sort.  Keys and payload are
// gathered by slot after the network.

template <int N>
__host__ __device__ constexpr int slot_bits() {
  return N <= 2 ? 1 : N <= 4 ? 2 : N <= 8 ? 3 : N <= 16 ? 4 : N <= 32 ? 5 : 6;
}

template <class K>
__device__ __forceinline__ int high_bit(K x) {
  if constexpr (sizeof(K) == 8)
    return x ? 63 - __clzll(static_cast<long long>(x)) : -1;
  else
    return x ? 31 - __clz(static_cast<int>(x)) : -1;
}

// Shift that puts the highest differing bit at the top of a W-bit window.
template <class K>
__device__ __forceinline__ int window_shift(K diff, int W) {
  const int h = high_bit(diff);
  return h >= W ? h - (W - 1) : 0;
}

template <class K>
__device__ __forceinline__ uint32_t window_of(K a, int sh, int W) {
  return static_cast<uint32_t>(a >> sh) & ((1u << W) - 1u);
}

// Stable insertion sort of one segment in place in shared memory (by the
// encoded key, payload moved along): the exact fallback of the composites.
template <class K, bool kVals, bool kF>
__device__ __noinline__ void insertion_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L) {
  for (int i = 1; i < L; ++i) {
    const K x = kbuf[p + i];
    const K ex = key_enc<K, kF>(x);
    const uint32_t v = kVals ? vbuf[pv + i] : 0u;
    int j = i - 1;
    while (j >= 0 && key_enc<K, kF>(kbuf[p + j]) > ex) {
      kbuf[p + j + 1] = kbuf[p + j];
      if constexpr (kVals) vbuf[pv + j + 1] = vbuf[pv + j];
      --j;
    }
    kbuf[p + j + 1] = x;
    if constexpr (kVals) vbuf[pv + j + 1] = v;
  }
}

// One lane's segment of 2 <= L <= N items at kbuf[p..p+L), payload at
// vbuf[pv..pv+L), sorted in place through composites.
template <int N, class K, bool kVals, bool kF>
__device__ __forceinline__ void slot_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L) {
  constexpr int B = slot_bits<N>();
  constexpr int W = 32 - B;
  constexpr uint32_t kSlot = (1u << B) - 1u;
  K k[N];
#pragma unroll
  for (int q = 0; q < N; ++q) k[q] = q < L ? key_enc<K, kF>(kbuf[p + q]) : K(0);
  K diff = 0;
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q < L) diff |= k[q] ^ k[0];
  const int sh = window_shift(diff, W);
  uint32_t c[N];
#pragma unroll
  for (int q = 0; q < N; ++q)
    c[q] = (q < L ? window_of(k[q], sh, W) << B : ~kSlot) | static_cast<uint32_t>(q);
  Net<N>::run(c);
  if (sh > 0) {  // the window may miss differing bits: two keys may share it
    bool tie = false;
#pragma unroll
    for (int q = 0; q + 1 < N; ++q) tie |= (c[q] >> B) == (c[q + 1] >> B) && (c[q + 1] & kSlot) < static_cast<uint32_t>(L);
    if (tie) {
      insertion_segment<K, kVals, kF>(kbuf, vbuf, p, pv, L);
      return;
    }
  }
  // the first L composites are the real items in order: gather by slot
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q < L) k[q] = kbuf[p + (c[q] & kSlot)];
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q < L) kbuf[p + q] = k[q];
  if constexpr (kVals) {
    uint32_t v[N];
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < L) v[q] = vbuf[pv + (c[q] & kSlot)];
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < L) vbuf[pv + q] = v[q];
  }
}

// ------------------------------------------------------ per-lane networks --

// Segment of 2 <= L <= N items at kbuf[p..p+L) (payload at vbuf[pv..pv+L)):
// with a payload through composites (slot_segment), keys alone by the
// network itself, padded with +inf to N channels.  (Composites for 8-byte
// keys alone were measured slower: the gather and the extra registers cost
// more than the 64-bit min/max they replace.)
template <int N, class K, bool kVals, bool kF>
__device__ __forceinline__ void net_segment(K* kbuf, uint32_t* vbuf, int p, int pv, int L) {
  if constexpr (kVals) {
    slot_segment<N, K, kVals, kF>(kbuf, vbuf, p, pv, L);
  } else {
    K k[N];
#pragma unroll
    for (int q = 0; q < N; ++q) k[q] = q < L ? key_enc<K, kF>(kbuf[p + q]) : static_cast<K>(~static_cast<K>(0));
    Net<N>::run(k);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < L) kbuf[p + q] = key_dec<K, kF>(k[q]);
  }
}

// ---------------------------------------------------- 17..32 on two lanes --

// The smaller / larger of the lane's item `a` and its partner's `b`; on equal
// keys each lane keeps its own item, so the exchange stays a permutation.
template <class T>
__device__ __forceinline__ T lo_of(const T& a, const T& b) {
  return item_less(b, a) ? b : a;
}
template <class T>
__device__ __forceinline__ T hi_of(const T& a, const T& b) {
  return item_less(a, b) ? b : a;
}
__device__ __forceinline__ uint32_t lo_of(uint32_t a, uint32_t b) { return min(a, b); }
__device__ __forceinline__ uint32_t hi_of(uint32_t a, uint32_t b) { return max(a, b); }
__device__ __forceinline__ uint64_t lo_of(uint64_t a, uint64_t b) { return min(a, b); }
__device__ __forceinline__ uint64_t hi_of(uint64_t a, uint64_t b) { return max(a, b); }

// 32 channels on a lane pair: the even lane holds items 0..15, the odd lane
// 16..31; both sort with the 16-channel network, then a bitonic merge: the
// mirrored exchange x_i <-> partner x_{15-i} leaves the 16 smallest on the
// even lane and the 16 largest on the odd lane, each a bitonic sequence that
// four in-register half-cleaner levels sort.
template <class T>
__device__ __forceinline__ void pair_merge(T (&x)[16], bool upper) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const T a = shfl_xor(x[15 - q], 1);
    const T b = shfl_xor(x[q], 1);
    if (upper) {
      x[q] = hi_of(x[q], a);
      x[15 - q] = hi_of(x[15 - q], b);
    } else {
      x[q] = lo_of(x[q], a);
      x[15 - q] = lo_of(x[15 - q], b);
    }
  }
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if ((i & m) == 0) ce(x[i], x[i | m]);
  }
}

// The 16-channel path shared by two kinds of work item, so that the GPU runs
// one copy of the 16-channel network code for both:
//  * pair = false: the lane's own segment of L <= 16 items (padded to 16);
//  * pair = true:  a segment of 17..32 items on lanes (lane & ~1, lane | 1):
//    the even lane holds items 0..15, the odd lane 16..31; after the network
//    the lanes merge (pair_merge).  `pair` is warp-uniform.
// Lanes without a segment (active = false) still take part in the shuffles.
template <class K, bool kVals, bool kF>
__device__ __forceinline__ void seg16(K* kbuf, uint32_t* vbuf, int p, int pv, int L, bool active, bool pair,
                                      int lane) {
  const bool upper = pair && (lane & 1);
  const int base = upper ? 16 : 0;
  if constexpr (kVals) {
    // composites (see slot_segment) with 5-bit slots, one code path for both
    // kinds of work item: a lane's own segment (slots 0..15), or a lane
    // pair's (the even lane slots 0..15, the odd lane 16..31, merged after
    // the network by exchanging one 32-bit word per item)
    constexpr int B = 5, W = 27;
    K k[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) k[q] = (active && base + q < L) ? key_enc<K, kF>(kbuf[p + base + q]) : K(0);
    const K a0 = shfl_idx(k[0], pair ? (lane & ~1) : lane);  // the segment's first key
    K diff = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (active && base + q < L) diff |= k[q] ^ a0;
    const K partner_diff = shfl_xor(diff, 1);
    if (pair) diff |= partner_diff;
    const int sh = window_shift(diff, W);
    uint32_t c[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
      c[q] = ((active && base + q < L) ? window_of(k[q], sh, W) << B : ~31u) | static_cast<uint32_t>(base + q);
    Net<16>::run(c);
    if (pair) pair_merge(c, upper);
    bool tie = false;
    if (sh > 0) {  // two different keys may share a window: check neighbours
#pragma unroll
      for (int q = 0; q < 15; ++q) tie |= (c[q] >> B) == (c[q + 1] >> B) && (c[q + 1] & 31u) < static_cast<uint32_t>(L);
    }
    // the even lane's last item and the odd lane's first; the pair decides
    // together (every lane takes part in both shuffles)
    const uint32_t prev = __shfl_xor_sync(kFull, c[15], 1);
    if (pair && upper && sh > 0) tie |= (prev >> B) == (c[0] >> B) && (c[0] & 31u) < static_cast<uint32_t>(L);
    const int partner_tie = __shfl_xor_sync(kFull, tie ? 1 : 0, 1);
    tie = active && (tie || (pair && partner_tie != 0));
    const bool write = active && !tie;
    // gather by slot; both lanes of a pair gather before either writes
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (write && base + q < L) k[q] = kbuf[p + (c[q] & 31u)];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (write && base + q < L) kbuf[p + base + q] = k[q];
    uint32_t v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (write && base + q < L) v[q] = vbuf[pv + (c[q] & 31u)];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (write && base + q < L) vbuf[pv + base + q] = v[q];
    if (tie && !upper && L >= 2) insertion_segment<K, kVals, kF>(kbuf, vbuf, p, pv, L);
  } else {
    K x[16];
#pragma unroll
    for (int q = 0; q < 16; ++q)
      x[q] = (active && base + q < L) ? key_enc<K, kF>(kbuf[p + base + q]) : static_cast<K>(~static_cast<K>(0));
    Net<16>::run(x);
    if (pair) pair_merge(x, upper);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q)
      if (active && base + q < L) kbuf[p + base + q] = key_dec<K, kF>(x[q]);
  }
}

// --------------------------------------------------- Register Sample Sort --

// Bucket of c (<= N) items at rm[st..st+c), padded to N with +inf.
template <int N, class K, bool kVals>
__device__ __forceinline__ void bucket_network(const RssMem<K, kVals>& rm, int st, int c) {
  using IO = RssIO<K, kVals>;
  if constexpr (kVals && sizeof(K) == 8) {
    // 8-byte keys with positions: key-first network with the positions
    // carried; a (key, position) pass only when equal keys were left out of
    // position order
    KeyIdx<K> it[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const typename IO::T x = q < c ? rm.get(st + q) : IO::sentinel(q);
      it[q] = KeyIdx<K>{IO::key(x), IO::idx(x)};
    }
    Net<N>::run(it);
    bool tie = false;
#pragma unroll
    for (int q = 0; q + 1 < N; ++q) tie |= tie_misordered(it[q], it[q + 1], 0x10000u);  // sentinels: 0x10000 + slot
    if (tie) {
      typename IO::T full[N];
#pragma unroll
      for (int q = 0; q < N; ++q) full[q] = IO::make(it[q].k, it[q].ix);
      Net<N>::run(full);
#pragma unroll
      for (int q = 0; q < N; ++q) it[q] = KeyIdx<K>{IO::key(full[q]), IO::idx(full[q])};
    }
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < c) rm.set(st + q, IO::make(it[q].k, it[q].ix));
  } else {
    // bare keys (equal keys are interchangeable), or 4-byte keys packed with
    // their positions into one 64-bit word that a single min/max orders
    typename IO::T k[N];
#pragma unroll
    for (int q = 0; q < N; ++q) k[q] = q < c ? rm.get(st + q) : IO::sentinel(q);
    Net<N>::run(k);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q < c) rm.set(st + q, k[q]);
  }
}

// The network for the warp's largest bucket m <= 16: 4, 8, 12 or 16 channels
// for 4-byte keys; for 8-byte keys only 8 or 16 (their networks' code is
// twice as large, and with four sizes the warps, each in a different one,
// missed the instruction cache more than the smaller networks saved: u64 RSS
// range 2.02 -> 1.92 ms, while the same change made u32 2 % slower).
template <class K, bool kVals>
__device__ __forceinline__ void bucket_network_class(int m, const RssMem<K, kVals>& rm, int st, int c) {
  if constexpr (sizeof(K) == 8) {
    if (m <= 8)
      bucket_network<8, K, kVals>(rm, st, c);
    else
      bucket_network<16, K, kVals>(rm, st, c);
  } else {
    if (m <= 4)
      bucket_network<4, K, kVals>(rm, st, c);
    else if (m <= 8)
      bucket_network<8, K, kVals>(rm, st, c);
    else if (m <= 12)
      bucket_network<12, K, kVals>(rm, st, c);
    else
      bucket_network<16, K, kVals>(rm, st, c);
  }
}


// Warp-cooperative ascending bitonic sort of n <= 256 stored items at
// rm[st..st+n), padded virtually to the next power of two with +inf:
// comparators that reach past n are skipped.
template <class K, bool kVals>
__device__ __forceinline__ void warp_bitonic_smem(const RssMem<K, kVals>& rm, int st, int n, int lane) {
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
          if (item_less(b, a)) {
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

// Segments of 33..64 items outside the RSS-only calls (launch parameter
// net_classes bit 4): a 64-channel warp network, two items per lane
// (warp_sort64), in place of Register Sample Sort, whose sample sort and
// classification cost more than the whole network at this size.  With a
// payload, and for 8-byte keys, the network sorts 32-bit composites of a key
// window and a 6-bit slot (see slot_segment), exact (key, position) items
// only when two different keys share a window; keys and payload are then
// gathered by slot.
// kInPlace: gk / gv point into the staged copy itself (the results replace
// the segment where it is staged), so every lane gathers its payload before
// any lane writes.
template <class K, bool kVals, bool kF, bool kInPlace = false>
__device__ __forceinline__ void net64_segment(const K* kbuf, const uint32_t* vbuf, int p, int pv, int L, int lane,
                                              K* gk, uint32_t* gv) {
  const int e1 = 32 + lane;
  constexpr K kTop = static_cast<K>(~static_cast<K>(0));
  if constexpr (kVals || sizeof(K) == 8) {
    // composites with 6-bit slots (see slot_segment); the exact fallback
    // sorts (key, position) items through the same network
    constexpr int B = 6, W = 26;
    const K klo = lane < L ? key_enc<K, kF>(kbuf[p + lane]) : K(0);
    const K khi = e1 < L ? key_enc<K, kF>(kbuf[p + e1]) : K(0);
    const K a0 = shfl_idx(klo, 0);
    K d = (lane < L ? klo ^ a0 : K(0)) | (e1 < L ? khi ^ a0 : K(0));
    if constexpr (sizeof(K) == 8) {
      const uint32_t dl = __reduce_or_sync(kFull, static_cast<uint32_t>(d));
      const uint32_t dh = __reduce_or_sync(kFull, static_cast<uint32_t>(d >> 32));
      d = (static_cast<K>(dh) << 32) | dl;
    } else {
      d = __reduce_or_sync(kFull, d);
    }
    const int sh = window_shift(d, W);
    uint32_t clo = (lane < L ? window_of(klo, sh, W) << B : ~63u) | static_cast<uint32_t>(lane);
    uint32_t chi = (e1 < L ? window_of(khi, sh, W) << B : ~63u) | static_cast<uint32_t>(e1);
    warp_sort64(clo, chi, lane);
    bool tie = false;
    if (sh > 0) {  // two different keys may share a window: check neighbouring slots
      const uint32_t lo_prev = __shfl_sync(kFull, clo, (lane + 31) & 31);
      const uint32_t hi_prev = __shfl_sync(kFull, chi, (lane + 31) & 31);
      auto same = [&](uint32_t x, uint32_t y) {
        return (x >> B) == (y >> B) && (y & 63u) < static_cast<uint32_t>(L);
      };
      tie = lane > 0 ? (same(lo_prev, clo) || same(hi_prev, chi)) : same(lo_prev, chi);
    }
    if (__any_sync(kFull, tie)) {
      using FI = ItemOf<K>;
      typename FI::T a = lane < L ? FI::make(klo, static_cast<uint32_t>(lane)) : FI::sentinel(lane);
      typename FI::T b = e1 < L ? FI::make(khi, static_cast<uint32_t>(e1)) : FI::sentinel(e1);
      warp_sort64(a, b, lane);
      clo = FI::idx(a);
      chi = FI::idx(b);
    } else {
      clo &= 63u;
      chi &= 63u;
    }
    // gather by slot from the staged copy; every lane before any lane writes
    const K olo = lane < L ? kbuf[p + clo] : K(0), ohi = e1 < L ? kbuf[p + chi] : K(0);
    uint32_t vlo = 0, vhi = 0;
    if constexpr (kVals) {
      vlo = lane < L ? vbuf[pv + clo] : 0u;
      vhi = e1 < L ? vbuf[pv + chi] : 0u;
    }
    if constexpr (kInPlace) __syncwarp();
    if (lane < L) {
      gk[lane] = olo;
      if constexpr (kVals) gv[lane] = vlo;
    }
    if (e1 < L) {
      gk[e1] = ohi;
      if constexpr (kVals) gv[e1] = vhi;
    }
  } else {
    using IO = RssIO<K, kVals>;
    using It = typename IO::T;
    It lo = lane < L ? IO::make(key_enc<K, kF>(kbuf[p + lane]), static_cast<uint32_t>(lane))
                     : IO::sentinel(static_cast<uint32_t>(lane));
    It hi = e1 < L ? IO::make(key_enc<K, kF>(kbuf[p + e1]), static_cast<uint32_t>(e1))
                   : IO::sentinel(static_cast<uint32_t>(e1));
    warp_sort64(lo, hi, lane);
    uint32_t vlo = 0, vhi = 0;
    if constexpr (kVals) {
      if (lane < L) vlo = vbuf[pv + IO::idx(lo)];
      if (e1 < L) vhi = vbuf[pv + IO::idx(hi)];
    }
    if constexpr (kInPlace) __syncwarp();
    if (lane < L) {
      gk[lane] = key_dec<K, kF>(IO::key(lo));
      if constexpr (kVals) gv[lane] = vlo;
    }
    if (e1 < L) {
      gk[e1] = key_dec<K, kF>(IO::key(hi));
      if constexpr (kVals) gv[e1] = vhi;
    }
  }
}

// Register Sample Sort of one segment of L (17..256) items by one warp
// (Sec. 3).  Splitters and classification use the keys alone; the buckets
// then hold (key, position-in-segment) items and are sorted by both, so equal
// keys end in input order.
//
//  1. sample: a*32 keys at equidistant positions (a = 1, or 2 above
//     `two_min` items), sorted in registers by the 32-lane warp network
//     (two halves merged for a = 2);
//  2. splitters s_j = S_{j*a}, j = 1..31, as a heap-ordered tree held one node
//     per lane (lane t holds node t) and broadcast by __shfl;
//  3. classify: every key descends j <- 2j + [t_j < e] five times, so bucket
//     b = j - 32 holds s_b < e <= s_{b+1}; all keys equal to a splitter fall
//     into one bucket; the rank inside the bucket comes from a shared-memory
//     counter (any order will do: each bucket is sorted afterwards);
//  4. bucket starts by a warp scan (lane b owns bucket b);
//  5. scatter the (key, position) items into the shared item buffer;
//  6. lane b sorts bucket b with a network padded to the warp's largest bucket
//     of at most 16 items (4, 8, 12 or 16 channels; 8 or 16 for 8-byte keys);
//     buckets above 16 items (rare unless keys repeat) are sorted by the whole
//     warp (32-lane network, or a bitonic pass in shared memory above 32);
//  7. write back (payload gathered by original position).
//  kInPlace: gk / gv point into the staged copy itself; the payload words are
//  then parked in the item buffer first and written once every lane has
//  gathered its own.
template <class K, bool kVals, bool kF, bool kInPlace = false>
__device__ __forceinline__ void rss_segment(const K* kbuf, const uint32_t* vbuf, int p, int pv, int L,
                                            const RssMem<K, kVals>& rm, int lane, int two_min, K* gk,
                                            uint32_t* gv) {
  using IO = RssIO<K, kVals>;
  using It = typename IO::T;
  constexpr K kTop = static_cast<K>(~static_cast<K>(0));
  const int rounds = (L + 31) >> 5;

  // 0. keys in registers (item e = 32 r + lane).  Sample, splitters and
  //    classification work on a 32-bit window of the encoded key: the key
  //    itself for 4-byte keys; for 8-byte keys the 32 bits from the highest
  //    bit in which the segment's keys differ down (every key agrees above
  //    it, so the window's order never contradicts the key order, and a
  //    bucket still holds a contiguous range of keys).  The buckets are then
  //    sorted by the full key.
  K xk[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int e = (r << 5) + lane;
    xk[r] = (r < rounds && e < L) ? key_enc<K, kF>(kbuf[p + e]) : kTop;
  }
  int sh = 0;
  if constexpr (sizeof(K) == 8) {
    const K k0 = shfl_idx(xk[0], 0);
    K diff = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
      if (r < rounds && (r << 5) + lane < L) diff |= xk[r] ^ k0;
    const uint32_t dl = __reduce_or_sync(kFull, static_cast<uint32_t>(diff));
    const uint32_t dh = __reduce_or_sync(kFull, static_cast<uint32_t>(diff >> 32));
    sh = window_shift((static_cast<K>(dh) << 32) | dl, 32);
  }
  auto win = [&](K x) -> uint32_t { return static_cast<uint32_t>(x >> sh); };

  // 1. sorted sample windows: slot q < 32 in s0 of lane q, slot 32 + q in s1 of lane q
  const bool two = L > two_min;
  uint32_t s0, s1 = 0xFFFFFFFFu;
  {
    // slot q of a*32 sits at position floor((2q + 1) L / (2 a 32))
    const int sh2 = two ? 7 : 6;
    s0 = win(key_enc<K, kF>(kbuf[p + (((2 * lane + 1) * L) >> sh2)]));
    if (!two) {
      warp_network32(s0, lane);
    } else {
      s1 = win(key_enc<K, kF>(kbuf[p + (((2 * (32 + lane) + 1) * L) >> sh2)]));
      warp_network32x2(s0, s1, lane);
      // merge two ascending halves: slot l meets slot 63 - l; the smaller
      // keys form a bitonic lower half, the larger a bitonic upper half
      // (in reversed lane order, still bitonic), each sorted by the
      // half-cleaners 16, 8, 4, 2, 1
      const uint32_t y = shfl_idx(s1, 31 - lane);
      uint32_t lo = pick(s0, y, true), hi = pick(s0, y, false);
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        const bool keep_min = lane < (lane ^ m);
        lo = pick(lo, shfl_xor(lo, m), keep_min);
        hi = pick(hi, shfl_xor(hi, m), keep_min);
      }
      s0 = lo;
      s1 = hi;
    }
  }

  // 2. tree node t (depth d, position p_d) = splitter (2 p_d + 1) * 2^(4 - d)
  //    = sample slot a * that - 1
  uint32_t tree;
  {
    const int t = lane > 0 ? lane : 1;
    const int d = 31 - __clz(t);
    const int rank = (2 * (t - (1 << d)) + 1) << (4 - d);
    const int slot = two ? 2 * rank - 1 : rank - 1;
    const uint32_t from0 = shfl_idx(s0, slot & 31);
    tree = from0;
    if (two) {
      const uint32_t from1 = shfl_idx(s1, slot & 31);
      tree = slot >= 32 ? from1 : from0;
    }
  }
  rm.cnt[lane] = 0;
  __syncwarp();

  // 3. classify the register-resident keys by their windows: every window
  //    descends j <- 2j + [t_j < w] five times (bucket b = j - 32 holds
  //    s_b < w <= s_{b+1}).  The top levels have few distinct nodes: they are
  //    broadcast once per segment and picked with selects (nodes 1..7); the
  //    deeper levels read node j of lane j.
  int j[8];
  uint32_t wk[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) wk[r] = win(xk[r]);
  const uint32_t n1 = shfl_idx(tree, 1), n2 = shfl_idx(tree, 2), n3 = shfl_idx(tree, 3);
  const uint32_t n4 = shfl_idx(tree, 4), n5 = shfl_idx(tree, 5), n6 = shfl_idx(tree, 6), n7 = shfl_idx(tree, 7);
  // The descent has no branch inside: it runs over 4 or all 8 rounds (keys
  // past the segment are +inf, sink to the last bucket and are never
  // counted), so the independent rounds interleave.  (Descents over 2, 4, 6
  // or 8 rounds did fewer instructions but ran 4 % slower: two more unrolled
  // copies in the instruction working set.)
  auto descend = [&](auto R_) {
    constexpr int R = decltype(R_)::value;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      j[r] = 2 + (n1 < wk[r] ? 1 : 0);
      j[r] = 2 * j[r] + ((j[r] & 1 ? n3 : n2) < wk[r] ? 1 : 0);
    }
#pragma unroll
    for (int lv = 2; lv < 5; ++lv) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        uint32_t t;
        if (lv == 2)  // the same on every lane (an unrolled loop index)
          t = j[r] & 2 ? (j[r] & 1 ? n7 : n6) : (j[r] & 1 ? n5 : n4);
        else
          t = shfl_idx(tree, j[r]);
        j[r] = 2 * j[r] + (t < wk[r] ? 1 : 0);
      }
    }
  };
#pragma unroll
  for (int r = 0; r < 8; ++r) j[r] = 32;
  if (rounds <= 4)
    descend(std::integral_constant<int, 4>{});
  else
    descend(std::integral_constant<int, 8>{});
  uint32_t rank_in[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    rank_in[r] = 0;
    if (r < rounds && (r << 5) + lane < L) rank_in[r] = atomicAdd(&rm.cnt[j[r] - 32], 1u);
  }
  __syncwarp();

  // 4. bucket starts (lane b owns bucket b)
  const uint32_t c = rm.cnt[lane];
  uint32_t incl = c;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t start = incl - c;

  // 5. scatter into the item buffer
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (r < rounds) {
      const uint32_t st = __shfl_sync(kFull, start, (j[r] - 32) & 31);
      const int e = (r << 5) + lane;
      if (e < L) rm.set(static_cast<int>(st + rank_in[r]), IO::make(xk[r], static_cast<uint32_t>(e)));
    }
  }
  __syncwarp();

  // 6. one bucket per lane, network padded to the warp's largest bucket <= 16
  const uint32_t m = __reduce_max_sync(kFull, c <= 16 ? c : 0u);
  if (m >= 2 && c <= 16) bucket_network_class<K, kVals>(static_cast<int>(m), rm, static_cast<int>(start),
                                                        static_cast<int>(c));
  __syncwarp();
  unsigned big = __ballot_sync(kFull, c > 16);
  while (big) {
    const int b = __ffs(big) - 1;
    big &= big - 1;
    const int st = static_cast<int>(__shfl_sync(kFull, start, b));
    const int cb = static_cast<int>(__shfl_sync(kFull, c, b));
    if (cb <= 32) {
      It y = lane < cb ? rm.get(st + lane) : IO::sentinel(lane);
      warp_network32(y, lane);
      __syncwarp();
      if (lane < cb) rm.set(st + lane, y);
    } else {
      warp_bitonic_smem<K, kVals>(rm, st, cb, lane);
    }
    __syncwarp();
  }

  // 7. write the sorted segment straight to its place in global memory
  //    (coalesced: lane l writes items 32 r + l; payload gathered by
  //    original position from the staged copy)
  if constexpr (kInPlace && kVals) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) {
        const It y = rm.get(e);
        gk[e] = key_dec<K, kF>(IO::key(y));
        rm.stash(e, vbuf[pv + IO::idx(y)]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) gv[e] = rm.unstash(e);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = (r << 5) + lane;
      if (r < rounds && e < L) {
        const It y = rm.get(e);
        gk[e] = key_dec<K, kF>(IO::key(y));
        if constexpr (kVals) gv[e] = vbuf[pv + IO::idx(y)];
      }
    }
  }
  __syncwarp();
}

// ------------------------------------------------- staged range stores -----

// Write items [e0, e0 + n) from the staged copy (granule-aligned, element
// e0 at index shift) back to `dst`: bulk store for the whole 16-byte granules
// (issued by lane 0 into the current bulk group), plain stores by the calling
// warp's lanes for the partial granules at both ends.
template <class T>
__device__ __forceinline__ void store_range(T* dst, const T* staged, uint32_t shift, uint32_t e0, uint32_t n,
                                            int lane) {
  if (n == 0) return;
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst + e0), z = reinterpret_cast<uintptr_t>(dst + e0 + n);
  const uintptr_t ia = (a + 15) & ~uintptr_t(15), iz = z & ~uintptr_t(15);
  uint32_t head = n, tail = n;
  if (ia < iz) {
    head = static_cast<uint32_t>((ia - a) / sizeof(T));
    tail = static_cast<uint32_t>((iz - a) / sizeof(T));
    if (lane == 0) bulk_s2g(reinterpret_cast<void*>(ia), staged + shift + head, static_cast<uint32_t>(iz - ia));
  }
  for (uint32_t e = lane; e < head; e += 32) dst[e0 + e] = staged[shift + e];
  for (uint32_t e = tail + lane; e < n; e += 32) dst[e0 + e] = staged[shift + e];
}

// ----------------------------------------------------------- tile kernel ---

// Task ring slots: at least the work items of kMaxStages staged tiles plus
// one stop item per consumer warp (tile_fits checks the tile shape against it).
constexpr int kRing = 512;
constexpr uint32_t kRingDone = 0xFFFFFFFFu;

struct TileTasks {
  uint32_t npair, pair_tasks, ntasks, b16, b12, b8, b4, b2;
};

// Work items of a staged tile: 16 pair segments per item, then the network
// list (classes 16, 12, 8, 4, 2 in that order) in chunks of 32 lanes; a chunk
// that spans two classes uses the larger network for all its lanes.
__device__ __forceinline__ TileTasks tile_tasks(const uint16_t* cnt) {
  TileTasks t;
  t.npair = cnt[kPair];
  t.b16 = t.npair + cnt[kNet16];
  t.b12 = t.b16 + cnt[kNet12];
  t.b8 = t.b12 + cnt[kNet8];
  t.b4 = t.b8 + cnt[kNet4];
  t.b2 = t.b4 + cnt[kNet2];
  t.pair_tasks = (t.npair + 15) / 16;
  t.ntasks = t.pair_tasks + (t.b2 - t.npair + 31) / 32;
  return t;
}

// Resident blocks per SM the register budget is sized for.  Ring kernel
// (16 warps a block): the (key, position) networks of payload sorts need
// about 128 registers a thread (1 block), keys-only networks 64 (2 blocks).
// Synchronous kernel (8 warps): 2 blocks with payload, 3 (u64) or 4 (u32)
// keys-only; more blocks keep more tiles in flight.
template <class K, bool kVals>
constexpr int tile_min_blocks() {
  return kVals ? 1 : 2;
}
template <class K, bool kVals>
constexpr int sync_min_blocks() {
  return kVals ? 2 : (sizeof(K) == 4 ? 4 : 3);
}

template <class K, bool kVals, int kStages, bool kF>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<K, kVals>())
    seg_tile_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ offsets,
                    const Plan* plan, const uint32_t* __restrict__ tile_first, const uint16_t* __restrict__ counts,
                    const uint16_t* __restrict__ order, uint32_t E, unsigned* status) {
  const RingLayout<K, kVals> lay(E);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  __shared__ TileMeta meta[kStages];
  __shared__ uint32_t ntasks_of[kStages], done_ctr[kStages];
  __shared__ uint32_t ring[kRing];
  __shared__ uint32_t ring_head, ring_tail;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      done_ctr[s] = 0;
    }
    ring_head = 0;
    ring_tail = 0;
    fence_mbar_init();
  }
  __syncthreads();

  // ------------------------------------------------------------ producer --
  // Tiles blockIdx.x + j * gridDim.x, j = 0, 1, ...; lane i reads the
  // metadata of tile j = 32 m + i.  The warp stages tiles into the two stages
  // as they free up and, as each staged copy lands, pushes the tile's work
  // items onto the ring.
  if (warp == kTileWarps) {
    const uint32_t ntiles = plan->bad ? 0u : plan->ntiles;
    const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
    const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);
    const uintptr_t ob = reinterpret_cast<uintptr_t>(offsets);
    const uintptr_t rb = reinterpret_cast<uintptr_t>(order);
    uint32_t chunk = blockIdx.x;
    bool more = chunk < ntiles;
    unsigned avail = 0;
    uint32_t t = 0, s0 = 0, s1 = 0, e0 = 0, e1 = 0;
    uint32_t issued = 0, pushed = 0, tail = 0;
    bool failed = false;
    unsigned long long idle_since = 0;
    for (;;) {
      if (avail == 0 && more) {
        t = chunk + lane * gridDim.x;
        bool has = false;
        if (t < ntiles) {
          const uint2 c03 = *reinterpret_cast<const uint2*>(counts + 8ull * t);
          const uint32_t c45 = *reinterpret_cast<const uint32_t*>(counts + 8ull * t + 4);
          has = (c03.x | c03.y | c45) != 0;
          if (has) {
            s0 = tile_first[t];
            s1 = tile_first[t + 1];
            e0 = offsets[s0];
            e1 = offsets[s1];
          }
        }
        avail = __ballot_sync(kFull, has);
        chunk += 32u * gridDim.x;
        more = chunk < ntiles;
        continue;
      }
      if (avail == 0 && !more && pushed == issued) break;
      bool progress = false;
      // stage the next tile when its stage is free (lane 0 tests, all lanes follow)
      bool can_issue = false;
      if (lane == 0)
        can_issue = avail != 0 && (issued < kStages || mbar_test(&empty[issued % kStages],
                                                                   ((issued / kStages) - 1) & 1u));
      can_issue = __shfl_sync(kFull, can_issue, 0);
      if (can_issue) {
        const int j = __ffs(avail) - 1;
        avail &= avail - 1;
        const uint32_t tj = __shfl_sync(kFull, t, j), s0j = __shfl_sync(kFull, s0, j),
                       s1j = __shfl_sync(kFull, s1, j), e0j = __shfl_sync(kFull, e0, j),
                       e1j = __shfl_sync(kFull, e1, j);
        bool staged = true;
        if (lane == 0) {
          const int s = static_cast<int>(issued % kStages);
          unsigned char* stage = smem + s * lay.stage_bytes;
          // granule-rounded source ranges (a 16-byte granule never crosses a
          // page, so reading its unused part cannot fault; it is discarded)
          const uintptr_t oa = (ob + 4ull * s0j) & ~uintptr_t(15);
          const uintptr_t oz = (ob + 4ull * (s1j + 1) + 15) & ~uintptr_t(15);
          const uintptr_t ra = (rb + 2ull * s0j) & ~uintptr_t(15);
          const uintptr_t rz = (rb + 2ull * s1j + 15) & ~uintptr_t(15);
          const uintptr_t ka = (kb + sizeof(K) * e0j) & ~uintptr_t(15);
          const uintptr_t kz = (kb + sizeof(K) * e1j + 15) & ~uintptr_t(15);
          TileMeta& m = meta[s];
          m.tile = tj;
          m.s0 = s0j;
          m.s1 = s1j;
          m.e0 = e0j;
          m.e1 = e1j;
          m.off_shift = static_cast<uint32_t>((ob + 4ull * s0j - oa) / 4);
          m.ord_shift = static_cast<uint32_t>((rb + 2ull * s0j - ra) / 2);
          m.key_shift = static_cast<uint32_t>((kb + sizeof(K) * e0j - ka) / sizeof(K));
          const bool has_items = e1j > e0j;
          uintptr_t va = 0, vz = 0;
          if constexpr (kVals) {
            va = (vb + 4ull * e0j) & ~uintptr_t(15);
            vz = (vb + 4ull * e1j + 15) & ~uintptr_t(15);
            m.val_shift = static_cast<uint32_t>((vb + 4ull * e0j - va) / 4);
          } else {
            m.val_shift = 0;
          }
          // packed regions: offsets at 0, then bins, counts, keys, payload
          // (every size a multiple of 16, so every region starts aligned)
          const size_t off_bytes = oz - oa, ord_bytes = rz - ra;
          const size_t key_bytes = has_items ? kz - ka : 0, val_bytes = kVals && has_items ? vz - va : 0;
          const size_t ord_at = off_bytes, cnt_at = ord_at + ord_bytes, key_at = cnt_at + 16;
          const size_t val_at = key_at + key_bytes, end = val_at + val_bytes;
          // self-check of every copy's range against the stage
          const bool args_ok = s1j > s0j && s1j - s0j <= E && e1j >= e0j && e1j - e0j <= E + kMaxSeg &&
                               end <= lay.stage_bytes &&
                               ((reinterpret_cast<uintptr_t>(counts) + 16ull * tj) & 15) == 0;
          if (!args_ok) {
            atomicOr(status, kStatusInternal | kCheckCopyArgs);
            staged = false;  // skip the tile; its data stays untouched
          } else {
          m.ord_at = static_cast<uint32_t>(ord_at);
          m.cnt_at = static_cast<uint32_t>(cnt_at);
          m.key_at = static_cast<uint32_t>(key_at);
          m.val_at = static_cast<uint32_t>(val_at);
          m.key_cap = static_cast<uint32_t>(key_bytes / sizeof(K));
          m.val_cap = kVals ? static_cast<uint32_t>(val_bytes / 4) : 0xFFFFFFFFu;
          mbar_arrive_expect_tx(&full[s], static_cast<uint32_t>(end));
          if (test_flags(status) & kTestSkipTileCopy) {
            // test hook: the stage's barrier is armed, no copy is issued
          } else {
          bulk_g2s(stage, reinterpret_cast<const void*>(oa), static_cast<uint32_t>(off_bytes), &full[s]);
          bulk_g2s(stage + ord_at, reinterpret_cast<const void*>(ra), static_cast<uint32_t>(ord_bytes), &full[s]);
          bulk_g2s(stage + cnt_at, counts + 8ull * tj, 16, &full[s]);
          if (has_items) {
            bulk_g2s(stage + key_at, reinterpret_cast<const void*>(ka), static_cast<uint32_t>(key_bytes), &full[s]);
            if constexpr (kVals)
              bulk_g2s(stage + val_at, reinterpret_cast<const void*>(va), static_cast<uint32_t>(val_bytes),
                       &full[s]);
          }
          }
          }
        }
        staged = __shfl_sync(kFull, staged, 0);
        if (staged) ++issued;
        progress = true;
      }
      // publish the work items of the oldest staged tile once it has landed
      bool can_push = false;
      if (lane == 0) can_push = pushed < issued && mbar_test(&full[pushed % kStages], (pushed / kStages) & 1u);
      can_push = __shfl_sync(kFull, can_push, 0);
      if (can_push) {
        const int s = static_cast<int>(pushed % kStages);
        // only lane 0 observed the copy's completion, so only lane 0 reads the
        // staged counts; the task count is broadcast
        uint32_t ntasks = 0;
        if (lane == 0)
          ntasks = tile_tasks(reinterpret_cast<const uint16_t*>(smem + s * lay.stage_bytes + meta[s].cnt_at)).ntasks;
        ntasks = __shfl_sync(kFull, ntasks, 0);
        const TileTasks tt{0, 0, ntasks, 0, 0, 0, 0, 0};
        // item = stage << 17 | phase parity of this use of the stage << 16 | index
        const uint32_t tag = (static_cast<uint32_t>(s) << 17) | (((pushed / kStages) & 1u) << 16);
        for (uint32_t i = lane; i < tt.ntasks; i += 32) ring[(tail + i) & (kRing - 1)] = tag | i;
        if (lane == 0) ntasks_of[s] = tt.ntasks;
        __syncwarp();
        tail += tt.ntasks;
        if (lane == 0) st_release_smem(&ring_tail, tail);
        ++pushed;
        progress = true;
      }
      if (progress) {
        idle_since = 0;
      } else {
        const unsigned long long now = global_ns();
        if (idle_since == 0) idle_since = now;
        if (now - idle_since > wait_limit_ns(status)) {
          failed = true;
          break;
        }
        __nanosleep(64);
      }
    }
    if (failed && lane == 0) {
      atomicOr(status, kStatusTimeout);
      // staged tiles whose work was never published: let their copies land
      // (bounded waits) before the block can exit
      for (uint32_t x = pushed; x < issued; ++x) (void)mbar_wait(&full[x % kStages], (x / kStages) & 1u, status);
    }
    // one stop item per consumer warp
    for (uint32_t i = lane; i < kTileWarps; i += 32) ring[(tail + i) & (kRing - 1)] = kRingDone;
    __syncwarp();
    if (lane == 0) st_release_smem(&ring_tail, tail + kTileWarps);
    return;
  }

  // ----------------------------------------------------------- consumers --
  bool stored = false;
  for (;;) {
    uint32_t desc = kRingDone;
    if (lane == 0) {
      const uint32_t pos = atomicAdd(&ring_head, 1u);
      const unsigned long long t0 = global_ns();
      const unsigned long long limit = wait_limit_ns(status);
      bool ok = true;
      while (ld_acquire_smem(&ring_tail) <= pos) {
        if (global_ns() - t0 > limit) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      if (ok) {
        desc = ring[pos & (kRing - 1)];
      } else {
        atomicOr(status, kStatusTimeout);
      }
    }
    desc = __shfl_sync(kFull, desc, 0);
    if (desc == kRingDone) break;
    const int s = static_cast<int>(desc >> 17);
    const uint32_t task = desc & 0xFFFFu;
    if (s >= kStages) {  // a malformed work item: report, never index with it
      if (lane == 0) atomicOr(status, kStatusInternal);
      break;
    }
    // Bulk-copy writes are visible to the threads that observe the mbarrier
    // phase, so every lane waits on the stage itself (the phase has completed;
    // the stage cannot move on while this item is outstanding).
    if (!__all_sync(kFull, mbar_wait(&full[s], (desc >> 16) & 1u, status))) {
      if (lane == 0) atomicOr(status, kStatusTimeout);
      break;
    }
    const TileMeta m = meta[s];  // copy: checked against the stage again before the store
    unsigned char* stage = smem + s * lay.stage_bytes;
    const uint32_t* obuf = reinterpret_cast<const uint32_t*>(stage) + m.off_shift;
    const uint16_t* ord = reinterpret_cast<const uint16_t*>(stage + m.ord_at) + m.ord_shift;
    K* kbuf = reinterpret_cast<K*>(stage + m.key_at);
    uint32_t* vbuf = reinterpret_cast<uint32_t*>(stage + m.val_at);
    const TileTasks tt = tile_tasks(reinterpret_cast<const uint16_t*>(stage + m.cnt_at));
    const uint32_t e0 = m.e0, key_shift = m.key_shift, val_shift = m.val_shift;
    const uint32_t ns = m.s1 - m.s0;
    if (task >= tt.ntasks || tt.b2 > ns || ns > E) {
      if (lane == 0) atomicOr(status, kStatusInternal);
      break;
    }

    // self-check: a segment's staged span must lie inside the stage buffers
    const uint32_t key_cap = m.key_cap;
    const uint32_t val_cap = m.val_cap;
    auto span_ok = [&](uint32_t i, uint32_t& o, uint32_t& L) -> bool {
      if (i >= ns) return false;
      o = obuf[i];
      const uint32_t o1 = obuf[i + 1];
      if (o < e0 || o1 < o || o1 > m.e1 || o1 - o > 32) return false;
      L = o1 - o;
      return o1 - e0 + key_shift <= key_cap && o1 - e0 + val_shift <= val_cap;
    };
    // every work item: the lane's segment, its class and its staged position
    const bool pair = task < tt.pair_tasks;
    bool active = false;
    int p = 0, pv = 0, L = 0, cls = 16;
    {
      uint32_t slot, first = 0;
      if (pair) {
        slot = task * 16 + (lane >> 1);
        active = slot < tt.npair;
      } else {
        first = tt.npair + (task - tt.pair_tasks) * 32;
        slot = first + lane;
        active = slot < tt.b2;
        cls = first < tt.b16 ? 16 : first < tt.b12 ? 12 : first < tt.b8 ? 8 : first < tt.b4 ? 4 : 2;
      }
      if (active) {
        uint32_t o = 0, l = 0;
        if (span_ok(ord[slot], o, l) && (pair || l <= 16)) {
          L = static_cast<int>(l);
          p = static_cast<int>(o - e0 + key_shift);
          pv = static_cast<int>(o - e0 + val_shift);
        } else {
          atomicOr(status, kStatusInternal | kCheckSegment);
          active = false;
        }
      }
    }
    if (cls == 16) {
      seg16<K, kVals, kF>(kbuf, vbuf, p, pv, L, active, pair, lane);
    } else if (active) {
      if (cls == 12)
        net_segment<12, K, kVals, kF>(kbuf, vbuf, p, pv, L);
      else if (cls == 8)
        net_segment<8, K, kVals, kF>(kbuf, vbuf, p, pv, L);
      else if (cls == 4)
        net_segment<4, K, kVals, kF>(kbuf, vbuf, p, pv, L);
      else
        net_segment<2, K, kVals, kF>(kbuf, vbuf, p, pv, L);
    }

    // completion: the warp that finishes a tile's last item stores the tile
    // and releases its stage
    fence_proxy_async_smem();
    __syncwarp();
    uint32_t fin = 0;
    if (lane == 0) {
      const uint32_t total = ntasks_of[s];
      fin = (atom_add_acq_rel_smem(&done_ctr[s], 1u) + 1 == total) ? 1u : 0u;
    }
    fin = __shfl_sync(kFull, fin, 0);
    if (fin) {
      // self-check: the stage must still hold this work item's tile
      const TileMeta now = meta[s];
      if (now.tile != m.tile || now.e0 != m.e0 || now.e1 != m.e1 || m.e1 - e0 > E + kMaxSeg) {
        if (lane == 0) atomicOr(status, kStatusInternal | kCheckStageMoved);
        break;
      }
      store_range<K>(keys, kbuf, key_shift, e0, m.e1 - e0, lane);
      if constexpr (kVals) store_range<uint32_t>(vals, vbuf, val_shift, e0, m.e1 - e0, lane);
      stored = true;
      __syncwarp();  // every lane's reads of the stage are done
      if (lane == 0) {
        bulk_commit();
        bulk_wait_read<0>();
        done_ctr[s] = 0;
        mbar_arrive(&empty[s]);
      }
      __syncwarp();
    }
  }
  if (stored && lane == 0) bulk_wait_all<0>();
}

// ------------------------------------------------ synchronous tile kernel --
//
// The second tile-kernel mode (launch parameter tile_mode = 1), built like the
// fixed-size kernel: every warp of the block works on the same staged tile,
// with no task ring.  Thread j of the block takes segments j, j + 256, ... of
// the tile: a segment of 2..16 items is sorted by the lane's network, padded
// to the largest such segment among the warp's 32 (a warp-uniform choice among
// the enabled classes); segments of 17..32 items in the warp's window are
// gathered by ballot and sorted two lanes each; longer ones are left to the
// RSS kernel.  The block then stores the tile and stages its tile kStages
// ahead into the freed buffer.
constexpr int kSyncThreads = 256;

// Bit position of the (n+1)-th set bit of m, -1 if m has at most n set bits.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
  if (__popc(m) <= n) return -1;
  for (int q = 0; q < n; ++q) m &= m - 1;
  return __ffs(m) - 1;
}

template <class K, bool kVals, int kStages, bool kF>
__global__ void __launch_bounds__(kSyncThreads, sync_min_blocks<K, kVals>())
    seg_sync_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ offsets,
                    const Plan* plan, const uint32_t* __restrict__ tile_first, uint32_t E, uint32_t net_mask,
                    bool rss_only, unsigned* status) {
  const TileLayout<K, kVals> lay(E);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ TileMeta meta[kStages];
  __shared__ int issue_failed;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t ntiles = plan->bad ? 0u : plan->ntiles;
  const uint32_t my = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
  const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);
  const uintptr_t ob = reinterpret_cast<uintptr_t>(offsets);

  // Stage this block's tile number i into stage s (thread 0).  Source ranges
  // are rounded out to 16-byte granules (a granule never crosses a page; the
  // extra elements are read, not used, and never written back).
  struct Where {
    uint32_t s0, s1, e0, e1;
  };
  auto locate = [&](uint32_t i) -> Where {  // global loads: tile bounds, then item bounds
    const uint32_t t = blockIdx.x + i * gridDim.x;
    Where w;
    w.s0 = tile_first[t];
    w.s1 = tile_first[t + 1];
    w.e0 = offsets[w.s0];
    w.e1 = offsets[w.s1];
    return w;
  };
  auto issue = [&](uint32_t i, int s, const Where& w) -> bool {
    const uint32_t t = blockIdx.x + i * gridDim.x;
    const uint32_t s0 = w.s0, s1 = w.s1, e0 = w.e0, e1 = w.e1;
    unsigned char* stage = smem + s * lay.stage_bytes;
    const uintptr_t oa = (ob + 4ull * s0) & ~uintptr_t(15), oz = (ob + 4ull * (s1 + 1) + 15) & ~uintptr_t(15);
    const uintptr_t ka = (kb + sizeof(K) * e0) & ~uintptr_t(15), kz = (kb + sizeof(K) * e1 + 15) & ~uintptr_t(15);
    uintptr_t va = 0, vz = 0;
    TileMeta& m = meta[s];
    m.tile = t;
    m.s0 = s0;
    m.s1 = s1;
    m.e0 = e0;
    m.e1 = e1;
    m.off_shift = static_cast<uint32_t>((ob + 4ull * s0 - oa) / 4);
    m.key_shift = static_cast<uint32_t>((kb + sizeof(K) * e0 - ka) / sizeof(K));
    m.ord_shift = 0;
    m.val_shift = 0;
    const bool has_items = e1 > e0;
    uint32_t bytes = static_cast<uint32_t>(oz - oa) + (has_items ? static_cast<uint32_t>(kz - ka) : 0u);
    if constexpr (kVals) {
      va = (vb + 4ull * e0) & ~uintptr_t(15);
      vz = (vb + 4ull * e1 + 15) & ~uintptr_t(15);
      m.val_shift = static_cast<uint32_t>((vb + 4ull * e0 - va) / 4);
      if (has_items) bytes += static_cast<uint32_t>(vz - va);
    }
    // self-check of every copy against its staging buffer
    const bool ok = s1 > s0 && s1 - s0 <= E && e1 >= e0 && e1 - e0 <= E + kMaxSeg &&
                    (oz - oa) <= lay.key_at - lay.off_at && (!has_items || (kz - ka) <= lay.val_at - lay.key_at) &&
                    (!kVals || !has_items || (vz - va) <= lay.ord_at - lay.val_at);
    if (!ok) {
      atomicOr(status, kStatusInternal | kCheckCopyArgs);
      return false;
    }
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_g2s(stage + lay.off_at, reinterpret_cast<const void*>(oa), static_cast<uint32_t>(oz - oa), &full[s]);
    if (has_items) {
      bulk_g2s(stage + lay.key_at, reinterpret_cast<const void*>(ka), static_cast<uint32_t>(kz - ka), &full[s]);
      if constexpr (kVals)
        bulk_g2s(stage + lay.val_at, reinterpret_cast<const void*>(va), static_cast<uint32_t>(vz - va), &full[s]);
    }
    return true;
  };

  uint32_t issued = 0;  // tiles staged so far (thread 0)
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    bool ok = true;
    while (issued < static_cast<uint32_t>(kStages) && issued < my && ok) {
      ok = issue(issued, static_cast<int>(issued), locate(issued));
      if (ok) ++issued;
    }
    issue_failed = ok ? 0 : 1;
    if (!ok)  // let the copies already issued land, then leave
      for (uint32_t t = 0; t < issued; ++t) (void)mbar_wait(&full[t], 0, status);
  }
  __syncthreads();
  if (issue_failed) return;

  const uint32_t key_cap = static_cast<uint32_t>((lay.val_at - lay.key_at) / sizeof(K));
  bool failed = false;
  uint32_t i = 0;
  for (; i < my; ++i) {
    const int s = static_cast<int>(i % kStages);
    const bool ok = mbar_wait(&full[s], (i / kStages) & 1u, status);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const TileMeta m = meta[s];
    // thread 0 fetches the bounds of the tile that refills this stage now, so
    // that the refill can be issued as soon as the store has read the stage
    Where next{};
    if (tid == 0 && i + kStages < my) next = locate(i + kStages);
    unsigned char* stage = smem + s * lay.stage_bytes;
    const uint32_t* obuf = reinterpret_cast<const uint32_t*>(stage + lay.off_at) + m.off_shift;
    K* kbuf = reinterpret_cast<K*>(stage + lay.key_at);
    uint32_t* vbuf = reinterpret_cast<uint32_t*>(stage + lay.val_at);
    const uint32_t ns = m.s1 - m.s0;
    for (uint32_t base = static_cast<uint32_t>(warp) * 32; base < ns; base += kSyncThreads) {
      const uint32_t j = base + lane;
      uint32_t o = m.e0, L = 0;
      if (j < ns) {
        o = obuf[j];
        L = obuf[j + 1] - o;
        // self-check: the segment lies in the tile's staged items
        if (o < m.e0 || obuf[j + 1] > m.e1 || obuf[j + 1] - m.e0 + m.key_shift > key_cap || L > kMaxSeg) {
          atomicOr(status, kStatusInternal | kCheckSegment);
          L = 0;
        }
      }
      const int p = static_cast<int>(o - m.e0 + m.key_shift), pv = static_cast<int>(o - m.e0 + m.val_shift);
      const bool net = L >= 2 && L <= 16;
      const uint32_t mx = __reduce_max_sync(kFull, net ? L : 0u);
      if (mx >= 2) {
        const int cls = (mx <= 2 && (net_mask & 1u))    ? 2
                        : (mx <= 4 && (net_mask & 2u))  ? 4
                        : (mx <= 8 && (net_mask & 4u))  ? 8
                        : (mx <= 12 && (net_mask & 8u)) ? 12
                                                        : 16;
        if (cls == 16) {
          seg16<K, kVals, kF>(kbuf, vbuf, p, pv, static_cast<int>(L), net, false, lane);
        } else if (net) {
          if (cls == 12)
            net_segment<12, K, kVals, kF>(kbuf, vbuf, p, pv, static_cast<int>(L));
          else if (cls == 8)
            net_segment<8, K, kVals, kF>(kbuf, vbuf, p, pv, static_cast<int>(L));
          else if (cls == 4)
            net_segment<4, K, kVals, kF>(kbuf, vbuf, p, pv, static_cast<int>(L));
          else
            net_segment<2, K, kVals, kF>(kbuf, vbuf, p, pv, static_cast<int>(L));
        }
      }
      // 17..32: the warp's such segments, 16 at a time on lane pairs
      unsigned pm = __ballot_sync(kFull, !rss_only && L >= 17 && L <= 32);
      while (pm) {
        const int src = nth_set_bit(pm, lane >> 1);
        const bool act = src >= 0;
        const uint32_t po = __shfl_sync(kFull, o, act ? src : 0);
        const uint32_t pL = __shfl_sync(kFull, L, act ? src : 0);
        seg16<K, kVals, kF>(kbuf, vbuf, static_cast<int>(po - m.e0 + m.key_shift),
                            static_cast<int>(po - m.e0 + m.val_shift), act ? static_cast<int>(pL) : 0, act, true,
                            lane);
        for (int q = 0; q < 16 && pm; ++q) pm &= pm - 1;
      }
    }
    fence_proxy_async_smem();  // this thread's writes, before the bulk store reads them
    __syncthreads();
    if (warp == 0) {
      store_range<K>(keys, kbuf, m.key_shift, m.e0, m.e1 - m.e0, lane);
      if constexpr (kVals) store_range<uint32_t>(vals, vbuf, m.val_shift, m.e0, m.e1 - m.e0, lane);
      __syncwarp();
      if (lane == 0) {
        bulk_commit();
        if (i + kStages < my) {
          bulk_wait_read<0>();  // the store has read the stage
          if (issue(i + kStages, s, next))
            ++issued;
          else
            failed = true;
        }
      }
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      ++i;
      break;
    }
  }
  if (tid == 0) {
    bulk_wait_all<0>();
    if (failed) {
      atomicOr(status, kStatusTimeout);
      // let staged copies that were issued but not consumed land before exit
      for (uint32_t t = i; t < issued; ++t) (void)mbar_wait(&full[t % kStages], (t / kStages) & 1u, status);
    }
  }
}

// ------------------------------------------------------------ RSS kernel ---

// Stage items [e0, e0 + L) (keys and payload) into staging buffer b of the
// calling warp; called by lane 0, completion counted on `bar`.
template <class K, bool kVals>
__device__ __forceinline__ void rss_issue(unsigned char* wbase, int b, uint64_t* bar, const K* keys,
                                          const uint32_t* vals, uint32_t e0, uint32_t L, bool skip_copy) {
  using WL = RssWarpLayout<K, kVals>;
  const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
  const uintptr_t ka = (kb + sizeof(K) * e0) & ~uintptr_t(15);
  const uintptr_t kz = (kb + sizeof(K) * (e0 + L) + 15) & ~uintptr_t(15);
  uint32_t bytes = static_cast<uint32_t>(kz - ka);
  uintptr_t va = 0, vz = 0;
  if constexpr (kVals) {
    const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);
    va = (vb + 4ull * e0) & ~uintptr_t(15);
    vz = (vb + 4ull * (e0 + L) + 15) & ~uintptr_t(15);
    bytes += static_cast<uint32_t>(vz - va);
  }
  mbar_arrive_expect_tx(bar, bytes);
  if (skip_copy) return;  // test hook: the barrier is armed, no copy is issued
  bulk_g2s(wbase + WL::kKeys + b * WL::kKeyCap, reinterpret_cast<const void*>(ka), static_cast<uint32_t>(kz - ka),
           bar);
  if constexpr (kVals)
    bulk_g2s(wbase + WL::kVals_ + b * WL::kValCap, reinterpret_cast<const void*>(va),
             static_cast<uint32_t>(vz - va), bar);
}

// Resident RSS blocks per SM the register budget is sized for: the kernel is
// latency-bound (shuffle and shared-memory round trips), so as many warps as
// fit without spills (4-byte bare keys 62 registers a thread, 4-byte keys with
// payload and 8-byte bare keys about 80, 8-byte keys with payload 116).
template <class K, bool kVals>
constexpr int rss_min_blocks() {
  return sizeof(K) == 4 ? (kVals ? 3 : 4) : (kVals ? 2 : 3);
}

template <class K, bool kVals, bool kF>
__global__ void __launch_bounds__(kRssThreads, rss_min_blocks<K, kVals>())
    seg_rss_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ offsets,
                   const Plan* plan, const uint32_t* __restrict__ tile_first, const uint16_t* __restrict__ counts,
                   const uint16_t* __restrict__ order, int two_min, bool net64, unsigned* status) {
  using WL = RssWarpLayout<K, kVals>;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  unsigned char* wbase = smem + warp * WL::kBytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wbase + WL::kBar);
  const RssMem<K, kVals> rm(wbase + WL::kScratch);
  if (lane == 0) {
    for (int b = 0; b < kRssBufs; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const uint32_t ntiles = plan->bad ? 0u : plan->ntiles;
  const bool skip_copy = lane == 0 && (test_flags(status) & kTestSkipRssCopy);
  const uint32_t gw = blockIdx.x * kRssWarps + warp;
  const uint32_t W = gridDim.x * kRssWarps;

  // Segment number d of this warp lives in staging buffer d % kRssBufs; its
  // mbarrier phase is (d / kRssBufs) & 1, and lane d % kRssBufs keeps its
  // start and length.  Segment d is sorted just before segment d + kRssBufs
  // is staged into the same buffer, so kRssBufs - 1 segments load while one
  // is sorted; results go straight to global memory, so a buffer is free as
  // soon as its sort ends.
  uint32_t issued = 0, sorted = 0;
  bool failed = false;
  uint32_t q_e0 = 0, q_L = 0;

  auto sort_staged = [&](uint32_t d) {  // sort segment number d of this warp
    const int b = static_cast<int>(d % kRssBufs);
    const uint32_t pe0 = __shfl_sync(kFull, q_e0, b), pL = __shfl_sync(kFull, q_L, b);
    // every lane waits itself (bulk-copy data is visible to the lanes that
    // observe the phase); a timeout anywhere fails the whole warp
    if (!__all_sync(kFull, mbar_wait(&bar[b], (d / kRssBufs) & 1u, status))) {
      if (lane == 0) atomicOr(status, kStatusTimeout);
      failed = true;
      return;
    }
    const K* kbuf = reinterpret_cast<const K*>(wbase + WL::kKeys + b * WL::kKeyCap);
    const uint32_t* vbuf = reinterpret_cast<const uint32_t*>(wbase + WL::kVals_ + b * WL::kValCap);
    const uint32_t ks = static_cast<uint32_t>((reinterpret_cast<uintptr_t>(keys + pe0) & 15) / sizeof(K));
    const uint32_t vs = kVals ? static_cast<uint32_t>((reinterpret_cast<uintptr_t>(vals + pe0) & 15) / 4) : 0u;
    uint32_t* gv = kVals ? vals + pe0 : nullptr;
    if (net64 && pL <= 64)
      net64_segment<K, kVals, kF>(kbuf, vbuf, static_cast<int>(ks), static_cast<int>(vs), static_cast<int>(pL), lane,
                                  keys + pe0, gv);
    else
      rss_segment<K, kVals, kF>(kbuf, vbuf, static_cast<int>(ks), static_cast<int>(vs), static_cast<int>(pL), rm,
                                lane, two_min, keys + pe0, gv);
    // every lane's reads of the staged copy are done (the results went
    // straight to global memory), so the buffer may be staged again
    __syncwarp();
    sorted = d + 1;
  };

  for (uint32_t chunk = gw; chunk < ntiles && !failed; chunk += 32u * W) {
    const uint32_t t = chunk + lane * W;
    uint32_t rc = 0, s0 = 0, base = 0;
    if (t < ntiles) {
      const uint4 c = *reinterpret_cast<const uint4*>(counts + 8ull * t);
      rc = c.w & 0xFFFFu;  // counts[8t + 6]
      if (rc) {
        base = (c.x & 0xFFFFu) + (c.x >> 16) + (c.y & 0xFFFFu) + (c.y >> 16) + (c.z & 0xFFFFu) + (c.z >> 16);
        s0 = tile_first[t];
      }
    }
    // The chunk's RSS segments form one list (lane i's tile contributing rc_i
    // entries after those of lanes < i); batches of 32 entries are fetched one
    // per lane, each lane finding its entry's tile by a binary search over the
    // inclusive scan, so one round trip finds up to 32 segments however they
    // are spread over the tiles.  The segments found are staged and sorted in
    // list order.
    uint32_t incl = rc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    for (uint32_t b0 = 0; b0 < total && !failed; b0 += 32) {
      const uint32_t k = b0 + static_cast<uint32_t>(lane);
      int i = 0;  // lanes before the entry's tile: those with incl <= k
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1)
        if (__shfl_sync(kFull, incl, i + step - 1) <= k) i += step;
      const uint32_t s0i = __shfl_sync(kFull, s0, i), basei = __shfl_sync(kFull, base, i);
      const uint32_t firsti = __shfl_sync(kFull, incl - rc, i);
      uint32_t e0q = 0, Lq = 0;
      const bool has = k < total;
      if (has) {
        const uint32_t local = order[s0i + basei + (k - firsti)];
        e0q = offsets[s0i + local];
        Lq = offsets[s0i + local + 1] - e0q;
      }
      unsigned m = __ballot_sync(kFull, has);
      while (m && !failed) {
        const int r = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t ne0 = __shfl_sync(kFull, e0q, r), nL = __shfl_sync(kFull, Lq, r);
        // free the buffer (sort its segment), then stage segment `issued` into it
        if (issued >= static_cast<uint32_t>(kRssBufs)) {
          sort_staged(issued - kRssBufs);
          if (failed) break;
        }
        const int nb = static_cast<int>(issued % kRssBufs);
        if (lane == 0) rss_issue<K, kVals>(wbase, nb, &bar[nb], keys, vals, ne0, nL, skip_copy);
        if (lane == nb) {
          q_e0 = ne0;
          q_L = nL;
        }
        ++issued;
      }
    }
  }
  for (uint32_t d = issued > static_cast<uint32_t>(kRssBufs) ? issued - kRssBufs : 0u; d < issued && !failed; ++d)
    sort_staged(d);
  if (lane == 0) {
    // after a failure, let staged copies that were never sorted land (bounded waits)
    if (failed)
      for (uint32_t x = sorted; x < issued; ++x) (void)mbar_wait(&bar[x % kRssBufs], (x / kRssBufs) & 1u, status);
  }
}

// ------------------------------------------------------------ host side ----

constexpr int kCacheDevices = 64;
constexpr int kCacheTileSizes = 9;  // tile_units 512, 1024, 2048, 3072, 4096, 6144, 8192, 12288, 16384; others are not cached

// Cache entry of a launch shape for device d, tile size E and staging depth
// (null: do not cache).
inline std::atomic<int>* cache_slot(std::atomic<int>* cache, const DeviceInfo& d, uint32_t E, int stages) {
  int t = 0;
  if (E) {
    static const uint32_t kSizes[kCacheTileSizes] = {512, 1024, 2048, 3072, 4096, 6144, 8192, 12288, 16384};
    t = -1;
    for (int q = 0; q < kCacheTileSizes; ++q)
      if (kSizes[q] == E) t = q;
    if (t < 0) return nullptr;
  }
  if (d.device < 0 || d.device >= kCacheDevices || stages < 1 || stages > kMaxStages) return nullptr;
  return &cache[(d.device * kCacheTileSizes + t) * kMaxStages + (stages - 1)];
}

// Dynamic shared memory a tile-kernel block may take (the 227 KB per-block
// limit less a margin for the kernel's static shared memory).
constexpr size_t kTileSmemLimit = 232448 - 4096;

// Whether `stages` stages of E-unit tiles fit in a block's shared memory:
// packed stages for the ring kernel (mode 0), fixed ones for the synchronous
// kernel (mode 1).
template <class K, bool kVals>
bool tile_fits(int E, int stages, int mode) {
  if (E < 512 || E > 16384 || stages < 2 || stages > kMaxStages) return false;
  const uint32_t e = static_cast<uint32_t>(E);
  const size_t bytes = mode == 1 ? TileLayout<K, kVals>(e).total(stages) : RingLayout<K, kVals>(e).total(stages);
  // work items of one tile: a network item holds 32 segments of >= 3 units
  // (offset + 2 items), a pair item 16 of >= 18 units; the network list is
  // one run (a chunk may span two classes), so at most (E + 256) / 96 + 2
  const int items_per_tile = (E + kMaxSeg) / 96 + 2;
  return bytes <= kTileSmemLimit && stages * items_per_tile + kTileWarps <= kRing;
}

// Resident blocks per SM of `kern` with `smem` bytes of dynamic shared
// memory; the attribute set-up (to `attr_smem`, the most any launch of the
// kernel uses, so that one launch's set-up never lowers another's limit) and
// the occupancy query run once per cache entry (0 = not yet known), so later
// calls make no runtime queries.
template <class Kern>
cudaError_t blocks_per_sm(Kern kern, int threads, int smem, int attr_smem, std::atomic<int>* cached, int* out) {
  int per_sm = cached ? cached->load(std::memory_order_relaxed) : 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, attr_smem);
    if (e != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    if (cached) cached->store(per_sm, std::memory_order_relaxed);
  }
  *out = per_sm;
  return cudaSuccess;
}

template <class K, bool kVals, bool kF>
cudaError_t launch_all(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, bool rss_only,
                       void* scratch, const SegTuning& tun, cudaStream_t stream, const DeviceInfo& d) {
  const uint32_t E = static_cast<uint32_t>(tun.tile_units);
  const ScratchLayout sl(nseg, E);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  Plan* plan = reinterpret_cast<Plan*>(base + sl.plan_at);
  uint32_t* tile_first = reinterpret_cast<uint32_t*>(base + sl.tile_first_at);
  uint16_t* counts = reinterpret_cast<uint16_t*>(base + sl.counts_at);
  uint16_t* order = reinterpret_cast<uint16_t*>(base + sl.order_at);
  uint32_t* cls = reinterpret_cast<uint32_t*>(base + sl.cls_at);

  cudaError_t e = cudaMemsetAsync(plan, 0, sizeof(Plan), stream);
  if (e != cudaSuccess) return e;
  // a thread per group of four offsets, kPlanU groups per step; at most one
  // wave of 8 blocks per SM
  const uint64_t want = (nseg / 4 + 2 + 256 * kPlanU - 1) / (256 * kPlanU);
  const unsigned g1 = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(want, 8ull * d.sm_count)));
  TileDiv tdiv{__builtin_ctz(E), 0, E};
  tdiv.m = E >> tdiv.k;
  if (tdiv.m == 3 && tdiv.k < 8) tdiv.m = 0;  // keep u >> k within 32 bits: the general division
  seg_plan_kernel<<<g1, 256, 0, stream>>>(offsets, nseg, tdiv, plan, tile_first, sl.cap, cls, rss_only,
                                          tun.net_classes, d.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const unsigned g2 = static_cast<unsigned>(std::max<uint64_t>(
      1, std::min<uint64_t>(sl.cap - 1, 8ull * d.sm_count)));
  seg_bin_kernel<<<g2, kBinWarps * 32, 0, stream>>>(cls, offsets, plan, tile_first, counts, order);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  if (tun.tile_mode == 1) {
    const TileLayout<K, kVals> lay(E);
    const int smem_bytes = static_cast<int>(lay.total(tun.tile_stages));
    auto kern = tun.tile_stages == 2   ? seg_sync_kernel<K, kVals, 2, kF>
                : tun.tile_stages == 3 ? seg_sync_kernel<K, kVals, 3, kF>
                                       : seg_sync_kernel<K, kVals, 4, kF>;
    static std::atomic<int> cache[kCacheDevices * kCacheTileSizes * kMaxStages];
    int per_sm = 0;
    if ((e = blocks_per_sm(kern, kSyncThreads, smem_bytes, static_cast<int>(kTileSmemLimit),
                           cache_slot(cache, d, E, tun.tile_stages), &per_sm)) != cudaSuccess)
      return e;
    const unsigned g3 = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>(sl.cap - 1, static_cast<uint64_t>(d.sm_count) * per_sm)));
    kern<<<g3, kSyncThreads, smem_bytes, stream>>>(keys, vals, offsets, plan, tile_first, E, tun.net_classes,
                                                   rss_only, d.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    const RingLayout<K, kVals> lay(E);
    const int smem_bytes = static_cast<int>(lay.total(tun.tile_stages));
    auto kern = tun.tile_stages == 2   ? seg_tile_kernel<K, kVals, 2, kF>
                : tun.tile_stages == 3 ? seg_tile_kernel<K, kVals, 3, kF>
                                       : seg_tile_kernel<K, kVals, 4, kF>;
    static std::atomic<int> cache[kCacheDevices * kCacheTileSizes * kMaxStages];
    int per_sm = 0;
    if ((e = blocks_per_sm(kern, kTileThreads, smem_bytes, static_cast<int>(kTileSmemLimit),
                           cache_slot(cache, d, E, tun.tile_stages), &per_sm)) != cudaSuccess)
      return e;
    const unsigned g3 = static_cast<unsigned>(
        std::max<uint64_t>(1, std::min<uint64_t>(sl.cap - 1, static_cast<uint64_t>(d.sm_count) * per_sm)));
    kern<<<g3, kTileThreads, smem_bytes, stream>>>(keys, vals, offsets, plan, tile_first, counts, order, E,
                                                   d.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  {
    using WL = RssWarpLayout<K, kVals>;
    const int smem_bytes = static_cast<int>(kRssWarps * WL::kBytes);
    auto kern = seg_rss_kernel<K, kVals, kF>;
    static std::atomic<int> cache[kCacheDevices * kCacheTileSizes * kMaxStages];
    int per_sm = 0;
    if ((e = blocks_per_sm(kern, kRssThreads, smem_bytes, smem_bytes, cache_slot(cache, d, 0, 2), &per_sm)) !=
        cudaSuccess)
      return e;
    const uint64_t tiles_cap = sl.cap - 1;
    const unsigned g4 = static_cast<unsigned>(std::max<uint64_t>(
        1, std::min<uint64_t>((tiles_cap + kRssWarps - 1) / kRssWarps, static_cast<uint64_t>(d.sm_count) * per_sm)));
    kern<<<g4, kRssThreads, smem_bytes, stream>>>(keys, vals, offsets, plan, tile_first, counts, order,
                                                   tun.rss_two_min, !rss_only && (tun.net_classes & 0x10u),
                                                   d.status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace seg
}  // namespace sn

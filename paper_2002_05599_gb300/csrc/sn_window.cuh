// Segmented sorting in one persistent launch: warp windows.
//
// The batching layer of the paper's future-work suggestion (Sec. 5: bucket
// base cases by size, solve batches of equal size), without a separate
// planning or binning pass over the batch:
//
// * Every warp works on its own.  It takes groups of 32 consecutive segments
//   (group g = segments [32 g, 32 g + 32)) round-robin over the grid's warps;
//   lane i holds offsets[32 g + i] and offsets[32 g + i + 1] in registers, and
//   the next group's offsets are fetched while the current one is worked on.
// * From a group the warp cuts windows: runs of consecutive segments whose
//   items fit the staging capacity C (a ballot over the lanes finds where the
//   next segment would not fit).  A window's keys (and payload) are staged in
//   shared memory by 1-D bulk copies, `nbuf` windows in flight per warp, each
//   completing on its own mbarrier.
// * A landed window is sorted in place:
//     - segments of 2..16 items one per lane, by the network of the largest
//       such segment of the window (2, 4, 8, 12 or 16 channels, padded with
//       the maximum key), Sec. 2;
//     - 17..32 items on lane pairs (16-channel networks and a bitonic merge
//       through shuffles), 16 segments per pass;
//     - 33..64 items by the 64-item warp network (a launch parameter), and up
//       to 256 by Register Sample Sort (Sec. 3) on the whole warp, one segment
//       after another;
//   in RSS-only mode every segment over 16 items takes Register Sample Sort.
// * The window is written back with coalesced stores (16-byte stores for its
//   whole granules), so its buffer can be refilled at once.
//
// Offsets are validated by a pass of their own before (seg_validate_kernel):
// a batch with a decreasing offset or a segment over 256 items is left
// untouched and reported as kStatusRange.
#pragma once

#include "sn_segments.cuh"

namespace sn {
namespace seg {
namespace {

constexpr int kWinWarps = 4;
constexpr int kWinThreads = kWinWarps * 32;

// Window capacity limits (items): a window holds at least one whole segment.
constexpr uint32_t kWinMinItems = 512;
constexpr uint32_t kWinMaxItems = 4096;

struct WinMeta {
  uint32_t e0;         // first item of the window
  uint32_t n;          // items in the window
  uint32_t key_shift;  // index of keys[e0] in the staged keys
  uint32_t val_shift;  // index of vals[e0] in the staged payload
  uint32_t k;          // segments in the window
  uint32_t pad[3];
};

// Per-warp shared memory: nbuf mbarriers, window records, per-window segment
// tables (one word per segment: offset in the window << 9 | length), the
// Register Sample Sort scratch, and nbuf staging buffers (keys, payload).
template <class K, bool kVals>
struct WinLayout {
  size_t bars_at, meta_at, tab_at, rss_at, buf_at, key_cap, val_cap, buf_bytes, warp_bytes;
  __host__ __device__ WinLayout(uint32_t C, int nbuf) {
    bars_at = 0;
    meta_at = align16(8 * static_cast<size_t>(nbuf));
    tab_at = align16(meta_at + sizeof(WinMeta) * nbuf);
    rss_at = align16(tab_at + 128 * static_cast<size_t>(nbuf));
    buf_at = align128(rss_at + RssMem<K, kVals>::kBytes);
    key_cap = align16((static_cast<size_t>(C) + 2 * (16 / sizeof(K))) * sizeof(K));
    val_cap = kVals ? align16((static_cast<size_t>(C) + 8) * 4) : 0;
    buf_bytes = key_cap + val_cap;
    warp_bytes = align128(buf_at + buf_bytes * nbuf);
  }
};

// Resident blocks (of kWinWarps warps) per SM the register budget is sized
// for: 64 registers a thread for 4-byte keys alone, 80 for 4-byte keys with
// payload or 8-byte keys, 128 for 8-byte keys with payload.
template <class K, bool kVals>
constexpr int win_min_blocks() {
  return sizeof(K) == 4 ? (kVals ? 6 : 8) : (kVals ? 4 : 6);
}

// Offsets check before any data is touched: non-decreasing, every segment at
// most 256 items.  One atomic per warp that found a violation.
__global__ void __launch_bounds__(256)
    seg_validate_kernel(const uint32_t* __restrict__ offsets, uint64_t nseg, unsigned* bad, unsigned* status) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool b = false;
  constexpr int kU = 4;
  for (uint64_t sb = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; sb < nseg; sb += kU * stride) {
    uint32_t o[kU], o1[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint64_t s = sb + u * stride;
      o[u] = o1[u] = 0;
      if (s < nseg) {
        o[u] = offsets[s];
        o1[u] = offsets[s + 1];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (o1[u] < o[u] || o1[u] - o[u] > kMaxSeg) b = true;
  }
  if (__any_sync(kFull, b) && (threadIdx.x & 31) == 0) {
    atomicOr(bad, 1u);
    atomicOr(status, kStatusRange);
  }
}

// Items [0, n) of a staged window back to dst (dst[0] is staged[shift]; the
// staged buffer starts at the 16-byte granule holding dst[0]): whole
// granules with 16-byte stores, the partial granules at both ends with
// element stores.
template <class T>
__device__ __forceinline__ void store_window(T* dst, const T* staged, uint32_t shift, uint32_t n, int lane) {
  if (n == 0) return;
  const uintptr_t a = reinterpret_cast<uintptr_t>(dst), z = reinterpret_cast<uintptr_t>(dst + n);
  const uintptr_t ia = (a + 15) & ~uintptr_t(15), iz = z & ~uintptr_t(15);
  if (ia < iz) {
    const uint32_t head = static_cast<uint32_t>((ia - a) / sizeof(T));
    const uint32_t tail = static_cast<uint32_t>((iz - a) / sizeof(T));
    const uint32_t ng = static_cast<uint32_t>((iz - ia) / 16);
    const uint4* src = reinterpret_cast<const uint4*>(staged + shift + head);
    uint4* out = reinterpret_cast<uint4*>(ia);
    for (uint32_t j = lane; j < ng; j += 32) out[j] = src[j];
    if (static_cast<uint32_t>(lane) < head) dst[lane] = staged[shift + lane];
    if (tail + lane < n) dst[tail + lane] = staged[shift + tail + lane];
  } else {
    for (uint32_t e = lane; e < n; e += 32) dst[e] = staged[shift + e];
  }
}

template <class K, bool kVals, bool kF>
__global__ void __launch_bounds__(kWinThreads, win_min_blocks<K, kVals>())
    seg_window_kernel(K* __restrict__ keys, uint32_t* __restrict__ vals, const uint32_t* __restrict__ offsets,
                      uint64_t nseg, const unsigned* __restrict__ bad, uint32_t C, int nbuf, uint32_t net_mask,
                      bool rss_only, bool net64, int two_min, unsigned* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (*bad) return;  // the offsets failed validation: leave the batch untouched
  const WinLayout<K, kVals> lay(C, nbuf);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  unsigned char* wb = smem + warp * lay.warp_bytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(wb + lay.bars_at);
  WinMeta* meta = reinterpret_cast<WinMeta*>(wb + lay.meta_at);
  uint32_t* tab = reinterpret_cast<uint32_t*>(wb + lay.tab_at);
  const RssMem<K, kVals> rm(wb + lay.rss_at);
  auto kbuf_of = [&](int b) { return reinterpret_cast<K*>(wb + lay.buf_at + b * lay.buf_bytes); };
  auto vbuf_of = [&](int b) {
    return reinterpret_cast<uint32_t*>(wb + lay.buf_at + b * lay.buf_bytes + lay.key_cap);
  };
  if (lane == 0) {
    for (int b = 0; b < nbuf; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncwarp();
  const bool skip_copy = lane == 0 && (test_flags(status) & kTestSkipTileCopy);

  const uint64_t ngroups = (nseg + 31) >> 5;
  const uint64_t W = static_cast<uint64_t>(gridDim.x) * kWinWarps;
  uint64_t g = static_cast<uint64_t>(blockIdx.x) * kWinWarps + warp;
  auto fetch = [&](uint64_t gg, uint32_t& l, uint32_t& h) {
    const uint64_t s = gg * 32 + lane;
    l = h = 0;
    if (gg < ngroups && s < nseg) {
      l = offsets[s];
      h = offsets[s + 1];
    }
  };
  auto valid_of = [&](uint64_t gg) -> int {
    return gg < ngroups ? static_cast<int>(nseg - gg * 32 < 32 ? nseg - gg * 32 : 32) : 0;
  };
  uint32_t lo, hi, nlo, nhi;
  fetch(g, lo, hi);
  fetch(g + W, nlo, nhi);
  int nv = valid_of(g);
  int st = 0;  // first segment of the group not yet in a window
  bool more = nv > 0;
  const uintptr_t kb = reinterpret_cast<uintptr_t>(keys);
  const uintptr_t vb = reinterpret_cast<uintptr_t>(vals);

  // Cut the next window from the current group and stage it into buffer b.
  auto issue = [&](int b) {
    const uint32_t base = __shfl_sync(kFull, lo, st);
    const bool fit = lane >= st && lane < nv && hi - base <= C;
    const int k = __popc(__ballot_sync(kFull, fit));  // >= 1: one segment always fits
    const uint32_t end = __shfl_sync(kFull, hi, st + k - 1);
    if (lane >= st && lane < st + k) tab[b * 32 + (lane - st)] = ((lo - base) << 9) | (hi - lo);
    if (lane == 0) {
      const uintptr_t ka = (kb + sizeof(K) * base) & ~uintptr_t(15);
      const uintptr_t kz = (kb + sizeof(K) * end + 15) & ~uintptr_t(15);
      const uint32_t kbytes = end > base ? static_cast<uint32_t>(kz - ka) : 0u;
      uintptr_t va = 0, vz = 0;
      uint32_t vbytes = 0;
      if constexpr (kVals) {
        va = (vb + 4ull * base) & ~uintptr_t(15);
        vz = (vb + 4ull * end + 15) & ~uintptr_t(15);
        vbytes = end > base ? static_cast<uint32_t>(vz - va) : 0u;
      }
      WinMeta m;
      m.e0 = base;
      m.n = end - base;
      m.key_shift = static_cast<uint32_t>((kb + sizeof(K) * base - ka) / sizeof(K));
      m.val_shift = kVals ? static_cast<uint32_t>((vb + 4ull * base - va) / 4) : 0u;
      m.k = static_cast<uint32_t>(k);
      // self-check of both copies against the buffer
      if (end < base || end - base > C || kbytes > lay.key_cap || vbytes > lay.val_cap) {
        atomicOr(status, kStatusInternal | kCheckCopyArgs);
        m.n = 0;
        m.k = 0;
        mbar_arrive(&bar[b]);  // an empty window: nothing to wait for, nothing to store
      } else {
        mbar_arrive_expect_tx(&bar[b], kbytes + vbytes);
        if (!skip_copy) {  // (the test hook arms the barrier and issues no copy)
          if (kbytes) bulk_g2s(kbuf_of(b), reinterpret_cast<const void*>(ka), kbytes, &bar[b]);
          if constexpr (kVals)
            if (vbytes) bulk_g2s(vbuf_of(b), reinterpret_cast<const void*>(va), vbytes, &bar[b]);
        }
      }
      meta[b] = m;
    }
    st += k;
    if (st >= nv) {  // on to the next group; fetch the one after it
      g += W;
      lo = nlo;
      hi = nhi;
      nv = valid_of(g);
      st = 0;
      more = nv > 0;
      if (more) fetch(g + W, nlo, nhi);
    }
    __syncwarp();  // the window record and table before any lane reads them
  };

  // Sort the landed window of buffer b in place, then write it back.
  auto process = [&](int b) {
    const WinMeta m = meta[b];
    K* kbuf = kbuf_of(b);
    uint32_t* vbuf = vbuf_of(b);
    const bool mine = static_cast<uint32_t>(lane) < m.k;
    const uint32_t t = mine ? tab[b * 32 + lane] : 0u;
    const int L = static_cast<int>(t & 511u);
    const int p = static_cast<int>((t >> 9) + m.key_shift);
    const int pv = static_cast<int>((t >> 9) + m.val_shift);
    // 2..16 items: one segment per lane, the window's largest class
    const bool net = mine && L >= 2 && L <= 16;
    const uint32_t mx = __reduce_max_sync(kFull, net ? static_cast<uint32_t>(L) : 0u);
    if (mx >= 2) {
      const int cls = (mx <= 2 && (net_mask & 1u))    ? 2
                      : (mx <= 4 && (net_mask & 2u))  ? 4
                      : (mx <= 8 && (net_mask & 4u))  ? 8
                      : (mx <= 12 && (net_mask & 8u)) ? 12
                                                      : 16;
      if (cls == 16) {
        seg16<K, kVals, kF>(kbuf, vbuf, p, pv, L, net, false, lane);
      } else if (net) {
        if (cls == 12)
          net_segment<12, K, kVals, kF>(kbuf, vbuf, p, pv, L);
        else if (cls == 8)
          net_segment<8, K, kVals, kF>(kbuf, vbuf, p, pv, L);
        else if (cls == 4)
          net_segment<4, K, kVals, kF>(kbuf, vbuf, p, pv, L);
        else
          net_segment<2, K, kVals, kF>(kbuf, vbuf, p, pv, L);
      }
    }
    // 17..32 items: 16 segments per pass on lane pairs
    if (!rss_only) {
      unsigned pm = __ballot_sync(kFull, mine && L >= 17 && L <= 32);
      while (pm) {
        const int src = nth_set_bit(pm, lane >> 1);
        const bool act = src >= 0;
        const int from = act ? src : 0;
        const int pp = __shfl_sync(kFull, p, from), ppv = __shfl_sync(kFull, pv, from);
        const int pL = __shfl_sync(kFull, L, from);
        seg16<K, kVals, kF>(kbuf, vbuf, pp, ppv, act ? pL : 0, act, true, lane);
        for (int q = 0; q < 16 && pm; ++q) pm &= pm - 1;
      }
    }
    // longer segments on the whole warp, one after another
    unsigned bm = __ballot_sync(kFull, mine && (rss_only ? L > 16 : L > 32));
    while (bm) {
      const int src = __ffs(bm) - 1;
      bm &= bm - 1;
      const int bp = __shfl_sync(kFull, p, src), bpv = __shfl_sync(kFull, pv, src);
      const int bL = __shfl_sync(kFull, L, src);
      if (net64 && !rss_only && bL <= 64)
        net64_segment<K, kVals, kF, true>(kbuf, vbuf, bp, bpv, bL, lane, kbuf + bp, vbuf + bpv);
      else
        rss_segment<K, kVals, kF, true>(kbuf, vbuf, bp, bpv, bL, rm, lane, two_min, kbuf + bp, vbuf + bpv);
    }
    __syncwarp();
    store_window<K>(keys + m.e0, kbuf, m.key_shift, m.n, lane);
    if constexpr (kVals) store_window<uint32_t>(vals + m.e0, vbuf, m.val_shift, m.n, lane);
    // this lane's shared-memory writes before the next bulk copy into the buffer
    fence_proxy_async_smem();
    __syncwarp();
  };

  uint32_t issued = 0, done = 0;
  while (issued < static_cast<uint32_t>(nbuf) && more) {
    issue(static_cast<int>(issued % nbuf));
    ++issued;
  }
  bool failed = false;
  while (done < issued) {
    const int b = static_cast<int>(done % nbuf);
    // every lane waits itself (bulk-copy data is visible to the lanes that
    // observe the phase); a timeout anywhere fails the whole warp
    if (!__all_sync(kFull, mbar_wait(&bar[b], (done / nbuf) & 1u, status))) {
      failed = true;
      break;
    }
    process(b);
    ++done;
    if (more) {
      issue(static_cast<int>(issued % nbuf));
      ++issued;
    }
  }
  if (failed && lane == 0) {
    atomicOr(status, kStatusTimeout);
    // let copies that were issued but never consumed land before the warp leaves
    for (uint32_t x = done; x < issued; ++x) (void)mbar_wait(&bar[x % nbuf], (x / nbuf) & 1u, status);
  }
}

// ------------------------------------------------------------ host side ----

// Whether nbuf buffers of C-item windows fit in shared memory (kWinWarps
// warps per block).
template <class K, bool kVals>
bool window_fits(int C, int nbuf) {
  if (C < static_cast<int>(kWinMinItems) || C > static_cast<int>(kWinMaxItems) || nbuf < 2 || nbuf > kMaxStages)
    return false;
  return kWinWarps * WinLayout<K, kVals>(static_cast<uint32_t>(C), nbuf).warp_bytes <= kTileSmemLimit;
}

template <class K, bool kVals, bool kF>
cudaError_t launch_window(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, bool rss_only,
                          void* scratch, const SegTuning& tun, cudaStream_t stream, const DeviceInfo& d) {
  const uint32_t C = static_cast<uint32_t>(tun.tile_units);
  const int nbuf = tun.tile_stages;
  unsigned* bad = &reinterpret_cast<Plan*>(scratch)->bad;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return e;
  const uint64_t want = (nseg + 1023) / 1024;
  const unsigned g1 = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(want, 8ull * d.sm_count)));
  seg_validate_kernel<<<g1, 256, 0, stream>>>(offsets, nseg, bad, d.status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const WinLayout<K, kVals> lay(C, nbuf);
  const int smem_bytes = static_cast<int>(kWinWarps * lay.warp_bytes);
  auto kern = seg_window_kernel<K, kVals, kF>;
  static std::atomic<int> cache[kCacheDevices * kCacheTileSizes * kMaxStages];
  int per_sm = 0;
  if ((e = blocks_per_sm(kern, kWinThreads, smem_bytes, static_cast<int>(kTileSmemLimit),
                         cache_slot(cache, d, C, nbuf), &per_sm)) != cudaSuccess)
    return e;
  const uint64_t ngroups = (nseg + 31) / 32;
  const unsigned g2 = static_cast<unsigned>(std::max<uint64_t>(
      1, std::min<uint64_t>((ngroups + kWinWarps - 1) / kWinWarps, static_cast<uint64_t>(d.sm_count) * per_sm)));
  kern<<<g2, kWinThreads, smem_bytes, stream>>>(keys, vals, offsets, nseg, bad, C, nbuf, tun.net_classes, rss_only,
                                                !rss_only && (tun.net_classes & 0x10u), tun.rss_two_min, d.status);
  return cudaGetLastError();
}

// Shared-memory fit of a parameter set: tile_mode 2 is the window kernel
// (tile_units = window capacity C in items, tile_stages = windows in flight
// per warp), modes 0 and 1 the tile kernels.
template <class K, bool kVals>
bool seg_fits(int E, int stages, int mode) {
  return mode == 2 ? window_fits<K, kVals>(E, stages) : tile_fits<K, kVals>(E, stages, mode);
}

template <class K, bool kF = false>
cudaError_t launch_segments(K* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, SegMode mode,
                            void* scratch, size_t scratch_bytes, const SegTuning& t, cudaStream_t s,
                            const DeviceInfo& d) {
  if (t.tile_units < 512 || t.rss_two_min < 16 || t.rss_two_min > kMaxSeg || t.net_classes > 0x1Fu ||
      t.tile_mode < 0 || t.tile_mode > 2)
    return cudaErrorInvalidValue;
  if (!(vals ? seg_fits<K, true>(t.tile_units, t.tile_stages, t.tile_mode)
             : seg_fits<K, false>(t.tile_units, t.tile_stages, t.tile_mode)))
    return cudaErrorInvalidValue;
  const bool rss = mode == SegMode::kRssOnly;
  if (t.tile_mode == 2) {
    if (scratch_bytes < sizeof(Plan)) return cudaErrorInvalidValue;
    return vals ? launch_window<K, true, kF>(keys, vals, offsets, nseg, rss, scratch, t, s, d)
                : launch_window<K, false, kF>(keys, vals, offsets, nseg, rss, scratch, t, s, d);
  }
  if (scratch_bytes < ScratchLayout(nseg, static_cast<uint32_t>(t.tile_units)).total) return cudaErrorInvalidValue;
  return vals ? launch_all<K, true, kF>(keys, vals, offsets, nseg, rss, scratch, t, s, d)
              : launch_all<K, false, kF>(keys, vals, offsets, nseg, rss, scratch, t, s, d);
}

}  // namespace
}  // namespace seg
}  // namespace sn

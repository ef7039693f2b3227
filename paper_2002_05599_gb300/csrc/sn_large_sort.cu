// Sorting one large array with this library's small-set sorters as the base
// case (include/smallsort.h: sn_sort_large).  The paper evaluates its sorters
// as base cases of Quicksort and IPS4o (Sec. 4.5, 4.6); this is the GPU
// counterpart: one sample-sort partition of the array into buckets of about
// 128 keys, then every bucket sorted by the segmented path.
//
// One level, for n keys:
//   1. sample: S = 4k items at equidistant positions, k = ceil(n / 128)
//      buckets; the sample is sorted by a recursive call (it is 32 times
//      smaller); splitters are every 4th sample item;
//   2. classify: each key finds its bucket by binary search over the k - 1
//      splitters (bucket b holds s_{b-1} < x <= s_b) and counts it;
//   3. exclusive scans give bucket starts and the base-case layout; keys are
//      scattered into a scratch copy, bucket by bucket;
//   4. base case: buckets of <= 256 keys go to the segmented sort (network /
//      warp network / Register Sample Sort) as CSR segments; buckets of
//      257..4096 are cut into 256-key segments there and then sorted whole by
//      the long-segment kernel; larger buckets (rare) recurse;
//   5. the sorted copy is copied back.
// u32 keys are classified as (key, position) pairs packed into 64 bits, so
// every element is distinct and duplicates cannot gather in one bucket; the
// sample of such pairs is sorted as distinct u64 values.  The call reads a few
// counts back to the host at each level, so it returns when the sort is done.
#include <algorithm>
#include <vector>

#include "smallsort.h"
#include "sn_common.cuh"
#include "sn_internal.h"

namespace sn {
namespace {

constexpr uint64_t kBucketTarget = 128;
constexpr uint32_t kOversample = 4;
constexpr uint32_t kBaseMax = SN_MAX_SEGMENT;
constexpr uint32_t kLongMax = SN_MAX_SEGMENT_LARGE;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr uint64_t kScanTile = static_cast<uint64_t>(kScanThreads) * kScanItems;

// Classification value: (key, position) for u32 keys, the key itself for the
// distinct u64 values of a sample.
__device__ __forceinline__ uint64_t class_value(uint32_t key, uint64_t pos) {
  return (static_cast<uint64_t>(key) << 32) | pos;
}
__device__ __forceinline__ uint64_t class_value(uint64_t key, uint64_t) { return key; }

template <class K>
__global__ void sample_kernel(const K* __restrict__ keys, uint64_t n, uint64_t S, uint64_t* __restrict__ sample) {
  for (uint64_t q = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < S;
       q += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t p = ((2 * q + 1) * n) / (2 * S);
    sample[q] = class_value(keys[p], p);
  }
}

// Bucket of every key: the number of splitters below its value, splitter j
// being sample[(j + 1) * a - 1]; counted into counts[].
template <class K>
__global__ void classify_kernel(const K* __restrict__ keys, uint64_t n, const uint64_t* __restrict__ sample,
                                uint32_t a, uint32_t nspl, uint32_t* __restrict__ bucket,
                                uint32_t* __restrict__ counts) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t x = class_value(keys[i], i);
    uint32_t lo = 0, hi = nspl;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sample[static_cast<uint64_t>(mid + 1) * a - 1] < x)
        lo = mid + 1;
      else
        hi = mid;
    }
    bucket[i] = lo;
    atomicAdd(&counts[lo], 1u);
  }
}

template <class K>
__global__ void scatter_kernel(const K* __restrict__ keys, uint64_t n, const uint32_t* __restrict__ bucket,
                               const uint32_t* __restrict__ starts, uint32_t* __restrict__ fill,
                               K* __restrict__ out) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint32_t b = bucket[i];
    out[starts[b] + atomicAdd(&fill[b], 1u)] = keys[i];
  }
}

// Per bucket: base-case segments (1, or ceil(c / 256) for c > 256; an empty
// bucket still takes one empty segment), and flags for the long-segment and
// recursion lists.
__global__ void layout_counts_kernel(const uint32_t* __restrict__ counts, uint32_t k, uint32_t* __restrict__ nsegs,
                                     uint32_t* __restrict__ long_flag, uint32_t* __restrict__ big_flag) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += gridDim.x * blockDim.x) {
    const uint32_t c = counts[b];
    nsegs[b] = c <= kBaseMax ? 1u : (c + kBaseMax - 1) / kBaseMax;
    long_flag[b] = (c > kBaseMax && c <= kLongMax) ? 1u : 0u;
    big_flag[b] = c > kLongMax ? 1u : 0u;
  }
}

__global__ void layout_write_kernel(const uint32_t* __restrict__ counts, const uint32_t* __restrict__ starts,
                                    uint32_t k, const uint32_t* __restrict__ seg_at, const uint32_t* __restrict__ long_at,
                                    const uint32_t* __restrict__ big_at, uint32_t* __restrict__ csr,
                                    uint32_t* __restrict__ long_start, uint32_t* __restrict__ long_end,
                                    uint32_t* __restrict__ big_start, uint32_t* __restrict__ big_end) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < k; b += gridDim.x * blockDim.x) {
    const uint32_t c = counts[b], st = starts[b];
    const uint32_t m = c <= kBaseMax ? 1u : (c + kBaseMax - 1) / kBaseMax;
    for (uint32_t j = 0; j < m; ++j) csr[seg_at[b] + j] = st + j * kBaseMax;
    if (c > kBaseMax && c <= kLongMax) {
      long_start[long_at[b]] = st;
      long_end[long_at[b]] = st + c;
    } else if (c > kLongMax) {
      big_start[big_at[b]] = st;
      big_end[big_at[b]] = st + c;
    }
  }
}

__global__ void set_word_kernel(uint32_t* p, uint32_t v) { *p = v; }

// ---- exclusive scan of u32 (out[i] = sum in[0..i), out[n] = total) ----

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, d);
      if (lane >= d) wi += y;
    }
    warp_sums[lane] = wi - w;
    if (lane == 31) *total = wi;
  }
  __syncthreads();
  const uint32_t r = warp_sums[warp] + incl - v;
  __syncthreads();
  return r;
}

// Tile t of kScanTile items: exclusive scan into out (plus offsets[t] when
// given), tile total into sums[t] (when given).
__global__ void __launch_bounds__(kScanThreads)
    scan_tiles_kernel(const uint32_t* __restrict__ in, uint64_t n, uint32_t* __restrict__ out,
                      const uint32_t* __restrict__ offsets, uint32_t* __restrict__ sums) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t total;
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanTile + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = base + q < n ? in[base + q] : 0u;
    s += v[q];
  }
  uint32_t run = block_exclusive_scan(s, warp_sums, &total) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
  if (sums && threadIdx.x == 0) sums[blockIdx.x] = total;
}

struct Pool {
  cudaMemPool_t pool;
  cudaStream_t s;
  std::vector<void*> live;
  bool failed = false;
  template <class T>
  T* get(uint64_t count) {
    void* p = nullptr;
    if (failed || cudaMallocFromPoolAsync(&p, std::max<uint64_t>(count, 1) * sizeof(T) + 256, pool, s) != cudaSuccess) {
      cudaGetLastError();
      failed = true;
      return nullptr;
    }
    live.push_back(p);
    return static_cast<T*>(p);
  }
  ~Pool() {
    for (void* p : live) cudaFreeAsync(p, s);
  }
};

unsigned grid_for(uint64_t items, const DeviceInfo& d, unsigned threads = 256) {
  return static_cast<unsigned>(
      std::max<uint64_t>(1, std::min<uint64_t>((items + threads - 1) / threads, 16ull * d.sm_count)));
}

// out[0..n] = exclusive scan of in[0..n) with out[n] = total (n >= 1).
cudaError_t exclusive_scan(const uint32_t* in, uint64_t n, uint32_t* out, Pool& pool, const DeviceInfo& d) {
  const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    scan_tiles_kernel<<<1, kScanThreads, 0, pool.s>>>(in, n, out, nullptr, out + n);
    return cudaGetLastError();
  }
  uint32_t* sums = pool.get<uint32_t>(tiles + 1);
  if (!sums) return cudaErrorMemoryAllocation;
  scan_tiles_kernel<<<static_cast<unsigned>(tiles), kScanThreads, 0, pool.s>>>(in, n, out, nullptr, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint32_t* sums_scan = pool.get<uint32_t>(tiles + 1);
  if (!sums_scan) return cudaErrorMemoryAllocation;
  if ((e = exclusive_scan(sums, tiles, sums_scan, pool, d)) != cudaSuccess) return e;
  scan_tiles_kernel<<<static_cast<unsigned>(tiles), kScanThreads, 0, pool.s>>>(in, n, out, sums_scan, nullptr);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the total
  return cudaMemcpyAsync(out + n, sums_scan + tiles, sizeof(uint32_t), cudaMemcpyDeviceToDevice, pool.s);
}

template <class K>
cudaError_t launch_base_segments(K* keys, const uint32_t* csr, uint64_t nseg, Pool& pool, const DeviceInfo& d);
template <>
cudaError_t launch_base_segments<uint32_t>(uint32_t* keys, const uint32_t* csr, uint64_t nseg, Pool& pool,
                                           const DeviceInfo& d) {
  const SegTuning tun = current_tuning(d.device, 4, false);
  const size_t bytes = segments_scratch_bytes(nseg, tun);
  void* scratch = pool.get<unsigned char>(bytes);
  if (!scratch) return cudaErrorMemoryAllocation;
  return launch_segments_u32(keys, nullptr, csr, nseg, SegMode::kNetworkWarpRss, scratch, bytes, tun, pool.s, d);
}
template <>
cudaError_t launch_base_segments<uint64_t>(uint64_t* keys, const uint32_t* csr, uint64_t nseg, Pool& pool,
                                           const DeviceInfo& d) {
  const SegTuning tun = current_tuning(d.device, 8, false);
  const size_t bytes = segments_scratch_bytes(nseg, tun);
  void* scratch = pool.get<unsigned char>(bytes);
  if (!scratch) return cudaErrorMemoryAllocation;
  return launch_segments_u64(keys, nullptr, csr, nseg, SegMode::kNetworkWarpRss, scratch, bytes, tun, pool.s, d);
}

cudaError_t launch_long(uint32_t* keys, const uint32_t* st, const uint32_t* en, uint64_t m, void* flag,
                        cudaStream_t s, const DeviceInfo& d) {
  return launch_large_u32(keys, nullptr, st, en, m, flag, s, d);
}
cudaError_t launch_long(uint64_t* keys, const uint32_t* st, const uint32_t* en, uint64_t m, void* flag,
                        cudaStream_t s, const DeviceInfo& d) {
  return launch_large_u64(keys, nullptr, st, en, m, flag, s, d);
}

template <class K>
cudaError_t sort_large(K* keys, uint64_t n, cudaMemPool_t mp, cudaStream_t s, const DeviceInfo& d, int depth) {
  if (n <= 1) return cudaSuccess;
  if (depth > 16) return cudaErrorInvalidValue;  // cannot happen: every level shrinks the problem
  Pool pool{mp, s};
  if (n <= kLongMax) {  // one long segment
    uint32_t* se = pool.get<uint32_t>(2);
    void* flag = pool.get<unsigned char>(16);
    if (pool.failed) return cudaErrorMemoryAllocation;
    set_word_kernel<<<1, 1, 0, s>>>(se, 0);
    set_word_kernel<<<1, 1, 0, s>>>(se + 1, static_cast<uint32_t>(n));
    return launch_long(keys, se, se + 1, 1, flag, s, d);
  }
  const uint64_t k = (n + kBucketTarget - 1) / kBucketTarget;
  const uint64_t S = std::min<uint64_t>(n, kOversample * k);
  uint64_t* sample = pool.get<uint64_t>(S);
  if (pool.failed) return cudaErrorMemoryAllocation;
  sample_kernel<K><<<grid_for(S, d), 256, 0, s>>>(keys, n, S, sample);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = sort_large<uint64_t>(sample, S, mp, s, d, depth + 1)) != cudaSuccess) return e;

  const uint32_t a = static_cast<uint32_t>(S / k);  // splitter j = sample[(j + 1) a - 1]
  const uint32_t nspl = static_cast<uint32_t>(k - 1);
  uint32_t* bucket = pool.get<uint32_t>(n);
  uint32_t* counts = pool.get<uint32_t>(k);
  uint32_t* starts = pool.get<uint32_t>(k + 1);
  uint32_t* fill = pool.get<uint32_t>(k);
  K* tmp = pool.get<K>(n);
  if (pool.failed) return cudaErrorMemoryAllocation;
  if ((e = cudaMemsetAsync(counts, 0, k * 4, s)) != cudaSuccess || (e = cudaMemsetAsync(fill, 0, k * 4, s)) != cudaSuccess)
    return e;
  classify_kernel<K><<<grid_for(n, d), 256, 0, s>>>(keys, n, sample, a, nspl, bucket, counts);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = exclusive_scan(counts, k, starts, pool, d)) != cudaSuccess) return e;
  scatter_kernel<K><<<grid_for(n, d), 256, 0, s>>>(keys, n, bucket, starts, fill, tmp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // base-case layout
  uint32_t* nsegs = pool.get<uint32_t>(k);
  uint32_t* long_flag = pool.get<uint32_t>(k);
  uint32_t* big_flag = pool.get<uint32_t>(k);
  uint32_t* seg_at = pool.get<uint32_t>(k + 1);
  uint32_t* long_at = pool.get<uint32_t>(k + 1);
  uint32_t* big_at = pool.get<uint32_t>(k + 1);
  if (pool.failed) return cudaErrorMemoryAllocation;
  layout_counts_kernel<<<grid_for(k, d), 256, 0, s>>>(counts, static_cast<uint32_t>(k), nsegs, long_flag, big_flag);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = exclusive_scan(nsegs, k, seg_at, pool, d)) != cudaSuccess) return e;
  if ((e = exclusive_scan(long_flag, k, long_at, pool, d)) != cudaSuccess) return e;
  if ((e = exclusive_scan(big_flag, k, big_at, pool, d)) != cudaSuccess) return e;
  uint32_t tot[3];
  if ((e = cudaMemcpyAsync(&tot[0], seg_at + k, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&tot[1], long_at + k, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&tot[2], big_at + k, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return e;
  const uint64_t nseg = tot[0], nlong = tot[1], nbig = tot[2];
  uint32_t* csr = pool.get<uint32_t>(nseg + 1);
  uint32_t* long_start = pool.get<uint32_t>(nlong);
  uint32_t* long_end = pool.get<uint32_t>(nlong);
  uint32_t* big_start = pool.get<uint32_t>(nbig);
  uint32_t* big_end = pool.get<uint32_t>(nbig);
  void* flag = pool.get<unsigned char>(16);
  if (pool.failed) return cudaErrorMemoryAllocation;
  layout_write_kernel<<<grid_for(k, d), 256, 0, s>>>(counts, starts, static_cast<uint32_t>(k), seg_at, long_at,
                                                     big_at, csr, long_start, long_end, big_start, big_end);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  set_word_kernel<<<1, 1, 0, s>>>(csr + nseg, static_cast<uint32_t>(n));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  if ((e = launch_base_segments<K>(tmp, csr, nseg, pool, d)) != cudaSuccess) return e;
  if (nlong && (e = launch_long(tmp, long_start, long_end, nlong, flag, s, d)) != cudaSuccess) return e;
  if (nbig) {
    std::vector<uint32_t> bs(nbig), be(nbig);
    if ((e = cudaMemcpyAsync(bs.data(), big_start, nbig * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(be.data(), big_end, nbig * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return e;
    for (uint64_t j = 0; j < nbig; ++j)
      if ((e = sort_large<K>(tmp + bs[j], be[j] - bs[j], mp, s, d, depth + 1)) != cudaSuccess) return e;
  }
  return cudaMemcpyAsync(keys, tmp, n * sizeof(K), cudaMemcpyDeviceToDevice, s);
}

}  // namespace

cudaError_t sort_large_u32(uint32_t* keys, uint64_t n, cudaStream_t s, const DeviceInfo& d) {
  const cudaError_t e = sort_large<uint32_t>(keys, n, d.pool, s, d, 0);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace sn

// Device primitives shared by the sorting kernels (sm_103a).
//
// Compare-exchange follows the comparator of Sec. 2.1: after it, the lower
// channel holds the smaller value.  On the GPU it is a pair of integer
// min/max (keys only) or one compare and selects (key + index items): no
// branches, all registers, the GPU counterpart of the paper's conditional-move
// swaps (Sec. 2.2.2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "networks_gen.h"

namespace sn {

// ---- status bits written by kernels into the per-device status word ----
constexpr unsigned kStatusRange = 1u;    // bad offsets / segment too long
constexpr unsigned kStatusTimeout = 2u;  // a bounded wait ran out
constexpr unsigned kStatusInternal = 4u; // an internal consistency check failed
// finer internal-check bits (reported together as an internal failure)
constexpr unsigned kCheckStageMoved = 8u;    // a tile's metadata changed while a work item was in flight
constexpr unsigned kCheckCopyArgs = 16u;     // a bulk copy's range or alignment was invalid
constexpr unsigned kCheckSegment = 32u;      // a segment's staged span left its buffer

// Per-device control block in device memory.  Kernels receive the address of
// its first word as `unsigned* status`:
//   status bits   OR-ed by kernels (kStatus*, kCheck*), read and cleared by
//                 sn_check / sn_get_last_cuda_error;
//   test flags    kTestSkip* below, zero in normal use (set only by the test
//                 hook sn_test_set_flags);
//   wait limit    every bounded wait gives up after this many nanoseconds of
//                 %globaltimer, reports kStatusTimeout and lets the kernel
//                 return (sn_set_wait_limit; two seconds by default).
struct alignas(16) DevCtl {
  unsigned status;
  unsigned test_flags;
  unsigned long long wait_limit_ns;
};
constexpr unsigned long long kDefaultWaitLimitNs = 2000000000ull;

// Test flags: the kernel arms its copy-completion barrier but issues no copy,
// so its own bounded wait runs out (the host-side way of exercising the
// timeout path; nothing faults, nothing waits forever).
constexpr unsigned kTestSkipFixedCopy = 1u;  // fixed-size kernel
constexpr unsigned kTestSkipTileCopy = 2u;   // segmented tile kernel (producer warp)
constexpr unsigned kTestSkipRssCopy = 4u;    // Register Sample Sort kernel

__device__ __forceinline__ unsigned long long wait_limit_ns(const unsigned* status) {
  return reinterpret_cast<const volatile DevCtl*>(status)->wait_limit_ns;
}
__device__ __forceinline__ unsigned test_flags(const unsigned* status) {
  return reinterpret_cast<const volatile DevCtl*>(status)->test_flags;
}

// ------------------------------------------------------------ items -------

// Key + original position, ordered lexicographically: this makes every item
// distinct and gives a stable result.  For u32 keys it is packed into one u64
// (key in the high half), so one 64-bit min/max orders it.
template <class K> struct ItemOf;
template <> struct ItemOf<uint32_t> {
  using T = uint64_t;
  static __device__ __forceinline__ T make(uint32_t key, uint32_t idx) {
    return (static_cast<uint64_t>(key) << 32) | idx;
  }
  static __device__ __forceinline__ uint32_t key(T it) { return static_cast<uint32_t>(it >> 32); }
  static __device__ __forceinline__ uint32_t idx(T it) { return static_cast<uint32_t>(it); }
  static __device__ __forceinline__ T sentinel(uint32_t slot) { return make(0xFFFFFFFFu, 0x10000u + slot); }
};

struct Item64 {
  uint64_t key;
  uint32_t idx;
};
template <> struct ItemOf<uint64_t> {
  using T = Item64;
  static __device__ __forceinline__ T make(uint64_t key, uint32_t idx) { return Item64{key, idx}; }
  static __device__ __forceinline__ uint64_t key(T it) { return it.key; }
  static __device__ __forceinline__ uint32_t idx(T it) { return it.idx; }
  static __device__ __forceinline__ T sentinel(uint32_t slot) {
    return Item64{0xFFFFFFFFFFFFFFFFull, 0x10000u + slot};
  }
};

__device__ __forceinline__ bool item_less(uint32_t a, uint32_t b) { return a < b; }
__device__ __forceinline__ bool item_less(uint64_t a, uint64_t b) { return a < b; }
__device__ __forceinline__ bool item_less(const Item64& a, const Item64& b) {
  return a.key < b.key || (a.key == b.key && a.idx < b.idx);
}

// ------------------------------------------------------ compare-exchange --

__device__ __forceinline__ void ce(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b);
  b = max(a, b);
  a = lo;
}
__device__ __forceinline__ void ce(uint64_t& a, uint64_t& b) {
  const uint64_t lo = min(a, b);
  b = max(a, b);
  a = lo;
}
__device__ __forceinline__ void ce(Item64& a, Item64& b) {
  const bool swap = item_less(b, a);
  const Item64 lo{swap ? b.key : a.key, swap ? b.idx : a.idx};
  const Item64 hi{swap ? a.key : b.key, swap ? a.idx : b.idx};
  a = lo;
  b = hi;
}

// A key with its position, ordered by the key alone: the first network pass of
// the payload paths.  Equal keys may end out of position order; a check of
// adjacent items finds that, and a (key, position) pass then fixes it.
template <class K>
struct KeyIdx {
  K k;
  uint32_t ix;
};
template <class K>
__device__ __forceinline__ bool item_less(const KeyIdx<K>& a, const KeyIdx<K>& b) {
  return a.k < b.k;
}
template <class K>
__device__ __forceinline__ void ce(KeyIdx<K>& a, KeyIdx<K>& b) {
  const bool swap = b.k < a.k;
  const KeyIdx<K> lo{swap ? b.k : a.k, swap ? b.ix : a.ix};
  const KeyIdx<K> hi{swap ? a.k : b.k, swap ? a.ix : b.ix};
  a = lo;
  b = hi;
}
// Adjacent items with equal keys out of position order, where the later one
// is a real item (position below `real`): padding items share the maximum key
// and may end in any order among themselves, which does not matter.
template <class K>
__device__ __forceinline__ bool tie_misordered(const KeyIdx<K>& a, const KeyIdx<K>& b, uint32_t real) {
  return a.k == b.k && a.ix > b.ix && b.ix < real;
}

// Min/max of two items for the warp network: `keep_min` selects the result.
__device__ __forceinline__ uint32_t pick(uint32_t mine, uint32_t other, bool keep_min) {
  return keep_min ? min(mine, other) : max(mine, other);
}
__device__ __forceinline__ uint64_t pick(uint64_t mine, uint64_t other, bool keep_min) {
  return keep_min ? min(mine, other) : max(mine, other);
}
__device__ __forceinline__ Item64 pick(const Item64& mine, const Item64& other, bool keep_min) {
  // the partner's item only if strictly on the wanted side (equal items: keep mine)
  const bool take = keep_min ? item_less(other, mine) : item_less(mine, other);
  return take ? other : mine;
}
template <class K>
__device__ __forceinline__ KeyIdx<K> pick(const KeyIdx<K>& mine, const KeyIdx<K>& other, bool keep_min) {
  // by key alone; on equal keys each lane keeps its own item, so a lane
  // exchange stays a permutation
  const bool take = keep_min ? other.k < mine.k : mine.k < other.k;
  return take ? other : mine;
}

// -------------------------------------------------------- networks --------

// Order-preserving codes of IEEE-754 bit patterns held as unsigned words:
// negative values get all bits flipped, non-negative ones the sign bit set, so
// the unsigned order of the codes is the standard's totalOrder (-NaN < -inf <
// ... < -0 < +0 < ... < +inf < +NaN).  Identity for integer keys (kF false).
template <class K, bool kF>
__device__ __forceinline__ K key_enc(K x) {
  if constexpr (kF) {
    constexpr K top = static_cast<K>(1) << (8 * sizeof(K) - 1);
    return (x & top) ? static_cast<K>(~x) : static_cast<K>(x | top);
  } else {
    return x;
  }
}
template <class K, bool kF>
__device__ __forceinline__ K key_dec(K x) {
  if constexpr (kF) {
    constexpr K top = static_cast<K>(1) << (8 * sizeof(K) - 1);
    return (x & top) ? static_cast<K>(x & ~top) : static_cast<K>(~x);
  } else {
    return x;
  }
}

// Net<N>::run applies the generated N-channel network to a register array.
template <int N> struct Net;
template <> struct Net<0> {
  template <class T> __device__ __forceinline__ static void run(T*) {}
};
template <> struct Net<1> {
  template <class T> __device__ __forceinline__ static void run(T*) {}
};
#define SN_CE_(i, j) ce(k[i], k[j]);
#define SN_DEFINE_NET(n)                                          \
  template <> struct Net<n> {                                     \
    template <class T> __device__ __forceinline__ static void run(T* k) { \
      SN_NET_##n(SN_CE_)                                          \
    }                                                             \
  };
SN_DEFINE_NET(2)
SN_DEFINE_NET(3)
SN_DEFINE_NET(4)
SN_DEFINE_NET(5)
SN_DEFINE_NET(6)
SN_DEFINE_NET(7)
SN_DEFINE_NET(8)
SN_DEFINE_NET(9)
SN_DEFINE_NET(10)
SN_DEFINE_NET(11)
SN_DEFINE_NET(12)
SN_DEFINE_NET(13)
SN_DEFINE_NET(14)
SN_DEFINE_NET(15)
SN_DEFINE_NET(16)
#undef SN_DEFINE_NET

// NetBN<N>::run applies Bose and Nelson's recursively constructed N-channel
// network (the family the paper compares against the best known networks).
template <int N> struct NetBN;
#define SN_DEFINE_BN(n)                                           \
  template <> struct NetBN<n> {                                   \
    template <class T> __device__ __forceinline__ static void run(T* k) { \
      SN_BN_##n(SN_CE_)                                           \
    }                                                             \
  };
SN_DEFINE_BN(2)
SN_DEFINE_BN(3)
SN_DEFINE_BN(4)
SN_DEFINE_BN(5)
SN_DEFINE_BN(6)
SN_DEFINE_BN(7)
SN_DEFINE_BN(8)
SN_DEFINE_BN(9)
SN_DEFINE_BN(10)
SN_DEFINE_BN(11)
SN_DEFINE_BN(12)
SN_DEFINE_BN(13)
SN_DEFINE_BN(14)
SN_DEFINE_BN(15)
SN_DEFINE_BN(16)
#undef SN_DEFINE_BN
#undef SN_CE_

// ------------------------------------------------ warp shuffles -----------

__device__ __forceinline__ uint32_t shfl_xor(uint32_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ uint64_t shfl_xor(uint64_t v, int m) { return __shfl_xor_sync(0xFFFFFFFFu, v, m); }
__device__ __forceinline__ Item64 shfl_xor(const Item64& v, int m) {
  return Item64{__shfl_xor_sync(0xFFFFFFFFu, v.key, m), __shfl_xor_sync(0xFFFFFFFFu, v.idx, m)};
}
template <class K>
__device__ __forceinline__ KeyIdx<K> shfl_xor(const KeyIdx<K>& v, int m) {
  return KeyIdx<K>{shfl_xor(v.k, m), __shfl_xor_sync(0xFFFFFFFFu, v.ix, m)};
}

__device__ __forceinline__ uint32_t shfl_idx(uint32_t v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }
__device__ __forceinline__ uint64_t shfl_idx(uint64_t v, int src) { return __shfl_sync(0xFFFFFFFFu, v, src); }
__device__ __forceinline__ Item64 shfl_idx(const Item64& v, int src) {
  return Item64{__shfl_sync(0xFFFFFFFFu, v.key, src), __shfl_sync(0xFFFFFFFFu, v.idx, src)};
}
template <class K>
__device__ __forceinline__ KeyIdx<K> shfl_idx(const KeyIdx<K>& v, int src) {
  return KeyIdx<K>{shfl_idx(v.k, src), __shfl_sync(0xFFFFFFFFu, v.ix, src)};
}

// 32-lane warp network (generated schedule): lane l meets lane l ^ M at every
// step; the lower lane keeps the smaller item.
template <class T>
__device__ __forceinline__ void warp_network32(T& x, int lane) {
#define SN_WARP_STEP_(M) { const T o = shfl_xor(x, M); x = pick(x, o, lane < (lane ^ (M))); }
  SN_WARP32_SCHEDULE(SN_WARP_STEP_)
#undef SN_WARP_STEP_
}

// Two independent columns through the same network, step by step, so that
// their shuffles and compares interleave.
template <class T>
__device__ __forceinline__ void warp_network32x2(T& x, T& y, int lane) {
#define SN_WARP_STEP2_(M)                        \
  {                                              \
    const T ox = shfl_xor(x, M);                 \
    const T oy = shfl_xor(y, M);                 \
    const bool keep_min = lane < (lane ^ (M));   \
    x = pick(x, ox, keep_min);                   \
    y = pick(y, oy, keep_min);                   \
  }
  SN_WARP32_SCHEDULE(SN_WARP_STEP2_)
#undef SN_WARP_STEP2_
}

// 64 items on a warp, slot 32 r + lane in register r (lo: r = 0, hi: r = 1),
// sorted ascending: each column by the 32-lane network; then slot l meets
// slot 63 - l in one compare-exchange (so equal keys stay a permutation),
// leaving the 32 smallest as a bitonic sequence in lo and the 32 largest as
// one in hi (lane order); the half-cleaners 16, 8, 4, 2, 1 sort each.
template <class T>
__device__ __forceinline__ void warp_sort64(T& lo, T& hi, int lane) {
  warp_network32x2(lo, hi, lane);
  {
    const T y = shfl_idx(hi, 31 - lane);
    const bool sw = item_less(y, lo);
    hi = sw ? lo : y;
    lo = sw ? y : lo;
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    const bool keep_min = (lane & m) == 0;
    const T a = shfl_xor(lo, m), b = shfl_xor(hi, m);
    lo = pick(lo, a, keep_min);
    hi = pick(hi, b, keep_min);
  }
}

// Comparator `c` of the step with XOR mask `mask` of the ascending bitonic
// sorter (mask = k-1 for the mirrored first step of a merge of size k, else a
// power of two): returns the lower slot; the partner is slot ^ mask.
__device__ __forceinline__ int bitonic_slot(int c, int mask) {
  const int h = (mask & (mask + 1)) == 0 ? (mask + 1) >> 1 : mask;  // highest bit of the pair distance
  const int b = __ffs(h) - 1;
  return ((c >> b) << (b + 1)) | (c & (h - 1));
}

// ------------------------------------------------ async-proxy PTX ---------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// CTA-scope release store / acquire load / acq_rel add on shared memory.
__device__ __forceinline__ void st_release_smem(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire_smem(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t atom_add_acq_rel_smem(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v)
               : "memory");
  return old;
}

// Wait for the phase with the given parity to complete; false once the
// device's wait limit (read from the control block at `status`) has passed
// without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long limit = wait_limit_ns(status);
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit) return false;
  return true;
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes).
// dst, src and bytes must be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// 1-D bulk copy shared -> global in the current bulk group.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N bulk groups are incomplete (writes performed).
template <int N>
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Named barrier over `count` threads (multiple of 32).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

}  // namespace sn

/*
 * smallsort.h -- C ABI of the GB300 small-set sorting library (libsmallsort.so).
 *
 * Sorts huge batches of independent small integer arrays on one GPU with the
 * methods of Bingmann, Marianczuk and Sanders, "Engineering Faster Sorters for
 * Small Sets of Items": branch-free sorting networks (compare-exchange as
 * min/max, Sec. 2) for n <= 16, a 32-lane warp network for 17..32 items, and
 * Register Sample Sort (Sec. 3) for segments of up to 256 items.
 *
 * Conventions shared by every call:
 *   - Pointers named keys / vals / offsets are DEVICE pointers owned by the
 *     caller.  The library never frees them and keeps no reference after the
 *     call's stream work completes.  Elements must be naturally aligned
 *     (4 bytes for u32, 8 bytes for u64).
 *   - Every call is asynchronous on `stream` (NULL = legacy default stream).
 *     Argument errors are returned synchronously, before anything is launched.
 *     Errors found on the device (offsets, timeouts) are recorded in a
 *     per-device status word and returned by sn_check().
 *   - Sorting is ascending by unsigned key.  With payloads, equal keys keep
 *     their input order (the result is ordered by (key, original position)),
 *     so every output is unique and deterministic.
 *   - Calls are thread-safe; concurrent calls on different streams are allowed.
 */
#ifndef SMALLSORT_H
#define SMALLSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *sn_stream_t;

/* Status codes.  Every entry point returns SN_OK (0) or one of these. */
enum {
    SN_OK = 0,
    SN_EINVAL = -1,       /* null pointer with work to do, n outside 2..16   */
    SN_ERANGE = -2,       /* size overflow; segment longer than 256 or
                             offsets decreasing (device-detected)            */
    SN_ENOMEM = -3,       /* device scratch allocation failed                */
    SN_ECUDA = -4,        /* CUDA runtime / launch error                     */
    SN_ETIMEOUT = -5,     /* a bounded device-side wait ran out              */
    SN_EUNSUPPORTED = -6  /* the current device is not an sm_103 GPU          */
};

/* Longest segment the segmented calls accept. */
#define SN_MAX_SEGMENT 256

/*
 * Fixed-size arrays (Sec. 2.2.1: an entry method takes an array A and its size
 * n; Sec. 4.3 ArrayInRow: many arrays stored back to back).
 *
 * keys:  `count` contiguous arrays of `n` keys each (count*n keys), sorted
 *        ascending in place.  16-byte-aligned `keys` take the TMA-staged path;
 *        other alignments take a slower direct path, never an error.
 * n:     2..16, else SN_EINVAL.
 * count: number of arrays; 0 returns SN_OK without launching.
 *        count*n must stay below 2^62, else SN_ERANGE.
 */
int sn_sort_fixed(uint32_t *keys, int n, uint64_t count, sn_stream_t stream);
int sn_sort_fixed_u64(uint64_t *keys, int n, uint64_t count, sn_stream_t stream);

/*
 * Network families for the fixed-size calls (Sec. 2.2.1): the best known
 * networks (sizes 1, 3, 5, 9, 12, 16, 19, 25, 29, 35, 39, 45, 51, 56, 60 for
 * n = 2..16), or Bose and Nelson's recursive construction (BN-L of the paper:
 * 65 comparators at n = 16).  Both sort every input; they differ in size,
 * depth and locality only.
 */
#define SN_NETWORK_BEST 0
#define SN_NETWORK_BOSE_NELSON 1

/* sn_sort_fixed with a choice of network family (SN_EINVAL for another value). */
int sn_sort_fixed_family(uint32_t *keys, int n, uint64_t count, int family, sn_stream_t stream);

/*
 * The paper's item type (Sec. 4.1: a 64-bit key and a 64-bit reference that
 * travels with it, 16 bytes), in `count` contiguous arrays of n items
 * (array-of-structs, the ArrayInRow layout).  Each array is sorted in place
 * by key; items with equal keys keep their order in the array, so the result
 * is unique.  Same n, count and alignment rules as sn_sort_fixed (items must
 * be 8-byte aligned; 16-byte-aligned arrays take the bulk-copy path).
 */
typedef struct {
    uint64_t key;
    uint64_t ref;
} sn_item64;
int sn_sort_fixed_items(sn_item64 *items, int n, uint64_t count, int family, sn_stream_t stream);

/*
 * Floating-point keys: the same calls for IEEE-754 single and double keys,
 * ordered by the standard's totalOrder: -NaN < -inf < negative numbers < -0
 * < +0 < positive numbers < +inf < +NaN (NaNs ordered by their payload
 * bits).  Keys are sorted as their bit patterns through an order-preserving
 * code applied in registers, so the bits of every key come back unchanged.
 * Conventions as for the u32 / u64 calls (payload ties by original position).
 */
int sn_sort_fixed_f32(float *keys, int n, uint64_t count, sn_stream_t stream);
int sn_sort_fixed_f64(double *keys, int n, uint64_t count, sn_stream_t stream);
int sn_sort_segments_f32(float *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg,
                         sn_stream_t stream);
int sn_sort_segments_f64(double *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg,
                         sn_stream_t stream);

/*
 * CSR segments (the batching layer: the paper's Sec. 5 suggests bucketing
 * base cases by size and solving batches of equal size).
 *
 * offsets: nseg+1 u32 entries; segment i is keys[offsets[i] .. offsets[i+1]).
 *          Must be non-decreasing with every length <= 256.  A violation is
 *          detected on the device: the call then leaves keys and vals
 *          untouched and sn_check() reports SN_ERANGE.
 * keys:    sorted ascending within each segment, in place.
 * vals:    optional (may be NULL) u32 payload, permuted with the keys; ties
 *          are broken by original position inside the segment.
 * nseg:    0 returns SN_OK without launching; keys/offsets must be non-NULL
 *          otherwise (SN_EINVAL).
 * Routing: segments of 2..16 items use the n-item sorting network,
 *          17..32 the 32-lane warp network, 33..256 Register Sample Sort,
 *          all inside one persistent launch that bins segments by size.
 * Scratch: a few MB of stream-ordered device memory from a library-owned pool
 *          (SN_ENOMEM if that allocation fails).
 */
int sn_sort_segments(uint32_t *keys, uint32_t *vals, const uint32_t *offsets,
                     uint64_t nseg, sn_stream_t stream);
int sn_sort_segments_u64(uint64_t *keys, uint32_t *vals, const uint32_t *offsets,
                         uint64_t nseg, sn_stream_t stream);

/*
 * Same contract as sn_sort_segments, but every segment longer than 16 items
 * goes through Register Sample Sort (Sec. 3: splitters from a sorted sample,
 * branch-free classification into buckets, a network per bucket), with the
 * networks of Sec. 2 as the base case for segments and buckets of <= 16.
 */
int rss_sort_segments(uint32_t *keys, uint32_t *vals, const uint32_t *offsets,
                      uint64_t nseg, sn_stream_t stream);
int rss_sort_segments_u64(uint64_t *keys, uint32_t *vals, const uint32_t *offsets,
                          uint64_t nseg, sn_stream_t stream);

/*
 * sn_sort_segments_u64 without any allocation.  (Library addition: the paper
 * has no counterpart.)  For callers that cannot allocate device memory at the
 * time they sort -- a process that reserved its whole device budget up front,
 * a thread that must not enter the allocator (a real-time loop, a callback
 * running under the allocator's lock), a framework that only hands out buffers
 * it manages.  Same contract and results as sn_sort_segments_u64, with these
 * differences:
 *   - scratch is a fixed device array inside the library (about 1.45 MB per GPU
 *     that loads the library, kept until the process exits); no cudaMalloc,
 *     cudaFree or pool allocation happens in the call;
 *   - nseg must be at most SN_NOALLOC_MAX_SEGMENTS, else SN_ERANGE (nothing
 *     is launched);
 *   - the first call on each device does a one-time set-up on the calling
 *     thread (it looks up the device addresses of that array and of the status
 *     word, which may load the library's device code); make that first call
 *     before any stream capture on the device;
 *   - every call on a device uses the same array, and the last call's plan
 *     stays in it; calls whose work overlaps on the GPU (different streams
 *     without ordering between them) race on it and give wrong results --
 *     order such calls on one stream or with events.
 * Device-detected errors land in the status word that sn_check() reports.
 */
#define SN_NOALLOC_MAX_SEGMENTS 262144
int sn_sort_segments_u64_noalloc(uint64_t *keys, uint32_t *vals, const uint32_t *offsets,
                                 uint64_t nseg, sn_stream_t stream);

/*
 * Launch parameters of the segmented calls, and their autotuner.  (Library
 * addition: the paper's CPU sorters have no launch parameters.)  Each device
 * keeps one parameter set per key type and payload kind (u32 / u64 keys,
 * with / without payload); sn_sort_segments*, rss_sort_segments* and the
 * request server read it at every call.  Parameters change speed only, never
 * results.
 */
typedef struct {
    int tile_units;        /* segments + items per tile of the network kernel: 512..16384 (default 4096) */
    unsigned net_classes;  /* padded network sizes for 2..16-item segments: bit 0 = 2, bit 1 = 4,
                              bit 2 = 8, bit 3 = 12 channels; 16 channels always.  Bit 4: segments
                              of 33..64 items take a 64-channel warp network instead of Register
                              Sample Sort (sn_sort_segments* and the server only; the rss_* calls
                              always use Register Sample Sort).  Default 0x1F */
    int rss_two_min;       /* Register Sample Sort: segments longer than this draw a 64-item sample,
                              shorter ones 32 (16..256, default 160) */
    int tile_stages;       /* staging depth of the network kernel: 2..4 tiles in flight per block
                              (default 2); tile_stages x tile size must fit in shared memory */
    int tile_mode;         /* network kernel: 0 = warps take work items from a task ring (default),
                              1 = all warps of a block work through each staged tile together,
                              2 = one launch without binning: every warp stages windows of
                              consecutive segments (tile_units = items per window, 512..4096;
                              tile_stages = windows in flight per warp, 2..4) and sorts every
                              segment of a window itself, Register Sample Sort included */
} sn_tuning;

/* Current parameters of the current device for (key_bytes = 4 or 8, with_vals = 0 or 1). */
int sn_tuning_get(int key_bytes, int with_vals, sn_tuning *out);
/* Installs parameters (SN_EINVAL if out of range, or if tile_stages tiles of
   tile_units do not fit in shared memory for this key type, payload kind and
   tile_mode: the ring kernel packs each stage into max(6, key + payload bytes)
   per unit of tile_units + 256, e.g. at most two 8192-unit or four 4096-unit
   stages for u64 keys with payload; the synchronous kernel's fixed regions take
   more: two 8192-unit stages fit only for u32 keys without payload). */
int sn_tuning_set(int key_bytes, int with_vals, const sn_tuning *t);
/*
 * Autotuner: times sn_sort_segments on the caller's batch (device pointers,
 * same contract as sn_sort_segments / _u64 with key_bytes 4 / 8) under
 * candidate parameters -- a coordinate search over net_classes, (tile_units,
 * tile_stages) and rss_two_min with tile_mode 0, then a few window shapes
 * with tile_mode 2 (tile_mode 1 only through sn_tuning_set), best of three
 * runs each, the input restored from a device copy before every run --
 * installs the fastest set for this key type and
 * payload kind on the current device and copies it to `out` (may be NULL).
 * Synchronous: returns after the search; the batch is left sorted.
 * Needs device memory for one copy of keys and payload (SN_ENOMEM if not).
 * `best_ms`, if not NULL, receives the time of one sort with the chosen set.
 */
int sn_tune_segments(void *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg, int key_bytes,
                     sn_stream_t stream, sn_tuning *out, float *best_ms);
/* The same search timing rss_sort_segments / rss_sort_segments_u64 instead
   (same arguments, same parameter table). */
int sn_tune_rss_segments(void *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg, int key_bytes,
                         sn_stream_t stream, sn_tuning *out, float *best_ms);
/*
 * Writes every parameter set that was set or tuned in this process to a text
 * file (one line per device, key type and payload kind), and reads such a file
 * back, installing the sets of devices present.  SN_EINVAL on I/O or format
 * errors.
 */
int sn_tuning_save(const char *path);
int sn_tuning_load(const char *path);

/*
 * Tuning in one call.  If `path` names a readable file written by
 * sn_tuning_save, loads it (sn_tuning_load's result).  Otherwise runs
 * sn_tune_segments for u32 and u64 keys, each with and without payload, on a
 * built-in synthetic batch (2^20 segments, lengths geometric(0.15) capped at
 * 256, uniform keys; about 60 MB of device memory allocated and freed with
 * cudaMalloc / cudaFree, so the call synchronises the device), installs the
 * four sets on the current device and, if `path` is not NULL, writes them to
 * it with sn_tuning_save.  The file format is sn_tuning_save's text format.
 * Returns SN_OK or the first failing step's status.
 */
int sn_tune(const char *path);

/*
 * Segments longer than 256 items (library addition; the paper names merging
 * networks as the way beyond its 256-item range, Sec. 5).  Same contract as
 * sn_sort_segments / _u64, for lengths 0..SN_MAX_SEGMENT_LARGE: one thread
 * block per segment sorts the (key, position) items in shared memory with the
 * bitonic sorting network on the next power of two channels.  A length above
 * the limit or decreasing offsets are detected on the device first: keys and
 * payload stay untouched and sn_check() reports SN_ERANGE.  Meant for batches
 * of long segments; batches of segments <= 256 are faster through
 * sn_sort_segments.  Scratch: one device word from the library's pool.
 */
#define SN_MAX_SEGMENT_LARGE 4096
int sn_sort_segments_large(uint32_t *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg,
                           sn_stream_t stream);
int sn_sort_segments_large_u64(uint64_t *keys, uint32_t *vals, const uint32_t *offsets, uint64_t nseg,
                               sn_stream_t stream);

/*
 * One large array of n u32 keys sorted ascending, with this library's small
 * sorters as the base case (library addition; the paper measures its sorters
 * as base cases of Quicksort and IPS4o, Sec. 4.5 / 4.6).  One sample-sort
 * partition splits the keys into buckets of about 128 (splitters from a
 * sorted 4x oversample; keys classified as (key, position) pairs, so equal
 * keys cannot pile up in one bucket); buckets of <= 256 keys are sorted by
 * the segmented path, 257..4096 by the long-segment kernel, larger ones
 * recursively.  Scratch: about 2n * 4 bytes plus small arrays from the
 * library's pool (SN_ENOMEM if that fails).  The call synchronises `stream`
 * (bucket counts are read back) and returns when the keys are sorted.
 * n must be below 2^32 (SN_ERANGE); n <= 1 returns SN_OK.
 */
int sn_sort_large(uint32_t *keys, uint64_t n, sn_stream_t stream);

/*
 * Synchronises `stream`, then returns and clears the device status word of the
 * current device: SN_ERANGE if a segmented call met bad offsets, SN_ETIMEOUT
 * if a bounded device wait ran out, SN_ECUDA if the stream reported a CUDA
 * error, else SN_OK.  The word is shared by all calls on the device, so errors
 * of concurrent calls on other streams are reported together.
 */
int sn_check(sn_stream_t stream);

/*
 * The device-wide form of sn_check: synchronises the current device (every
 * stream), then returns and clears its status word with the same mapping as
 * sn_check; SN_ECUDA if the device or an earlier asynchronous launch reported
 * a CUDA error.  For callers that do not track which stream a failed call
 * used.
 */
int sn_get_last_cuda_error(void);

/*
 * Limit of the bounded device waits (a library safeguard; the paper's CPU
 * code has no device waits).  Every wait inside this library's kernels -- for
 * a staged copy, a work item, a free staging buffer -- gives up after `ns`
 * nanoseconds of GPU time (2 s by default), records SN_ETIMEOUT in the status
 * word and lets its kernel return, so no library kernel can spin forever.
 * Applies to the current device; `ns` in [1000, 6e10], else SN_EINVAL.
 * Synchronous (a 16-byte copy to the device); call it while no library work
 * runs on the device.  A limit shorter than a kernel's normal waits makes
 * calls fail with SN_ETIMEOUT and leaves their data partly sorted.
 */
int sn_set_wait_limit(uint64_t ns);

/* Short English description of a status code (static storage). */
const char *sn_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SMALLSORT_H */

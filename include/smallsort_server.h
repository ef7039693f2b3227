/*
 * smallsort_server.h -- request server over the segmented sort of
 * libsmallsort.so (library addition; the paper has no serving layer).
 *
 * A server owns one resident device buffer of `budget_bytes` and a few CUDA
 * streams ("slots").  Clients submit sort requests (CSR segments of u32 or u64
 * keys in HOST memory, optional u32 payload) from any thread.  A dispatcher
 * thread admits pending requests in arrival order as soon as a slot is free
 * and their device memory fits in the budget, coalesces them into one batch,
 * and runs the batch as one segmented sort: host->device copies, an offsets
 * rebase, the plan/bin/sort launches of sn_sort_segments, device->host copies
 * of the results.  Batches on different slots overlap on the GPU (the copies
 * of one with the sort of another).  A request's result is the same whether
 * it ran alone or coalesced with others: every segment is sorted on its own,
 * ascending, ties (with payload) in input order.
 *
 * Host buffers passed to sn_server_submit must stay valid and unmodified
 * until the request completes.  Pinned (page-locked) host memory makes the
 * copies asynchronous; pageable memory works but serialises the copies with
 * the host thread.
 */
#ifndef SMALLSORT_SERVER_H
#define SMALLSORT_SERVER_H

#include <stdint.h>

#include "smallsort.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sn_server sn_server;

typedef struct {
    uint64_t budget_bytes;       /* device memory for admitted requests: keys, payload, offsets and
                                    sort scratch of every batch in flight (allocated once, at create) */
    int key_bytes;               /* 4 (uint32 keys) or 8 (uint64 keys) */
    int slots;                   /* batches in flight at once, one stream each: 1..16 (0 = 4) */
    uint64_t max_batch_keys;     /* coalescing limit per batch (0 = 2^27); a larger request runs alone */
    uint64_t max_batch_segments; /* coalescing limit per batch (0 = 2^24) */
    uint32_t max_batch_requests; /* coalescing limit per batch: 1..65536 (0 = 4096) */
} sn_server_config;

typedef struct {
    uint64_t submitted;          /* accepted by sn_server_submit */
    uint64_t completed;          /* finished (successfully or not) */
    uint64_t failed;             /* finished with a CUDA error */
    uint64_t batches;            /* batches (segmented sorts) issued */
    uint64_t keys_completed;
    uint64_t segments_completed;
    uint64_t max_batch_requests_seen; /* most requests coalesced into one batch */
    uint32_t max_inflight_seen;  /* most batches on the GPU at once */
    uint32_t pad;
    uint64_t peak_device_bytes;  /* most budget bytes held at once */
    double latency_p50_us;       /* arrival -> results in host memory, completed requests */
    double latency_p99_us;
    double latency_max_us;
    double latency_mean_us;
    double span_s;               /* first arrival -> last completion */
    double keys_per_s;           /* keys_completed / span_s */
} sn_server_stats;

/*
 * Creates a server on the current device.  SN_EINVAL for a bad config,
 * SN_ENOMEM if the budget cannot be allocated, SN_EUNSUPPORTED on a device
 * other than sm_103.
 */
int sn_server_create(const sn_server_config *cfg, sn_server **out);

/*
 * Queues one request; returns at once.
 *   keys_in:   host keys (key_bytes each); segment i is keys_in[offsets[i] .. offsets[i+1]).
 *   vals_in:   optional host u32 payload with the same indexing (NULL = keys only).
 *   offsets:   host array of nseg+1 u32, non-decreasing, every length <= 256;
 *              checked here (SN_ERANGE if violated, nothing queued).
 *   keys_out:  host buffer receiving the sorted keys at the same indices
 *              (may equal keys_in); vals_out likewise (required iff vals_in).
 *   arrival_ns: arrival time on the sn_server_now_ns() clock, for latency
 *              statistics (0 = now).
 *   ticket:    receives the request id for sn_server_wait.
 * SN_ERANGE also when the request alone needs more device memory than the
 * budget.  nseg == 0 completes at once.
 */
int sn_server_submit(sn_server *srv, const void *keys_in, const uint32_t *vals_in, const uint32_t *offsets,
                     uint64_t nseg, void *keys_out, uint32_t *vals_out, int64_t arrival_ns,
                     uint64_t *ticket);

/*
 * Waits up to timeout_ns (0 = poll, negative = forever) for request `ticket`.
 * Returns its status once it has completed, and forgets the ticket: SN_OK;
 * SN_ERANGE if the device found its batch's offsets invalid; SN_ECUDA if its
 * batch failed (a CUDA error, a bounded device wait that ran out, an internal
 * check) -- every request of a batch gets the batch's status, which comes from
 * a status word of the batch's own, so failures of other batches or calls do
 * not leak into it.  SN_ETIMEOUT if it is still running; SN_EINVAL for an
 * unknown or already collected ticket (also when another thread waiting on the
 * same ticket collected it first).
 */
int sn_server_wait(sn_server *srv, uint64_t ticket, int64_t timeout_ns);

/* Waits until every submitted request has completed (tickets stay collectable). */
int sn_server_drain(sn_server *srv);

/* Copies the statistics; reset != 0 clears the counters and latency samples. */
int sn_server_stats_get(sn_server *srv, sn_server_stats *out, int reset);

/* Drains, stops the dispatcher and frees the device buffer and streams. */
int sn_server_destroy(sn_server *srv);

/* Monotonic clock of the latency statistics, in nanoseconds. */
int64_t sn_server_now_ns(void);

#ifdef __cplusplus
}
#endif

#endif /* SMALLSORT_SERVER_H */

// Request server of libsmallsort.so (declared in include/smallsort_server.h).
//
// Continuous batching over the segmented sort: client threads queue requests
// (host CSR batches); one dispatcher thread turns the head of the queue into a
// batch whenever a slot (stream) is free and the batch's device memory fits in
// the resident budget, and issues it without waiting for earlier batches:
//
//   H2D keys / payload / offsets of every request  ->  rebase kernel (request
//   offsets -> batch offsets)  ->  plan / bin / tile / RSS launches of the
//   segmented sort  ->  D2H results  ->  host callback (completion, frees).
//
// Batches on different slots overlap on the GPU.  The completion callback
// runs on CUDA's callback thread and makes no CUDA calls: it only updates the
// server state under the lock and wakes the dispatcher and the waiters.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "smallsort.h"
#include "smallsort_server.h"
#include "sn_arena.h"
#include "sn_internal.h"

namespace {

constexpr int kMaxSlots = 16;
constexpr int kRunning = 1;  // ticket state while queued or on the GPU (status codes are <= 0)
constexpr uint64_t kMaxBatchKeysLimit = 1ull << 31;

int64_t clock_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t ticket;
  const unsigned char* keys_in;
  const uint32_t* vals_in;
  const uint32_t* offsets;
  uint64_t nseg;
  unsigned char* keys_out;
  uint32_t* vals_out;
  uint32_t first;  // offsets[0]
  uint32_t nkeys;  // offsets[nseg] - offsets[0]
  int64_t arrival;
};

// One entry per request of a batch: its first segment in the batch, its
// offsets[0] and its first key in the batch.
struct RebaseEntry {
  uint64_t seg_base;
  uint32_t raw0;
  uint32_t key_base;
};
static_assert(sizeof(RebaseEntry) == 16, "table entry layout");

// Batch offsets: entry i of request r was copied verbatim from the request's
// offsets; it becomes key_base[r] + (raw - offsets_r[0]).  The final entry is
// the batch's key count.
__global__ void rebase_offsets_kernel(uint32_t* off, uint64_t total_segs, uint32_t total_keys,
                                      const RebaseEntry* tab, uint32_t nreq) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i <= total_segs; i += stride) {
    if (i == total_segs) {
      off[i] = total_keys;
      continue;
    }
    uint32_t lo = 0, hi = nreq;  // last request whose seg_base <= i
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (tab[mid].seg_base <= i)
        lo = mid;
      else
        hi = mid;
    }
    off[i] = off[i] - tab[lo].raw0 + tab[lo].key_base;
  }
}

struct BatchLayout {
  uint64_t keys_at = 0, vals_at = 0, off_at = 0, tab_at = 0, scratch_at = 0, scratch_bytes = 0, total = 0;
};

BatchLayout batch_layout(uint64_t nkeys, uint64_t nseg, uint64_t nreq, int key_bytes, bool vals,
                         const sn::SegTuning& tun) {
  using sn::RangeArena;
  BatchLayout L;
  uint64_t a = 0;
  L.keys_at = a;
  a += RangeArena::round_up(nkeys * key_bytes);
  L.vals_at = a;
  if (vals) a += RangeArena::round_up(nkeys * 4);
  L.off_at = a;
  a += RangeArena::round_up((nseg + 1) * 4);
  L.tab_at = a;
  a += RangeArena::round_up(nreq * sizeof(RebaseEntry));
  L.scratch_at = a;
  L.scratch_bytes = sn::segments_scratch_bytes(nseg, tun);
  a += RangeArena::round_up(L.scratch_bytes);
  L.total = a;
  return L;
}

// A slot's batch reports device-detected failures (bad offsets, a bounded
// wait that ran out, an internal check) through its own control block: the
// kernels of that batch get `ctl` as their status word, and the word is read
// back into `hstatus` behind the batch's results.
struct Slot {
  cudaStream_t stream = nullptr;
  RebaseEntry* htab = nullptr;  // pinned, max_batch_requests entries
  unsigned char* ctl = nullptr;  // device control block (kDevCtlBytes)
  unsigned* hstatus = nullptr;   // pinned copy of the batch's status word
  bool busy = false;
};

struct Batch;

}  // namespace

struct sn_server {
  sn_server_config cfg{};
  int device = 0;
  const sn::DeviceInfo* dev = nullptr;
  unsigned char* dbuf = nullptr;
  sn::RangeArena arena;
  int nslots = 0;
  Slot slots[kMaxSlots];
  unsigned char* dctl = nullptr;  // the slots' control blocks

  std::mutex mu;
  std::condition_variable cv_dispatch, cv_done;
  std::deque<Request> pending;
  std::unordered_map<uint64_t, int> state;  // ticket -> kRunning or final status
  uint64_t next_ticket = 1;
  uint64_t outstanding = 0;
  uint64_t completions = 0;  // batches finished (wakes an admission that waits for memory)
  int inflight = 0;
  bool stop = false;
  std::thread dispatcher;

  // statistics
  uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, keys_done = 0, segs_done = 0;
  uint64_t max_batch_reqs = 0, peak_bytes = 0;
  uint32_t max_inflight = 0;
  int64_t first_arrival = INT64_MAX, last_completion = 0;
  std::vector<int64_t> lat_ns;
};

namespace {

struct Batch {
  sn_server* srv;
  std::vector<Request> reqs;
  uint64_t arena_at;
  uint64_t nkeys, nseg;
  int slot;
  int status;
  sn::SegTuning tuning;
};

// Completion bookkeeping for a batch (lock held by the caller).
void finish_locked(sn_server* s, Batch* b, int64_t t) {
  for (const Request& r : b->reqs) {
    auto it = s->state.find(r.ticket);
    if (it != s->state.end()) it->second = b->status;
    s->lat_ns.push_back(t - r.arrival);
    s->first_arrival = std::min(s->first_arrival, r.arrival);
    ++s->completed;
    if (b->status != SN_OK) ++s->failed;
  }
  s->keys_done += b->nkeys;
  s->segs_done += b->nseg;
  s->last_completion = std::max(s->last_completion, t);
  s->outstanding -= b->reqs.size();
  s->arena.release(b->arena_at);
  s->slots[b->slot].busy = false;
  --s->inflight;
  ++s->completions;
}

void CUDART_CB batch_done(void* p) {
  Batch* b = static_cast<Batch*>(p);
  sn_server* s = b->srv;
  const int64_t t = clock_ns();
  // the batch's device status word, copied back behind its sorts; a bounded
  // device wait that ran out is a failed batch (SN_ECUDA): SN_ETIMEOUT from
  // sn_server_wait means "still running"
  int dev_status = sn::status_from_word(*s->slots[b->slot].hstatus);
  if (dev_status == SN_ETIMEOUT) dev_status = SN_ECUDA;
  if (b->status == SN_OK) b->status = dev_status;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    finish_locked(s, b, t);
  }
  s->cv_dispatch.notify_all();
  s->cv_done.notify_all();
  delete b;
}

// Enqueues the whole batch on its slot's stream (no lock held).
cudaError_t issue(sn_server* s, Batch* b, const BatchLayout& L) {
  const Slot& sl = s->slots[b->slot];
  const cudaStream_t st = sl.stream;
  const int kb = s->cfg.key_bytes;
  const bool vals = b->reqs.front().vals_in != nullptr;
  unsigned char* base = s->dbuf + b->arena_at;
  cudaError_t e = cudaSuccess;
  uint64_t kpos = 0, spos = 0;
  for (size_t i = 0; i < b->reqs.size(); ++i) {
    const Request& r = b->reqs[i];
    sl.htab[i] = RebaseEntry{spos, r.first, static_cast<uint32_t>(kpos)};
    if (r.nkeys) {
      if ((e = cudaMemcpyAsync(base + L.keys_at + kpos * kb, r.keys_in + static_cast<uint64_t>(r.first) * kb,
                               static_cast<uint64_t>(r.nkeys) * kb, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
      if (vals && (e = cudaMemcpyAsync(base + L.vals_at + kpos * 4, r.vals_in + r.first,
                                       static_cast<uint64_t>(r.nkeys) * 4, cudaMemcpyHostToDevice, st)) !=
                      cudaSuccess)
        return e;
    }
    if ((e = cudaMemcpyAsync(base + L.off_at + spos * 4, r.offsets, r.nseg * 4, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return e;
    kpos += r.nkeys;
    spos += r.nseg;
  }
  const RebaseEntry* dtab = reinterpret_cast<const RebaseEntry*>(base + L.tab_at);
  if ((e = cudaMemcpyAsync(base + L.tab_at, sl.htab, b->reqs.size() * sizeof(RebaseEntry), cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return e;
  // the batch's control block: the device's wait limit and flags, a clear status word
  if ((e = cudaMemcpyAsync(sl.ctl, s->dev->status, sn::kDevCtlBytes, cudaMemcpyDeviceToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(sl.ctl, 0, sizeof(unsigned), st)) != cudaSuccess)
    return e;
  sn::DeviceInfo di = *s->dev;
  di.status = reinterpret_cast<unsigned*>(sl.ctl);
  uint32_t* doff = reinterpret_cast<uint32_t*>(base + L.off_at);
  const uint64_t blocks = std::min<uint64_t>((spos + 1 + 255) / 256, 4ull * s->dev->sm_count);
  rebase_offsets_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(doff, spos, static_cast<uint32_t>(kpos), dtab,
                                                                      static_cast<uint32_t>(b->reqs.size()));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  uint32_t* dvals = vals ? reinterpret_cast<uint32_t*>(base + L.vals_at) : nullptr;
  if (kb == 4)
    e = sn::launch_segments_u32(reinterpret_cast<uint32_t*>(base + L.keys_at), dvals, doff, spos,
                                sn::SegMode::kNetworkWarpRss, base + L.scratch_at, L.scratch_bytes, b->tuning, st,
                                di);
  else
    e = sn::launch_segments_u64(reinterpret_cast<uint64_t*>(base + L.keys_at), dvals, doff, spos,
                                sn::SegMode::kNetworkWarpRss, base + L.scratch_at, L.scratch_bytes, b->tuning, st,
                                di);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(sl.hstatus, sl.ctl, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return e;
  kpos = 0;
  for (const Request& r : b->reqs) {
    if (r.nkeys) {
      if ((e = cudaMemcpyAsync(r.keys_out + static_cast<uint64_t>(r.first) * kb, base + L.keys_at + kpos * kb,
                               static_cast<uint64_t>(r.nkeys) * kb, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return e;
      if (vals && (e = cudaMemcpyAsync(r.vals_out + r.first, base + L.vals_at + kpos * 4,
                                       static_cast<uint64_t>(r.nkeys) * 4, cudaMemcpyDeviceToHost, st)) !=
                      cudaSuccess)
        return e;
    }
    kpos += r.nkeys;
  }
  return cudaLaunchHostFunc(st, batch_done, b);
}

int free_slot(const sn_server* s) {
  for (int i = 0; i < s->nslots; ++i)
    if (!s->slots[i].busy) return i;
  return -1;
}

void dispatch_loop(sn_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_dispatch.wait(lk, [&] { return (s->stop && s->pending.empty()) || (!s->pending.empty() && free_slot(s) >= 0); });
    if (s->pending.empty()) break;  // stop requested and nothing queued
    const int slot = free_slot(s);

    // Coalesce from the head of the queue (same payload kind, within limits).
    std::vector<Request> reqs;
    uint64_t nk = 0, ns = 0;
    const bool vals = s->pending.front().vals_in != nullptr;
    while (!s->pending.empty() && reqs.size() < s->cfg.max_batch_requests) {
      const Request& r = s->pending.front();
      if ((r.vals_in != nullptr) != vals) break;
      if (!reqs.empty() && (nk + r.nkeys > s->cfg.max_batch_keys || ns + r.nseg > s->cfg.max_batch_segments)) break;
      nk += r.nkeys;
      ns += r.nseg;
      reqs.push_back(r);
      s->pending.pop_front();
    }
    // Admission by device memory: give requests back from the tail until the
    // batch fits; if even the head does not fit, wait for a batch to finish.
    BatchLayout L;
    uint64_t at = sn::RangeArena::kFail;
    const sn::SegTuning tun = sn::current_tuning(s->device, s->cfg.key_bytes, vals);
    for (;;) {
      L = batch_layout(nk, ns, reqs.size(), s->cfg.key_bytes, vals, tun);
      at = s->arena.alloc(L.total);
      if (at != sn::RangeArena::kFail || reqs.size() == 1) break;
      nk -= reqs.back().nkeys;
      ns -= reqs.back().nseg;
      s->pending.push_front(reqs.back());
      reqs.pop_back();
    }
    if (at == sn::RangeArena::kFail) {
      s->pending.push_front(reqs.front());
      const uint64_t seen = s->completions;
      s->cv_dispatch.wait(lk, [&] { return s->completions != seen || s->inflight == 0; });
      continue;
    }
    Batch* b = new Batch{s, std::move(reqs), at, nk, ns, slot, SN_OK, tun};
    s->slots[slot].busy = true;
    ++s->inflight;
    ++s->batches;
    s->max_inflight = std::max<uint32_t>(s->max_inflight, static_cast<uint32_t>(s->inflight));
    s->max_batch_reqs = std::max<uint64_t>(s->max_batch_reqs, b->reqs.size());
    s->peak_bytes = std::max(s->peak_bytes, s->arena.used());
    lk.unlock();
    const cudaError_t e = issue(s, b, L);
    if (e != cudaSuccess) {
      // nothing of this batch will complete through the callback: wait for
      // what was enqueued, then finish it here as failed
      cudaGetLastError();
      cudaStreamSynchronize(s->slots[slot].stream);
      cudaGetLastError();
      b->status = SN_ECUDA;
      const int64_t t = clock_ns();
      lk.lock();
      finish_locked(s, b, t);
      delete b;
      s->cv_done.notify_all();
      continue;
    }
    lk.lock();
  }
}

void destroy_resources(sn_server* s) {
  for (int i = 0; i < s->nslots; ++i) {
    if (s->slots[i].stream) cudaStreamDestroy(s->slots[i].stream);
    if (s->slots[i].htab) cudaFreeHost(s->slots[i].htab);
    if (s->slots[i].hstatus) cudaFreeHost(s->slots[i].hstatus);
  }
  if (s->dctl) cudaFree(s->dctl);
  if (s->dbuf) cudaFree(s->dbuf);
}

}  // namespace

extern "C" {

int64_t sn_server_now_ns(void) { return clock_ns(); }

int sn_server_create(const sn_server_config* cfg, sn_server** out) {
  if (cfg == nullptr || out == nullptr) return SN_EINVAL;
  *out = nullptr;
  sn_server_config c = *cfg;
  if (c.key_bytes != 4 && c.key_bytes != 8) return SN_EINVAL;
  if (c.slots == 0) c.slots = 4;
  if (c.slots < 1 || c.slots > kMaxSlots) return SN_EINVAL;
  if (c.max_batch_keys == 0) c.max_batch_keys = 1ull << 27;
  if (c.max_batch_segments == 0) c.max_batch_segments = 1ull << 24;
  if (c.max_batch_requests == 0) c.max_batch_requests = 4096;
  if (c.max_batch_keys > kMaxBatchKeysLimit || c.max_batch_segments > kMaxBatchKeysLimit ||
      c.max_batch_requests > 65536 || c.budget_bytes < sn::RangeArena::kAlign)
    return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  sn_server* s = new (std::nothrow) sn_server;
  if (s == nullptr) return SN_ENOMEM;
  s->cfg = c;
  s->device = d->device;
  s->dev = d;
  if (cudaMalloc(&s->dbuf, c.budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    s->dbuf = nullptr;
    delete s;
    return SN_ENOMEM;
  }
  s->arena.reset(c.budget_bytes);
  s->nslots = c.slots;
  if (cudaMalloc(&s->dctl, kMaxSlots * sn::kDevCtlBytes) != cudaSuccess) {
    cudaGetLastError();
    s->dctl = nullptr;
    destroy_resources(s);
    delete s;
    return SN_ENOMEM;
  }
  for (int i = 0; i < c.slots; ++i) {
    s->slots[i].ctl = s->dctl + i * sn::kDevCtlBytes;
    if (cudaStreamCreateWithFlags(&s->slots[i].stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s->slots[i].htab), c.max_batch_requests * sizeof(RebaseEntry),
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(reinterpret_cast<void**>(&s->slots[i].hstatus), sizeof(unsigned), cudaHostAllocDefault) !=
            cudaSuccess) {
      cudaGetLastError();
      destroy_resources(s);
      delete s;
      return SN_ECUDA;
    }
  }
  try {
    s->dispatcher = std::thread(dispatch_loop, s);
  } catch (...) {
    destroy_resources(s);
    delete s;
    return SN_ECUDA;
  }
  *out = s;
  return SN_OK;
}

int sn_server_submit(sn_server* srv, const void* keys_in, const uint32_t* vals_in, const uint32_t* offsets,
                     uint64_t nseg, void* keys_out, uint32_t* vals_out, int64_t arrival_ns, uint64_t* ticket) {
  if (srv == nullptr || ticket == nullptr) return SN_EINVAL;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return SN_EINVAL;
  if (nseg > 0 && (keys_in == nullptr || offsets == nullptr || keys_out == nullptr)) return SN_EINVAL;
  if (nseg >= (1ull << 32)) return SN_ERANGE;
  uint32_t first = 0, nkeys = 0;
  if (nseg > 0) {
    for (uint64_t i = 0; i < nseg; ++i)
      if (offsets[i + 1] < offsets[i] || offsets[i + 1] - offsets[i] > SN_MAX_SEGMENT) return SN_ERANGE;
    first = offsets[0];
    nkeys = offsets[nseg] - offsets[0];
    sn::SegTuning worst;  // the smallest tile size needs the most scratch
    worst.tile_units = 512;
    const BatchLayout L = batch_layout(nkeys, nseg, 1, srv->cfg.key_bytes, vals_in != nullptr, worst);
    if (!srv->arena.fits_at_all(L.total)) return SN_ERANGE;
  }
  const int64_t arrival = arrival_ns ? arrival_ns : clock_ns();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->stop) return SN_EINVAL;
    const uint64_t t = srv->next_ticket++;
    *ticket = t;
    ++srv->submitted;
    if (nseg == 0) {
      srv->state[t] = SN_OK;
      ++srv->completed;
      return SN_OK;
    }
    srv->state[t] = kRunning;
    srv->pending.push_back(Request{t, static_cast<const unsigned char*>(keys_in), vals_in, offsets, nseg,
                                   static_cast<unsigned char*>(keys_out), vals_out, first, nkeys, arrival});
    ++srv->outstanding;
  }
  srv->cv_dispatch.notify_one();
  return SN_OK;
}

int sn_server_wait(sn_server* srv, uint64_t ticket, int64_t timeout_ns) {
  if (srv == nullptr) return SN_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->state.find(ticket);
  if (it == srv->state.end()) return SN_EINVAL;
  // done, or gone: another thread waiting on the same ticket collected it
  auto done = [&] {
    const auto f = srv->state.find(ticket);
    return f == srv->state.end() || f->second != kRunning;
  };
  if (timeout_ns < 0)
    srv->cv_done.wait(lk, done);
  else if (timeout_ns > 0)
    srv->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done);
  it = srv->state.find(ticket);
  if (it == srv->state.end()) return SN_EINVAL;
  if (it->second == kRunning) return SN_ETIMEOUT;
  const int st = it->second;
  srv->state.erase(it);
  return st;
}

int sn_server_drain(sn_server* srv) {
  if (srv == nullptr) return SN_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->cv_done.wait(lk, [&] { return srv->outstanding == 0; });
  return SN_OK;
}

int sn_server_stats_get(sn_server* srv, sn_server_stats* out, int reset) {
  if (srv == nullptr || out == nullptr) return SN_EINVAL;
  std::vector<int64_t> lat;
  sn_server_stats st;
  std::memset(&st, 0, sizeof(st));
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    st.submitted = srv->submitted;
    st.completed = srv->completed;
    st.failed = srv->failed;
    st.batches = srv->batches;
    st.keys_completed = srv->keys_done;
    st.segments_completed = srv->segs_done;
    st.max_batch_requests_seen = srv->max_batch_reqs;
    st.max_inflight_seen = srv->max_inflight;
    st.peak_device_bytes = srv->peak_bytes;
    if (srv->last_completion > srv->first_arrival)
      st.span_s = 1e-9 * static_cast<double>(srv->last_completion - srv->first_arrival);
    lat.swap(srv->lat_ns);
    if (!reset) srv->lat_ns = lat;
    if (reset) {
      srv->submitted = srv->completed = srv->failed = srv->batches = srv->keys_done = srv->segs_done = 0;
      srv->max_batch_reqs = 0;
      srv->max_inflight = 0;
      srv->peak_bytes = srv->arena.used();
      srv->first_arrival = INT64_MAX;
      srv->last_completion = 0;
    }
  }
  if (!lat.empty()) {
    auto pct = [&](double q) {
      const size_t k = std::min(lat.size() - 1, static_cast<size_t>(q * static_cast<double>(lat.size() - 1) + 0.5));
      std::nth_element(lat.begin(), lat.begin() + k, lat.end());
      return 1e-3 * static_cast<double>(lat[k]);
    };
    double sum = 0;
    int64_t mx = 0;
    for (int64_t v : lat) {
      sum += static_cast<double>(v);
      mx = std::max(mx, v);
    }
    st.latency_mean_us = 1e-3 * sum / static_cast<double>(lat.size());
    st.latency_max_us = 1e-3 * static_cast<double>(mx);
    st.latency_p50_us = pct(0.50);
    st.latency_p99_us = pct(0.99);
  }
  if (st.span_s > 0) st.keys_per_s = static_cast<double>(st.keys_completed) / st.span_s;
  *out = st;
  return SN_OK;
}

int sn_server_destroy(sn_server* srv) {
  if (srv == nullptr) return SN_EINVAL;
  sn_server_drain(srv);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_dispatch.notify_all();
  if (srv->dispatcher.joinable()) srv->dispatcher.join();
  for (int i = 0; i < srv->nslots; ++i) cudaStreamSynchronize(srv->slots[i].stream);
  destroy_resources(srv);
  delete srv;
  return SN_OK;
}

}  // extern "C"

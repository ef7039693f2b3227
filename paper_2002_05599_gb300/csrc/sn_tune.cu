// Launch-parameter table and autotuner of the segmented calls (declared in
// include/smallsort.h: sn_tuning_*, sn_tune_segments).
//
// The table holds one SegTuning per (device, key type, payload kind).  The
// tuner is a coordinate search: starting from the installed set (with the
// ring tile kernel, tile_mode 0) it sweeps one
// parameter at a time over its candidates with the others fixed (skipping
// tile shapes whose staging does not fit in shared memory), keeps a candidate
// only if it is more than 1% faster, and makes two passes; then it times the
// window kernel (tile_mode 2) over a few window shapes and, if that wins,
// sweeps the network classes and the sample threshold once more.  Every
// timing restores the caller's batch from a device copy, then times one
// sn_sort_segments launch sequence with CUDA events on the caller's stream;
// the best of three runs counts.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "smallsort.h"
#include "sn_internal.h"

namespace sn {
namespace {

constexpr int kDevs = 64;
std::mutex g_mu;
SegTuning g_table[kDevs][2][2];  // [device][u64 keys][payload]
bool g_touched[kDevs][2][2];

}  // namespace

bool tuning_valid(const SegTuning& t) {
  return t.tile_units >= 512 && t.tile_units <= 16384 && t.net_classes <= 0x1Fu && t.rss_two_min >= 16 &&
         t.rss_two_min <= SN_MAX_SEGMENT && t.tile_stages >= 2 && t.tile_stages <= 4 && t.tile_mode >= 0 &&
         t.tile_mode <= 2;
}

SegTuning current_tuning(int device, int key_bytes, bool vals) {
  if (device < 0 || device >= kDevs) return SegTuning{};
  std::lock_guard<std::mutex> lk(g_mu);
  return g_table[device][key_bytes == 8][vals ? 1 : 0];
}

namespace {

void install(int device, int key_bytes, bool vals, const SegTuning& t) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[device][key_bytes == 8][vals ? 1 : 0] = t;
  g_touched[device][key_bytes == 8][vals ? 1 : 0] = true;
}

sn_tuning to_c(const SegTuning& t) {
  sn_tuning c;
  c.tile_units = t.tile_units;
  c.net_classes = t.net_classes;
  c.rss_two_min = t.rss_two_min;
  c.tile_stages = t.tile_stages;
  c.tile_mode = t.tile_mode;
  return c;
}

SegTuning from_c(const sn_tuning& c) {
  SegTuning t;
  t.tile_units = c.tile_units;
  t.net_classes = c.net_classes;
  t.rss_two_min = c.rss_two_min;
  t.tile_stages = c.tile_stages;
  t.tile_mode = c.tile_mode;
  return t;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

struct DevBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() {
    if (p) {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  }
};

}  // namespace
}  // namespace sn

extern "C" {

int sn_tuning_get(int key_bytes, int with_vals, sn_tuning* out) {
  if (out == nullptr || (key_bytes != 4 && key_bytes != 8)) return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  *out = sn::to_c(sn::current_tuning(d->device, key_bytes, with_vals != 0));
  return SN_OK;
}

int sn_tuning_set(int key_bytes, int with_vals, const sn_tuning* t) {
  if (t == nullptr || (key_bytes != 4 && key_bytes != 8)) return SN_EINVAL;
  const sn::SegTuning st = sn::from_c(*t);
  if (!sn::tuning_valid(st) || !sn::tile_fits(key_bytes, with_vals != 0, st.tile_units, st.tile_stages, st.tile_mode))
    return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  sn::install(d->device, key_bytes, with_vals != 0, st);
  return SN_OK;
}

}  // extern "C"

namespace {

// The search of sn_tune_segments / sn_tune_rss_segments: `mode` is the call
// whose time is minimised (the two calls share the parameter table).
int tune(void* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, int key_bytes, sn_stream_t stream,
         sn_tuning* out, float* best_ms, sn::SegMode mode) {
  if (key_bytes != 4 && key_bytes != 8) return SN_EINVAL;
  if (nseg == 0 || keys == nullptr || offsets == nullptr) return SN_EINVAL;
  if (nseg >= (1ull << 32)) return SN_ERANGE;
  if (reinterpret_cast<uintptr_t>(keys) % key_bytes != 0 || reinterpret_cast<uintptr_t>(offsets) % 4 != 0 ||
      reinterpret_cast<uintptr_t>(vals) % 4 != 0)
    return SN_EINVAL;
  int err = SN_OK;
  const sn::DeviceInfo* d = sn::device_info(&err);
  if (d == nullptr) return err;
  const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool with_vals = vals != nullptr;

  uint32_t first = 0, last = 0;
  if (cudaMemcpyAsync(&first, offsets, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&last, offsets + nseg, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return SN_ECUDA;
  if (last < first) return SN_ERANGE;
  const uint64_t nk = last - first;
  const uint64_t key_b = nk * key_bytes, val_b = with_vals ? nk * 4 : 0;
  unsigned char* kbase = static_cast<unsigned char*>(keys) + static_cast<uint64_t>(first) * key_bytes;
  uint32_t* vbase = with_vals ? vals + first : nullptr;

  sn::SegTuning small;
  small.tile_units = 512;  // the largest scratch of any candidate
  const size_t scratch_b = sn::segments_scratch_bytes(nseg, small);
  sn::DevBuf copy, scratch;
  copy.s = scratch.s = s;
  if (cudaMallocFromPoolAsync(&copy.p, key_b + val_b + 16, d->pool, s) != cudaSuccess ||
      cudaMallocFromPoolAsync(&scratch.p, scratch_b, d->pool, s) != cudaSuccess) {
    cudaGetLastError();
    return SN_ENOMEM;
  }
  unsigned char* ck = static_cast<unsigned char*>(copy.p);
  if (cudaMemcpyAsync(ck, kbase, key_b, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return SN_ECUDA;
  if (with_vals && cudaMemcpyAsync(ck + key_b, vbase, val_b, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SN_ECUDA;
  sn::Timer tm;
  if (cudaEventCreate(&tm.a) != cudaSuccess || cudaEventCreate(&tm.b) != cudaSuccess) return SN_ECUDA;

  auto restore = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(kbase, ck, key_b, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && with_vals) e = cudaMemcpyAsync(vbase, ck + key_b, val_b, cudaMemcpyDeviceToDevice, s);
    return e;
  };
  auto run = [&](const sn::SegTuning& t) -> cudaError_t {
    return key_bytes == 4
               ? sn::launch_segments_u32(static_cast<uint32_t*>(keys), vals, offsets, nseg, mode, scratch.p,
                                         scratch_b, t, s, *d)
               : sn::launch_segments_u64(static_cast<uint64_t*>(keys), vals, offsets, nseg, mode, scratch.p,
                                         scratch_b, t, s, *d);
  };
  bool failed = false;
  auto time_of = [&](const sn::SegTuning& t) -> float {
    float best = 1e30f;
    for (int rep = 0; rep < 3 && !failed; ++rep) {
      float ms = 0;
      if (restore() != cudaSuccess || cudaEventRecord(tm.a, s) != cudaSuccess || run(t) != cudaSuccess ||
          cudaEventRecord(tm.b, s) != cudaSuccess || cudaEventSynchronize(tm.b) != cudaSuccess ||
          cudaEventElapsedTime(&ms, tm.a, tm.b) != cudaSuccess) {
        failed = true;
        break;
      }
      best = std::min(best, ms);
    }
    return best;
  };

  sn::SegTuning best = sn::current_tuning(d->device, key_bytes, with_vals);
  // The search keeps the ring tile kernel (tile_mode 0): the synchronous
  // kernel stages every tile, with tile work or not, so a batch that times
  // well with it under sn_sort_segments can be slower under rss_sort_segments,
  // which shares the parameter set; it stays available through sn_tuning_set.
  best.tile_mode = 0;
  float best_t = time_of(best);
  static const int kTiles[] = {512, 1024, 2048, 3072, 4096, 6144, 8192, 12288, 16384};
  static const int kStagesC[] = {2, 3, 4};
  static const int kTwo[] = {32, 64, 96, 128, 160, 192, 224, 256};
  for (int pass = 0; pass < 2 && !failed; ++pass) {
    for (unsigned mask = 0; mask <= 0xFu && !failed; ++mask) {  // the 2..16-item classes
      sn::SegTuning c = best;
      c.net_classes = mask | (best.net_classes & 0x10u);
      if (c.net_classes == best.net_classes) continue;
      const float t = time_of(c);
      if (t < 0.99f * best_t) best = c, best_t = t;
    }
    if (!failed) {  // 33..64 items: 64-channel warp network or Register Sample Sort
      sn::SegTuning c = best;
      c.net_classes = best.net_classes ^ 0x10u;
      const float t = time_of(c);
      if (t < 0.99f * best_t) best = c, best_t = t;
    }
    for (int tu : kTiles) {
      for (int st : kStagesC) {
        if (failed || (tu == best.tile_units && st == best.tile_stages) ||
            !sn::tile_fits(key_bytes, with_vals, tu, st, best.tile_mode))
          continue;
        sn::SegTuning c = best;
        c.tile_units = tu;
        c.tile_stages = st;
        const float t = time_of(c);
        if (t < 0.99f * best_t) best = c, best_t = t;
      }
    }
    for (int two : kTwo) {
      if (failed || two == best.rss_two_min) continue;
      sn::SegTuning c = best;
      c.rss_two_min = two;
      const float t = time_of(c);
      if (t < 0.99f * best_t) best = c, best_t = t;
    }
  }
  // The one-launch window kernel (tile_mode 2) over a few window shapes, with
  // the classes and sample threshold found above; if it wins, those two are
  // searched once more under it.
  static const int kWin[][2] = {{512, 2}, {512, 3}, {1024, 2}, {1024, 3}, {2048, 2}};
  bool window_won = false;
  for (const auto& w : kWin) {
    if (failed || !sn::tile_fits(key_bytes, with_vals, w[0], w[1], 2)) continue;
    sn::SegTuning c = best;
    c.tile_mode = 2;
    c.tile_units = w[0];
    c.tile_stages = w[1];
    const float t = time_of(c);
    if (t < 0.99f * best_t) best = c, best_t = t, window_won = true;
  }
  if (window_won) {
    for (unsigned mask = 0; mask <= 0x1Fu && !failed; ++mask) {
      sn::SegTuning c = best;
      c.net_classes = mask;
      if (c.net_classes == best.net_classes) continue;
      const float t = time_of(c);
      if (t < 0.99f * best_t) best = c, best_t = t;
    }
    for (int two : kTwo) {
      if (failed || two == best.rss_two_min) continue;
      sn::SegTuning c = best;
      c.rss_two_min = two;
      const float t = time_of(c);
      if (t < 0.99f * best_t) best = c, best_t = t;
    }
  }
  if (failed) {
    cudaGetLastError();
    return SN_ECUDA;
  }
  // leave the batch sorted with the chosen set
  if (restore() != cudaSuccess || run(best) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return SN_ECUDA;
  sn::install(d->device, key_bytes, with_vals, best);
  if (out) *out = sn::to_c(best);
  if (best_ms) *best_ms = best_t;
  return SN_OK;
}

}  // namespace

extern "C" {

int sn_tune_segments(void* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, int key_bytes,
                     sn_stream_t stream, sn_tuning* out, float* best_ms) {
  return tune(keys, vals, offsets, nseg, key_bytes, stream, out, best_ms, sn::SegMode::kNetworkWarpRss);
}

int sn_tune_rss_segments(void* keys, uint32_t* vals, const uint32_t* offsets, uint64_t nseg, int key_bytes,
                         sn_stream_t stream, sn_tuning* out, float* best_ms) {
  return tune(keys, vals, offsets, nseg, key_bytes, stream, out, best_ms, sn::SegMode::kRssOnly);
}

int sn_tuning_save(const char* path) {
  if (path == nullptr) return SN_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (f == nullptr) return SN_EINVAL;
  bool ok = std::fprintf(f, "smallsort-tuning 3\n") > 0;
  {
    std::lock_guard<std::mutex> lk(sn::g_mu);
    for (int dev = 0; dev < sn::kDevs; ++dev)
      for (int u64 = 0; u64 < 2; ++u64)
        for (int v = 0; v < 2; ++v)
          if (sn::g_touched[dev][u64][v]) {
            const sn::SegTuning& t = sn::g_table[dev][u64][v];
            ok = ok && std::fprintf(f, "%d %d %d %d %u %d %d %d\n", dev, u64 ? 8 : 4, v, t.tile_units,
                                    t.net_classes, t.rss_two_min, t.tile_stages, t.tile_mode) > 0;
          }
  }
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SN_OK : SN_EINVAL;
}

int sn_tuning_load(const char* path) {
  if (path == nullptr) return SN_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (f == nullptr) return SN_EINVAL;
  int version = 0;
  if (std::fscanf(f, "smallsort-tuning %d\n", &version) != 1 || version != 3) {
    std::fclose(f);
    return SN_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    ndev = 0;
  }
  int dev, kb, v, tu, two, st, mode;
  unsigned mask;
  int rc = SN_OK, n;
  while ((n = std::fscanf(f, "%d %d %d %d %u %d %d %d", &dev, &kb, &v, &tu, &mask, &two, &st, &mode)) == 8) {
    sn::SegTuning t;
    t.tile_units = tu;
    t.net_classes = mask;
    t.rss_two_min = two;
    t.tile_stages = st;
    t.tile_mode = mode;
    if (dev < 0 || dev >= sn::kDevs || (kb != 4 && kb != 8) || (v != 0 && v != 1) || !sn::tuning_valid(t) ||
        !sn::tile_fits(kb, v != 0, t.tile_units, t.tile_stages, t.tile_mode)) {
      rc = SN_EINVAL;
      break;
    }
    if (dev < ndev) sn::install(dev, kb, v != 0, t);
  }
  if (rc == SN_OK && n != EOF) rc = SN_EINVAL;
  std::fclose(f);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// sn_tune: load a saved parameter table, or tune every key type and payload
// kind on a built-in synthetic batch.
// ---------------------------------------------------------------------------

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): the synthetic batch's random numbers.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Tunes (key_bytes, payload) on 2^20 segments with geometric(0.15) lengths
// capped at 256 (the shape of the library's uneven-batch workload), keys
// uniform, built on the host and copied to the device.
int tune_synthetic(int key_bytes, bool with_vals) {
  constexpr uint64_t kSeg = 1ull << 20;
  uint64_t rng = 0x5EEDull + key_bytes * 2 + (with_vals ? 1 : 0);
  std::vector<uint32_t> off(kSeg + 1);
  off[0] = 0;
  for (uint64_t i = 0; i < kSeg; ++i) {
    uint32_t len = 1;  // geometric on {1, 2, ...}: P(len = k) = 0.15 * 0.85^(k-1)
    while (len < SN_MAX_SEGMENT && (splitmix(rng) >> 11) * (1.0 / 9007199254740992.0) >= 0.15) ++len;
    off[i + 1] = off[i] + len;
  }
  const uint64_t nk = off[kSeg];
  std::vector<uint64_t> keys(nk);
  for (auto& k : keys) k = splitmix(rng);
  std::vector<uint32_t> vals;
  if (with_vals) {
    vals.resize(nk);
    for (uint64_t i = 0; i < nk; ++i) vals[i] = static_cast<uint32_t>(i);
  }
  void *dk = nullptr, *dv = nullptr, *doff = nullptr;
  int rc = SN_OK;
  if (cudaMalloc(&dk, nk * key_bytes) != cudaSuccess || cudaMalloc(&doff, (kSeg + 1) * 4) != cudaSuccess ||
      (with_vals && cudaMalloc(&dv, nk * 4) != cudaSuccess)) {
    cudaGetLastError();
    rc = SN_ENOMEM;
  }
  if (rc == SN_OK) {
    bool ok = cudaMemcpy(doff, off.data(), (kSeg + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (key_bytes == 8) {
      ok = ok && cudaMemcpy(dk, keys.data(), nk * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    } else {
      std::vector<uint32_t> k32(nk);
      for (uint64_t i = 0; i < nk; ++i) k32[i] = static_cast<uint32_t>(keys[i] >> 32);
      ok = ok && cudaMemcpy(dk, k32.data(), nk * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    }
    if (with_vals) ok = ok && cudaMemcpy(dv, vals.data(), nk * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    rc = ok ? sn_tune_segments(dk, static_cast<uint32_t*>(dv), static_cast<const uint32_t*>(doff), kSeg, key_bytes,
                               nullptr, nullptr, nullptr)
            : SN_ECUDA;
  }
  if (dk) cudaFree(dk);
  if (dv) cudaFree(dv);
  if (doff) cudaFree(doff);
  return rc;
}

}  // namespace

extern "C" int sn_tune(const char* path) {
  if (path != nullptr) {
    if (FILE* f = std::fopen(path, "r")) {
      std::fclose(f);
      return sn_tuning_load(path);
    }
  }
  int err = SN_OK;
  if (sn::device_info(&err) == nullptr) return err;
  for (int kb : {4, 8})
    for (bool v : {false, true}) {
      const int rc = tune_synthetic(kb, v);
      if (rc != SN_OK) return rc;
    }
  return path != nullptr ? sn_tuning_save(path) : SN_OK;
}

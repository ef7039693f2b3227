// Randomised check of sn::RangeArena (the request server's device-memory
// allocator) against a brute-force model: a bitmap of 256-byte units where an
// allocation of u units lands at the lowest start of a maximal free run of at
// least u units (first fit over address-ordered, fully merged free ranges).
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "sn_arena.h"

namespace {

uint64_t rng_state = 0x9E3779B97F4A7C15ull;
uint64_t next_rand() {  // SplitMix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int fail(const char* what, long step) {
  std::printf("FAIL %s at step %ld\n", what, step);
  return 1;
}

}  // namespace

int main() {
  const uint64_t kUnit = sn::RangeArena::kAlign;
  for (int round = 0; round < 4; ++round) {
    const uint64_t units = 64 + 97 * round;
    sn::RangeArena a(units * kUnit + 17);  // capacity rounds down to whole units
    if (a.capacity() != units * kUnit) return fail("capacity", -1);
    std::vector<int> owner(units, -1);  // model: unit -> allocation id
    std::vector<uint64_t> live_at, live_units;
    for (long step = 0; step < 20000; ++step) {
      const bool do_alloc = live_at.empty() || (next_rand() % 100) < 55;
      if (do_alloc) {
        const uint64_t bytes = next_rand() % (units * kUnit / 6 + 1);
        const uint64_t need = bytes ? (bytes + kUnit - 1) / kUnit : 1;
        uint64_t expect = sn::RangeArena::kFail;
        for (uint64_t s = 0; s < units;) {  // maximal free runs in address order
          if (owner[s] != -1) { ++s; continue; }
          uint64_t e = s;
          while (e < units && owner[e] == -1) ++e;
          if (e - s >= need) { expect = s * kUnit; break; }
          s = e;
        }
        const uint64_t got = a.alloc(bytes);
        if (got != expect) return fail("first fit", step);
        if (got != sn::RangeArena::kFail) {
          for (uint64_t u = 0; u < need; ++u) owner[got / kUnit + u] = static_cast<int>(step);
          live_at.push_back(got);
          live_units.push_back(need);
        }
      } else {
        const size_t k = next_rand() % live_at.size();
        if (live_units[k] > 1 && a.release(live_at[k] + kUnit)) return fail("release inside a range", step);
        if (!a.release(live_at[k])) return fail("release", step);
        if (a.release(live_at[k])) return fail("double release", step);
        for (uint64_t u = 0; u < live_units[k]; ++u) owner[live_at[k] / kUnit + u] = -1;
        live_at[k] = live_at.back();
        live_units[k] = live_units.back();
        live_at.pop_back();
        live_units.pop_back();
      }
      uint64_t used = 0;
      for (int o : owner) used += o != -1 ? kUnit : 0;
      if (a.used() != used) return fail("used", step);
      if (!a.check()) return fail("invariants", step);
      if (a.live_ranges() != live_at.size()) return fail("live count", step);
    }
    while (!live_at.empty()) {
      a.release(live_at.back());
      live_at.pop_back();
    }
    if (a.used() != 0 || a.free_ranges() != 1 || a.largest_free() != units * kUnit) return fail("all freed", -2);
  }
  std::printf("ok\n");
  return 0;
}

// Device scratch of one segmented call: a plan header, the tile table, the
// per-tile class counts (16 bytes per tile), the per-tile index lists (u16
// per segment, grouped by class, Register Sample Sort entries last) and the
// segments' class bytes (one per segment, in 4-byte words aligned like the
// offsets' 16-byte groups).  Every region starts on a 256-byte boundary.
#pragma once

#include <cstddef>
#include <cstdint>

namespace sn {
namespace seg {

struct Plan {
  unsigned bad;     // offsets failed validation
  unsigned ntiles;  // tiles of the batch
  unsigned pad[14];
};

struct ScratchLayout {
  uint64_t cap;  // entries of the tile tables (an upper bound on tiles + 1)
  size_t plan_at, tile_first_at, counts_at, order_at, cls_at, total;

  static constexpr size_t up256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

  // nseg segments, tiles of E units (segments + items).  For valid offsets
  // segment s starts at unit u_s <= 257 s, so at most 257 (nseg - 1) / E + 1
  // tiles exist.
  constexpr ScratchLayout(uint64_t nseg, uint32_t E)
      : cap(nseg ? (257ull * (nseg - 1)) / E + 2 : 2),
        plan_at(0),
        tile_first_at(up256(sizeof(Plan))),
        counts_at(up256(tile_first_at + cap * 4)),
        order_at(up256(counts_at + cap * 16)),
        cls_at(up256(order_at + (nseg + 8) * 2)),
        total(up256(cls_at + nseg + 8)) {}
};

}  // namespace seg
}  // namespace sn

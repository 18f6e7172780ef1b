// Host-side packing of the tensor-core multi-RHS product (layout: uh_panel.h).
#include "uh_panel_pack.h"

#include <algorithm>
#include <cstring>
#include <functional>
#include <queue>
#include <utility>

namespace uh {
namespace {

uint32_t bits_of(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
float float_of(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
// Round to the nearest TF32 value (10 explicit mantissa bits), ties to even.
float to_tf32(float f) {
  uint32_t u = bits_of(f);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0xfffu + ((u >> 13) & 1u);
  return float_of(u & 0xffffe000u);
}
// Round to the nearest BF16 value, ties to even.
uint16_t to_bf16(float f) {
  uint32_t u = bits_of(f);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(u >> 16);
}
float bf16_value(uint16_t h) { return float_of(static_cast<uint32_t>(h) << 16); }

// Byte offset of element (row, k) of a K-major operand with 128-byte swizzle: 128-byte row
// segments of `per_seg` elements, 8-row groups of 1024 bytes, 16-byte chunk index XOR row % 8;
// segment columns of `rows` x 128 bytes.
size_t swizzled(int row, int k, int rows, int esz) {
  const int per_seg = 128 / esz;
  const int seg = k / per_seg, byte = (k % per_seg) * esz;
  return static_cast<size_t>(seg) * rows * 128 + static_cast<size_t>(row / 8) * 1024 + (row % 8) * 128 +
         (((byte / 16) ^ (row % 8)) * 16) + byte % 16;
}

// Schedule cost of an item. A CTA's time over a pass grows with the number of its items and
// hardly with their bytes (measured on GB300 with per-CTA clock stamps, N = 32768 sphere, both
// modes: about 7 us + 0.85 us per item, the spread of bytes per CTA explaining none of the rest):
// the per-item path of the MMA issuer (operand waits, then the item's MMAs) sets the pace. The
// operand-B bytes only break ties.
constexpr int64_t kItemCost = int64_t{1} << 20;
int64_t item_cost(int64_t b_bytes) { return kItemCost + b_bytes; }

}  // namespace

void PanelBuilder::pack_item(PanelItem& it, int h, const std::vector<const ColSpec*>& spec,
                             const std::vector<int64_t>& q) {
  const int n = it.n;
  // TF32: one 128-byte K segment per 32 columns; BF16: the hi and the lo plane (K <= 64).
  const size_t bytes = static_cast<size_t>(panel_tile_bytes(mode_, n, it.nrows));
  it.tile_off = static_cast<int64_t>(tiles.size());
  for (int r = 0; r < it.nruns; ++r)
    if (it.runs[r].src != kPSrcXP) it.flags |= it.runs[r].src == kPSrcZ1 ? kPItemDepZ1 : kPItemDepZ2;
  streamed_bytes += static_cast<int64_t>(bytes);
  mma_flops += int64_t{2} * 128 * n * it.nrows * (mode_ == kPanelTF32 ? 1 : 3);
  tiles.resize(tiles.size() + bytes, 0);
  unsigned char* t = tiles.data() + it.tile_off;
  for (int k = 0; k < it.nrows; ++k) {
    if (!spec[k]) continue;  // zero column
    const ColSpec& c = *spec[k];
    for (int i = 0; i < h; ++i) {
      const int64_t idx = c.rowoff ? c.rowoff[i] + q[k] * c.colstep : c.off + q[k] * c.colstep + i * c.rowstep;
      cd v = c.mat->at(idx);
      if (c.conj) v = std::conj(v);
      const float part[2] = {static_cast<float>(v.real()), static_cast<float>(v.imag())};
      for (int b = 0; b < 2; ++b) {
        const int row = 2 * i + b;
        if (mode_ == kPanelTF32) {
          const uint32_t u = bits_of(to_tf32(part[b]));
          std::memcpy(t + swizzled(row, k, n, 4), &u, 4);
        } else {
          const uint16_t hi = to_bf16(part[b]);
          const uint16_t lo = to_bf16(part[b] - bf16_value(hi));
          std::memcpy(t + swizzled(row, k, n, 2), &hi, 2);
          std::memcpy(t + static_cast<size_t>(n) * 128 + swizzled(row, k, n, 2), &lo, 2);
        }
      }
    }
  }
}

void PanelBuilder::add_chunk(int phase, int16_t kind, int64_t out, int h, const std::vector<ColSpec>& cols) {
  Chunk ch;
  ch.phase = phase;
  ch.cost = 0;
  const int16_t n = static_cast<int16_t>((2 * h + 15) / 16 * 16);
  std::vector<const ColSpec*> spec;
  std::vector<int64_t> q;
  auto fresh = [&]() {
    PanelItem it{};
    it.out = static_cast<int32_t>(out);
    it.n = n;
    it.h = static_cast<int16_t>(h);
    it.kind = kind;
    return it;
  };
  PanelItem cur = fresh();
  auto flush = [&]() {
    // K up to a multiple of the MMA's K with a run of the zero block of XP
    while (cur.nrows % kmma_) {
      cur.runs[cur.nruns++] = PanelRun{static_cast<int32_t>(zero_row_), static_cast<int16_t>(C_), kPSrcXP, 0};
      cur.nrows = static_cast<int16_t>(cur.nrows + C_);
      for (int e = 0; e < C_; ++e) {
        spec.push_back(nullptr);
        q.push_back(0);
      }
    }
    pack_item(cur, h, spec, q);
    ch.cost += item_cost(panel_tile_bytes(mode_, cur.n, cur.nrows));
    ch.items.push_back(cur);
    cur = fresh();
    spec.clear();
    q.clear();
  };
  // One block of C panel rows [p, p + C) of source src; column e comes from segment specs
  // covering p + e, or is zero. Room is kept for the zero runs that complete the MMA's K.
  const int max_data_runs = kPanelMaxRuns - kmma_ / C_ + 1;
  auto add_block = [&](int src, int64_t p, const std::vector<const ColSpec*>& seg) {
    if (cur.nrows + C_ > kPanelK) flush();
    PanelRun* last = cur.nruns ? &cur.runs[cur.nruns - 1] : nullptr;
    const bool extend = last && last->src == src && last->start + last->len == p && last->len + C_ <= 32767;
    if (!extend && cur.nruns == max_data_runs) flush();
    last = cur.nruns ? &cur.runs[cur.nruns - 1] : nullptr;
    if (last && last->src == src && last->start + last->len == p && last->len + C_ <= 32767) {
      last->len = static_cast<int16_t>(last->len + C_);
    } else {
      cur.runs[cur.nruns++] = PanelRun{static_cast<int32_t>(p), static_cast<int16_t>(C_), static_cast<int8_t>(src), 0};
    }
    for (int e = 0; e < C_; ++e) {
      const int64_t pos = p + e;
      const ColSpec* hit = nullptr;
      for (const ColSpec* c : seg)
        if (pos >= c->start && pos < c->start + c->len) {
          hit = c;
          break;
        }
      spec.push_back(hit);
      q.push_back(hit ? pos - hit->start : 0);
    }
    cur.nrows = static_cast<int16_t>(cur.nrows + C_);
  };
  // Consecutive specs that continue each other in the same panel form one segment, widened to
  // block boundaries.
  size_t k0 = 0;
  std::vector<const ColSpec*> seg;
  while (k0 < cols.size()) {
    if (cols[k0].len <= 0) {
      ++k0;
      continue;
    }
    size_t k1 = k0 + 1;
    while (k1 < cols.size() && cols[k1].len > 0 && cols[k1].src == cols[k0].src &&
           cols[k1].start == cols[k1 - 1].start + cols[k1 - 1].len)
      ++k1;
    seg.clear();
    for (size_t k = k0; k < k1; ++k) seg.push_back(&cols[k]);
    const int64_t lo = cols[k0].start, hi = cols[k1 - 1].start + cols[k1 - 1].len;
    for (int64_t p = lo / C_ * C_; p < hi; p += C_) add_block(cols[k0].src, p, seg);
    k0 = k1;
  }
  if (cur.nrows > 0 || ch.items.empty()) flush();  // a chunk without columns writes zeros
  ch.items.front().flags |= kPItemFirst;
  ch.items.back().flags |= kPItemLast;
  if (kind == kPOutZ1 || kind == kPOutZ2) ++z_chunks[kind];
  chunks_.push_back(std::move(ch));
}

const char* PanelBuilder::finalize() {
  items.clear();
  begin.assign(ncta_ + 1, 0);
  using Entry = std::pair<int64_t, int>;
  std::vector<std::vector<int>> per_cta(ncta_);
  // Phase 0 on its own (every coupling item waits until all of Z1 is written, so the CTAs start
  // phase 1 together); phases 1 and 2 together, phase 2 on the loads phase 1 left (its near
  // field does not wait for Z2, so a CTA runs the two back to back).
  std::vector<int64_t> load(ncta_, 0);
  for (int phase = 0; phase < 3; ++phase) {
    std::vector<int> ids;
    for (size_t c = 0; c < chunks_.size(); ++c)
      if (chunks_[c].phase == phase) ids.push_back(static_cast<int>(c));
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return chunks_[a].cost > chunks_[b].cost; });
    if (phase < 2) load.assign(ncta_, 0);
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    for (int b = 0; b < ncta_; ++b) pq.push({load[b], b});
    for (int c : ids) {
      auto [l, b] = pq.top();
      pq.pop();
      per_cta[b].push_back(c);
      load[b] = l + chunks_[c].cost;
      pq.push({load[b], b});
    }
  }
  for (int b = 0; b < ncta_; ++b) {
    begin[b] = static_cast<int32_t>(items.size());
    for (int c : per_cta[b]) items.insert(items.end(), chunks_[c].items.begin(), chunks_[c].items.end());
    if (items.size() > static_cast<size_t>(INT32_MAX)) return "too many work items";
  }
  begin[ncta_] = static_cast<int32_t>(items.size());
  // The CTA's operand-B ring, items placed in list order and freed in list order (the MMAs
  // consume them in order): B goes at the head, or at the ring's start when it does not fit
  // before the end (the skipped tail is held with the item); an empty ring starts over. Before
  // its copy, the item waits for the consumption of the last item that has to be freed to make
  // room, and of the item kPanelSlots before it (whose barriers it reuses): the last item freed
  // so far, since another copy worker may copy it before the copies of the items before it.
  std::vector<int> charge;
  for (int b = 0; b < ncta_; ++b) {
    const int n = begin[b + 1] - begin[b];
    PanelItem* its = items.data() + begin[b];
    charge.assign(static_cast<size_t>(n), 0);
    int head = 0, used = 0, oldest = 0;
    for (int j = 0; j < n; ++j) {
      for (; oldest <= j - kPanelSlots; ++oldest) used -= charge[oldest];
      const int sz = panel_tile_bytes(mode_, its[j].n, its[j].nrows);
      if (used == 0) head = 0;
      bool wrap = head + sz > kPanelBRing;
      while (used + (wrap ? kPanelBRing - head : 0) + sz > kPanelBRing) {
        used -= charge[oldest];
        ++oldest;
        if (used == 0) {
          head = 0;
          wrap = false;
        }
      }
      const int off = wrap ? 0 : head;
      charge[j] = (wrap ? kPanelBRing - head : 0) + sz;
      used += charge[j];
      head = off + sz;
      its[j].boff = off;
      its[j].room = oldest - 1;
    }
  }
  return nullptr;
}

const char* PanelBuilder::self_check(const int64_t src_rows[3], const int64_t out_rows[3]) const {
  for (int k = 0; k < 3; ++k)
    if (src_rows[k] % C_) return "panel height not a multiple of the block rows";
  if (zero_row_ % C_ || zero_row_ + C_ > src_rows[kPSrcXP]) return "zero block outside XP";
  {
    for (int b = 0; b < ncta_; ++b) {
      const int32_t i0 = begin[b], i1 = begin[b + 1];
      if (i0 > i1 || i1 > static_cast<int32_t>(items.size())) return "item range";
      bool open = false;
      // Every wait ends: in a CTA's list, no item reads Z1 (Z2) before its last item that
      // writes Z1 (Z2), so its own chunks of a panel never wait on the panel.
      bool read_z[2] = {false, false};
      for (int32_t j = i0; j < i1; ++j) {
        const PanelItem& it = items[j];
        if (it.kind != kPOutY && read_z[it.kind]) return "a CTA reads a panel before it has written its part";
        for (int r = 0; r < it.nruns; ++r)
          if (it.runs[r].src != kPSrcXP) read_z[it.runs[r].src - 1] = true;
        if (it.n < 16 || it.n > 2 * kPanelMaxH || it.n % 16) return "MMA N";
        if (it.h < 1 || it.h > kPanelMaxH || 2 * it.h > it.n) return "chunk height";
        if (it.nrows < 0 || it.nrows > kPanelK || it.nrows % kmma_ || it.nruns < 0 || it.nruns > kPanelMaxRuns)
          return "item size";
        const int bytes = panel_tile_bytes(mode_, it.n, it.nrows);
        if (bytes > kPanelTileMax) return "operand B size";
        if (it.tile_off < 0 || it.tile_off % 1024 || it.tile_off + static_cast<int64_t>(bytes) > static_cast<int64_t>(tiles.size()))
          return "tile outside the packed tiles or misaligned";
        // Operand B in the ring: inside it, 1024-aligned, copied only after the item whose
        // barrier slot it reuses is consumed, and disjoint from every earlier item that can still
        // hold its bytes (one consumed after this item's room is free).
        const int jj = j - i0;
        if (it.boff < 0 || it.boff % 1024 || it.boff + bytes > kPanelBRing) return "operand B outside its ring";
        if (it.room >= jj || it.room < jj - kPanelSlots || (jj >= kPanelSlots && it.room < 0))
          return "operand B room";
        for (int q = std::max(0, it.room + 1); q < jj; ++q) {
          const PanelItem& o = items[i0 + q];
          const int ob = panel_tile_bytes(mode_, o.n, o.nrows);
          if (o.boff < it.boff + bytes && it.boff < o.boff + ob) return "operand B overlaps an item in flight";
        }
        int deps = 0;
        for (int r = 0; r < it.nruns; ++r)
          if (it.runs[r].src != kPSrcXP) deps |= it.runs[r].src == kPSrcZ1 ? kPItemDepZ1 : kPItemDepZ2;
        if ((it.flags & (kPItemDepZ1 | kPItemDepZ2)) != deps) return "panel dependencies";
        int64_t rows = 0;
        for (int r = 0; r < it.nruns; ++r) {
          const PanelRun& run = it.runs[r];
          if (run.src < 0 || run.src > 2 || run.len < C_ || run.len % C_ || run.start < 0 || run.start % C_ ||
              static_cast<int64_t>(run.start) + run.len > src_rows[static_cast<int>(run.src)])
            return "run outside its panel or not whole blocks";
          rows += run.len;
        }
        if (rows != it.nrows) return "run lengths";
        if (it.kind < kPOutZ1 || it.kind > kPOutY || it.out < 0) return "chunk output";
        if (it.kind == kPOutY ? int64_t{it.out} + it.h > out_rows[it.kind]
                              : (it.out % C_ || int64_t{it.out} + (it.h + C_ - 1) / C_ * C_ > out_rows[it.kind]))
          return "chunk outside its output or misaligned";
        if ((it.flags & kPItemFirst) == open) return "chunk boundaries";
        open = !(it.flags & kPItemLast);
      }
      if (open) return "unfinished chunk";
    }
  }
  return nullptr;
}

}  // namespace uh

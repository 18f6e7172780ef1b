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

constexpr int64_t kItemOverhead = 8192;  // schedule cost of an item beyond its bytes

}  // namespace

void PanelBuilder::pack_item(PanelItem& it, int h, const std::vector<const ColSpec*>& spec,
                             const std::vector<int64_t>& q) {
  const int n = it.n;
  const size_t bytes = static_cast<size_t>(256) * n;
  it.tile_off = static_cast<int64_t>(tiles.size());
  tiles.resize(tiles.size() + bytes, 0);
  unsigned char* t = tiles.data() + it.tile_off;
  for (int k = 0; k < it.nrows; ++k) {
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
    it.out = out;
    it.n = n;
    it.h = static_cast<int16_t>(h);
    it.kind = kind;
    return it;
  };
  PanelItem cur = fresh();
  auto flush = [&]() {
    pack_item(cur, h, spec, q);
    ch.cost += 256 * static_cast<int64_t>(n) + static_cast<int64_t>(cur.nrows) * kPanelRowBytes + kItemOverhead;
    ch.items.push_back(cur);
    cur = fresh();
    spec.clear();
    q.clear();
  };
  for (const ColSpec& c : cols) {
    for (int64_t j = 0; j < c.len; ++j) {
      const int64_t row = c.start + j;
      if (cur.nrows == kPanelK) flush();
      PanelRun* last = cur.nruns ? &cur.runs[cur.nruns - 1] : nullptr;
      const bool extend = last && last->src == c.src && last->start + last->len == row && last->len < 32767;
      if (!extend && cur.nruns == kPanelMaxRuns) flush();
      last = cur.nruns ? &cur.runs[cur.nruns - 1] : nullptr;
      if (last && last->src == c.src && last->start + last->len == row && last->len < 32767) {
        last->len++;
      } else {
        cur.runs[cur.nruns++] = PanelRun{static_cast<int32_t>(row), 1, static_cast<int8_t>(c.src), 0};
      }
      spec.push_back(&c);
      q.push_back(j);
      cur.nrows++;
    }
  }
  if (cur.nrows > 0 || ch.items.empty()) flush();  // a chunk without columns writes zeros
  ch.items.front().flags |= kPItemFirst;
  ch.items.back().flags |= kPItemLast;
  chunks_.push_back(std::move(ch));
}

const char* PanelBuilder::finalize() {
  items.clear();
  begin.assign(3 * (ncta_ + 1), 0);
  using Entry = std::pair<int64_t, int>;
  for (int phase = 0; phase < 3; ++phase) {
    std::vector<int> ids;
    for (size_t c = 0; c < chunks_.size(); ++c)
      if (chunks_[c].phase == phase) ids.push_back(static_cast<int>(c));
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return chunks_[a].cost > chunks_[b].cost; });
    std::vector<std::vector<int>> per_cta(ncta_);
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    for (int b = 0; b < ncta_; ++b) pq.push({0, b});
    for (int c : ids) {
      auto [l, b] = pq.top();
      pq.pop();
      per_cta[b].push_back(c);
      pq.push({l + chunks_[c].cost, b});
    }
    for (int b = 0; b < ncta_; ++b) {
      begin[phase * (ncta_ + 1) + b] = static_cast<int32_t>(items.size());
      for (int c : per_cta[b]) items.insert(items.end(), chunks_[c].items.begin(), chunks_[c].items.end());
    }
    begin[phase * (ncta_ + 1) + ncta_] = static_cast<int32_t>(items.size());
    if (items.size() > static_cast<size_t>(INT32_MAX)) return "too many work items";
  }
  return nullptr;
}

const char* PanelBuilder::self_check(const int64_t src_rows[3], const int64_t out_rows[3]) const {
  for (int phase = 0; phase < 3; ++phase) {
    for (int b = 0; b < ncta_; ++b) {
      const int32_t i0 = begin[phase * (ncta_ + 1) + b], i1 = begin[phase * (ncta_ + 1) + b + 1];
      if (i0 > i1 || i1 > static_cast<int32_t>(items.size())) return "item range";
      bool open = false;
      for (int32_t j = i0; j < i1; ++j) {
        const PanelItem& it = items[j];
        if (it.n < 16 || it.n > 2 * kPanelMaxH || it.n % 16) return "MMA N";
        if (it.h < 1 || it.h > kPanelMaxH || 2 * it.h > it.n) return "chunk height";
        if (it.tile_off < 0 || it.tile_off % 256 || it.tile_off + 256 * static_cast<int64_t>(it.n) >
                                                       static_cast<int64_t>(tiles.size()))
          return "tile outside the packed tiles";
        if (it.nrows < 0 || it.nrows > kPanelK || it.nruns < 0 || it.nruns > kPanelMaxRuns) return "item size";
        int64_t rows = 0;
        for (int r = 0; r < it.nruns; ++r) {
          const PanelRun& run = it.runs[r];
          if (run.src < 0 || run.src > 2 || run.len < 1 || run.start < 0 ||
              static_cast<int64_t>(run.start) + run.len > src_rows[static_cast<int>(run.src)])
            return "run outside its panel";
          rows += run.len;
        }
        if (rows != it.nrows) return "run lengths";
        if (it.kind < kPOutZ1 || it.kind > kPOutY || it.out < 0 || it.out + it.h > out_rows[it.kind])
          return "chunk outside its output";
        if ((it.flags & kPItemFirst) == open) return "chunk boundaries";
        open = !(it.flags & kPItemLast);
      }
      if (open) return "unfinished chunk";
    }
  }
  return nullptr;
}

}  // namespace uh

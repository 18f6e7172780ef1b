// Host-side packing of a matvec into the streaming kernel's device program (uh_program.h).
#include "uh_program.h"

#include <algorithm>
#include <numeric>
#include <queue>
#include <utility>

namespace uh {

ProgramBuilder::ProgramBuilder(bool c128, int64_t n, int ncta)
    : c128_(c128), n_(n), ncta_(ncta), A_(c128 ? 1 : 2), eb_(c128 ? 16 : 8) {}

int ProgramBuilder::add_chunk(int kind, int64_t dst, int h, int group, int counter) {
  OutChunk c{};
  c.dst = dst;
  c.h = h;
  c.kind = static_cast<int16_t>(kind);
  c.counter = static_cast<int16_t>(counter);
  chunks.push_back(c);
  group_.push_back(group);
  base_of_.push_back(-1);
  bytes_.push_back(0);
  chunk_items_.emplace_back();
  if (counter >= 0) counter_total_[counter]++;
  return static_cast<int>(chunks.size()) - 1;
}

namespace {
// Scheduling costs of an item and of a chunk end, in bytes streamed in the same time (GB300
// traces: a CTA streams ~45 GB/s; consumers spend ~0.1 us of fixed cost per item beyond the
// streaming and ~1 us per chunk end).
constexpr int64_t kItemCost = 4096;
constexpr int64_t kChunkCost = 49152;
int counter_of_source(int src) {
  return src == kSrcXp ? kCounterPermute : src == kSrcZ1 ? kCounterForward : src == kSrcZ2 ? kCounterCoupling : -1;
}
}  // namespace

void ProgramBuilder::add_columns(int chunk, const std::vector<ColSpec>& cols, int base_chunk) {
  const int h = chunks[chunk].h;
  const int64_t hp = chunks[chunk].kind == kPermute ? A_ : std::max<int64_t>(A_, round_up(h, A_));
  // an item's tile (hp x ncols) and its inputs (ncols) share one stage buffer
  int64_t maxcols = std::min<int64_t>(kStreamMaxCols, std::min<int64_t>(kTileBytes / (hp * eb_), kStageBytes / ((hp + 1) * eb_)));
  maxcols = maxcols / A_ * A_;
  auto& out = chunk_items_[chunk];
  WorkItem cur{};
  bool open = false;
  auto start_item = [&]() {
    cur = WorkItem{};
    cur.tile_off = static_cast<int64_t>(M.size());
    cur.hp = static_cast<int32_t>(hp);
    cur.chunk = chunk;
    open = true;
  };
  auto close_item = [&]() {
    if (!open) return;
    out.push_back(cur);
    bytes_[chunk] += static_cast<int64_t>(cur.ncols) * (hp + 1) * eb_ + kItemCost;
    tile_bytes_total += static_cast<int64_t>(cur.ncols) * hp * eb_;
    input_bytes_total += static_cast<int64_t>(cur.ncols) * eb_;
    open = false;
  };
  // Consecutive specs that continue each other in the same input vector form one run (one copy),
  // padded to 16 bytes only at its two ends.
  size_t k0 = 0;
  while (k0 < cols.size()) {
    if (cols[k0].len <= 0) {
      ++k0;
      continue;
    }
    size_t k1 = k0 + 1;
    while (k1 < cols.size() && cols[k1].len > 0 && cols[k1].src == cols[k0].src &&
           cols[k1].start == cols[k1 - 1].start + cols[k1 - 1].len)
      ++k1;
    const int src = cols[k0].src;
    const int64_t lo = cols[k0].start, hi = cols[k1 - 1].start + cols[k1 - 1].len;
    const int64_t a = lo / A_ * A_;
    const int64_t b = round_up(hi, A_);
    size_t spec = k0;  // spec holding the current position
    int64_t p = a;
    while (p < b) {
      if (!open) start_item();
      const int64_t room = maxcols - cur.ncols;
      if (room <= 0 || cur.nruns == kMaxRuns) {
        close_item();
        continue;
      }
      const int64_t take = std::min(b - p, room);
      Run run{};
      run.start = static_cast<int32_t>(p);
      run.len = static_cast<int16_t>(take);
      run.src = static_cast<int8_t>(src);
      cur.runs[cur.nruns++] = run;
      const int ctr = counter_of_source(src);
      if (ctr >= 0) cur.flags |= static_cast<int16_t>(1 << (kDepShift + ctr));
      // tile columns for input positions p .. p + take - 1
      const size_t base = M.size();
      M.resize(base + static_cast<size_t>(take * hp), cd(0, 0));
      for (int64_t q = 0; q < take; ++q) {
        const int64_t pos = p + q;
        if (pos < lo || pos >= hi) continue;  // alignment padding column
        while (pos >= cols[spec].start + cols[spec].len) ++spec;
        const ColSpec& cs = cols[spec];
        cd* col = M.data() + base + static_cast<size_t>(q * hp);
        const int64_t q0 = (pos - cs.start) * cs.colstep;
        for (int i = 0; i < h; ++i) {
          const cd v = cs.mat->at(cs.rowoff ? cs.rowoff[i] + q0 : cs.off + q0 + i * cs.rowstep);
          col[i] = cs.conj ? std::conj(v) : v;
        }
      }
      cur.ncols += static_cast<int32_t>(take);
      p += take;
    }
    k0 = k1;
  }
  close_item();
  if (out.empty()) {  // no columns: one empty item writes zeros (or, for a permutation slice, runs it)
    start_item();
    close_item();
  }
  out.front().flags |= kItemFirst;
  out.back().flags |= kItemLast;
  bytes_[chunk] += kChunkCost;
  if (base_chunk >= 0) {
    for (WorkItem& it : out) {
      it.flags |= kItemBaseAll;
      it.aux = static_cast<int32_t>(chunks[base_chunk].dst);
    }
    out.back().flags |= kItemBase;
    base_of_[chunk] = base_chunk;
  }
}

void ProgramBuilder::add_scatter(int chunk, int64_t dst, int lo, int hi) {
  OutChunk& c = chunks[chunk];
  if (c.nscat == 0) c.scat0 = static_cast<int32_t>(scatter.size());
  Scatter e{};
  e.dst = static_cast<int32_t>(dst);
  e.lo = static_cast<int16_t>(lo);
  e.hi = static_cast<int16_t>(hi);
  scatter.push_back(e);
  c.nscat++;
}

const char* ProgramBuilder::finalize() {
  const int nchunk = static_cast<int>(chunks.size());
  std::vector<std::vector<int>> per_cta(ncta_);
  std::vector<int64_t> load(ncta_, 0);
  cta_of_.assign(nchunk, -1);
  using Entry = std::pair<int64_t, int>;  // (load, cta), smallest first
  for (int g = 0; g < kNumGroups; ++g) {
    std::vector<int> ids;
    for (int c = 0; c < nchunk; ++c)
      if (group_[c] == g) ids.push_back(c);
    if (g == kGroupPermute) {
      for (size_t j = 0; j < ids.size(); ++j) {
        const int b = static_cast<int>(j % ncta_);
        per_cta[b].push_back(ids[j]);
        cta_of_[ids[j]] = b;
        load[b] += bytes_[ids[j]];
      }
      continue;
    }
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return bytes_[a] > bytes_[b]; });
    for (int c : ids) {  // chunks with a base go to their base chunk's CTA
      if (base_of_[c] < 0) continue;
      const int b = cta_of_[base_of_[c]];
      per_cta[b].push_back(c);
      cta_of_[c] = b;
      load[b] += bytes_[c];
    }
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    for (int b = 0; b < ncta_; ++b) pq.push({load[b], b});
    for (int c : ids) {
      if (base_of_[c] >= 0) continue;
      auto [l, b] = pq.top();
      pq.pop();
      per_cta[b].push_back(c);
      cta_of_[c] = b;
      load[b] = l + bytes_[c];
      pq.push({load[b], b});
    }
  }
  items.clear();
  cta_begin.assign(ncta_ + 1, 0);
  for (int b = 0; b < ncta_; ++b) {
    cta_begin[b] = static_cast<int32_t>(items.size());
    for (int c : per_cta[b])
      for (WorkItem it : chunk_items_[c]) {
        it.dst = chunks[c].dst;
        it.h = chunks[c].h;
        it.kind = chunks[c].kind;
        it.counter = chunks[c].counter;
        if (chunks[c].kind == kScatterZ1 || chunks[c].kind == kScatterZ2) {
          it.aux = chunks[c].scat0;
          it.naux = chunks[c].nscat;
        }
        items.push_back(it);
      }
  }
  cta_begin[ncta_] = static_cast<int32_t>(items.size());
  if (items.size() > static_cast<size_t>(INT32_MAX)) return "too many work items";
  return nullptr;
}

const char* ProgramBuilder::self_check() const {
  const int nchunk = static_cast<int>(chunks.size());
  if (static_cast<int>(cta_begin.size()) != ncta_ + 1 || cta_begin[0] != 0 ||
      cta_begin[ncta_] != static_cast<int32_t>(items.size()))
    return "CTA item ranges";
  for (int b = 0; b < ncta_; ++b)
    if (cta_begin[b] > cta_begin[b + 1]) return "CTA item ranges not monotone";
  const int64_t msize = static_cast<int64_t>(M.size());
  std::vector<int> seen(nchunk, 0);
  for (int b = 0; b < ncta_; ++b) {
    int open_chunk = -1;
    for (int32_t k = cta_begin[b]; k < cta_begin[b + 1]; ++k) {
      const WorkItem& it = items[k];
      if (it.chunk < 0 || it.chunk >= nchunk) return "item chunk out of range";
      const OutChunk& ch = chunks[it.chunk];
      if (it.dst != ch.dst || it.h != ch.h || it.kind != ch.kind || it.counter != ch.counter)
        return "item does not carry its chunk's output fields";
      if ((ch.kind == kScatterZ1 || ch.kind == kScatterZ2) && (it.aux != ch.scat0 || it.naux != ch.nscat))
        return "item does not carry its chunk's scatter list";
      // chunk items contiguous inside one CTA, first/last marks
      if (it.flags & kItemFirst) {
        if (open_chunk >= 0 || seen[it.chunk]) return "chunk items not contiguous";
        open_chunk = it.chunk;
        seen[it.chunk] = 1;
      }
      if (open_chunk != it.chunk) return "item outside its chunk's range";
      if (it.flags & kItemLast) open_chunk = -1;
      if (it.hp < A_ || it.hp > kStreamHpMax || it.hp % A_ || (ch.kind != kPermute && it.hp < ch.h))
        return "item height";
      if (it.ncols < 0 || it.ncols > kStreamMaxCols ||
          static_cast<int64_t>(it.ncols) * it.hp * eb_ > kTileBytes ||
          static_cast<int64_t>(it.ncols) * (it.hp + 1) * eb_ > kStageBytes)
        return "item tile size";
      if (it.tile_off < 0 || (it.tile_off * eb_) % 16 || it.tile_off + static_cast<int64_t>(it.ncols) * it.hp > msize)
        return "item tile outside the packed buffer or misaligned";
      if (it.nruns < 0 || it.nruns > kMaxRuns) return "item run count";
      int64_t cols = 0;
      uint32_t deps = 0;
      for (int r = 0; r < it.nruns; ++r) {
        const Run& run = it.runs[r];
        if (run.src < 0 || run.src > 2 || run.len <= 0 || run.len % A_ || run.start < 0 || run.start % A_ ||
            run.start + static_cast<int64_t>(run.len) > src_len_[run.src])
          return "run outside its input vector or misaligned";
        deps |= 1u << counter_of_source(run.src);
        cols += run.len;
      }
      if (cols != it.ncols) return "item runs do not match its columns";
      if (((static_cast<uint32_t>(it.flags) >> kDepShift) & 7u) != deps) return "item dependency bits";
      // a group waits only on groups that every CTA runs before it
      const int dep_group[kNumCounters] = {kGroupPermute, kGroupForward, kGroupCoupling};
      for (int g = 0; g < kNumCounters; ++g)
        if (((deps >> g) & 1u) && dep_group[g] >= group_[it.chunk]) return "item waits on a later group";
      if (((it.flags & kItemBaseAll) != 0) != (base_of_[it.chunk] >= 0)) return "base flag on the wrong chunk";
      if (it.flags & kItemBase) {
        if (!(it.flags & kItemLast)) return "base on an item that does not end its chunk";
        const int bc = base_of_[it.chunk];
        if (bc < 0 || cta_of_[bc] != b || cta_of_[it.chunk] != b || chunks[bc].kind != kToZ3 ||
            chunks[bc].dst != it.aux || chunks[bc].h != ch.h || !seen[bc] || group_[bc] >= group_[it.chunk])
          return "near-field base not written earlier in the same CTA";
        if (it.aux < 0 || it.aux + static_cast<int64_t>(ch.h) > src_len_[kSrcZ3]) return "base outside z3";
      }
    }
    if (open_chunk >= 0) return "chunk not closed in its CTA";
  }
  for (int c = 0; c < nchunk; ++c) {
    if (!seen[c]) return "chunk without items";
    const OutChunk& ch = chunks[c];
    if (ch.h < 1 || ch.dst < 0) return "chunk size";
    switch (ch.kind) {
      case kToZ1:
        if (ch.dst + ch.h > src_len_[kSrcZ1]) return "chunk outside z1";
        break;
      case kToZ2:
        if (ch.dst + ch.h > src_len_[kSrcZ2]) return "chunk outside z2";
        break;
      case kToZ3:
        if (ch.dst + ch.h > src_len_[kSrcZ3]) return "chunk outside z3";
        break;
      case kToY:
        if (ch.dst + ch.h > n_) return "chunk outside y";
        break;
      case kScatterZ1:
      case kScatterZ2: {
        const int64_t len = src_len_[ch.kind == kScatterZ1 ? kSrcZ1 : kSrcZ2];
        if (ch.nscat < 1 || ch.scat0 < 0 || ch.scat0 + static_cast<int64_t>(ch.nscat) > static_cast<int64_t>(scatter.size()))
          return "scatter list";
        for (int k = 0; k < ch.nscat; ++k) {
          const Scatter& e = scatter[ch.scat0 + k];
          if (e.lo < 0 || e.hi > ch.h || e.lo >= e.hi || e.dst < 0 || e.dst + static_cast<int64_t>(e.hi - e.lo) > len)
            return "scatter entry outside its vector";
        }
        break;
      }
      case kPermute:
        if (ch.dst + ch.h > n_ || ch.dst + ch.h > src_len_[kSrcXp]) return "permutation slice outside x";
        break;
      default:
        return "chunk kind";
    }
  }
  return nullptr;
}

}  // namespace uh

// Host-side packing of a matvec into the streaming kernel's device program (uh_program.h).
#include "uh_program.h"

#include <algorithm>
#include <numeric>
#include <queue>
#include <utility>

namespace uh {

ProgramBuilder::ProgramBuilder(bool c128, int64_t n, int ncta, const PackParams& params)
    : c128_(c128), n_(n), ncta_(ncta), prm_(params), geom_(params.ctas_per_sm == 2 ? kGeomDual : kGeomOne),
      A_(c128 ? 1 : 2), eb_(c128 ? 16 : 8) {
  prm_.tile_bytes = std::min<int64_t>(prm_.tile_bytes, geom_.tile_bytes);
}

int ProgramBuilder::add_chunk(int kind, int64_t dst, int h, int group, int counter) {
  OutChunk c{};
  c.dst = dst;
  c.h = h;
  c.kind = static_cast<int16_t>(kind);
  if (kind == kToZ3) {  // a near-field partial: releases a flag of its own
    counter = kCounterFlag;
    c.flag = static_cast<int32_t>(nflags_++);
  }
  c.counter = static_cast<int16_t>(counter);
  chunks.push_back(c);
  group_.push_back(group);
  base_of_.push_back(-1);
  bytes_.push_back(0);
  chunk_items_.emplace_back();
  if (counter >= 0 && counter < kNumCounters) counter_total_[counter]++;
  return static_cast<int>(chunks.size()) - 1;
}

namespace {
// The default scheduling costs (PackParams) of an item and of a chunk end are bytes streamed in
// the same time (GB300 traces: a CTA streams ~45 GB/s; consumers spend ~0.1 us of fixed cost per
// item beyond the streaming and ~1 us per chunk end); consecutive pool chunks share a ticket up
// to pool_unit (a ticket costs the producer about 2 us of latency, hidden only behind enough
// staged work).
int counter_of_source(int src) {
  return src == kSrcXp ? kCounterPermute : src == kSrcZ1 ? kCounterForward : src == kSrcZ2 ? kCounterCoupling
       : src == kSrcZ4 ? kCounterCouplingY : -1;
}
}  // namespace

void ProgramBuilder::add_columns(int chunk, const std::vector<ColSpec>& cols, int base_chunk) {
  const int h = chunks[chunk].h;
  const int64_t hp = std::max<int64_t>(A_, round_up(h, A_));
  // an item's tile (hp x ncols) and its inputs (ncols) share one stage buffer
  int64_t maxcols = std::min<int64_t>(kStreamMaxCols, std::min<int64_t>(prm_.tile_bytes / (hp * eb_), geom_.stage_bytes / ((hp + 1) * eb_)));
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
    bytes_[chunk] += static_cast<int64_t>(cur.ncols) * (hp + 1) * eb_ + prm_.item_cost;
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
  if (out.empty()) {  // no columns: one empty item writes zeros
    start_item();
    close_item();
  }
  if (base_chunk >= 0) {
    // The near-field partial, staged after the last item's inputs (an extra item without columns
    // when the last one has no room for it).
    const int64_t hb = round_up(h, A_);
    const WorkItem& last = out.back();
    if (last.nruns == kMaxRuns || (static_cast<int64_t>(last.ncols) * (hp + 1) + hb) * eb_ > geom_.stage_bytes) {
      start_item();
      close_item();
    }
    WorkItem& it = out.back();
    Run run{};
    run.start = static_cast<int32_t>(chunks[base_chunk].dst);
    run.len = static_cast<int16_t>(hb);
    run.src = kSrcZ3;
    it.runs[it.nruns++] = run;
    it.flags |= kItemBase;
    it.aux = static_cast<int32_t>(chunks[base_chunk].dst);
    it.naux = chunks[base_chunk].flag;
    bytes_[chunk] += hb * eb_;
    input_bytes_total += hb * eb_;
    base_of_[chunk] = base_chunk;
  }
  out.front().flags |= kItemFirst;
  out.back().flags |= kItemLast;
  bytes_[chunk] += prm_.chunk_cost;
}

bool ProgramBuilder::covered_by_cta(int reader, const std::vector<int>& list, int base_pos) const {
  const uint32_t deps = static_cast<uint32_t>((chunk_items_[reader].back().flags >> kDepShift)) & ((1u << kNumCounters) - 1u);
  for (size_t k = static_cast<size_t>(base_pos) + 1; k < list.size(); ++k) {
    const int ctr = chunks[list[k]].counter;
    if (ctr >= 0 && ctr < kNumCounters && ((deps >> ctr) & 1u)) return true;
  }
  return false;
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
  pool_pos_.assign(nchunk, -1);
  std::vector<int> pool_order, order_pos(nchunk, -1);
  using Entry = std::pair<int64_t, int>;  // (load, cta), smallest first
  for (int g = 0; g < kNumGroups; ++g) {
    std::vector<int> ids;
    for (int c = 0; c < nchunk; ++c)
      if (group_[c] == g) ids.push_back(c);
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return bytes_[a] > bytes_[b]; });
    if (g >= kFirstPoolGroup) {
      // Largest first; a chunk whose near-field partial comes from the pool goes after every chunk
      // whose partial was written in the static part, in the order its partial was handed out
      // (so that it is likely complete when the chunk is taken).
      auto key = [&](int c) -> int64_t {
        const int b = base_of_[c];
        return b >= 0 && order_pos[b] >= 0 ? 1 + order_pos[b] : 0;
      };
      std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) { return key(a) < key(b); });
      for (int c : ids) {
        order_pos[c] = static_cast<int>(pool_order.size());
        pool_order.push_back(c);
      }
      continue;
    }
    std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> pq;
    for (int b = 0; b < ncta_; ++b) pq.push({load[b], b});
    for (int c : ids) {
      auto [l, b] = pq.top();
      pq.pop();
      per_cta[b].push_back(c);
      cta_of_[c] = b;
      load[b] = l + bytes_[c];
      pq.push({load[b], b});
    }
  }
  // A reader of a static near-field partial needs no flag when the partial's CTA publishes, later
  // in its list, a chunk of a group the reader waits for: that release also publishes the partial
  // (the same consumer threads stored it earlier).
  std::vector<char> covered(nchunk, 0);
  {
    std::vector<int> pos_in_cta(nchunk, -1);
    for (int b = 0; b < ncta_; ++b)
      for (size_t k = 0; k < per_cta[b].size(); ++k) pos_in_cta[per_cta[b][k]] = static_cast<int>(k);
    for (int c = 0; c < nchunk; ++c) {
      const int bc = base_of_[c];
      if (bc < 0 || cta_of_[bc] < 0) continue;
      covered[c] = covered_by_cta(c, per_cta[cta_of_[bc]], pos_in_cta[bc]);
    }
  }
  items.clear();
  auto emit = [&](int c) {
    for (WorkItem it : chunk_items_[c]) {
      it.dst = chunks[c].dst;
      it.h = chunks[c].h;
      it.kind = chunks[c].kind;
      it.counter = chunks[c].counter;
      if (is_scatter(chunks[c].kind)) {
        it.aux = chunks[c].scat0;
        it.naux = chunks[c].nscat;
      }
      if (chunks[c].counter == kCounterFlag) it.naux = chunks[c].flag;
      if ((it.flags & kItemBase) && covered[c]) it.naux = -1;
      items.push_back(it);
    }
  };
  cta_begin.assign(ncta_ + 1, 0);
  for (int b = 0; b < ncta_; ++b) {
    cta_begin[b] = static_cast<int32_t>(items.size());
    for (int c : per_cta[b]) emit(c);
  }
  cta_begin[ncta_] = static_cast<int32_t>(items.size());
  pool.clear();
  first_item_.assign(nchunk, -1);
  for (int32_t k = 0; k < cta_begin[ncta_]; ++k)
    if (items[k].flags & kItemFirst) first_item_[items[k].chunk] = k;
  for (size_t k = 0; k < pool_order.size();) {
    PoolRange r{};
    r.begin = static_cast<int32_t>(items.size());
    int64_t cost = 0;
    while (k < pool_order.size() && cost < prm_.pool_unit) {
      const int c = pool_order[k++];
      pool_pos_[c] = static_cast<int>(pool.size());
      cost += bytes_[c];
      first_item_[c] = static_cast<int32_t>(items.size());
      emit(c);
    }
    r.end = static_cast<int32_t>(items.size());
    pool.push_back(r);
  }
  if (items.size() > static_cast<size_t>(INT32_MAX)) return "too many work items";
  return nullptr;
}

const char* ProgramBuilder::self_check() const {
  const int nchunk = static_cast<int>(chunks.size());
  // the kernel permutes positions [0, perm_n) of x into xp, one slice per CTA, each CTA releasing
  // the permutation counter once
  if (perm_n_ < 0 || perm_n_ > src_len_[kSrcXp] || counter_total_[kCounterPermute] != ncta_)
    return "permutation";
  if (static_cast<int>(cta_begin.size()) != ncta_ + 1 || cta_begin[0] != 0) return "CTA item ranges";
  for (int b = 0; b < ncta_; ++b)
    if (cta_begin[b] > cta_begin[b + 1]) return "CTA item ranges not monotone";
  if (static_cast<int>(pool_pos_.size()) != nchunk || static_cast<int>(cta_of_.size()) != nchunk) return "placement";
  // Where each counter's chunks are: the latest static group, the latest pool position.
  int last_static[kNumCounters], last_pool[kNumCounters];
  for (int g = 0; g < kNumCounters; ++g) last_static[g] = last_pool[g] = -1;
  for (int c = 0; c < nchunk; ++c) {
    const int ctr = chunks[c].counter;
    if ((ctr < -1 || ctr >= kNumCounters) && ctr != kCounterFlag) return "chunk counter";
    if (ctr == kCounterPermute) return "a chunk releasing the permutation counter";
    if ((ctr == kCounterFlag) != (chunks[c].kind == kToZ3)) return "flag of a chunk that is no near-field partial";
    if (ctr == kCounterFlag && (chunks[c].flag < 0 || chunks[c].flag >= nflags_)) return "chunk flag";
    if (ctr < 0 || ctr == kCounterFlag) continue;
    if (pool_pos_[c] >= 0) last_pool[ctr] = std::max(last_pool[ctr], pool_pos_[c]);
    else last_static[ctr] = std::max(last_static[ctr], group_[c]);
  }
  const int64_t msize = static_cast<int64_t>(M.size());
  std::vector<int> seen(nchunk, 0);
  // Checks of one item of chunk list position `pos` (a static CTA: -1, the pool: its ticket).
  auto check_item = [&](const WorkItem& it, int pos) -> const char* {
    if (it.chunk < 0 || it.chunk >= nchunk) return "item chunk out of range";
    const OutChunk& ch = chunks[it.chunk];
    if (it.dst != ch.dst || it.h != ch.h || it.kind != ch.kind || it.counter != ch.counter)
      return "item does not carry its chunk's output fields";
    if (is_scatter(ch.kind) && (it.aux != ch.scat0 || it.naux != ch.nscat))
      return "item does not carry its chunk's scatter list";
    if (it.hp < A_ || it.hp > (ch.kind == kScatterZ4 ? kStreamHpTall : kStreamHpMax) || it.hp % A_ || it.hp < ch.h)
      return "item height";
    if (it.nruns < 0 || it.nruns > kMaxRuns) return "item run count";
    const bool has_base = (it.flags & kItemBase) != 0;
    if (has_base && (!(it.flags & kItemLast) || it.nruns < 1)) return "base on an item that does not end its chunk";
    if (ch.counter == kCounterFlag && it.naux != ch.flag) return "item does not carry its chunk's flag";
    int64_t cols = 0, staged = 0;
    uint32_t deps = 0;
    for (int r = 0; r < it.nruns; ++r) {
      const Run& run = it.runs[r];
      if (has_base && r == it.nruns - 1) {
        const int bc = base_of_[it.chunk];
        if (bc < 0 || chunks[bc].kind != kToZ3 || chunks[bc].h != ch.h ||
            run.src != kSrcZ3 || run.start != chunks[bc].dst || it.aux != run.start || run.len != round_up(ch.h, A_))
          return "near-field base run";
        if (it.naux != chunks[bc].flag) {
          // no flag: the base's CTA must publish a group this item waits for after the base
          if (it.naux != -1 || cta_of_[bc] < 0) return "near-field base flag";
          const int b = cta_of_[bc];
          bool after = false, cov = false;
          for (int32_t k = cta_begin[b]; k < cta_begin[b + 1]; ++k) {
            const WorkItem& o = items[k];
            if (o.chunk == bc && (o.flags & kItemLast)) after = true;
            else if (after && (o.flags & kItemLast) && o.counter >= 0 && o.counter < kNumCounters &&
                     ((it.flags >> (kDepShift + o.counter)) & 1))
              cov = true;
          }
          if (!cov) return "near-field base neither flagged nor published by a later group";
        }
        // the flag's chunk is static, or handed out before this one (or earlier by the same
        // ticket: the same consumers finish it first); static chunks wait on no flag
        if (pos < 0 || pool_pos_[bc] > pos) return "near-field base handed out after its reader";
        if (pool_pos_[bc] == pos && first_item_[bc] > first_item_[it.chunk]) return "near-field base after its reader";
        if (run.start < 0 || run.start + static_cast<int64_t>(run.len) > src_len_[kSrcZ3]) return "base outside z3";
      } else {
        if (run.src < 0 || run.src >= kNumSources || run.src == kSrcZ3 || run.len <= 0 || run.len % A_ || run.start < 0 || run.start % A_ ||
            run.start + static_cast<int64_t>(run.len) > src_len_[run.src])
          return "run outside its input vector or misaligned";
        cols += run.len;
      }
      if (counter_of_source(run.src) >= 0) deps |= 1u << counter_of_source(run.src);
      staged += run.len;
    }
    if (cols != it.ncols) return "item runs do not match its columns";
    if (it.ncols < 0 || it.ncols > kStreamMaxCols || static_cast<int64_t>(it.ncols) * it.hp * eb_ > geom_.tile_bytes ||
        (static_cast<int64_t>(it.ncols) * it.hp + staged) * eb_ > geom_.stage_bytes)
      return "item tile size";
    // the extended-precision variant stages the same complex64 tile with 16-byte inputs
    if (eb_ == 8 && static_cast<int64_t>(it.ncols) * it.hp * 8 + staged * 16 > geom_.stage_bytes_mixed)
      return "item tile size (extended-precision stage)";
    if (it.tile_off < 0 || (it.tile_off * eb_) % 16 || it.tile_off + static_cast<int64_t>(it.ncols) * it.hp > msize)
      return "item tile outside the packed buffer or misaligned";
    if (((static_cast<uint32_t>(it.flags) >> kDepShift) & ((1u << kNumCounters) - 1u)) != deps ||
        (static_cast<uint32_t>(it.flags) >> (kDepShift + kNumCounters)) != 0)
      return "item dependency bits";
    // every wait ends: static items wait on static groups run earlier in every CTA; pool items on
    // those and on chunks handed out before them
    for (int g = 0; g < kNumCounters; ++g) {
      if (!((deps >> g) & 1u)) continue;
      if (pos < 0 ? (last_pool[g] >= 0 || last_static[g] >= group_[it.chunk]) : last_pool[g] >= pos)
        return "item waits on a later group";
    }
    return nullptr;
  };
  // static lists
  for (int b = 0; b < ncta_; ++b) {
    int open_chunk = -1;
    for (int32_t k = cta_begin[b]; k < cta_begin[b + 1]; ++k) {
      const WorkItem& it = items[k];
      if (const char* e = check_item(it, -1)) return e;
      if (pool_pos_[it.chunk] >= 0 || cta_of_[it.chunk] != b) return "static item of a chunk placed elsewhere";
      if (it.flags & kItemFirst) {
        if (open_chunk >= 0 || seen[it.chunk]) return "chunk items not contiguous";
        open_chunk = it.chunk;
        seen[it.chunk] = 1;
      }
      if (open_chunk != it.chunk) return "item outside its chunk's range";
      if (it.flags & kItemLast) open_chunk = -1;
    }
    if (open_chunk >= 0) return "chunk not closed in its CTA";
  }
  // pool: consecutive ranges after the static items, each one or more whole chunks
  int32_t at = cta_begin[ncta_];
  for (size_t t = 0; t < pool.size(); ++t) {
    const PoolRange& r = pool[t];
    if (r.begin != at || r.end <= r.begin) return "pool ranges";
    at = r.end;
    int open_chunk = -1;
    for (int32_t k = r.begin; k < r.end; ++k) {
      const WorkItem& it = items[k];
      if (it.chunk < 0 || it.chunk >= nchunk || pool_pos_[it.chunk] != static_cast<int>(t)) return "pool chunk";
      if (const char* e = check_item(it, static_cast<int>(t))) return e;
      if (it.flags & kItemFirst) {
        if (open_chunk >= 0 || seen[it.chunk]) return "pool chunk items not contiguous";
        open_chunk = it.chunk;
        seen[it.chunk] = 1;
      }
      if (open_chunk != it.chunk) return "item outside its pool chunk";
      if (it.flags & kItemLast) open_chunk = -1;
    }
    if (open_chunk >= 0) return "pool chunk not closed in its range";
  }
  if (at != static_cast<int32_t>(items.size())) return "items after the pool";
  for (int c = 0; c < nchunk; ++c) {
    if (!seen[c]) return "chunk without items";
    const OutChunk& ch = chunks[c];
    if (ch.h < 1 || ch.dst < 0) return "chunk size";
    if ((base_of_[c] >= 0) != ((chunk_items_[c].back().flags & kItemBase) != 0)) return "base flag on the wrong chunk";
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
      case kScatterZ2:
      case kScatterZ4: {
        const int64_t len = src_len_[ch.kind == kScatterZ1 ? kSrcZ1 : ch.kind == kScatterZ2 ? kSrcZ2 : kSrcZ4];
        if (ch.nscat < 1 || ch.scat0 < 0 || ch.scat0 + static_cast<int64_t>(ch.nscat) > static_cast<int64_t>(scatter.size()))
          return "scatter list";
        for (int k = 0; k < ch.nscat; ++k) {
          const Scatter& e = scatter[ch.scat0 + k];
          if (e.lo < 0 || e.hi > ch.h || e.lo >= e.hi || e.dst < 0 || e.dst + static_cast<int64_t>(e.hi - e.lo) > len)
            return "scatter entry outside its vector";
        }
        break;
      }
      default:
        return "chunk kind";
    }
  }
  return nullptr;
}

}  // namespace uh

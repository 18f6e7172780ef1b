// Host-side packing of a matvec into the streaming kernel's device program (uh_stream.h).
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

#include "uh_stream.h"

namespace uh {

using cd = std::complex<double>;

// Complex source array of either element type, read as complex<double>.
struct Src {
  const void* p = nullptr;
  int type = 0;  // 0: complex128, 1: complex64
  cd at(int64_t i) const {
    if (type == 0) return static_cast<const cd*>(p)[i];
    const std::complex<float> f = static_cast<const std::complex<float>*>(p)[i];
    return cd(f.real(), f.imag());
  }
};

// Consecutive input positions [start, start + len) of vector `src`; tile column q (for input
// position start + q) holds rows i = 0..h-1 of mat[off + q * colstep + i * rowstep], or, with a
// row offset table, mat[rowoff[i] + q * colstep] (conjugated if conj).
struct ColSpec {
  int src;
  int64_t start, len;
  const Src* mat;
  bool conj;
  int64_t off, colstep, rowstep;
  const int64_t* rowoff = nullptr;
};

// Schedule groups. The first six are static (a list per CTA, in this group order; the permutation
// group has no chunks: every CTA permutes a slice of x at entry); the last two form the pool, in
// this order, handed out by ticket. An item only waits on counters whose
// chunks are static and in earlier groups, or earlier in the pool.
enum Group { kGroupPermute = 0, kGroupForward = 1, kGroupNearA = 2, kGroupCouplingY = 3, kGroupNearA2 = 4,
             kGroupCoupling = 5, kGroupNearB = 6, kGroupBackward = 7, kNumGroups = 8 };
constexpr int kFirstPoolGroup = kGroupNearB;

// Packing and scheduling parameters (the defaults were chosen by sweeps on the N = 32768 sphere):
// the largest tile of an item (capped by the geometry's), the schedule's cost of an item and of a
// chunk end in bytes streamed in the same time, the cost that consecutive pool chunks share a
// ticket up to, and the CTAs per SM (1: kGeomOne, 2: kGeomDual; 0 = automatic,
// resolved by the caller before packing).
struct PackParams {
  int64_t tile_bytes = kTileBytes;
  int64_t item_cost = 4096;
  int64_t chunk_cost = 49152;
  int64_t pool_unit = 131072;
  int64_t ctas_per_sm = 0;
};

class ProgramBuilder {
 public:
  ProgramBuilder(bool c128, int64_t n, int ncta, const PackParams& params = PackParams());

  int64_t align() const { return A_; }
  const StreamGeometry& geometry() const { return geom_; }
  static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

  // Input vector lengths (elements, multiples of align()).
  void set_source_len(int src, int64_t len) { src_len_[src] = len; }

  // x in cluster order: the kernel permutes positions [0, n) into xp at entry, one slice per CTA,
  // and every CTA releases the permutation counter once.
  void set_permutation(int64_t n) {
    perm_n_ = n;
    counter_total_[kCounterPermute] = ncta_;
  }
  int64_t permutation_length() const { return perm_n_; }

  // counter: the group counter the chunk's completion is added to (kCounter*), or -1. A kToZ3
  // chunk (a near-field partial) releases a flag of its own instead.
  int add_chunk(int kind, int64_t dst, int h, int group, int counter = -1);
  // The columns of one chunk, in order. base_chunk >= 0: the chunk adds the outputs of that
  // (near-field, kToZ3) chunk, staged as an extra run of its last item.
  void add_columns(int chunk, const std::vector<ColSpec>& cols, int base_chunk = -1);

  // Scatter kinds: outputs lo <= r < hi of `chunk` also go to z[dst + r - lo].
  void add_scatter(int chunk, int64_t dst, int lo, int hi);

  // Assign the static chunks to CTAs (groups in order, longest processing time first within a
  // group), order the pool (each pool group largest first) and lay the items out: static by CTA,
  // then the pool.
  const char* finalize();
  // Checks every address the kernel derives from the program. Returns nullptr if all hold.
  const char* self_check() const;
  // Chunks feeding each group counter (the kernel waits for epoch * count).
  int64_t counter_total(int c) const { return counter_total_[c]; }
  // Flags released by near-field partials (each once per call).
  int64_t flag_count() const { return nflags_; }

  // Results.
  std::vector<WorkItem> items;        // by CTA
  std::vector<int32_t> cta_begin;     // ncta + 1 (static items)
  std::vector<PoolRange> pool;        // pool tickets in order: each one or more whole chunks (items
                                      // after the static ones)
  std::vector<OutChunk> chunks;
  std::vector<cd> M;                  // packed tiles (converted to the element type at upload)
  std::vector<Scatter> scatter;       // scatter entries
  int64_t src_len_[kNumSources] = {};
  int64_t tile_bytes_total = 0, input_bytes_total = 0;

 private:
  bool c128_;
  int64_t n_;
  int ncta_;
  PackParams prm_;
  StreamGeometry geom_;
  int64_t A_;   // elements per 16 bytes
  int eb_;      // bytes per element
  std::vector<int> group_, base_of_, cta_of_, pool_pos_;
  std::vector<int32_t> first_item_;  // index of each chunk's first item
  std::vector<int64_t> bytes_;
  std::vector<std::vector<WorkItem>> chunk_items_;
  int64_t counter_total_[kNumCounters] = {0, 0, 0};
  // Whether `reader` (which adds the partial of the static chunk at base_pos in a CTA's list) is
  // covered by a later chunk of that list publishing a group the reader's last item waits for.
  bool covered_by_cta(int reader, const std::vector<int>& list, int base_pos) const;
  int64_t nflags_ = 0;
  int64_t perm_n_ = -1;
};

}  // namespace uh

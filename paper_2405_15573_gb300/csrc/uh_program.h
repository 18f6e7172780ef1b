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

// Schedule groups, in the order every CTA runs them. Flags only point to earlier groups.
enum Group { kGroupPermute = 0, kGroupForward = 1, kGroupNearA = 2, kGroupCoupling = 3, kGroupNearB = 4,
             kGroupBackward = 5, kNumGroups = 6 };

class ProgramBuilder {
 public:
  ProgramBuilder(bool c128, int64_t n, int ncta);

  int64_t align() const { return A_; }
  static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

  // Input vector lengths (elements, multiples of align()).
  void set_source_len(int src, int64_t len) { src_len_[src] = len; }

  // counter: the group counter the chunk's completion is added to (kCounter*), or -1.
  int add_chunk(int kind, int64_t dst, int h, int group, int counter = -1);
  // The columns of one chunk, in order. base_chunk >= 0: the chunk adds the outputs of that
  // (near-field, kToZ3) chunk, which is placed in the same CTA ahead of it.
  void add_columns(int chunk, const std::vector<ColSpec>& cols, int base_chunk = -1);

  // Scatter kinds: outputs lo <= r < hi of `chunk` also go to z[dst + r - lo].
  void add_scatter(int chunk, int64_t dst, int lo, int hi);

  // Assign chunks to CTAs (phase groups in order, longest processing time first within a group;
  // a chunk with a base goes to its base chunk's CTA) and lay the items out by CTA.
  const char* finalize();
  // Checks every address the kernel derives from the program. Returns nullptr if all hold.
  const char* self_check() const;
  // Chunks feeding each group counter (the kernel waits for epoch * count).
  int64_t counter_total(int c) const { return counter_total_[c]; }

  // Results.
  std::vector<WorkItem> items;        // by CTA
  std::vector<int32_t> cta_begin;     // ncta + 1
  std::vector<OutChunk> chunks;
  std::vector<cd> M;                  // packed tiles (converted to the element type at upload)
  std::vector<Scatter> scatter;       // scatter entries
  int64_t src_len_[4] = {0, 0, 0, 0};
  int64_t tile_bytes_total = 0, input_bytes_total = 0;

 private:
  bool c128_;
  int64_t n_;
  int ncta_;
  int64_t A_;   // elements per 16 bytes
  int eb_;      // bytes per element
  std::vector<int> group_, base_of_, cta_of_;
  std::vector<int64_t> bytes_;
  std::vector<std::vector<WorkItem>> chunk_items_;
  int64_t counter_total_[kNumCounters] = {0, 0, 0};
};

}  // namespace uh

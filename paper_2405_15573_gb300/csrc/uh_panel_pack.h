// Host-side packing of the tensor-core multi-RHS product into its device program (uh_panel.h).
#pragma once

#include <cstdint>
#include <vector>

#include "uh_panel.h"
#include "uh_program.h"

namespace uh {

class PanelBuilder {
 public:
  PanelBuilder(int mode, int ncta) : mode_(mode), ncta_(ncta) {}

  // One output chunk of phase `phase` (0: forward transform, 1: coupling, 2: near field and
  // backward transform): h <= kPanelMaxH outputs starting at row `out` of the kind's output; its
  // columns, in order, are `cols` (ColSpec sources are kPSrc* panels, positions are panel rows).
  void add_chunk(int phase, int16_t kind, int64_t out, int h, const std::vector<ColSpec>& cols);

  // Assign the chunks of each phase to CTAs (longest processing time first) and lay the items
  // out by phase and CTA.
  const char* finalize();
  // Checks every address the kernel derives from the program against the panel heights
  // (src_rows: rows of XP, Z1, Z2) and the output heights (out_rows: Z1, Z2, Y).
  const char* self_check(const int64_t src_rows[3], const int64_t out_rows[3]) const;

  std::vector<PanelItem> items;    // by phase, then CTA
  std::vector<int32_t> begin;      // [3][ncta + 1]
  std::vector<unsigned char> tiles;

 private:
  int mode_, ncta_;
  struct Chunk {
    int phase;
    std::vector<PanelItem> items;
    int64_t cost;
  };
  std::vector<Chunk> chunks_;
  void pack_item(PanelItem& it, int h, const std::vector<const ColSpec*>& spec, const std::vector<int64_t>& q);
};

}  // namespace uh

// Host-side packing of the tensor-core multi-RHS product into its device program (uh_panel.h).
#pragma once

#include <cstdint>
#include <vector>

#include "uh_panel.h"
#include "uh_program.h"

namespace uh {

class PanelBuilder {
 public:
  // zero_row: first row of a block of XP that is always zero (padding runs read it).
  PanelBuilder(int mode, int ncta, int64_t zero_row)
      : mode_(mode), ncta_(ncta), C_(panel_block_rows(mode)), kmma_(panel_mma_k(mode)), zero_row_(zero_row) {}

  // One output chunk of phase `phase` (0: forward transform, 1: coupling, 2: near field and
  // backward transform): h <= kPanelMaxH outputs starting at row `out` of the kind's output (a
  // multiple of the block rows for Z1 / Z2); its columns, in order, are `cols` (ColSpec sources
  // are kPSrc* panels, positions are panel rows). Runs are whole blocks of C panel rows: a
  // column range is widened to block boundaries, and the positions outside it get zero columns
  // in operand B.
  void add_chunk(int phase, int16_t kind, int64_t out, int h, const std::vector<ColSpec>& cols);

  // Assign the chunks to CTAs (longest processing time first: phase 0 on its own, phases 1 and 2
  // on shared loads) and lay the items out by CTA, each CTA's list phase by phase.
  const char* finalize();
  // Checks every address the kernel derives from the program against the panel heights
  // (src_rows: rows of XP, Z1, Z2, each a multiple of the block rows) and the output heights
  // (out_rows: Z1, Z2, Y).
  const char* self_check(const int64_t src_rows[3], const int64_t out_rows[3]) const;

  std::vector<PanelItem> items;    // by CTA, then phase
  std::vector<int32_t> begin;      // [ncta + 1]
  std::vector<unsigned char> tiles;
  int64_t streamed_bytes = 0;      // operand B bytes of one pass
  int64_t mma_flops = 0;           // tensor-core flops of one pass
  int64_t z_chunks[2] = {0, 0};    // chunks writing Z1, Z2

 private:
  int mode_, ncta_, C_, kmma_;
  int64_t zero_row_;
  struct Chunk {
    int phase;
    std::vector<PanelItem> items;
    int64_t cost;
  };
  std::vector<Chunk> chunks_;
  // Column k of the item: spec[k] (null for a zero column) at position q[k] of it.
  void pack_item(PanelItem& it, int h, const std::vector<const ColSpec*>& spec, const std::vector<int64_t>& q);
};

}  // namespace uh

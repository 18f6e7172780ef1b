// Internal declarations shared by the host side (packing, C ABI) and the CUDA kernels.
//
// Every phase of both products is one "segmented GEMV": a set of output chunks (at most
// kHpMax consecutive outputs each) and a set of work items. An item multiplies one packed,
// column-major tile of `hp` rows x `ncols` columns by the input values that its column index
// list names, and contributes the result to one chunk. A chunk fed by several items collects
// their partial results in a fixed slot order; the last item to finish sums them in that order,
// so results do not depend on scheduling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace uh {

constexpr int kThreads = 256;   // threads per CTA of the GEMV kernels
constexpr int kHpMax = 64;      // largest chunk height (outputs per chunk)
constexpr int kMaxCols = 512;   // largest column count of one item (shared-memory staging)

// One work item. The packed tile starts at element data_off of the phase's matrix buffer;
// column c holds hp elements (rows h..hp-1 are zero padding); its input is in0[idx] for
// idx >= 0 and in1[-idx-1] for idx < 0.
struct Item {
  int64_t data_off;
  int32_t hp;
  int32_t ncols;
  int32_t idx_off;   // first entry of this item's column index list
  int32_t chunk;     // output chunk
  int32_t part;      // partial slot, or -1 when the item is the chunk's only contributor
  int32_t pad;
};
static_assert(sizeof(Item) == 32, "Item layout");

// Output chunk: h consecutive outputs. kind 0 writes out_lin[dst + r]; kind 1 writes
// out_perm[perm[dst + r]] (row positions mapped back to original indices).
struct Chunk {
  int64_t dst;
  int32_t h;
  int32_t nparts;
  int32_t part_base;  // first partial slot of this chunk (slots part_base .. part_base+nparts-1)
  int32_t kind;
};
static_assert(sizeof(Chunk) == 24, "Chunk layout");

struct SegGemvParams {
  const Item* items;      // this launch's items
  int32_t item_count;
  const Chunk* chunks;    // all chunks of the program
  const void* M;          // packed matrices (element type of the op)
  const int32_t* colidx;  // column index lists
  const void* in0;        // input addressed by idx >= 0
  const void* in1;        // input addressed by idx < 0 (x, original ordering)
  void* out_lin;          // kind-0 destination
  void* out_perm;         // kind-1 destination (y, original ordering)
  const int32_t* perm;    // position -> original index
  void* partials;         // [slots][kHpMax] accumulator-type complex
  uint32_t* chunk_cnt;    // [chunks] arrival counters, zero between launches
  uint32_t* sched;        // [2] work counter and exit counter, zero between launches
};

// Records a message for uh_last_error() (calling thread) and returns `code`.
int set_error(int code, const char* fmt, ...);

// Launch the segmented GEMV for complex128 (fp64) or complex64 (fp32 accumulation) data.
cudaError_t launch_seg_gemv(bool c128, const SegGemvParams& p, int grid, cudaStream_t stream);

}  // namespace uh

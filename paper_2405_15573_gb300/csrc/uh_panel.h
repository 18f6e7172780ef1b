// Device program of the tensor-core multi-RHS product (uh_panel.cu), shared with the host packer
// (uh_panel_pack.cpp).
//
// Y = A^UH X for up to kPanelR right-hand sides per pass (Algorithm 6 applied to a block of
// columns): X is gathered into cluster order as a row-major panel XP (row i = the kPanelR values
// of point i); three launches then compute Z1 = Xhat (forward transform), Z2 = Yhat (coupling)
// and Y (near field + backward transform), each a list of output chunks of at most 64 rows.
//
// A chunk's output rows, times the panel, is a sum over work items of one real GEMM on the
// tensor cores: item = kPanelK columns of the chunk's complex matrix, as the real K-major
// operand B (N = 2h rows: row 2i holds Re, row 2i+1 Im of output row i), with the kPanelK panel
// rows its columns multiply (operand A, M = 2 kPanelR rows: row 2r holds Re, row 2r+1 Im of
// right-hand side r, built in shared memory from the staged panel rows). D = A B^T accumulates
// in tensor memory (M = 128 lanes x N columns, FP32) over the chunk's items, so that
//   Re Y[i][r] = D[2r][2i] - D[2r+1][2i+1],   Im Y[i][r] = D[2r+1][2i] + D[2r][2i+1],
// two neighbouring lanes of one warp. B is packed by the host in the swizzled K-major layout of
// the MMA (128-byte rows, 16-byte chunks XOR-ed with row % 8, 8-row groups of 1024 bytes), either
// as TF32 (rounded to nearest) or as a BF16 pair hi + lo (3 products: hi*hi + hi*lo + lo*hi).
#pragma once

#include <stdint.h>

namespace uh {

constexpr int kPanelR = 64;          // right-hand sides per pass (M = 2 kPanelR = 128)
constexpr int kPanelK = 64;          // columns (panel rows) per item
constexpr int kPanelMaxH = 64;       // outputs per chunk (N <= 128)
constexpr int kPanelMaxRuns = 8;     // contiguous runs of panel rows per item
constexpr int kPanelStages = 3;
constexpr int kPanelRowBytes = kPanelR * 8;                  // one panel row, complex64
constexpr int kPanelTileMax = 256 * 2 * kPanelMaxH;          // B bytes at N = 128 (32 KB)
constexpr int kPanelRawMax = kPanelK * kPanelRowBytes;       // staged panel rows (32 KB)
constexpr int kPanelABytes = 2 * kPanelR * kPanelK * 4;      // operand A (32 KB, either mode)

enum : int { kPanelTF32 = 0, kPanelBF16X3 = 1 };
// Panel sources (row-major, kPanelR complex64 per row) and outputs.
enum : int8_t { kPSrcXP = 0, kPSrcZ1 = 1, kPSrcZ2 = 2 };
enum : int16_t { kPOutZ1 = 0, kPOutZ2 = 1, kPOutY = 2 };
enum : int16_t { kPItemFirst = 1, kPItemLast = 2 };

struct PanelRun {
  int32_t start;  // first panel row in the source
  int16_t len;    // rows
  int8_t src;     // kPSrc*
  int8_t pad;
};
static_assert(sizeof(PanelRun) == 8, "PanelRun layout");

struct alignas(16) PanelItem {
  int64_t tile_off;  // byte offset of the item's B operand in the packed tiles (256 * n bytes)
  int64_t out;       // the chunk's first output row (Z1 / Z2 row, or Y position in cluster order)
  int16_t n;         // MMA N = 2h rounded up to 16
  int16_t h;         // the chunk's output rows
  int16_t kind;      // kPOut*
  int16_t flags;     // kPItem*
  int16_t nrows;     // panel rows of the item (sum of run lengths) <= kPanelK
  int16_t nruns;
  int32_t pad;
  PanelRun runs[kPanelMaxRuns];
};
static_assert(sizeof(PanelItem) == 96, "PanelItem layout");

// One phase (launch) of a pass.
struct PanelParams {
  const PanelItem* items;
  const int32_t* cta_begin;  // items of CTA b: [cta_begin[b], cta_begin[b + 1])
  const unsigned char* tiles;
  const void* src[3];        // XP, Z1, Z2 (row-major panels)
  void* zout[2];             // Z1, Z2
  void* y;                   // complex64, column-major n x nrhs, leading dimension ldy
  int64_t ldy;
  const int32_t* perm;       // cluster position -> original index
  int32_t rhs0;              // first right-hand side of this pass
  int32_t nb;                // right-hand sides in this pass (<= kPanelR)
  int32_t mode;              // kPanelTF32 or kPanelBF16X3
  uint32_t* status;          // nonzero after a bounded wait ran out
  long long timeout_cycles;
};

// Launches: X (complex64, column-major, ldx) -> XP rows for right-hand sides [rhs0, rhs0 + nb),
// zero beyond; then one phase of the pass.
int panel_gather(const void* x, int64_t ldx, int64_t n, const int32_t* perm, int32_t rhs0, int32_t nb,
                 void* xp, void* stream);
int panel_prepare();
int panel_launch(const PanelParams& p, int grid, void* stream);

}  // namespace uh

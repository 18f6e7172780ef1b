// Device program of the tensor-core multi-RHS product (uh_panel.cu), shared with the host packer
// (uh_panel_pack.cpp).
//
// Y = A^UH X for up to kPanelR right-hand sides per pass (Algorithm 6 applied to a block of
// columns): X is gathered into cluster order as the panel XP; one persistent launch then
// computes Z1 = Xhat (forward transform), Z2 = Yhat (coupling) and Y (near field + backward
// transform), three phases of output chunks of at most 64 rows. Every CTA runs its list phase by
// phase; an item whose operand A comes from Z1 or Z2 waits (before that copy only) until every
// chunk of the phase that writes it has been published on a monotonic counter.
//
// A chunk's output rows, times the panel, is a sum over work items of one real GEMM on the
// tensor cores: item = up to kPanelK columns of the chunk's complex matrix, as the real K-major
// operand B (N = 2h rows: row 2i holds Re, row 2i+1 Im of output row i), with the panel rows its
// columns multiply (operand A, M = 2 kPanelR rows: row 2r holds Re, row 2r+1 Im of right-hand
// side r). D = A B^T accumulates in tensor memory (M = 128 lanes x N columns, FP32) over the
// chunk's items; a pass of at most 32 right-hand sides runs MMAs of M = 64 on the first 64 rows
// of operand A (D row m then sits in lane 32 (m / 16) + m % 16: the lanes 0-15 of each 32-lane
// quarter), so that
//   Re Y[i][r] = D[2r][2i] - D[2r+1][2i+1],   Im Y[i][r] = D[2r+1][2i] + D[2r][2i+1],
// two neighbouring lanes of one warp.
//
// Operand formats. B is packed by the host in the 128-byte-swizzled K-major layout (128-byte
// rows, 16-byte chunks XOR-ed with row % 8, 8-row groups of 1024 bytes; K segments of 128 bytes,
// n * 128 bytes apart), as TF32 (rounded to nearest) or as a BF16 pair hi + lo (segment 0 the hi
// plane, segment 1 the lo plane; 3 products hi*hi + hi*lo + lo*hi). The panels XP, Z1 and Z2 are
// kept in global memory already in the layout of operand A: the K-major layout without swizzle,
// in blocks of C consecutive panel rows (C = 4 for TF32, 8 for BF16). A block holds, for every
// A row m (0..127), the C values of rows [C g, C g + C) as one 16-byte core-matrix row, at
// (m / 8) * 128 + (m % 8) * 16; for BF16 the lo plane follows the hi plane 2048 bytes on. A block
// is C * kPanelRowBytes bytes, so panel row j starts at j * kPanelRowBytes for j % C == 0, and a
// run of whole blocks is one contiguous copy: operand A of an item is its runs copied back to
// back (descriptor: core matrices 128 bytes apart along M, one block apart along K). The gather
// writes XP in this layout and the epilogues write Z1 and Z2 in it, so no item converts its
// inputs.
#pragma once

#include <stdint.h>

namespace uh {

constexpr int kPanelR = 64;          // right-hand sides per pass (M = 2 kPanelR = 128)
constexpr int kPanelK = 64;          // panel rows (K) per item
constexpr int kPanelMaxH = 64;       // outputs per chunk (N <= 128)
constexpr int kPanelMaxRuns = 8;     // contiguous runs of panel blocks per item
constexpr int kPanelRowBytes = 512;                          // one panel row in operand-A layout
constexpr int kPanelTileMax = 2 * 128 * 2 * kPanelMaxH;      // B bytes at N = 128, two segments (32 KB)
constexpr int kPanelABytes = kPanelK * kPanelRowBytes;       // operand A of an item (32 KB)
// A CTA's operand-B ring in shared memory, and its items in flight (each has a slot of
// barriers). The packer places every item's B in the ring (PanelItem::boff) and names the item
// whose consumption frees that room and the item's slot (PanelItem::room), so the copies need
// no allocator on the device.
constexpr int kPanelBRing = 120 * 1024;
constexpr int kPanelSlots = 24;
// Bytes of a panel row in a pass: M = 128 rows of operand A, or the compact layout of M = 64
// (the same core-matrix pattern for rows 0-63, blocks of C * 256 bytes) for at most 32
// right-hand sides.
#ifndef UH_HOST_DEVICE
#ifdef __CUDACC__
#define UH_HOST_DEVICE __host__ __device__
#else
#define UH_HOST_DEVICE
#endif
#endif
UH_HOST_DEVICE constexpr int panel_row_bytes(int m64) { return m64 ? kPanelRowBytes / 2 : kPanelRowBytes; }

enum : int { kPanelTF32 = 0, kPanelBF16X3 = 1 };
// Panel rows per block of the operand-A layout, and the MMA's K per instruction.
constexpr int panel_block_rows(int mode) { return mode == kPanelTF32 ? 4 : 8; }
constexpr int panel_mma_k(int mode) { return mode == kPanelTF32 ? 8 : 16; }
// Panel sources and outputs.
enum : int8_t { kPSrcXP = 0, kPSrcZ1 = 1, kPSrcZ2 = 2 };
enum : int16_t { kPOutZ1 = 0, kPOutZ2 = 1, kPOutY = 2 };
// kPItemDepZ1 / kPItemDepZ2: the item's operand A reads Z1 / Z2.
enum : int16_t { kPItemFirst = 1, kPItemLast = 2, kPItemDepZ1 = 4, kPItemDepZ2 = 8 };

struct PanelRun {
  int32_t start;  // first panel row in the source (a multiple of the block rows)
  int16_t len;    // rows (likewise a multiple)
  int8_t src;     // kPSrc*
  int8_t pad;
};
static_assert(sizeof(PanelRun) == 8, "PanelRun layout");

struct alignas(16) PanelItem {
  int64_t tile_off;    // byte offset of the item's B operand in the packed tiles
  int32_t out;         // the chunk's first output row (Z1 / Z2 row, or Y position in cluster order)
  int32_t boff;        // byte offset of B in the CTA's operand-B ring
  int32_t room;        // B may be copied once the CTA's item `room` (index in its list) is consumed;
                       // -1: at once
  int16_t n;           // MMA N = 2h rounded up to 16
  int16_t h;           // the chunk's output rows
  int16_t kind;        // kPOut*
  int16_t flags;       // kPItem*
  int16_t nrows;       // K: panel rows of the item (sum of run lengths), a multiple of the MMA K
  int16_t nruns;
  PanelRun runs[kPanelMaxRuns];
};
static_assert(sizeof(PanelItem) == 96, "PanelItem layout");
// Bytes of an item's operand B: 128 * n per K segment (TF32: one per 32 panel rows; BF16: the hi
// and the lo plane).
UH_HOST_DEVICE constexpr int panel_tile_bytes(int mode, int n, int nrows) {
  return 128 * n * (mode == kPanelTF32 ? (nrows + 31) / 32 : 2);
}

// A pass (one launch).
struct PanelParams {
  const PanelItem* items;
  const int32_t* cta_begin;  // items of CTA b: [cta_begin[b], cta_begin[b + 1]), phase by phase
  const unsigned char* tiles;
  const void* src[3];        // XP, Z1, Z2 (operand-A layout)
  void* zout[2];             // Z1, Z2
  void* y;                   // complex64, column-major n x nrhs, leading dimension ldy
  int64_t ldy;
  const int32_t* perm;       // cluster position -> original index
  int32_t rhs0;              // first right-hand side of this pass
  int32_t nb;                // right-hand sides in this pass (<= kPanelR)
  int32_t mode;              // kPanelTF32 or kPanelBF16X3
  int32_t m64;               // 1: nb <= 32, MMAs of M = 64 on the first 64 operand-A rows
  unsigned long long* done;  // [2] monotonic: +1 per finished Z1 / Z2 chunk
  unsigned long long need[2];  // Z1 / Z2 complete in this pass when done[k] >= need[k]
  uint32_t* status;          // nonzero after a bounded wait ran out
  long long timeout_cycles;
};

// Launches: X (complex64, column-major, ldx) -> XP in operand-A layout for right-hand sides
// [rhs0, rhs0 + nb) (zero beyond nb), `rows` panel rows (a multiple of the block rows; rows
// >= n are zero); then one phase of the pass.
int panel_gather(const void* x, int64_t ldx, int64_t n, int64_t rows, const int32_t* perm, int32_t rhs0,
                 int32_t nb, int32_t mode, int32_t m64, void* xp, void* stream);
int panel_prepare();
// Cooperative launch of one pass: every CTA must be resident (the phases wait on each other).
int panel_launch(const PanelParams& p, int grid, void* stream);

}  // namespace uh

// Device program of the streaming matvec kernel (uh_stream.cu), shared with the host packer.
//
// One matvec (UH: Algorithm 6; H: Algorithm 5) is ONE persistent launch, one CTA per SM. Its work
// is a list of output chunks (at most 64 consecutive outputs each). Every chunk is owned by one
// CTA and streamed as a sequence of work items; an item is one column-major tile of `hp` rows x
// `ncols` columns (at most kTileBytes) together with the input values its columns multiply,
// given as up to kMaxRuns contiguous runs of an input vector. In each CTA a producer warp copies
// item tiles and input runs into a ring of kStages shared-memory stages with TMA bulk copies
// (cp.async.bulk, mbarrier transaction counts); eight consumer warps multiply and accumulate, and
// at the end of a chunk reduce the column groups and write the chunk's outputs.
//
// Dependencies are per phase group: an item that reads x in cluster order, xhat or yhat waits (in
// its producer, before copying those runs) until every chunk of the group that writes that vector
// has finished in this call, counted by a monotonic 64-bit counter per group. A producer checks a
// group once per call and then remembers it. The release that publishes a finished chunk to the
// other CTAs (red.release on the group counter) is issued by a publisher warp, fed through a ring
// of mbarriers, so that its wait for the chunk's stores is off the consumers' path.
//
// Every CTA first permutes its slice of x into cluster order (xp), at entry, without descriptors:
// positions [a_b, a_{b+1}) with a_b = floor(n b / grid) rounded down to 16 bytes, and publishes the
// permutation counter (one release per CTA). Work is then placed in two parts. The static part
// (forward transform, the first part of the near field, coupling) is a list per CTA, ordered by
// group; a group there only waits on earlier groups. Coefficient matrices stored factored,
// S_b = S_X,b S_Y,b^* (Section 4.2), add a static group between the forward transform and the
// coupling: t_b = S_Y,b^* xhat_sigma into z4, which the coupling reads with S_X,b. The pool (the second half of the near field,
// then the backward chunks) is one list of tickets in a fixed order, each one or more whole chunks,
// that the CTAs take from through a global counter once their static list is issued. A CTA whose
// static part ran slowly takes fewer tickets: the end times of the CTAs differ by about one
// ticket. A backward chunk adds its row tile's near-field partial, written by any CTA: every
// near-field chunk that writes a partial releases a flag of its own, and the backward chunk stages
// the partial like an input run once that flag is set in this call (or without a flag, when the
// partial's CTA published it through a later chunk of a group the backward chunk waits for). A
// pool chunk only waits on static groups and on flags of chunks handed out before it (or earlier
// in its own ticket), so every wait ends.
#pragma once

#include <stdint.h>

namespace uh {

constexpr int kStreamConsumerWarps = 8;
constexpr int kStreamConsumers = kStreamConsumerWarps * 32;
constexpr int kStreamThreads = kStreamConsumers + 64;  // + producer warp + publisher warp
constexpr int kPubRing = 16;  // group-counter releases in flight from consumers to the publisher
constexpr int kStages = 3;
constexpr int kTileBytes = 65536;       // largest tile of an item
constexpr int kStreamMaxCols = 512;     // largest column count of an item
constexpr int kStageBytes = 69632;      // an item's tile and inputs (inputs at the tile's end)
constexpr int kMaxRuns = 6;
constexpr int kStreamHpMax = 64;
// Rows of a chunk of t_b = S_Y,b^* xhat_sigma (kScatterZ4): up to one row per consumer thread, so
// that the stacked rows of a column cluster fill few chunks (their chunk ends scatter directly).
constexpr int kStreamHpTall = 256;
static_assert(kStreamHpTall <= kStreamConsumers, "one output row per consumer thread");
// Pool descriptors are fetched into the ring in segments of at most kPoolSeg items, one segment
// ahead of the items being issued.
constexpr int kPoolSeg = 16;

// Work-item descriptors are streamed into a ring of kDescRing entries, kDescBatch per copy.
// The consumers read the descriptors in the ring; a batch is refilled only after the producer
// has issued the whole next batch, when the consumers (at most kStages items behind) are past it.
constexpr int kDescBatch = 8;
constexpr int kDescBatches = 8;
constexpr int kDescRing = kDescBatch * kDescBatches;
static_assert(kStages < kDescBatch, "consumers must be past a batch when it is refilled");
static_assert(2 * kPoolSeg + kStages <= kDescRing, "a fetched pool segment must not overwrite live descriptors");

// The kernel comes in three variants over the same device program:
//  kVarC64    complex64 tiles, vectors and accumulation in FP32;
//  kVarC128   complex128 tiles, vectors and accumulation in FP64;
//  kVarMixed  complex64 tiles of a complex64 program, x and y in complex128, the intermediate
//             vectors and the accumulation in extended precision from pairs of FP32 values
//             (value = hi + lo, error-free transforms), 16 bytes per complex value. Its inputs
//             take twice the bytes of the complex64 ones, so it runs two stages of
//             kStageBytesMixed: a complex64 item with ncols columns and s staged values uses
//             ncols * hp * 8 + s * 8 <= kStageBytes bytes, hence ncols * hp * 8 + s * 16 <=
//             kStageBytes + 8 * (kStreamMaxCols + kStreamHpMax) = kStageBytesMixed.
// A program is packed for one of two geometries: one CTA per SM with kStages stages of
// kStageBytes (tiles up to kTileBytes), or two CTAs per SM with kStagesDual stages of
// kStageBytesDual (tiles up to kTileBytesDual). The second suits operators of many small chunks
// (low ranks, small leaves, batches of small operators), whose per-item and per-chunk latencies
// then overlap between the two CTAs of an SM; kVarC64Dual, kVarMixedDual and kVarC128Dual run
// such programs.
// kVarC64R2 / kVarC64R4 / kVarC64DualR2 run a complex64 program for 2 or 4 right-hand sides in one
// pass over the operator: every vector holds the R values of a position together, and an item's
// inputs take R times the bytes, so these run two stages of the geometry's stage plus
// (R - 1) * 8 * (kStreamMaxCols + kStreamHpMax) bytes (an item stages at most
// kStreamMaxCols + kStreamHpMax values).
enum StreamVariant : int {
  kVarC64 = 0, kVarC128 = 1, kVarMixed = 2, kVarC64Dual = 3, kVarMixedDual = 4,
  kVarC64R2 = 5, kVarC64R4 = 6, kVarC64DualR2 = 7, kVarC128Dual = 8
};
constexpr int stage_bytes_rhs(int stage_bytes, int r) { return stage_bytes + (r - 1) * 8 * (kStreamMaxCols + kStreamHpMax); }
constexpr int kStageBytesMixed = kStageBytes + 8 * (kStreamMaxCols + kStreamHpMax);
constexpr int kStagesMixed = 2;
constexpr int kStagesDual = 3;
constexpr int kTileBytesDual = 24576;
constexpr int kStageBytesDual = 26624;
constexpr int kStageBytesMixedDual = kStageBytesDual + 8 * (kStreamMaxCols + kStreamHpMax);

// The capacities a program is packed for.
struct StreamGeometry {
  int ctas_per_sm;
  int tile_bytes;          // largest tile of an item
  int stage_bytes;         // an item's tile and inputs
  int stage_bytes_mixed;   // the same item in the extended-precision variant
};
constexpr StreamGeometry kGeomOne{1, kTileBytes, kStageBytes, kStageBytesMixed};
constexpr StreamGeometry kGeomDual{2, kTileBytesDual, kStageBytesDual, kStageBytesMixedDual};

// Shared-memory layout of the kernel (bytes) for `Stages` stages of `StageBytes` and a per-thread
// reduction slot of `RedSlot` bytes. The chunk-end buffers are double-buffered by chunk parity,
// so a chunk end needs no barrier after its last use of them.
template <int Stages, int StageBytes, int RedSlot>
struct StreamSmem {
  static constexpr int stages = Stages;
  static constexpr int stage_bytes = StageBytes;
  static constexpr int red = Stages * StageBytes;                // group reduction [2], one slot per consumer thread
  static constexpr int desc = red + 2 * kStreamConsumers * RedSlot;  // descriptor ring, 96 B each
  static constexpr int scat = desc + kDescRing * 96;             // scatter entries of a chunk [2] (256 x 8 B)
  static constexpr int bars = scat + 2 * 256 * 8;                 // full, empty [Stages], desc [kDescBatches],
                                                                  // pub_full, pub_empty [kPubRing], pool [2]
  static constexpr int misc = bars + (2 * Stages + kDescBatches + 2 * kPubRing + 2) * 8;  // abort flag, decision words
  static constexpr int pub = misc + 32;                           // group counter of each release [kPubRing]
  static constexpr int bytes = pub + kPubRing * 4;
  static_assert(Stages <= kStages, "descriptor ring sized for at most kStages stages");
  static_assert(bytes <= 227 * 1024, "shared memory of one CTA");
};
using StreamSmemStd = StreamSmem<kStages, kStageBytes, 16>;
using StreamSmemMixed = StreamSmem<kStagesMixed, kStageBytesMixed, 32>;
using StreamSmemDual = StreamSmem<kStagesDual, kStageBytesDual, 16>;
using StreamSmemMixedDual = StreamSmem<kStagesMixed, kStageBytesMixedDual, 32>;
// two CTAs per SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
using StreamSmemR2 = StreamSmem<2, stage_bytes_rhs(kStageBytes, 2), 32>;
using StreamSmemR4 = StreamSmem<2, stage_bytes_rhs(kStageBytes, 4), 64>;
using StreamSmemDualR2 = StreamSmem<2, stage_bytes_rhs(kStageBytesDual, 2), 32>;
static_assert(2 * (StreamSmemDual::bytes + 1024) <= 228 * 1024, "two CTAs per SM");
static_assert(2 * (StreamSmemDualR2::bytes + 1024) <= 228 * 1024, "two CTAs per SM");
static_assert(2 * (StreamSmemMixedDual::bytes + 1024) <= 228 * 1024, "two CTAs per SM");

// Input vectors a run can read.
enum : int8_t { kSrcXp = 0, kSrcZ1 = 1, kSrcZ2 = 2, kSrcZ3 = 3, kSrcZ4 = 4 };
constexpr int kNumSources = 5;

struct Run {
  int32_t start;   // first element (a multiple of the 16-byte element count)
  int16_t len;     // elements (likewise a multiple)
  int8_t src;      // kSrc*
  int8_t pad;
};
static_assert(sizeof(Run) == 8, "Run layout");

// Item flags: chunk boundaries, near-field base, and the groups whose completion the item's runs
// need (bits kDepShift + counter index). kItemBase (on the last item of a chunk): the item's last
// run is not a column input but the chunk's near-field partial z3[aux .. aux + h), staged after
// the inputs, once flag naux is set (naux -1: the partial's CTA published it, before this item's
// group counters, through a later chunk of those groups), and added to the outputs.
enum : int16_t { kItemFirst = 1, kItemLast = 2, kItemBase = 4 };
constexpr int kDepShift = 8;
enum : int { kCounterPermute = 0, kCounterForward = 1, kCounterCoupling = 2, kCounterCouplingY = 3, kNumCounters = 4 };
// WorkItem::counter of a chunk that releases its own flag (number naux) instead of a group counter.
constexpr int kCounterFlag = 15;
// Layout of the counter array: group counters, the pool ticket, then the flags.
constexpr int kTicketIndex = kNumCounters;
constexpr int kFlagBase = kNumCounters + 1;

// Chunk outputs: kToZ1..kToZ3 write z[dst + r]; kToY writes y[perm[dst + r]]; kScatterZ1 / kScatterZ2 /
// kScatterZ4 write output r to z[e.dst + r - e.lo] for every scatter entry e with e.lo <= r < e.hi (the chunk's entries are
// scatter[aux .. aux + naux)): each consumer chunk then finds its inputs in one contiguous run.
// counter >= 0: the chunk's completion is added to that group counter.
// kEnd: written by a CTA's producer after its last item (never packed).
enum : int16_t { kToZ1 = 0, kToZ2 = 1, kToZ3 = 2, kToY = 3, kScatterZ1 = 5, kScatterZ2 = 6, kEnd = 7, kScatterZ4 = 8 };
#ifndef UH_HOST_DEVICE
#ifdef __CUDACC__
#define UH_HOST_DEVICE __host__ __device__
#else
#define UH_HOST_DEVICE
#endif
#endif
UH_HOST_DEVICE constexpr bool is_scatter(int kind) {
  return kind == kScatterZ1 || kind == kScatterZ2 || kind == kScatterZ4;
}

struct Scatter {
  int32_t dst;
  int16_t lo, hi;
};
static_assert(sizeof(Scatter) == 8, "Scatter layout");

struct alignas(16) WorkItem {
  int64_t tile_off;  // element offset of the tile in the packed matrix buffer
  int64_t dst;       // the chunk's output offset (see kind)
  int32_t hp;        // rows of the tile = padded chunk height
  int32_t ncols;     // tile columns = staged input values (sum of the run lengths)
  int32_t h;         // the chunk's height
  int16_t kind;      // the chunk's output kind (kTo*, kScatter*)
  int16_t counter;   // the chunk's group counter, or -1
  int16_t nruns;
  int16_t flags;     // kItem* | dependency bits
  int32_t aux;       // kItemBase: the chunk adds z3[aux + r] to output r; scatter kinds: first
                     // scatter entry
  int32_t chunk;     // chunk number (host bookkeeping)
  int32_t naux;      // scatter kinds: number of scatter entries; kCounterFlag chunks: their flag;
                     // kItemBase: the flag of the near-field partial
  Run runs[kMaxRuns];
};
static_assert(sizeof(WorkItem) == 96, "WorkItem layout");

// Host-side record of a chunk.
struct OutChunk {
  int64_t dst;
  int32_t h;
  int16_t kind;
  int16_t counter;
  int32_t scat0 = 0, nscat = 0;  // scatter entries of scatter kinds
  int32_t flag = -1;             // near-field partials (kToZ3): the flag the chunk releases
};

struct PoolRange {
  int32_t begin, end;  // items of a pool ticket: [begin, end), one or more whole chunks
};

struct StreamParams {
  const WorkItem* items;
  const int32_t* cta_begin;  // static items of CTA b: [cta_begin[b], cta_begin[b + 1])
  const PoolRange* pool;     // [pool_chunks] item ranges (one or more whole chunks each), in the
                             // order the tickets hand them out
  int64_t pool_chunks;
  unsigned long long* group_done;  // counters, monotonic over calls: [kNumCounters] group counters,
                                   // [kTicketIndex] the pool ticket (every call adds pool_chunks +
                                   // grid: one failed take per CTA), [kFlagBase + f] flag f (every
                                   // call adds 1)
  unsigned long long need[kNumCounters];  // a group is complete when its counter >= need
  unsigned long long ticket_base;  // ticket value at the start of this call
  unsigned long long flag_need;    // a flag is set in this call when it is >= flag_need
  const void* M;             // packed tiles
  const void* x;             // input, original ordering (complex128 in the mixed variant)
  int64_t n;                 // positions permuted into xp (all operators of the program)
  void* y;                   // output, original ordering (complex128 in the mixed variant)
  const int32_t* perm;       // position -> original index
  const Scatter* scatter;    // scatter entries of the scatter kinds
  void* xp;                  // x in cluster order (kSrcXp)
  void* z1;                  // xhat (UH) or t_b (H) (kSrcZ1)
  void* z2;                  // yhat (kSrcZ2)
  void* z3;                  // near-field partials of row tiles (base of the backward chunks)
  void* z4;                  // t_b = S_Y,b^* xhat_sigma of the blocks stored factored (kSrcZ4)
  const void* xr[4];         // several right-hand sides (R > 1): x and y of right-hand side r
  void* yr[4];               // (x and y above are unused then)
  uint32_t* status;          // nonzero after a bounded wait ran out
  long long timeout_cycles;  // bound of every wait, in SM clock cycles
};

}  // namespace uh

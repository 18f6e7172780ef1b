// Tensor-core multi-RHS product (sm_103a): one persistent cooperative launch per pass of up to 64
// right-hand sides (MMAs of M = 128; of M = 64 on a compact panel layout for up to 32), one CTA
// per SM. Layout of the work and of the operands: uh_panel.h.
//
// Roles in a CTA of 448 threads (14 warps). No thread allocates operand space: the packer has
// placed every item's operand B in the CTA's B ring and named the item whose consumption frees
// that room (PanelItem boff, room), and the items' descriptors stream into a ring of 32 that
// every role reads.
//  - copy workers (lane 0 of warps 11-13, items in turn): copy operand B of their items (the
//    packed operator, from HBM) once the room is free, up to 6 items ahead, so that operator
//    tiles keep streaming while an operand A waits for the previous phase; and operand A (runs
//    of panel blocks, already in the MMA's layout, from L2) into one of 3 fixed buffers (6 of half
//    the size in a pass of M = 64) once the item's panel is complete in this pass (Z1 / Z2
//    counters). Both copies arrive on the item's one full barrier. A thread issues about two
//    barrier-armed bulk copies per microsecond whatever their size, so the copies are spread over
//    three threads.
//  - MMA issuer (lane 0 of warp 1; warp 1 also allocates and frees the tensor memory): issues
//    the descriptor copies (TMA bulk copies of 8, refilled as the items are consumed); per item
//    waits for its operands, at a chunk's first item for the accumulator (all 512 columns of
//    tensor memory, taken in turn by the chunks: four of 128 columns for TF32, two of 256 for
//    BF16x3) and hands the chunk's output record to the epilogue, issues the
//    item's tcgen05.mma instructions and commits them to the barriers that free the slot (its B
//    bytes and A buffer) and, at a chunk's end, the accumulator for the epilogue.
//  - epilogue (warps 2-9, each on its own): per chunk reads its part of the finished accumulator
//    (tcgen05.ld; warp w reads the 32-lane quarter w % 4 and half of the column blocks), combines
//    the real products into complex outputs and writes them: Z1 / Z2 in the operand-A layout of
//    the next phase (TF32, or BF16 hi and lo), Y as complex64 in original ordering. Each warp
//    releases the accumulator on its own (an mbarrier of 8 arrivals), so no epilogue warp waits
//    for another and none of them stalls the copy workers or the MMA issuer. After its part of a Z1
//    or Z2 chunk is stored, each warp arrives on the chunk's entry of a publication ring.
//  - publisher (lane 0 of warp 10): per Z1 / Z2 chunk, once all 8 epilogue warps have arrived,
//    adds 1 to the pass's counter of that panel with red.release.gpu. The release waits for the
//    stores to be performed (about a microsecond under full HBM load); that wait is here, not on
//    the epilogue warps' path.
// Every wait is bounded (timeout_cycles); when one runs out the CTA records it in `status`, stops,
// lets its copies and MMAs in flight finish, frees the tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "uh.h"
#include "uh_internal.h"
#include "uh_panel.h"

namespace uh {
namespace {

constexpr int kAProducers = 3;          // copy-worker threads (one per warp)
constexpr int kBAhead = 6;              // a worker's B copies run at most this many items past its A
// (warp 0 unused), MMA issuer, 8 epilogue warps, publisher, copy workers
constexpr int kThreads = 32 * (11 + kAProducers);
constexpr int kPubRing = 16;            // Z1 / Z2 chunk publications in flight
constexpr int kEpiWarps = 8;
constexpr int kDescBatch = 8;           // descriptors per bulk copy
constexpr int kDescBatches = 4;         // batches in the descriptor ring
constexpr int kDescRing = kDescBatches * kDescBatch;
constexpr int kAccCols = 128;          // one accumulator of a TF32 pass: N <= 128 FP32 columns
constexpr int kAccs = 4;               // accumulators, chunk after chunk (all 512 columns)
constexpr uint32_t kTmemCols = kAccs * kAccCols;
constexpr int kSlots = kPanelSlots;    // items in flight: full / empty barriers
constexpr int kASlots = 3;             // operand-A buffers of 32 KB (twice as many of 16 KB at M = 64)
constexpr int kBRing = kPanelBRing;    // operand-B byte ring (B sizes are multiples of 2 KB)

// Shared memory (bytes from a 1024-aligned base).
constexpr int kOffA = 0;                                        // operand A [kASlots]
constexpr int kOffB = kASlots * kPanelABytes;                   // operand-B ring (1024-aligned)
constexpr int kOffRing = kOffB + kBRing;                        // descriptor ring [kDescRing]
constexpr int kOffRec = kOffRing + kDescRing * 96;              // chunk records [kAccs], one per accumulator
constexpr int kOffPub = kOffRec + kAccs * 16;                   // panel of each publication [kPubRing]
constexpr int kOffBars = kOffPub + kPubRing * 4;
// barriers: full[kSlots] (operands B and A landed: two arrivals with their bytes), empty[kSlots],
// accfull[A], accempty[A], desc[kDescBatches], recfull[A], done, pubfull[P], pubempty[P]
constexpr int kNumBars = 2 * kSlots + 3 * kAccs + kDescBatches + 1 + 2 * kPubRing;
static_assert(kOffB % 1024 == 0 && kBRing % 2048 == 0, "operand-B ring alignment");
static_assert(kASlots >= 2 && 2 * kASlots < kSlots, "operand-A buffers");
// A slot's barriers are reused kSlots items on: a drained B copy (item j - nA - kAProducers up
// to j + kBAhead + kAProducers, nA <= 2 kASlots buffers) must not alias an item of the same slot.
static_assert(2 * kASlots + 2 * kAProducers + kBAhead < kSlots, "slots");
// A copy worker at item j has seen item j - nA - kAProducers consumed; the descriptors it reads
// (up to j + kBAhead) must lie in the batches issued by then.
static_assert(kBAhead + 2 * kASlots + kAProducers + 2 * kDescBatch <= kDescRing, "descriptor ring");
// Operand-A buffers of a pass: kASlots of a whole operand A, or at M = 64 (compact panel rows of
// half the bytes) twice as many in the same space.
__device__ __forceinline__ int a_buffers(int m64) { return m64 ? 2 * kASlots : kASlots; }
__device__ __forceinline__ int a_buffer_bytes(int m64) { return m64 ? kPanelABytes / 2 : kPanelABytes; }
// A BF16x3 pass accumulates hi*[hi; lo] in 2 N columns: two accumulators of 256 columns.
__device__ __forceinline__ int acc_count(bool bf) { return bf ? kAccs / 2 : kAccs; }
__device__ __forceinline__ int acc_cols(bool bf) { return bf ? 2 * kAccCols : kAccCols; }
constexpr int kOffMisc = kOffBars + kNumBars * 8;              // tmem base, abort flag
constexpr int kSmemBytes = kOffMisc + 64 + 1024;               // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory of one CTA");
static_assert(kOffRec % 16 == 0 && kOffBars % 8 == 0, "alignment");

// A chunk's output, handed from the producer to the epilogue.
struct ChunkRec {
  int64_t out;
  int16_t h, n, kind, pad;
};
static_assert(sizeof(ChunkRec) == 16, "ChunkRec layout");

struct Bars {
  uint64_t *full, *empty, *accfull, *accempty, *desc, *recfull, *done, *pubfull, *pubempty;
};
__device__ __forceinline__ Bars bars_of(unsigned char* sm) {
  uint64_t* b = reinterpret_cast<uint64_t*>(sm + kOffBars);
  Bars r;
  r.full = b;
  r.empty = b + kSlots;
  r.accfull = r.empty + kSlots;
  r.accempty = r.accfull + kAccs;
  r.desc = r.accempty + kAccs;
  r.recfull = r.desc + kDescBatches;
  r.done = r.recfull + kAccs;
  r.pubfull = r.done + 1;
  r.pubempty = r.pubfull + kPubRing;
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test of an mbarrier phase (try_wait may hold the thread for a while before it
// returns false).
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false if it ran out or the CTA is aborting.
__device__ bool wait_parity(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31u) == 0) {
      if (*abort_flag) return false;
      if (clock64() - t0 > budget) return false;
    }
  }
}
// Like wait_parity, but ignores the abort flag (used to drain work already in flight).
__device__ void drain(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity) && clock64() - t0 < budget) {
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// TMA bulk copy global -> shared with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(1024 >> 4) << 32) |
         (static_cast<uint64_t>(1) << 46) | (static_cast<uint64_t>(2) << 61);
}
// Shared-memory matrix descriptor: K-major without swizzle, core matrices of 8 rows x 16 bytes,
// `kstep` bytes apart along K (leading-dimension offset) and 128 bytes apart along M (stride
// offset). Checked against a host product for TF32 and BF16 operands.
__device__ __forceinline__ uint64_t plain_desc(uint32_t saddr, uint32_t kstep) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>((kstep >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>(128 >> 4) << 32) | (static_cast<uint64_t>(1) << 46);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ uint32_t tf32_rna(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}


__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Descriptors of items [8 batch, 8 batch + 8) of the CTA's list (from global index i0) into
// their batch of the descriptor ring.
__device__ void issue_desc_batch(const PanelParams& p, int i0, int n, int batch, unsigned char* sm, const Bars& bar) {
  const int first = batch * kDescBatch;
  if (first >= n) return;
  const int cnt = n - first < kDescBatch ? n - first : kDescBatch;
  PanelItem* ring = reinterpret_cast<PanelItem*>(sm + kOffRing);
  uint64_t* b = &bar.desc[batch % kDescBatches];
  mbar_arrive_expect_tx(b, static_cast<uint32_t>(cnt * sizeof(PanelItem)));
  bulk_g2s(ring + (batch % kDescBatches) * kDescBatch, p.items + i0 + first, static_cast<uint32_t>(cnt * sizeof(PanelItem)), b);
}
__device__ __forceinline__ uint64_t* desc_bar(const Bars& bar, int j) { return &bar.desc[(j / kDescBatch) % kDescBatches]; }
__device__ __forceinline__ uint32_t desc_parity(int j) { return static_cast<uint32_t>(j / kDescBatch / kDescBatches) & 1u; }

// Copy worker `a` of kAProducers (one thread each): items j = a, a + kAProducers, ... in order,
// their descriptors read from the ring: copies operand B to its place in the B ring once the
// item named by its room is consumed, running up to kBAhead items ahead; then waits for the
// item's A buffer (item j - nA consumed, nA buffers) and, for runs in Z1 / Z2, the panel complete
// in this pass, and copies the runs. Both copies arrive on the item's full barrier (two
// arrivals, with their bytes).
__device__ void producer_a(const PanelParams& p, int n, int a, unsigned char* sm, const Bars& bar,
                           volatile int* abort_flag) {
  const PanelItem* ring = reinterpret_cast<const PanelItem*>(sm + kOffRing);
  uint64_t keep;  // the panels stay in L2: every item's runs are read again by other items
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  // The operator is streamed once: its lines go first, so the panels stay.
  uint64_t stream_once;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_once));
  uint32_t ready = 0;  // panels Z1 (bit 0), Z2 (bit 1) known complete in this pass
  int j = a;
  bool ok = true;
  int jbq = a;  // this worker's next B copy
  const int na = a_buffers(p.m64), abytes = a_buffer_bytes(p.m64);
  auto copy_b = [&](const PanelItem& ib, int q) {
    const int sb = q % kSlots;
    const uint32_t bytes = static_cast<uint32_t>(panel_tile_bytes(p.mode, ib.n, ib.nrows));
    mbar_arrive_expect_tx(&bar.full[sb], bytes);
    bulk_g2s_hint(sm + kOffB + ib.boff, p.tiles + ib.tile_off, bytes, &bar.full[sb], stream_once);
  };
  // B of this worker's later items whose descriptors have landed and whose room is free (tests,
  // never waits).
  auto look_ahead = [&]() {
    while (jbq < n && jbq <= j + kBAhead && mbar_test(desc_bar(bar, jbq), desc_parity(jbq))) {
      const PanelItem& ib = ring[jbq % kDescRing];
      const int room = ib.room;
      if (room >= 0 && !mbar_test(&bar.empty[room % kSlots], static_cast<uint32_t>(room / kSlots) & 1u)) break;
      copy_b(ib, jbq);
      jbq += kAProducers;
    }
  };
  for (; j < n; j += kAProducers) {
    const int s = j % kSlots;
    if (!wait_parity(desc_bar(bar, j), desc_parity(j), p.timeout_cycles, abort_flag)) {
      ok = false;
      break;
    }
    const PanelItem& it = ring[j % kDescRing];
    if (jbq == j) {  // B of this item
      const int room = it.room;
      if (room >= 0 && !wait_parity(&bar.empty[room % kSlots], static_cast<uint32_t>(room / kSlots) & 1u,
                                    p.timeout_cycles, abort_flag)) {
        ok = false;
        break;
      }
      copy_b(it, j);
      jbq += kAProducers;
    }
    look_ahead();
    if (j >= na && !wait_parity(&bar.empty[(j - na) % kSlots], static_cast<uint32_t>((j - na) / kSlots) & 1u,
                                p.timeout_cycles, abort_flag)) {
      ok = false;
      break;
    }
    const uint32_t deps = static_cast<uint32_t>(it.flags / kPItemDepZ1) & 3u;
    if (deps & ~ready) {
      const long long t0 = clock64();
      for (;;) {
        for (int k = 0; k < 2; ++k)
          if (((deps & ~ready) >> k) & 1u)
            if (ld_acquire_u64(p.done + k) >= p.need[k]) ready |= 1u << k;
        if (!(deps & ~ready)) break;
        if (*abort_flag || clock64() - t0 > p.timeout_cycles) {
          ok = false;
          break;
        }
        __nanosleep(64);
      }
      if (!ok) break;
      fence_proxy_async();  // the acquires above before the bulk copies that read those panels
    }
    unsigned char* dst = sm + kOffA + (j % na) * abytes;
    const uint32_t rb = panel_row_bytes(p.m64);
    mbar_arrive_expect_tx(&bar.full[s], static_cast<uint32_t>(it.nrows) * rb);
    uint32_t row = 0;
    for (int r = 0; r < it.nruns; ++r) {
      const PanelRun run = it.runs[r];
      const unsigned char* src = static_cast<const unsigned char*>(p.src[run.src]);
      bulk_g2s_hint(dst + row * rb, src + static_cast<int64_t>(run.start) * rb, static_cast<uint32_t>(run.len) * rb,
                    &bar.full[s], keep);
      row += static_cast<uint32_t>(run.len);
    }
    look_ahead();
  }
  if (ok) return;
  if (!*abort_flag) {
    atomicOr(p.status, 64u);
    *abort_flag = 1;
  }
  // The copies of this worker still in flight: its items from j - nA - kAProducers (earlier ones
  // are consumed: the previous item's buffer wait) up to jbq. Items from j on have their B copy
  // but no A copy: the missing arrival (without bytes) lets their barrier complete when B lands.
  for (int q = j; q < jbq; q += kAProducers) mbar_arrive(&bar.full[q % kSlots]);
  for (int q = j - na - kAProducers; q < jbq; q += kAProducers)
    if (q >= 0) drain(&bar.full[q % kSlots], static_cast<uint32_t>(q / kSlots) & 1u, p.timeout_cycles);
}

// MMA issuer (one thread): issues the first descriptor batches; per item waits for its operands,
// at a chunk's first item for its accumulator (and writes the chunk's record for the epilogue),
// issues the item's tcgen05.mma instructions and commits them to the barriers that free the
// item's slot (its B bytes and A buffer) and, at a chunk's end, the accumulator; after the last
// item of a descriptor batch, refills that batch of the ring. After the last item an end record
// (kind -1).
__device__ void mma_issuer(const PanelParams& p, int i0, int n, unsigned char* sm, const Bars& bar, uint32_t tmem,
                           volatile int* abort_flag) {
  const PanelItem* ring = reinterpret_cast<const PanelItem*>(sm + kOffRing);
  ChunkRec* recs = reinterpret_cast<ChunkRec*>(sm + kOffRec);
  const uint32_t st_base = smem_u32(sm);
  const bool bf = p.mode == kPanelBF16X3;
  // D FP32; A, B TF32 (2) or BF16 (1); both K-major; M = 128, or 64 for a pass of at most 32
  // right-hand sides (the first 64 operand-A rows, the same layout).
  const uint32_t fmt = bf ? 1u : 2u;
  const uint32_t mdim = p.m64 ? 64u : 128u;
  const uint32_t rb = panel_row_bytes(p.m64);
  const uint32_t idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | ((mdim >> 4) << 24);
  const int na = a_buffers(p.m64), abytes = a_buffer_bytes(p.m64);
  const int nacc = acc_count(bf);
  int batches = 0;  // descriptor batches issued
  for (; batches < kDescBatches && batches * kDescBatch < n; ++batches) issue_desc_batch(p, i0, n, batches, sm, bar);
  int chunks = 0;
  bool issued = false, ok = true;
  auto give_up = [&]() {
    if (!*abort_flag) {
      atomicOr(p.status, 8u);
      *abort_flag = 1;
    }
    ok = false;
  };
  // The accumulator of chunk `k` is free (the epilogue is done with chunk k - nacc); then record.
  auto put_record = [&](int k, const ChunkRec& r) -> bool {
    const int c = k % nacc;
    if (k >= nacc &&
        !wait_parity(&bar.accempty[c], static_cast<uint32_t>(k / nacc - 1) & 1u, p.timeout_cycles, abort_flag))
      return false;
    recs[c] = r;
    mbar_arrive(&bar.recfull[c]);  // release: the record before the epilogue's acquire
    return true;
  };
  for (int j = 0; j < n; ++j) {
    const int s = j % kSlots;
    // (the batch's descriptors land together: one wait per batch)
    if ((j % kDescBatch == 0 && !wait_parity(desc_bar(bar, j), desc_parity(j), p.timeout_cycles, abort_flag)) ||
        !wait_parity(&bar.full[s], static_cast<uint32_t>(j / kSlots) & 1u, p.timeout_cycles, abort_flag)) {
      give_up();
      break;
    }
    const PanelItem& it = ring[j % kDescRing];
    const int nn = it.n, flags = it.flags, nrows = it.nrows;
    const int c = chunks % nacc;
    if (flags & kPItemFirst) {
      if (!put_record(chunks, ChunkRec{it.out, it.h, it.n, it.kind, 0})) {
        give_up();
        break;
      }
      tc_fence_after();  // the epilogue's reads of this accumulator before these MMAs
    }
    const uint32_t d = tmem + static_cast<uint32_t>(c * acc_cols(bf));
    const uint32_t idesc = idesc_base | (static_cast<uint32_t>(nn >> 3) << 17);
    // Descriptors of the item's A buffer and B bytes; a K step moves their start addresses (the
    // low 14 bits, in 16-byte units, which stay within shared memory).
    const uint64_t da = plain_desc(st_base + static_cast<uint32_t>(kOffA + (j % na) * abytes), (bf ? 8u : 4u) * rb);
    const uint64_t db = sw128_desc(st_base + static_cast<uint32_t>(kOffB + it.boff));
    uint32_t acc = (flags & kPItemFirst) ? 0u : 1u;
    if (!bf) {
      // K = 8 per instruction: two 4-row blocks of A (one block, 4 rb bytes, apart); B in 32-value
      // segments.
      for (int k0 = 0; k0 < nrows; k0 += 8) {
        const uint32_t bo = static_cast<uint32_t>((k0 >> 5) * nn * 128 + (k0 & 31) * 4);
        mma_tf32(d, da + ((static_cast<uint32_t>(k0) * rb) >> 4), db + (bo >> 4), idesc, acc);
        acc = 1u;
      }
    } else {
      // K = 16 per instruction: two 8-row blocks of A (8 rb bytes apart, lo plane 4 rb into each).
      // B's hi plane (segment 0) and lo plane (segment 1, n rows on) are one K-major operand of
      // 2 n rows: hi*[hi; lo] into columns [0, 2n), then lo*hi into [0, n); the epilogue adds
      // column n + i to column i (hi*hi + lo*hi + hi*lo).
      const uint32_t idesc2 = idesc_base | (static_cast<uint32_t>(nn >> 2) << 17);
      const uint64_t dalo = da + ((4u * rb) >> 4);
      for (int k0 = 0; k0 < nrows; k0 += 16) {
        const uint64_t ao = (static_cast<uint32_t>(k0) * rb) >> 4, bo = static_cast<uint32_t>(k0 * 2) >> 4;
        mma_bf16(d, da + ao, db + bo, idesc2, acc);
        acc = 1u;
        mma_bf16(d, dalo + ao, db + bo, idesc, 1u);
      }
    }
    issued = true;
    tc_commit(&bar.empty[s]);
    if (flags & kPItemLast) {
      tc_commit(&bar.accfull[c]);
      ++chunks;
    }
    // Done with this batch's ring entries (the copy workers read them before the copies this
    // item waited for): refill them with the batch kDescBatches on.
    if ((j % kDescBatch == kDescBatch - 1) && batches * kDescBatch < n) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_desc_batch(p, i0, n, batches, sm, bar);
      ++batches;
    }
  }
  if (ok && !put_record(chunks, ChunkRec{0, 0, 0, -1, 0})) give_up();
  // Let the descriptor copies already issued land before the CTA can exit.
  for (int b = batches > kDescBatches ? batches - kDescBatches : 0; b < batches; ++b)
    drain(&bar.desc[b % kDescBatches], static_cast<uint32_t>(b / kDescBatches) & 1u, p.timeout_cycles);
  // No MMA may be in flight when the tensor memory is freed.
  if (issued) {
    tc_commit(bar.done);
    drain(bar.done, 0u, p.timeout_cycles);
  }
}

// Every lane of the warp waits (each acquires the phase itself); false for all if any lane ran out.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, long long budget, volatile int* abort_flag) {
  const bool ok = wait_parity(bar, parity, budget, abort_flag);
  return __all_sync(0xffffffffu, ok) != 0;
}

// Epilogue warp (warps 2-9): chunk after chunk until the end record.
__device__ void epilogue(const PanelParams& p, unsigned char* sm, const Bars& bar, uint32_t tmem,
                         volatile int* abort_flag) {
  const ChunkRec* recs = reinterpret_cast<const ChunkRec*>(sm + kOffRec);
  volatile int* pub = reinterpret_cast<volatile int*>(sm + kOffPub);
  int np = 0;  // publications handed to the publisher
  // Hands panel `kind` (or -1: no more) to the publisher as publication np; after this warp's
  // stores (the warp barrier orders its lanes' stores before lane 0's arrive).
  auto publish = [&](int kind) -> bool {
    const int k = np % kPubRing;
    __syncwarp();
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
      if (np >= kPubRing)
        ok = wait_parity(&bar.pubempty[k], static_cast<uint32_t>(np / kPubRing - 1) & 1u, p.timeout_cycles, abort_flag);
      if (ok) {
        pub[k] = kind;
        mbar_arrive(&bar.pubfull[k]);
      } else if (!*abort_flag) {
        atomicOr(p.status, 16u);
        *abort_flag = 1;
      }
    }
    ++np;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
  };
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;            // tensor-memory lane quarter of this warp
  const int hf = (warp - 2) >> 2;    // which column blocks: 16 (2 b + hf) .. + 15
  // Accumulator row = operand-A row of the next phase: lane 32 q + l holds row 32 q + l (M = 128),
  // or row 16 q + l for l < 16 (M = 64; lanes 16-31 of a quarter hold no row).
  const bool live = !p.m64 || lane < 16;
  const int m = p.m64 ? 16 * q + (lane & 15) : 32 * q + lane;
  const int r = m >> 1, part = m & 1;
  const bool bf = p.mode == kPanelBF16X3;
  const int nacc = acc_count(bf);
  const int64_t rb = panel_row_bytes(p.m64);
  for (int k = 0;; ++k) {
    const int c = k % nacc;
    if (!warp_wait(&bar.recfull[c], static_cast<uint32_t>(k / nacc) & 1u, p.timeout_cycles, abort_flag)) {
      if (lane == 0 && !*abort_flag) {
        atomicOr(p.status, 2u);
        *abort_flag = 1;
      }
      return;
    }
    const ChunkRec rec = recs[c];
    if (rec.kind < 0) {
      publish(-1);
      return;
    }
    if (!warp_wait(&bar.accfull[c], static_cast<uint32_t>(k / nacc) & 1u, p.timeout_cycles, abort_flag)) {
      if (lane == 0 && !*abort_flag) {
        atomicOr(p.status, 4u);
        *abort_flag = 1;
      }
      return;
    }
    tc_fence_after();
    const int h = rec.h;
    int pm0 = 0, pm1 = 0;
    if (rec.kind == kPOutY) {
      if (lane < h) pm0 = p.perm[rec.out + lane];
      if (32 + lane < h) pm1 = p.perm[rec.out + 32 + lane];
    }
    const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(c * acc_cols(bf));
    for (int n0 = 16 * hf; n0 < rec.n; n0 += 32) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tbase + static_cast<uint32_t>(n0))
          : "memory");
      if (bf) {  // + hi*lo, n columns on
        uint32_t w[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7]),
              "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
            : "r"(tbase + static_cast<uint32_t>(n0 + rec.n))
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] = __float_as_uint(__uint_as_float(v[e]) + __uint_as_float(w[e]));
      } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
      // Re: D[2r][2i] - D[2r+1][2i+1]; Im: D[2r+1][2i] + D[2r][2i+1] (partner lane m ^ 1).
      float val[8];
#pragma unroll
      for (int ii = 0; ii < 8; ++ii) {
        const float other = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[2 * ii + 1]), 1);
        val[ii] = part ? __uint_as_float(v[2 * ii]) + other : __uint_as_float(v[2 * ii]) - other;
      }
      const int i0 = n0 / 2;  // first output row of these 8 (a multiple of 8)
      if (rec.kind == kPOutY) {
#pragma unroll
        for (int ii = 0; ii < 8; ++ii) {
          const int i = i0 + ii;
          if (i >= h) break;  // uniform over the warp
          const int pi = __shfl_sync(0xffffffffu, i < 32 ? pm0 : pm1, i & 31);
          if (live && r < p.nb)
            static_cast<float*>(p.y)[(static_cast<int64_t>(pi) + static_cast<int64_t>(p.rhs0 + r) * p.ldy) * 2 + part] =
                val[ii];
        }
      } else {
        // The next phase's operand A: blocks of C rows from row out + i0 (out and i0 multiples
        // of C); the zero rows of the accumulator past h complete the last block.
        unsigned char* z = static_cast<unsigned char*>(p.zout[rec.kind]) + (m / 8) * 128 + (m % 8) * 16;
        if (!bf) {
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            const int i = i0 + 4 * g;
            if (live && i < h)
              *reinterpret_cast<uint4*>(z + (rec.out + i) * rb) =
                  make_uint4(tf32_rna(val[4 * g]), tf32_rna(val[4 * g + 1]), tf32_rna(val[4 * g + 2]),
                             tf32_rna(val[4 * g + 3]));
          }
        } else if (i0 < h) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = make_float2(val[2 * e], val[2 * e + 1]);
            const __nv_bfloat162 hv = __float22bfloat162_rn(f);
            const float2 hf2 = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __float22bfloat162_rn(make_float2(f.x - hf2.x, f.y - hf2.y));
            hi[e] = *reinterpret_cast<const uint32_t*>(&hv);
            lo[e] = *reinterpret_cast<const uint32_t*>(&lv);
          }
          unsigned char* d = z + (rec.out + i0) * rb;
          if (live) {
            *reinterpret_cast<uint4*>(d) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(d + 4 * rb) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&bar.accempty[c]);  // the accumulator and the record are free
    if (rec.kind != kPOutY && !publish(rec.kind)) return;
  }
}

// Publisher (one thread): one release per Z1 / Z2 chunk, until the epilogue hands over -1.
__device__ void publisher(const PanelParams& p, unsigned char* sm, const Bars& bar, volatile int* abort_flag) {
  const volatile int* pub = reinterpret_cast<const volatile int*>(sm + kOffPub);
  for (int j = 0;; ++j) {
    const int k = j % kPubRing;
    if (!wait_parity(&bar.pubfull[k], static_cast<uint32_t>(j / kPubRing) & 1u, p.timeout_cycles, abort_flag)) {
      if (!*abort_flag) {
        atomicOr(p.status, 32u);
        *abort_flag = 1;
      }
      return;
    }
    const int kind = pub[k];
    mbar_arrive(&bar.pubempty[k]);
    if (kind < 0) return;
    // the epilogue warps' stores happen before their arrives, which this thread has acquired;
    // the release makes them visible to every CTA that acquires the counter
    red_release_add(p.done + kind, 1ull);
  }
}

__global__ void __launch_bounds__(kThreads, 1) panel_kernel(const PanelParams p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const Bars bar = bars_of(sm);
  volatile int* misc = reinterpret_cast<volatile int*>(sm + kOffMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 32);
  volatile int* abort_flag = misc;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&bar.full[s], 2);  // operand B and operand A
      mbar_init(&bar.empty[s], 1);  // MMA commit: both operands read
    }
    for (int q = 0; q < kAccs; ++q) {
      mbar_init(&bar.accfull[q], 1);
      mbar_init(&bar.accempty[q], kEpiWarps);
      mbar_init(&bar.recfull[q], 1);
    }
    for (int q = 0; q < kDescBatches; ++q) mbar_init(&bar.desc[q], 1);
    mbar_init(bar.done, 1);
    for (int q = 0; q < kPubRing; ++q) {
      mbar_init(&bar.pubfull[q], kEpiWarps);
      mbar_init(&bar.pubempty[q], 1);
    }
    for (int q = 0; q < 4; ++q) misc[q] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int i0 = p.cta_begin[blockIdx.x], n = p.cta_begin[blockIdx.x + 1] - i0;
  if (warp == 0) {
    // no role: the operand placement is precomputed by the packer
  } else if (warp == 1) {
    if (threadIdx.x == 32) mma_issuer(p, i0, n, sm, bar, tmem, abort_flag);
  } else if (warp < 2 + kEpiWarps) {
    epilogue(p, sm, bar, tmem, abort_flag);
  } else if (warp == 2 + kEpiWarps) {
    if (threadIdx.x == 32 * (2 + kEpiWarps)) publisher(p, sm, bar, abort_flag);
  } else if ((threadIdx.x & 31) == 0) {
    producer_a(p, n, warp - 3 - kEpiWarps, sm, bar, abort_flag);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// X (complex64, column-major) -> XP in operand-A layout: one thread per (block g, A row m),
// 2 blocks per 256 threads; rows >= n and right-hand sides >= nb are zero.
template <bool BF>
__global__ void gather_kernel(const float2* __restrict__ x, int64_t ldx, int64_t n, int64_t rows,
                              const int32_t* __restrict__ perm, int32_t rhs0, int32_t nb, int32_t m64,
                              unsigned char* __restrict__ xp) {
  constexpr int C = BF ? 8 : 4;
  const int64_t g = static_cast<int64_t>(blockIdx.x) * 2 + (threadIdx.x >> 7);
  const int m = threadIdx.x & 127;
  if (g * C >= rows || (m64 && m >= 64)) return;  // M = 64: the compact layout holds rows 0-63
  const int64_t rb = panel_row_bytes(m64);
  const int r = m >> 1, part = m & 1;
  float v[C];
#pragma unroll
  for (int t = 0; t < C; ++t) {
    const int64_t j = g * C + t;
    float f = 0.0f;
    if (j < n && r < nb) {
      const float2 z = x[perm[j] + static_cast<int64_t>(rhs0 + r) * ldx];
      f = part ? z.y : z.x;
    }
    v[t] = f;
  }
  unsigned char* d = xp + g * C * rb + (m / 8) * 128 + (m % 8) * 16;
  if (!BF) {
    *reinterpret_cast<uint4*>(d) = make_uint4(tf32_rna(v[0]), tf32_rna(v[1]), tf32_rna(v[2]), tf32_rna(v[3]));
  } else {
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = make_float2(v[2 * e], v[2 * e + 1]);
      const __nv_bfloat162 hv = __float22bfloat162_rn(f);
      const float2 hf2 = __bfloat1622float2(hv);
      const __nv_bfloat162 lv = __float22bfloat162_rn(make_float2(f.x - hf2.x, f.y - hf2.y));
      hi[e] = *reinterpret_cast<const uint32_t*>(&hv);
      lo[e] = *reinterpret_cast<const uint32_t*>(&lv);
    }
    *reinterpret_cast<uint4*>(d) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(d + 4 * rb) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

}  // namespace

int panel_gather(const void* x, int64_t ldx, int64_t n, int64_t rows, const int32_t* perm, int32_t rhs0, int32_t nb,
                 int32_t mode, int32_t m64, void* xp, void* stream) {
  const int C = panel_block_rows(mode);
  const int64_t blocks = (rows / C + 1) / 2;
  if (blocks > 0) {
    if (mode == kPanelBF16X3)
      gather_kernel<true><<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
          static_cast<const float2*>(x), ldx, n, rows, perm, rhs0, nb, m64, static_cast<unsigned char*>(xp));
    else
      gather_kernel<false><<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
          static_cast<const float2*>(x), ldx, n, rows, perm, rhs0, nb, m64, static_cast<unsigned char*>(xp));
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel gather launch: %s", cudaGetErrorString(e));
}

int panel_prepare() {
  const cudaError_t e = cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel kernel attributes: %s", cudaGetErrorString(e));
}

int panel_launch(const PanelParams& p, int grid, void* stream) {
  void* args[] = {const_cast<PanelParams*>(&p)};
  const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(panel_kernel), dim3(grid),
                                                    dim3(kThreads), args, kSmemBytes, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel kernel launch: %s", cudaGetErrorString(e));
}

}  // namespace uh

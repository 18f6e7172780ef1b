// Tensor-core multi-RHS product (sm_103a): one phase of a pass per launch, one CTA per SM.
// Layout of the work and of the operands: uh_panel.h.
//
// Roles in a CTA of 320 threads:
//  - producer (lane 0 of warp 0): streams the CTA's item descriptors into a shared-memory ring
//    (TMA bulk copies of 8); per item waits for a free stage, copies the descriptor into the
//    stage's slot, and copies the item's B operand (one bulk copy) and its panel rows (one bulk
//    copy per run) into the stage.
//  - MMA issuer (lane 0 of warp 1; warp 1 also allocates and frees the tensor memory): per item
//    waits for the converted A operand, issues the item's tcgen05.mma instructions into the
//    chunk's accumulator (two accumulators of 128 columns alternate between chunks) and commits
//    them to the barriers that free the stage and, at a chunk's end, the accumulator for the
//    epilogue.
//  - converters (warps 2-9; thread = one A-operand row x one half of K): per item read the
//    staged panel rows into registers and overwrite them with operand A (TF32 rounding, or a
//    BF16 hi/lo split) in the swizzled K-major layout, so a stage holds the item's two operands
//    and nothing else; after the first item of the next chunk has been handed to the MMA
//    issuer, read the finished accumulator (tcgen05.ld; each warp its 32-lane quarter and half
//    of the column blocks), combine the real products into complex outputs and write them.
// Every wait is bounded (timeout_cycles); when one runs out the CTA records it in `status`, stops,
// lets its copies and MMAs in flight finish, frees the tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "uh.h"
#include "uh_internal.h"
#include "uh_panel.h"

namespace uh {
namespace {

constexpr int kThreads = 320;
constexpr int kConverters = 256;
constexpr int kDescBatch = 8;
constexpr int kDescRing = 2 * kDescBatch;
constexpr int kAccCols = 128;          // one accumulator: N <= 128 FP32 columns
constexpr uint32_t kTmemCols = 2 * kAccCols;

// Shared memory (bytes from a 1024-aligned base).
constexpr int kStageTile = 0;                                   // B operand
constexpr int kStagePanel = kPanelTileMax;                      // staged panel rows, then operand A
constexpr int kStageBytes = kPanelTileMax + kPanelRawMax;       // 64 KB
static_assert(kPanelRawMax == kPanelABytes, "operand A replaces the staged panel rows");
constexpr int kOffSlots = kPanelStages * kStageBytes;           // item descriptor per stage
constexpr int kOffRing = kOffSlots + kPanelStages * 96;         // descriptor ring
constexpr int kOffBars = kOffRing + kDescRing * 96;
// barriers: full[S], empty[S], afull[S], accfull[2], accempty[2], desc[2], done
constexpr int kNumBars = 3 * kPanelStages + 2 + 2 + 2 + 1;
constexpr int kOffMisc = kOffBars + kNumBars * 8;              // tmem base, abort, go words
constexpr int kSmemBytes = kOffMisc + 64 + 1024;               // + alignment slack
static_assert(kSmemBytes <= 227 * 1024, "shared memory of one CTA");
struct Bars {
  uint64_t *full, *empty, *afull, *accfull, *accempty, *desc, *done;
};
__device__ __forceinline__ Bars bars_of(unsigned char* sm) {
  uint64_t* b = reinterpret_cast<uint64_t*>(sm + kOffBars);
  Bars r;
  r.full = b;
  r.empty = b + kPanelStages;
  r.afull = b + 2 * kPanelStages;
  r.accfull = r.afull + kPanelStages;
  r.accempty = r.accfull + 2;
  r.desc = r.accempty + 2;
  r.done = r.desc + 2;
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
__device__ __forceinline__ void converters_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kConverters) : "memory");
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

// Producer: descriptors into the ring, per item the descriptor into the stage slot and the
// operand B and panel rows into the stage.
__device__ void producer(const PanelParams& p, int i0, int n, unsigned char* sm, const Bars& bar,
                         volatile int* abort_flag) {
  PanelItem* ring = reinterpret_cast<PanelItem*>(sm + kOffRing);
  PanelItem* slots = reinterpret_cast<PanelItem*>(sm + kOffSlots);
  auto issue_batch = [&](int batch) {
    const int first = batch * kDescBatch;
    if (first >= n) return;
    const int cnt = n - first < kDescBatch ? n - first : kDescBatch;
    uint64_t* b = &bar.desc[batch & 1];
    mbar_arrive_expect_tx(b, static_cast<uint32_t>(cnt * sizeof(PanelItem)));
    bulk_g2s(ring + (batch & 1) * kDescBatch, p.items + i0 + first, static_cast<uint32_t>(cnt * sizeof(PanelItem)), b);
  };
  issue_batch(0);
  issue_batch(1);
  // The operator is streamed once: its lines go first, so the panels (read by many items) stay.
  uint64_t stream_once, keep;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_once));
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
  int j = 0;
  bool ok = true;
  for (; j < n; ++j) {
    const int batch = j / kDescBatch;
    if (j % kDescBatch == 0 &&
        !wait_parity(&bar.desc[batch & 1], static_cast<uint32_t>(batch >> 1) & 1u, p.timeout_cycles, abort_flag)) {
      ok = false;
      break;
    }
    const int s = j % kPanelStages;
    if (j >= kPanelStages &&
        !wait_parity(&bar.empty[s], static_cast<uint32_t>(j / kPanelStages - 1) & 1u, p.timeout_cycles, abort_flag)) {
      ok = false;
      break;
    }
    const PanelItem& it = ring[j % kDescRing];
    // Descriptor into the stage slot (generic stores, published by the arrive below).
    const uint4* from = reinterpret_cast<const uint4*>(&it);
    uint4* to = reinterpret_cast<uint4*>(slots + s);
#pragma unroll
    for (int w = 0; w < 6; ++w) to[w] = from[w];
    unsigned char* st = sm + s * kStageBytes;
    const uint32_t tile_bytes = 256u * static_cast<uint32_t>(it.n);
    mbar_arrive_expect_tx(&bar.full[s], tile_bytes + static_cast<uint32_t>(it.nrows) * kPanelRowBytes);
    bulk_g2s_hint(st + kStageTile, p.tiles + it.tile_off, tile_bytes, &bar.full[s], stream_once);
    uint32_t row = 0;
    for (int r = 0; r < it.nruns; ++r) {
      const PanelRun run = it.runs[r];
      const unsigned char* src = static_cast<const unsigned char*>(p.src[run.src]);
      bulk_g2s_hint(st + kStagePanel + row * kPanelRowBytes, src + static_cast<int64_t>(run.start) * kPanelRowBytes,
                    static_cast<uint32_t>(run.len) * kPanelRowBytes, &bar.full[s], keep);
      row += static_cast<uint32_t>(run.len);
    }
    if (j % kDescBatch == kDescBatch - 1) {
      // Done with this batch's ring entries (read through the generic proxy): refill them.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_batch(batch + 2);
    }
  }
  if (!ok) {
    if (!*abort_flag) {
      atomicOr(p.status, 1u);
      *abort_flag = 1;
    }
    // Let the copies already issued land before the CTA can exit.
    for (int q = (j >= kPanelStages ? j - kPanelStages + 1 : 0); q < j && q < n; ++q)
      drain(&bar.full[q % kPanelStages], static_cast<uint32_t>(q / kPanelStages) & 1u, p.timeout_cycles);
    const int b0 = j / kDescBatch;
    for (int b = b0; b < b0 + 2 && b * kDescBatch < n; ++b)
      drain(&bar.desc[b & 1], static_cast<uint32_t>(b >> 1) & 1u, p.timeout_cycles);
  }
}

// MMA issuer (one thread).
__device__ void mma_issuer(const PanelParams& p, int n, unsigned char* sm, const Bars& bar, uint32_t tmem,
                           volatile int* abort_flag) {
  const PanelItem* slots = reinterpret_cast<const PanelItem*>(sm + kOffSlots);
  const uint32_t st_base = smem_u32(sm);
  const bool bf = p.mode == kPanelBF16X3;
  // D FP32; A, B TF32 (2) or BF16 (1); both K-major; M = 128.
  const uint32_t fmt = bf ? 1u : 2u;
  const uint32_t idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(128 >> 4) << 24);
  int chunks = 0;
  bool issued = false;
  auto give_up = [&]() {
    if (!*abort_flag) {
      atomicOr(p.status, 8u);
      *abort_flag = 1;
    }
  };
  for (int j = 0; j < n; ++j) {
    const int s = j % kPanelStages;
    if (!wait_parity(&bar.afull[s], static_cast<uint32_t>(j / kPanelStages) & 1u, p.timeout_cycles, abort_flag) ||
        !wait_parity(&bar.full[s], static_cast<uint32_t>(j / kPanelStages) & 1u, p.timeout_cycles, abort_flag)) {
      give_up();
      break;
    }
    const PanelItem& it = slots[s];
    const int nn = it.n, flags = it.flags;
    const int c = chunks & 1;
    if ((flags & kPItemFirst) && chunks >= 2 &&
        !wait_parity(&bar.accempty[c], static_cast<uint32_t>((chunks >> 1) - 1) & 1u, p.timeout_cycles, abort_flag)) {
      give_up();
      break;
    }
    tc_fence_after();
    const uint32_t d = tmem + static_cast<uint32_t>(c * kAccCols);
    const uint32_t idesc = idesc_base | (static_cast<uint32_t>(nn >> 3) << 17);
    const uint32_t A = st_base + static_cast<uint32_t>(s * kStageBytes + kStagePanel);
    const uint32_t B = st_base + static_cast<uint32_t>(s * kStageBytes + kStageTile);
    uint32_t acc = (flags & kPItemFirst) ? 0u : 1u;
    if (!bf) {
      // K = 8 per instruction: 32-byte steps inside a 128-byte segment (32 TF32 values).
#pragma unroll
      for (int k0 = 0; k0 < kPanelK; k0 += 8) {
        const uint32_t ao = static_cast<uint32_t>((k0 / 32) * 128 * 128 + (k0 % 32) * 4);
        const uint32_t bo = static_cast<uint32_t>((k0 / 32) * nn * 128 + (k0 % 32) * 4);
        mma_tf32(d, sw128_desc(A + ao), sw128_desc(B + bo), idesc, acc);
        acc = 1u;
      }
    } else {
      // K = 16 per instruction; hi and lo planes: hi*hi + hi*lo + lo*hi.
      const uint32_t alo = 128u * 128u, blo = static_cast<uint32_t>(nn) * 128u;
#pragma unroll
      for (int k0 = 0; k0 < kPanelK; k0 += 16) {
        const uint32_t o = static_cast<uint32_t>(k0 * 2);
        mma_bf16(d, sw128_desc(A + o), sw128_desc(B + o), idesc, acc);
        acc = 1u;
        mma_bf16(d, sw128_desc(A + o), sw128_desc(B + blo + o), idesc, 1u);
        mma_bf16(d, sw128_desc(A + alo + o), sw128_desc(B + o), idesc, 1u);
      }
    }
    issued = true;
    tc_commit(&bar.empty[s]);
    if (flags & kPItemLast) {
      tc_commit(&bar.accfull[c]);
      ++chunks;
    }
  }
  // No MMA may be in flight when the tensor memory is freed.
  if (issued) {
    tc_commit(bar.done);
    drain(bar.done, 0u, p.timeout_cycles);
  }
}

template <bool BF>
__device__ __forceinline__ void convert_item(unsigned char* panel, int nrows, int t) {
  // Thread t builds half `hf` of row m of A: A[m][k] = component (m & 1) of right-hand side m / 2
  // in panel row k, i.e. raw[k * 2 kPanelR + m], for k in [32 hf, 32 hf + 32); rows k >= nrows
  // are zero. A replaces the staged rows in place: every thread reads its values before any
  // thread writes.
  const int m = t & 127, hf = t >> 7;
  const float* raw = reinterpret_cast<const float*>(panel);
  constexpr int kH = kPanelK / 2;
  float v[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) {
    const int kk = hf * kH + k;
    v[k] = kk < nrows ? raw[kk * 2 * kPanelR + m] : 0.0f;
  }
  converters_sync();
  unsigned char* rowbase = panel + (m / 8) * 1024 + (m % 8) * 128;
  if (!BF) {
    // 32 TF32 values = one 128-byte segment (segment hf).
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      unsigned char* dst = rowbase + hf * (128 * 128) + ((c ^ (m % 8)) * 16);
      *reinterpret_cast<uint4*>(dst) =
          make_uint4(tf32_rna(v[4 * c]), tf32_rna(v[4 * c + 1]), tf32_rna(v[4 * c + 2]), tf32_rna(v[4 * c + 3]));
    }
  } else {
    // 32 BF16 values = 16-byte chunks 4 hf .. 4 hf + 3 of the hi and lo planes.
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = make_float2(v[8 * c + 2 * e], v[8 * c + 2 * e + 1]);
        const __nv_bfloat162 h = __float22bfloat162_rn(f);
        const float2 hf2 = __bfloat1622float2(h);
        const __nv_bfloat162 l = __float22bfloat162_rn(make_float2(f.x - hf2.x, f.y - hf2.y));
        hi[e] = *reinterpret_cast<const uint32_t*>(&h);
        lo[e] = *reinterpret_cast<const uint32_t*>(&l);
      }
      unsigned char* dst = rowbase + (((4 * hf + c) ^ (m % 8)) * 16);
      *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(dst + 128 * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
}

struct Pending {
  int64_t out;
  int h, n, kind, c, use;
};

// Epilogue of one chunk by the 128 converter threads; false when aborting.
__device__ bool epilogue(const PanelParams& p, const Pending& ch, const Bars& bar, uint32_t tmem,
                         volatile int* abort_flag, volatile int* go, int t) {
  if (t == 0) {
    const bool ok = wait_parity(&bar.accfull[ch.c], static_cast<uint32_t>(ch.use) & 1u, p.timeout_cycles, abort_flag);
    if (!ok && !*abort_flag) {
      atomicOr(p.status, 2u);
      *abort_flag = 1;
    }
    go[2] = ok ? 1 : 0;
  }
  converters_sync();
  if (!go[2]) return false;
  tc_fence_after();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;            // tensor-memory lane quarter of this warp
  const int hf = (warp - 2) >> 2;    // which column blocks: 16 (2 b + hf) .. + 15
  const int m = 32 * q + lane;       // accumulator row
  const int r = m >> 1, part = m & 1;
  int pm0 = 0, pm1 = 0;
  if (ch.kind == kPOutY) {
    if (lane < ch.h) pm0 = p.perm[ch.out + lane];
    if (32 + lane < ch.h) pm1 = p.perm[ch.out + 32 + lane];
  }
  const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(ch.c * kAccCols);
  for (int n0 = 16 * hf; n0 < ch.n; n0 += 32) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(tbase + static_cast<uint32_t>(n0))
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int ii = 0; ii < 8; ++ii) {
      const int i = n0 / 2 + ii;
      if (i >= ch.h) break;  // uniform over the warp
      // Re: D[2r][2i] - D[2r+1][2i+1]; Im: D[2r+1][2i] + D[2r][2i+1] (partner lane m ^ 1).
      const float other = __shfl_xor_sync(0xffffffffu, __uint_as_float(v[2 * ii + 1]), 1);
      const float val = part ? __uint_as_float(v[2 * ii]) + other : __uint_as_float(v[2 * ii]) - other;
      if (ch.kind == kPOutY) {
        const int pi = __shfl_sync(0xffffffffu, i < 32 ? pm0 : pm1, i & 31);
        if (r < p.nb)
          static_cast<float*>(p.y)[(static_cast<int64_t>(pi) + static_cast<int64_t>(p.rhs0 + r) * p.ldy) * 2 + part] = val;
      } else {
        float* z = static_cast<float*>(p.zout[ch.kind]);
        z[(ch.out + i) * (2 * kPanelR) + m] = val;
      }
    }
  }
  tc_fence_before();
  converters_sync();
  if (t == 0) mbar_arrive(&bar.accempty[ch.c]);
  return true;
}

template <bool BF>
__device__ void converters(const PanelParams& p, int n, unsigned char* sm, const Bars& bar, uint32_t tmem,
                           volatile int* abort_flag, volatile int* go) {
  const int t = threadIdx.x - 64;  // 0 .. 255
  const PanelItem* slots = reinterpret_cast<const PanelItem*>(sm + kOffSlots);
  Pending pend{};
  bool pending = false;
  int chunks = 0;
  for (int j = 0; j < n; ++j) {
    const int s = j % kPanelStages;
    if (t == 0) {
      const bool ok = wait_parity(&bar.full[s], static_cast<uint32_t>(j / kPanelStages) & 1u, p.timeout_cycles, abort_flag);
      if (!ok && !*abort_flag) {
        atomicOr(p.status, 4u);
        *abort_flag = 1;
      }
      go[j & 1] = ok ? 1 : 0;
    }
    converters_sync();
    if (!go[j & 1]) return;
    // Everything needed from the stage slot, before the stage is released below.
    const PanelItem& it = slots[s];
    const int nrows = it.nrows, flags = it.flags;
    const Pending mine{it.out, it.h, it.n, it.kind, chunks & 1, chunks >> 1};
    convert_item<BF>(sm + s * kStageBytes + kStagePanel, nrows, t);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A writes before the MMA reads them
    converters_sync();
    if (t == 0) mbar_arrive(&bar.afull[s]);
    if ((flags & kPItemFirst) && pending) {
      if (!epilogue(p, pend, bar, tmem, abort_flag, go, t)) return;
      pending = false;
    }
    if (flags & kPItemLast) {
      pend = mine;
      pending = true;
      ++chunks;
    }
  }
  if (pending) epilogue(p, pend, bar, tmem, abort_flag, go, t);
}

__global__ void __launch_bounds__(kThreads, 1) panel_kernel(const PanelParams p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sm = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const Bars bar = bars_of(sm);
  volatile int* misc = reinterpret_cast<volatile int*>(sm + kOffMisc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 32);
  volatile int* abort_flag = misc;
  volatile int* go = misc + 1;  // go[0], go[1] by item parity, go[2] for epilogues
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPanelStages; ++s) {
      mbar_init(&bar.full[s], 1);
      mbar_init(&bar.empty[s], 1);  // MMA commit: both operands read
      mbar_init(&bar.afull[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bar.accfull[q], 1);
      mbar_init(&bar.accempty[q], 1);
      mbar_init(&bar.desc[q], 1);
    }
    mbar_init(bar.done, 1);
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
    if (threadIdx.x == 0) producer(p, i0, n, sm, bar, abort_flag);
  } else if (warp == 1) {
    if (threadIdx.x == 32) mma_issuer(p, n, sm, bar, tmem, abort_flag);
  } else if (p.mode == kPanelBF16X3) {
    converters<true>(p, n, sm, bar, tmem, abort_flag, go);
  } else {
    converters<false>(p, n, sm, bar, tmem, abort_flag, go);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

__global__ void gather_kernel(const float2* __restrict__ x, int64_t ldx, int64_t n, const int32_t* __restrict__ perm,
                              int32_t rhs0, int32_t nb, float2* __restrict__ xp) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * 4 + threadIdx.x / kPanelR;
  const int r = threadIdx.x % kPanelR;
  if (i >= n) return;
  xp[i * kPanelR + r] = r < nb ? x[perm[i] + static_cast<int64_t>(rhs0 + r) * ldx] : make_float2(0.f, 0.f);
}

}  // namespace

int panel_gather(const void* x, int64_t ldx, int64_t n, const int32_t* perm, int32_t rhs0, int32_t nb, void* xp,
                 void* stream) {
  const int64_t blocks = (n + 3) / 4;
  gather_kernel<<<static_cast<unsigned>(blocks), 4 * kPanelR, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float2*>(x), ldx, n, perm, rhs0, nb, static_cast<float2*>(xp));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel gather launch: %s", cudaGetErrorString(e));
}

int panel_prepare() {
  const cudaError_t e = cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel kernel attributes: %s", cudaGetErrorString(e));
}

int panel_launch(const PanelParams& p, int grid, void* stream) {
  panel_kernel<<<grid, kThreads, kSmemBytes, static_cast<cudaStream_t>(stream)>>>(p);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : set_error(UH_ECUDA, "panel kernel launch: %s", cudaGetErrorString(e));
}

}  // namespace uh

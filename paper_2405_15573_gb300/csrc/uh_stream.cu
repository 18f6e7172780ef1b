// Streaming matvec kernel (sm_103a): one persistent launch per UH or H matrix-vector product.
// Layout of the work and the dependency rules: uh_stream.h.
//
// Roles in a CTA of 320 threads:
//  - producer (lane 0 of warp 8): streams the CTA's item descriptors into a shared-memory ring
//    (its static list in batches, then pool tickets, in segments); per item waits
//    for its stage to be free, arms the stage's full barrier with the byte count, copies the tile
//    with one TMA bulk copy and, once every group the item's runs read from is complete (checked
//    once per group and call, then remembered), each input run with one more bulk copy into the
//    stage's input area. After its last item it marks the next ring slot as the end.
//  - consumers (warps 0-7): first gather the CTA's slice of x into cluster order and release the
//    permutation counter; then per item, wait for the stage, multiply the tile by the staged inputs
//    into per-thread accumulators (thread = 16-byte row slice x column group), release the
//    stage; at the end of a chunk reduce the column groups in a fixed tree order, add the staged
//    near-field partial if the chunk has one, write the outputs and, for chunks other CTAs wait on,
//    hand the group counter to the publisher (each warp arrives after its own stores).
//  - publisher (lane 0 of warp 9): per handed-over chunk, red.release on its group counter.
// Every wait is bounded (timeout_cycles); when one runs out the CTA records it in `status`,
// stops issuing, lets the copies in flight land, and returns.
#include <cuda_runtime.h>

#include "uh_internal.h"
#include "uh_stream.h"

namespace uh {
namespace {

// Variants (uh_stream.h): TM = tile element, TV = element of the intermediate vectors, of the
// staged inputs and of the accumulators, TX = element of x and y, L = shared-memory layout.
// kMinBlocks: CTAs per SM the variant is compiled for; R: right-hand sides of one product.
struct KC64 {
  using TM = float2;
  using TV = float2;
  using TX = float2;
  using L = StreamSmemStd;
  static constexpr int kMinBlocks = 1;
  static constexpr int R = 1;
};
struct KC128 {
  using TM = double2;
  using TV = double2;
  using TX = double2;
  using L = StreamSmemStd;
  static constexpr int kMinBlocks = 1;
  static constexpr int R = 1;
};
// TV = (re_hi, im_hi, re_lo, im_lo): the value re_hi + re_lo + i (im_hi + im_lo).
struct KMixed {
  using TM = float2;
  using TV = float4;
  using TX = double2;
  using L = StreamSmemMixed;
  static constexpr int kMinBlocks = 1;
  static constexpr int R = 1;
};
// Several right-hand sides of one complex64 program in one pass over the operator.
struct KC64R2 : KC64 {
  using L = StreamSmemR2;
  static constexpr int R = 2;
};
struct KC64R4 : KC64 {
  using L = StreamSmemR4;
  static constexpr int R = 4;
};
// The same with two CTAs per SM (programs packed for kGeomDual).
struct KC64Dual : KC64 {
  using L = StreamSmemDual;
  static constexpr int kMinBlocks = 2;
};
struct KMixedDual : KMixed {
  using L = StreamSmemMixedDual;
  static constexpr int kMinBlocks = 2;
};
struct KC128Dual : KC128 {
  using L = StreamSmemDual;
  static constexpr int kMinBlocks = 2;
};
struct KC64DualR2 : KC64Dual {
  using L = StreamSmemDualR2;
  static constexpr int R = 2;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// TMA bulk copy global -> shared, completion counted on `bar` (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same with an L2 eviction policy (createpolicy) for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kStreamConsumers) : "memory");
}

__device__ __forceinline__ void cfma(float2& a, float2 m, float2 v) {
  a.x = fmaf(m.x, v.x, fmaf(-m.y, v.y, a.x));
  a.y = fmaf(m.x, v.y, fmaf(m.y, v.x, a.y));
}
__device__ __forceinline__ void cfma(double2& a, double2 m, double2 v) {
  a.x = fma(m.x, v.x, fma(-m.y, v.y, a.x));
  a.y = fma(m.x, v.y, fma(m.y, v.x, a.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Extended precision from FP32 pairs. The round-to-nearest intrinsics keep the compiler from
// contracting a product and a sum into one fma, which would break the error-free transforms.
// (h, l) += p + pl, where p is a rounded value and pl a small correction: Knuth's two-sum gives
// the exact rounding error e of h + p, and the correction and e are added to the low word.
__device__ __forceinline__ void ff_acc(float& h, float& l, float p, float pl) {
  const float s = __fadd_rn(h, p);
  const float z = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(p, z));
  h = s;
  l = __fadd_rn(l, __fadd_rn(e, pl));
}
// a += m * v, m a complex64 tile element, v and a extended: each of the four real products
// m_i * v_hi is split exactly into its rounded value and error (fma), and m_i * v_lo joins the error.
__device__ __forceinline__ void cfma(float4& a, float2 m, float4 v) {
  float p = __fmul_rn(m.x, v.x);
  ff_acc(a.x, a.z, p, fmaf(m.x, v.z, fmaf(m.x, v.x, -p)));
  const float my = -m.y;
  p = __fmul_rn(my, v.y);
  ff_acc(a.x, a.z, p, fmaf(my, v.w, fmaf(my, v.y, -p)));
  p = __fmul_rn(m.x, v.y);
  ff_acc(a.y, a.w, p, fmaf(m.x, v.w, fmaf(m.x, v.y, -p)));
  p = __fmul_rn(m.y, v.x);
  ff_acc(a.y, a.w, p, fmaf(m.y, v.z, fmaf(m.y, v.x, -p)));
}
// (h, l) normalised: h = round(h + l), l the exact rest.
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}
__device__ __forceinline__ float4 cadd(float4 a, float4 b) {
  ff_acc(a.x, a.z, b.x, b.z);
  ff_acc(a.y, a.w, b.y, b.w);
  ff_norm(a.x, a.z);
  ff_norm(a.y, a.w);
  return a;
}
// Conversions between the x / y element and the vector element.
__device__ __forceinline__ float2 to_v(float2 a, float2*) { return a; }
__device__ __forceinline__ double2 to_v(double2 a, double2*) { return a; }
__device__ __forceinline__ float4 to_v(double2 a, float4*) {
  const float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
  return make_float4(rh, ih, __double2float_rn(a.x - static_cast<double>(rh)),
                     __double2float_rn(a.y - static_cast<double>(ih)));
}
__device__ __forceinline__ float2 to_x(float2 a, float2*) { return a; }
__device__ __forceinline__ double2 to_x(double2 a, double2*) { return a; }
__device__ __forceinline__ double2 to_x(float4 a, double2*) {
  return make_double2(static_cast<double>(a.x) + static_cast<double>(a.z),
                      static_cast<double>(a.y) + static_cast<double>(a.w));
}

__device__ __forceinline__ float2 shfl_xor(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int m) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}
__device__ __forceinline__ float4 shfl_xor(float4 v, int m) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m),
                     __shfl_xor_sync(0xffffffffu, v.z, m), __shfl_xor_sync(0xffffffffu, v.w, m));
}

__device__ __forceinline__ void lds16(const float2* p, float2 (&m)[2]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  m[0] = make_float2(q.x, q.y);
  m[1] = make_float2(q.z, q.w);
}
__device__ __forceinline__ void lds16(const double2* p, double2 (&m)[1]) { m[0] = *p; }

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

__device__ __forceinline__ const void* src_ptr(const StreamParams& p, int src) {
  return src == kSrcXp ? p.xp : src == kSrcZ1 ? p.z1 : src == kSrcZ2 ? p.z2 : src == kSrcZ3 ? p.z3 : p.z4;
}

struct Bars {
  uint64_t* full;       // tile and runs landed (1 arrival + their bytes)
  uint64_t* empty;      // stage consumed (one arrival per consumer warp)
  uint64_t* desc;       // descriptor batch landed
  uint64_t* pub_full;   // a finished chunk's outputs stored (one arrival per consumer warp)
  uint64_t* pub_empty;  // the publisher has taken the slot (1 arrival)
  uint64_t* pool;       // pool descriptor segment landed [2] (1 arrival + bytes)
};
template <class L>
__device__ __forceinline__ Bars bars_of(unsigned char* smem) {
  uint64_t* b = reinterpret_cast<uint64_t*>(smem + L::bars);
  uint64_t* q = b + 2 * L::stages + kDescBatches;
  return Bars{b, b + L::stages, b + 2 * L::stages, q, q + kPubRing, q + 2 * kPubRing};
}

// Consumers: hand counter `counter` (index in group_done, or -1: no more) to the publisher as
// release number `np`. Each warp arrives after its own stores (the warp barrier orders its lanes' stores before
// lane 0's arrive); thread 0 writes the counter first. Called by whole warps; false when aborting.
__device__ __forceinline__ bool publish(const Bars& bar, int* pub_ctr, int np, int counter, const StreamParams& p,
                                        volatile int* abort_flag) {
  const int k = np % kPubRing;
  __syncwarp();
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if (np >= kPubRing)
      ok = wait_parity(&bar.pub_empty[k], static_cast<uint32_t>(np / kPubRing - 1) & 1u, p.timeout_cycles, abort_flag);
    if (ok) {
      if (threadIdx.x == 0) *reinterpret_cast<volatile int*>(pub_ctr + k) = counter;
      mbar_arrive(&bar.pub_full[k]);
    } else if (!*abort_flag) {
      atomicOr(p.status, 16u);
      *abort_flag = 1;
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Publisher: releases until the consumers hand over -1 (or the CTA aborts).
template <class L>
__device__ void publisher(const StreamParams& p, unsigned char* smem) {
  const Bars bar = bars_of<L>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::misc);
  const volatile int* pub_ctr = reinterpret_cast<const volatile int*>(smem + L::pub);
  for (int j = 0;; ++j) {
    const int k = j % kPubRing;
    if (!wait_parity(&bar.pub_full[k], static_cast<uint32_t>(j / kPubRing) & 1u, p.timeout_cycles, abort_flag)) {
      if (!*abort_flag) {
        atomicOr(p.status, 32u);
        *abort_flag = 1;
      }
      return;
    }
    const int c = pub_ctr[k];
    mbar_arrive(&bar.pub_empty[k]);
    if (c < 0) return;
    // The consumers' stores happen before their arrives, which this thread has acquired; the
    // release makes them visible to every CTA that acquires the counter.
    red_release_add(p.group_done + c, 1ull);
  }
}


// Orders this thread's earlier generic-proxy accesses before its later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Bounded wait for the completion of an mbarrier phase on the way out of an aborted CTA (the
// copies in flight must land before the CTA exits).
__device__ __forceinline__ void drain(uint64_t* bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity) && clock64() - t0 < budget) {
  }
}

template <class K>
__device__ void producer(const StreamParams& p, int i0, int i1, unsigned char* smem) {
  using TM = typename K::TM;
  using TV = typename K::TV;
  using L = typename K::L;
  constexpr int R = K::R;  // values per vector position
  unsigned char* stages = smem;
  WorkItem* ring = reinterpret_cast<WorkItem*>(smem + L::desc);
  const Bars bar = bars_of<L>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::misc);
  const TM* M = static_cast<const TM*>(p.M);
  const int n = i1 - i0;
  int batches = 0;  // static descriptor batches issued
  auto issue_batch = [&](int batch) {
    const int first = batch * kDescBatch;
    if (first >= n) return;
    const int cnt = n - first < kDescBatch ? n - first : kDescBatch;
    const int q = batch % kDescBatches;
    mbar_arrive_expect_tx(&bar.desc[q], static_cast<uint32_t>(cnt * sizeof(WorkItem)));
    bulk_g2s(ring + q * kDescBatch, p.items + i0 + first, static_cast<uint32_t>(cnt * sizeof(WorkItem)),
             &bar.desc[q]);
    batches = batch + 1;
  };
  for (int b = 0; b < kDescBatches; ++b) issue_batch(b);  // batches 0 .. kDescBatches-1
  int seq = 0;      // items whose stage has been armed
  bool ok = true;
  uint32_t ready = 0;  // groups known complete in this call
  // Tiles are read once per call: first out of L2, so that the vectors (a few MB, read by every
  // call's input copies and permutation) stay in it across calls.
  uint64_t stream_once, keep;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream_once));
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));

  // Waits for the stage of item `sq` to be free.
  auto stage_free = [&](int sq) -> bool {
    const uint32_t k = static_cast<uint32_t>(sq / L::stages);
    if (k > 0 && !wait_parity(&bar.empty[sq % L::stages], (k - 1) & 1u, p.timeout_cycles, abort_flag)) {
      atomicOr(p.status, 2u);
      return false;
    }
    return true;
  };
  // Arms the stage of item `sq` (descriptor in its ring slot) and issues its copies. When a group
  // wait runs out the input copies are still issued (valid addresses, stale values), so that the
  // stage's barrier completes and the way out can wait for it.
  auto copy_item = [&](int sq) -> bool {
    // the descriptor in registers: six 16-byte shared loads issued together
    WorkItem it;
    {
      const uint4* src = reinterpret_cast<const uint4*>(ring + sq % kDescRing);
      uint4* w = reinterpret_cast<uint4*>(&it);
#pragma unroll
      for (int k = 0; k < static_cast<int>(sizeof(WorkItem) / 16); ++k) w[k] = src[k];
    }
    const int s = sq % L::stages;
    unsigned char* st = stages + static_cast<size_t>(s) * L::stage_bytes;
    const uint32_t tile_bytes = static_cast<uint32_t>(it.ncols) * static_cast<uint32_t>(it.hp) * sizeof(TM);
    uint32_t bytes = tile_bytes;
#pragma unroll
    for (int r = 0; r < kMaxRuns; ++r)
      if (r < it.nruns) bytes += static_cast<uint32_t>(it.runs[r].len) * sizeof(TV) * R;
    mbar_arrive_expect_tx(&bar.full[s], bytes);
    if (tile_bytes) bulk_g2s_hint(st, M + it.tile_off, tile_bytes, &bar.full[s], stream_once);
    const uint32_t deps = (static_cast<uint32_t>(it.flags) >> kDepShift) & ((1u << kNumCounters) - 1u);
    const bool flag = (it.flags & kItemBase) && it.naux >= 0;
    bool done = true;
    if ((deps & ~ready) || flag) {
      const long long t0 = clock64();
      bool flag_set = !flag;
      for (;;) {
        for (int g = 0; g < kNumCounters; ++g)
          if (((deps & ~ready) >> g) & 1u)
            if (ld_acquire_u64(p.group_done + g) >= p.need[g]) ready |= 1u << g;
        if (!flag_set) flag_set = ld_acquire_u64(p.group_done + kFlagBase + it.naux) >= p.flag_need;
        if (!(deps & ~ready) && flag_set) break;
        __nanosleep(100);
        if (*abort_flag || clock64() - t0 > p.timeout_cycles) {
          atomicOr(p.status, 4u);
          done = false;
          break;
        }
      }
      fence_proxy_async();  // the acquires above before the bulk copies that read those inputs
    }
    uint32_t col = 0;
#pragma unroll
    for (int r = 0; r < kMaxRuns; ++r) {
      if (r >= it.nruns) break;
      const Run run = it.runs[r];
      bulk_g2s_hint(st + tile_bytes + col * sizeof(TV) * R,
                    static_cast<const TV*>(src_ptr(p, run.src)) + static_cast<int64_t>(run.start) * R,
                    static_cast<uint32_t>(run.len) * sizeof(TV) * R, &bar.full[s], keep);
      col += static_cast<uint32_t>(run.len);
    }
    return done;
  };

  // ---- static list
  int waited = 0;  // static descriptor batches waited for
  while (seq < n) {
    const int batch = seq / kDescBatch;
    if (seq % kDescBatch == 0) {
      if (!wait_parity(&bar.desc[batch % kDescBatches], static_cast<uint32_t>(batch / kDescBatches) & 1u,
                       p.timeout_cycles, abort_flag)) {
        atomicOr(p.status, 8u);
        ok = false;
        break;
      }
      waited = batch + 1;
    }
    if (!stage_free(seq)) {
      ok = false;
      break;
    }
    if (seq % kDescBatch == kDescBatch - 1 && batch >= 1) {
      // The consumers have finished item seq - kStages (we waited for its stage), so they are
      // past batch - 1: refill its ring slots with the batch kDescBatches further on.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_batch(batch - 1 + kDescBatches);
    }
    if (!copy_item(seq++)) {
      ok = false;
      break;
    }
  }

  // ---- pool: a CTA takes tickets (each one or more whole chunks) until its first ticket past the
  // end. The next ticket is taken three items before the end of the current one and resolved after
  // its last item is issued (the atomic's latency is hidden behind those items); descriptors are
  // fetched into the ring one segment ahead.
  unsigned long long* ticket = p.group_done + kTicketIndex;
  const unsigned long long P = static_cast<unsigned long long>(p.pool_chunks);
  int fetched = 0, landed = 0;  // pool segments fetched / waited for
  int fseq = seq;               // ring position of the next fetched segment
  auto fetch = [&](int g, int end) {
    const int cnt = end - g < kPoolSeg ? end - g : kPoolSeg;
    uint64_t* fb = &bar.pool[fetched & 1];
    const int s0 = fseq % kDescRing;
    const int c0 = cnt < kDescRing - s0 ? cnt : kDescRing - s0;
    // the consumers' reads of these ring slots (observed through the stage barriers) before the copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(fb, static_cast<uint32_t>(cnt * sizeof(WorkItem)));
    bulk_g2s(ring + s0, p.items + g, static_cast<uint32_t>(c0 * sizeof(WorkItem)), fb);
    if (c0 < cnt) bulk_g2s(ring, p.items + g + c0, static_cast<uint32_t>((cnt - c0) * sizeof(WorkItem)), fb);
    fseq += cnt;
    ++fetched;
  };
  if (ok) {
    // ticket index in this call; a counter left short by an aborted call reads as past the end
    const unsigned long long t0 = atomicAdd(ticket, 1ull) - p.ticket_base;
    bool more = t0 < P;
    PoolRange r{0, 0};
    if (more) {
      r = p.pool[t0];
      fetch(r.begin, r.end);
    }
    while (more && ok) {
      const int take_at = r.end - 3 > r.begin ? r.end - 3 : r.begin;
      unsigned long long raw = 0ull;
      bool more1 = false;
      PoolRange r1{0, 0};
      for (int g = r.begin; g < r.end && ok; g += kPoolSeg) {
        const int cnt = r.end - g < kPoolSeg ? r.end - g : kPoolSeg;
        if (!wait_parity(&bar.pool[landed & 1], static_cast<uint32_t>(landed >> 1) & 1u, p.timeout_cycles,
                         abort_flag)) {
          atomicOr(p.status, 8u);
          ok = false;
          break;
        }
        ++landed;
        if (g + cnt < r.end) fetch(g + cnt, r.end);  // the chunk's next segment
        for (int j = 0; j < cnt; ++j) {
          if (!stage_free(seq)) {
            ok = false;
            break;
          }
          if (g + j == take_at) raw = atomicAdd(ticket, 1ull);
          if (!copy_item(seq++)) {
            ok = false;
            break;
          }
        }
      }
      if (!ok) break;
      // the next chunk: its range, and the first segment of its descriptors
      const unsigned long long t1 = raw - p.ticket_base;
      more1 = t1 < P;
      if (more1) {
        r1 = p.pool[t1];
        fetch(r1.begin, r1.end);
      }
      more = more1;
      r = r1;
    }
  }
  // ---- end mark: the next ring slot says kEnd; its stage's full barrier completes without bytes
  if (ok && stage_free(seq)) {
    reinterpret_cast<volatile int16_t*>(&ring[seq % kDescRing].kind)[0] = kEnd;
    mbar_arrive(&bar.full[seq % L::stages]);
    return;
  }
  *abort_flag = 1;
  // Let every bulk copy already issued land before the CTA can exit: bounded waits on the stages
  // of the last kStages armed items and on the descriptor copies in flight.
  for (int q = seq >= L::stages ? seq - L::stages : 0; q < seq; ++q)
    drain(&bar.full[q % L::stages], static_cast<uint32_t>(q / L::stages) & 1u, p.timeout_cycles);
  for (int b = waited; b < batches; ++b)
    drain(&bar.desc[b % kDescBatches], static_cast<uint32_t>(b / kDescBatches) & 1u, p.timeout_cycles);
  for (int f = landed; f < fetched; ++f)
    drain(&bar.pool[f & 1], static_cast<uint32_t>(f >> 1) & 1u, p.timeout_cycles);
}

template <class K>
__device__ void consumers(const StreamParams& p, unsigned char* smem) {
  using TM = typename K::TM;
  using T = typename K::TV;
  using TX = typename K::TX;
  using L = typename K::L;
  constexpr int EPL = 16 / sizeof(TM);  // tile elements per 16-byte row slice
  constexpr int R = K::R;               // right-hand sides: vectors hold R values per position
  const int tid = threadIdx.x;
  unsigned char* stages = smem;
  const WorkItem* ring = reinterpret_cast<const WorkItem*>(smem + L::desc);
  int* pub_ctr = reinterpret_cast<int*>(smem + L::pub);
  const Bars bar = bars_of<L>(smem);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::misc);
  volatile int* go = abort_flag + 1;  // go[0], go[1]: leader's decision, by item parity

  T acc[EPL][R];
  T base[R];
#pragma unroll
  for (int r = 0; r < R; ++r) base[r] = T{0, 0};
  int out_idx = 0;
  static_assert(kStreamConsumers >= 256, "a chunk's first 256 scatter entries, one per consumer thread");
  Scatter my_scat{};  // this thread's scatter entry of the current chunk (entry tid, if any)
  int need = 1, lanes = 1, groups = kStreamConsumers, lane = 0, g = tid, hpl = EPL;
  const int warp = tid >> 5;
  int nchunk = 0;  // reduced chunks so far: their parity selects the chunk-end buffers
  int np = 0;      // releases handed to the publisher
  {
    // This CTA's slice of the permutation, then its release (each warp after its own stores).
    constexpr int64_t EPV = 16 / sizeof(T) > 0 ? 16 / sizeof(T) : 1;  // vector elements per 16 bytes
    const int64_t b = blockIdx.x, nb = gridDim.x;
    const int64_t a = (p.n * b / nb) / EPV * EPV;
    const int64_t e = b == nb - 1 ? p.n : (p.n * (b + 1) / nb) / EPV * EPV;
    const TX* x = static_cast<const TX*>(p.x);
    T* xp = static_cast<T*>(p.xp);
    for (int64_t q = a + tid; q < e; q += kStreamConsumers) {
      const int64_t src = p.perm[q];
#pragma unroll
      for (int r = 0; r < R; ++r)
        xp[q * R + r] = to_v((R == 1 ? x : static_cast<const TX*>(p.xr[r]))[src], static_cast<T*>(nullptr));
    }
    publish(bar, pub_ctr, np++, kCounterPermute, p, abort_flag);
  }
  for (int seq = 0;; ++seq) {
    const int s = seq % L::stages;
    const uint32_t parity = static_cast<uint32_t>(seq / L::stages) & 1u;
    if (tid == 0) {
      const bool ok = wait_parity(&bar.full[s], parity, p.timeout_cycles, abort_flag);
      if (!ok && !*abort_flag) {
        atomicOr(p.status, 1u);
        *abort_flag = 1;
      }
      go[seq & 1] = ok ? 1 : 0;
    }
    consumer_sync();
    if (!go[seq & 1]) break;
    // The leader's acquire of the full barrier, then the consumer barrier, order the stage's
    // bulk-copied data before every consumer thread's reads.
    const WorkItem& sl = ring[seq % kDescRing];
    if (sl.kind == kEnd) break;
    const int flags = sl.flags;
    const int hp = sl.hp, nc = sl.ncols;
    const int kind = sl.kind, h = sl.h, counter = sl.counter, aux = sl.aux, naux = sl.naux;
    const int64_t dst = sl.dst;
    const unsigned char* st = stages + static_cast<size_t>(s) * L::stage_bytes;
    const int rb = nchunk & 1;
    T* sred = reinterpret_cast<T*>(smem + L::red) + rb * (kStreamConsumers * EPL * R);
    Scatter* sscat = reinterpret_cast<Scatter*>(smem + L::scat) + rb * 256;
    // The chunk's scatter entries (one per thread), loaded now into a register and stored to
    // shared memory at the chunk end, so that the load's latency overlaps the chunk's items.
    if ((flags & kItemFirst) && is_scatter(kind) && tid < naux && tid < 256) my_scat = p.scatter[aux + tid];
    // the output's original index: loaded now, used at the end of the chunk
    if ((flags & kItemFirst) && tid < h && kind == kToY) out_idx = p.perm[dst + tid];
    if (flags & kItemFirst) {
      need = hp / EPL;
      lanes = 1;
      while (lanes < need) lanes <<= 1;
      groups = kStreamConsumers / lanes;
      lane = tid & (lanes - 1);
      g = tid / lanes;
      hpl = lanes * EPL;
#pragma unroll
      for (int e = 0; e < EPL; ++e)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[e][r] = T{0, 0};
    }
    // the staged inputs, after the tile
    const T* vin = reinterpret_cast<const T*>(st + static_cast<size_t>(nc) * hp * sizeof(TM));
    if (lane < need) {
      const TM* tile = reinterpret_cast<const TM*>(st) + lane * EPL;
      int c = g;
      // columns in flight per iteration: 8, or fewer for several right-hand sides (registers)
      constexpr int U = R == 1 ? 8 : R == 2 ? 4 : 2;
      for (; c + (U - 1) * groups < nc; c += U * groups) {
        TM m[U][EPL];
        T v[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          lds16(tile + (c + u * groups) * hp, m[u]);
#pragma unroll
          for (int r = 0; r < R; ++r) v[u][r] = vin[(c + u * groups) * R + r];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int e = 0; e < EPL; ++e)
#pragma unroll
            for (int r = 0; r < R; ++r) cfma(acc[e][r], m[u][e], v[u][r]);
      }
      for (; c < nc; c += groups) {
        TM m0[EPL];
        lds16(tile + c * hp, m0);
#pragma unroll
        for (int e = 0; e < EPL; ++e)
#pragma unroll
          for (int r = 0; r < R; ++r) cfma(acc[e][r], m0[e], vin[c * R + r]);
      }
    }
    // the near-field partial of this row tile, staged after the inputs
    if ((flags & kItemBase) && tid < h)
#pragma unroll
      for (int r = 0; r < R; ++r) base[r] = vin[(nc + tid) * R + r];
    // The stage (tile, inputs, slot) has been read: release it to the producer.
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&bar.empty[s]);
    if (flags & kItemLast) {
      // Column groups in one warp (lanes < 32: groups g and g ^ (m / lanes) share a warp):
      // butterfly over the group bits of the lane index, fixed order.
      for (int m = lanes; m < 32; m <<= 1) {
#pragma unroll
        for (int e = 0; e < EPL; ++e)
#pragma unroll
          for (int r = 0; r < R; ++r) acc[e][r] = cadd(acc[e][r], shfl_xor(acc[e][r], m));
      }
      // One partial per warp (lanes <= 32) or per group (lanes >= 32): at most 8 of them, each
      // row's R values together.
      const int parts = lanes < 32 ? kStreamConsumerWarps : groups;
      const int part = lanes < 32 ? warp : g;
      if (lanes >= 32 || (tid & 31) < lanes) {
#pragma unroll
        for (int e = 0; e < EPL; ++e)
#pragma unroll
          for (int r = 0; r < R; ++r) sred[(part * hpl + lane * EPL + e) * R + r] = acc[e][r];
      }
      if (is_scatter(kind) && tid < naux && tid < 256) sscat[tid] = my_scat;
      consumer_sync();
      // Output row `row`, right-hand side r: its partials summed in a fixed order (at most 8 of
      // them; the loads are independent and issued together).
      auto row_sum = [&](int row, int r) -> T {
        T v = sred[row * R + r];
#pragma unroll
        for (int q = 1; q < kStreamConsumerWarps; ++q)
          if (q < parts) v = cadd(v, sred[(q * hpl + row) * R + r]);
        return v;
      };
      if (is_scatter(kind) && h <= kStreamHpMax) {
        // (entry, row) pairs over all consumer threads, each entry's rows consecutive; a thread
        // sums the row of each pair it stores, so no second barrier is needed.
        T* z = static_cast<T*>(kind == kScatterZ1 ? p.z1 : kind == kScatterZ2 ? p.z2 : p.z4);
        int k = tid / h, r = tid - k * h;
        const int dk = kStreamConsumers / h, dr = kStreamConsumers - dk * h;
        for (int w = tid; w < naux * h; w += kStreamConsumers) {
          const Scatter e = k < 256 ? sscat[k] : p.scatter[aux + k];
          if (r >= e.lo && r < e.hi)
#pragma unroll
            for (int q = 0; q < R; ++q) z[(static_cast<int64_t>(e.dst) + r - e.lo) * R + q] = row_sum(r, q);
          k += dk;
          r += dr;
          if (r >= h) {
            r -= h;
            ++k;
          }
        }
      } else if (tid < h) {
        T v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          v[r] = row_sum(tid, r);
          if (flags & kItemBase) v[r] = cadd(v[r], base[r]);
        }
        if (kind == kToY) {
#pragma unroll
          for (int r = 0; r < R; ++r)
            static_cast<TX*>(R == 1 ? p.y : p.yr[r])[out_idx] = to_x(v[r], static_cast<TX*>(nullptr));
        } else if (is_scatter(kind)) {
          // a tall chunk (t_b rows, up to kStreamHpTall): each thread stores its own row to every
          // scatter entry holding it (few entries: one per block in the chunk)
          T* z = static_cast<T*>(kind == kScatterZ1 ? p.z1 : kind == kScatterZ2 ? p.z2 : p.z4);
          for (int k = 0; k < naux; ++k) {
            const Scatter e = k < 256 ? sscat[k] : p.scatter[aux + k];
            if (tid >= e.lo && tid < e.hi)
#pragma unroll
              for (int r = 0; r < R; ++r) z[(static_cast<int64_t>(e.dst) + tid - e.lo) * R + r] = v[r];
          }
        } else {
          T* z = static_cast<T*>(kind == kToZ1 ? p.z1 : kind == kToZ2 ? p.z2 : p.z3);
#pragma unroll
          for (int r = 0; r < R; ++r) z[(dst + tid) * R + r] = v[r];
        }
      }
      // sred and sscat of this parity are next written two chunks on, after the next chunk end's
      // barrier.
      ++nchunk;
      // On failure the abort flag is set; the leader's next wait then ends the loop for all.
      if (counter >= 0)
        publish(bar, pub_ctr, np++, counter == kCounterFlag ? kFlagBase + naux : counter, p, abort_flag);
    }
  }
  // No more releases: let the publisher finish (skipped when aborting; decided per warp).
  if (__shfl_sync(0xffffffffu, *abort_flag ? 0 : 1, 0)) publish(bar, pub_ctr, np, -1, p, abort_flag);
}

template <class K>
__global__ void __launch_bounds__(kStreamThreads, K::kMinBlocks) stream_kernel(const StreamParams p) {
  using L = typename K::L;
  extern __shared__ __align__(128) unsigned char smem[];
  const Bars bar = bars_of<L>(smem);
  volatile int* misc = reinterpret_cast<volatile int*>(smem + L::misc);
  if (threadIdx.x == 0) {
    for (int s = 0; s < L::stages; ++s) {
      mbar_init(&bar.full[s], 1);
      mbar_init(&bar.empty[s], kStreamConsumerWarps);
    }
    for (int q = 0; q < kDescBatches; ++q) mbar_init(&bar.desc[q], 1);
    for (int q = 0; q < 2; ++q) mbar_init(&bar.pool[q], 1);
    for (int q = 0; q < kPubRing; ++q) {
      mbar_init(&bar.pub_full[q], kStreamConsumerWarps);
      mbar_init(&bar.pub_empty[q], 1);
    }
    for (int q = 0; q < 6; ++q) misc[q] = 0;  // abort, go[2], pf[2]
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x >= kStreamConsumers + 32) {
    if (threadIdx.x == kStreamConsumers + 32) publisher<L>(p, smem);
  } else if (threadIdx.x >= kStreamConsumers) {
    if (threadIdx.x == kStreamConsumers) producer<K>(p, p.cta_begin[blockIdx.x], p.cta_begin[blockIdx.x + 1], smem);
  } else {
    consumers<K>(p, smem);
  }
  __syncthreads();
}

}  // namespace

const void* stream_fn(int variant, int* smem_bytes) {
  switch (variant) {
    case kVarC64: *smem_bytes = KC64::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KC64>);
    case kVarC128: *smem_bytes = KC128::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KC128>);
    case kVarMixed: *smem_bytes = KMixed::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KMixed>);
    case kVarC64Dual: *smem_bytes = KC64Dual::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KC64Dual>);
    case kVarC128Dual:
      *smem_bytes = KC128Dual::L::bytes;
      return reinterpret_cast<const void*>(stream_kernel<KC128Dual>);
    case kVarC64R2: *smem_bytes = KC64R2::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KC64R2>);
    case kVarC64R4: *smem_bytes = KC64R4::L::bytes; return reinterpret_cast<const void*>(stream_kernel<KC64R4>);
    case kVarC64DualR2:
      *smem_bytes = KC64DualR2::L::bytes;
      return reinterpret_cast<const void*>(stream_kernel<KC64DualR2>);
    case kVarMixedDual:
      *smem_bytes = KMixedDual::L::bytes;
      return reinterpret_cast<const void*>(stream_kernel<KMixedDual>);
    default: *smem_bytes = 0; return nullptr;
  }
}

cudaError_t stream_prepare(int variant) {
  int smem = 0;
  const void* fn = stream_fn(variant, &smem);
  if (!fn) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t stream_occupancy(int variant, int* blocks_per_sm) {
  int smem = 0;
  const void* fn = stream_fn(variant, &smem);
  if (!fn) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kStreamThreads, smem);
}

cudaError_t stream_launch(int variant, const StreamParams& p, int grid, cudaStream_t stream) {
  int smem = 0;
  const void* fn = stream_fn(variant, &smem);
  if (!fn) return cudaErrorInvalidValue;
  void* args[] = {const_cast<StreamParams*>(&p)};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kStreamThreads), args, smem, stream);
}

}  // namespace uh

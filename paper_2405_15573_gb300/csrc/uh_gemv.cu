// Persistent segmented GEMV for the single-RHS products (sm_103a).
//
// Used by every phase of the UH matvec (Algorithm 6: forward transform, coupling, backward
// transform, near field) and of the H matvec (Algorithm 5). The host packs each phase into
// column-major tiles whose rows are the outputs, so one CTA streams a contiguous tile with
// 16-byte coalesced loads: thread (lane, group) loads the 16 bytes of rows [lane*EPL, lane*EPL+EPL)
// of every `groups`-th column and multiplies them by that column's input value, which the CTA
// staged in shared memory beforehand. Groups are then reduced in a fixed tree order, and chunks
// fed by several items are finished by the last arriving item (fixed slot order), so every result
// is bitwise reproducible. CTAs take items from an atomic work counter (items are sorted largest
// first on the host), which keeps all SMs streaming until the end of the phase.
#include "uh_internal.h"

namespace uh {
namespace {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; using V16 = float4; };
template <> struct Cx<double> { using T = double2; using V16 = double2; };

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

// 16-byte streaming load of `EPL` complex values (evict-first: the operator is read once).
__device__ __forceinline__ void load16(const float2* p, float2 (&m)[2]) {
  float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  m[0] = make_float2(q.x, q.y);
  m[1] = make_float2(q.z, q.w);
}
__device__ __forceinline__ void load16(const double2* p, double2 (&m)[1]) { m[0] = __ldcs(p); }

template <typename R>
__device__ __forceinline__ void write_out(const SegGemvParams& p, const Chunk& ch, int r,
                                          typename Cx<R>::T v) {
  using T = typename Cx<R>::T;
  if (ch.kind == 0) {
    reinterpret_cast<T*>(p.out_lin)[ch.dst + r] = v;
  } else {
    reinterpret_cast<T*>(p.out_perm)[p.perm[ch.dst + r]] = v;
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) seg_gemv_kernel(const SegGemvParams p) {
  using T = typename Cx<R>::T;
  constexpr int EPL = 16 / sizeof(T);  // complex values per 16-byte load
  __shared__ T sv[kMaxCols];
  __shared__ T sred[kThreads * EPL];
  __shared__ int s_item;
  __shared__ int s_last;

  const T* M = reinterpret_cast<const T*>(p.M);
  const T* in0 = reinterpret_cast<const T*>(p.in0);
  const T* in1 = reinterpret_cast<const T*>(p.in1);
  T* partials = reinterpret_cast<T*>(p.partials);
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_item = static_cast<int>(atomicAdd(&p.sched[0], 1u));
    __syncthreads();
    const int it = s_item;
    if (it >= p.item_count) break;
    const Item item = p.items[it];

    // Stage this item's input values.
    for (int c = tid; c < item.ncols; c += kThreads) {
      const int ix = p.colidx[item.idx_off + c];
      sv[c] = ix >= 0 ? in0[ix] : in1[-ix - 1];
    }
    __syncthreads();

    // lanes: power of two >= hp/EPL; groups = kThreads / lanes (power of two).
    const int need = item.hp / EPL;
    int lanes = 1;
    while (lanes < need) lanes <<= 1;
    const int groups = kThreads / lanes;
    const int lane = tid & (lanes - 1);
    const int g = tid / lanes;
    const int hpl = lanes * EPL;

    T acc[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) acc[e] = T{0, 0};
    if (lane < need) {
      const T* base = M + item.data_off + lane * EPL;
      const int64_t colstride = item.hp;
      int c = g;
      // Four independent loads in flight per thread per trip.
      for (; c + 3 * groups < item.ncols; c += 4 * groups) {
        T m0[EPL], m1[EPL], m2[EPL], m3[EPL];
        load16(base + (int64_t)c * colstride, m0);
        load16(base + (int64_t)(c + groups) * colstride, m1);
        load16(base + (int64_t)(c + 2 * groups) * colstride, m2);
        load16(base + (int64_t)(c + 3 * groups) * colstride, m3);
        const T v0 = sv[c], v1 = sv[c + groups], v2 = sv[c + 2 * groups], v3 = sv[c + 3 * groups];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          cfma(acc[e], m0[e], v0);
          cfma(acc[e], m1[e], v1);
          cfma(acc[e], m2[e], v2);
          cfma(acc[e], m3[e], v3);
        }
      }
      for (; c < item.ncols; c += groups) {
        T m0[EPL];
        load16(base + (int64_t)c * colstride, m0);
        const T v0 = sv[c];
#pragma unroll
        for (int e = 0; e < EPL; ++e) cfma(acc[e], m0[e], v0);
      }
    }
#pragma unroll
    for (int e = 0; e < EPL; ++e) sred[g * hpl + lane * EPL + e] = acc[e];
    __syncthreads();
    // Fixed-order tree reduction over the groups.
    for (int s = groups >> 1; s >= 1; s >>= 1) {
      if (g < s) {
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int k = g * hpl + lane * EPL + e;
          sred[k] = cadd(sred[k], sred[k + s * hpl]);
        }
      }
      __syncthreads();
    }

    const Chunk ch = p.chunks[item.chunk];
    if (item.part < 0) {
      if (tid < ch.h) write_out<R>(p, ch, tid, sred[tid]);
    } else {
      if (tid < ch.h) {
        __stcg(&partials[(int64_t)item.part * kHpMax + tid], sred[tid]);
        __threadfence();
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const unsigned old = atomicAdd(&p.chunk_cnt[item.chunk], 1u);
        s_last = (old == static_cast<unsigned>(ch.nparts - 1));
      }
      __syncthreads();
      if (s_last) {
        __threadfence();
        if (tid < ch.h) {
          T s = T{0, 0};
          for (int q = 0; q < ch.nparts; ++q)
            s = cadd(s, __ldcg(&partials[(int64_t)(ch.part_base + q) * kHpMax + tid]));
          write_out<R>(p, ch, tid, s);
        }
        if (tid == 0) p.chunk_cnt[item.chunk] = 0u;
      }
    }
    __syncthreads();
  }

  // The last CTA to leave resets the work counters for the next launch on this op.
  if (tid == 0) {
    __threadfence();
    const unsigned old = atomicAdd(&p.sched[1], 1u);
    if (old == gridDim.x - 1) {
      atomicExch(&p.sched[0], 0u);
      atomicExch(&p.sched[1], 0u);
    }
  }
}

}  // namespace

cudaError_t launch_seg_gemv(bool c128, const SegGemvParams& p, int grid, cudaStream_t stream) {
  if (p.item_count <= 0) return cudaSuccess;
  if (grid > p.item_count) grid = p.item_count;
  if (c128) {
    seg_gemv_kernel<double><<<grid, kThreads, 0, stream>>>(p);
  } else {
    seg_gemv_kernel<float><<<grid, kThreads, 0, stream>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace uh

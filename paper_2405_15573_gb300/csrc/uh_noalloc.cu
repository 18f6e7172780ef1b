// uh_block_apply_noalloc: one admissible block of a UH-matrix, y = U (S (V^* x)), computed in the
// forward / coupling / backward steps of the UH product without any device allocation. The
// intermediate vectors (partial sums of V^* x, and S V^* x) live in a fixed device array owned by
// this file. It exists for callers that cannot call cudaMalloc: code that runs while a stream is
// being captured into a CUDA graph, or that must stay inside device memory handed out by its own
// arena or by a framework's allocator. The paper has no counterpart to this entry point.
#include <mutex>

#include "uh.h"
#include "uh_internal.h"

namespace {

constexpr int kNaMaxRank = 256;     // largest l_tau and l_sigma accepted
constexpr int kNaMaxChunks = 64;    // row chunks of the forward step (partial sums per column)
constexpr int kNaMaxDevices = 64;
// Largest block height or width: keeps the backward grid ((m + 255) / 256 blocks) inside the
// 2^31 - 1 limit of a grid's x dimension.
constexpr int64_t kNaMaxRows = static_cast<int64_t>(0x7fffffff) * 256;
// Partial sums [kNaMaxChunks][kNaMaxRank] and yhat [kNaMaxRank], complex128-sized slots.
constexpr size_t kNaScratchBytes = static_cast<size_t>(kNaMaxChunks + 1) * kNaMaxRank * 16;

// The scratch. Every GPU that loads the library holds these 266,240 bytes until the process
// exits; all calls share them.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kNaMaxDevices] = {};

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

__device__ __forceinline__ float2 cmad(float2 a, float2 m, float2 v) {
  return make_float2(fmaf(m.x, v.x, fmaf(-m.y, v.y, a.x)), fmaf(m.x, v.y, fmaf(m.y, v.x, a.y)));
}
__device__ __forceinline__ double2 cmad(double2 a, double2 m, double2 v) {
  return make_double2(fma(m.x, v.x, fma(-m.y, v.y, a.x)), fma(m.x, v.y, fma(m.y, v.x, a.y)));
}
// a + conj(m) * v
__device__ __forceinline__ float2 cmad_conj(float2 a, float2 m, float2 v) {
  return make_float2(fmaf(m.x, v.x, fmaf(m.y, v.y, a.x)), fmaf(m.x, v.y, fmaf(-m.y, v.x, a.y)));
}
__device__ __forceinline__ double2 cmad_conj(double2 a, double2 m, double2 v) {
  return make_double2(fma(m.x, v.x, fma(m.y, v.y, a.x)), fma(m.x, v.y, fma(-m.y, v.x, a.y)));
}

// Forward step: partial[c][j] = sum_{r in chunk c} conj(V[r, j]) x[r]. One warp per column j,
// lanes over the rows of the chunk, fixed shuffle reduction.
template <typename R>
__global__ void na_forward(int64_t n, int ls, int nchunk, const typename Cx<R>::T* V, int64_t ldv,
                           const typename Cx<R>::T* x, typename Cx<R>::T* partial) {
  using T = typename Cx<R>::T;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.y * (blockDim.x / 32) + threadIdx.x / 32;
  const int c = blockIdx.x;
  if (j >= ls) return;
  const int64_t r0 = n * c / nchunk, r1 = n * (c + 1) / nchunk;
  T acc = T{0, 0};
  for (int64_t r = r0 + lane; r < r1; r += 32) acc = cmad_conj(acc, V[r + j * ldv], x[r]);
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) partial[static_cast<int64_t>(c) * kNaMaxRank + j] = acc;
}

// Coupling step: xhat = sum over chunks of the partials (fixed order), yhat = S xhat.
template <typename R>
__global__ void na_coupling(int lt, int ls, int nchunk, const typename Cx<R>::T* S, int64_t lds,
                            const typename Cx<R>::T* partial, typename Cx<R>::T* yhat) {
  using T = typename Cx<R>::T;
  __shared__ T xs[kNaMaxRank];
  for (int j = threadIdx.x; j < ls; j += blockDim.x) {
    T s = T{0, 0};
    for (int c = 0; c < nchunk; ++c) {
      const T v = partial[static_cast<int64_t>(c) * kNaMaxRank + j];
      s.x += v.x;
      s.y += v.y;
    }
    xs[j] = s;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < lt; i += blockDim.x) {
    T a = T{0, 0};
    for (int j = 0; j < ls; ++j) a = cmad(a, S[i + j * lds], xs[j]);
    yhat[i] = a;
  }
}

// Backward step: y[r] = sum_i U[r, i] yhat[i], one thread per row.
template <typename R>
__global__ void na_backward(int64_t m, int lt, const typename Cx<R>::T* U, int64_t ldu,
                            const typename Cx<R>::T* yhat, typename Cx<R>::T* y) {
  using T = typename Cx<R>::T;
  __shared__ T ys[kNaMaxRank];
  for (int i = threadIdx.x; i < lt; i += blockDim.x) ys[i] = yhat[i];
  __syncthreads();
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= m) return;
  T a = T{0, 0};
  for (int i = 0; i < lt; ++i) a = cmad(a, U[r + i * ldu], ys[i]);
  y[r] = a;
}

template <typename R>
cudaError_t na_run(int64_t m, int64_t n, int lt, int ls, const void* U, int64_t ldu, const void* S, int64_t lds,
                   const void* V, int64_t ldv, const void* x, void* y, void* scratch, cudaStream_t st) {
  using T = typename Cx<R>::T;
  T* partial = static_cast<T*>(scratch);
  T* yhat = partial + static_cast<int64_t>(kNaMaxChunks) * kNaMaxRank;
  int nchunk = static_cast<int>((n + 255) / 256);
  if (nchunk > kNaMaxChunks) nchunk = kNaMaxChunks;
  if (ls > 0) {
    dim3 grid(nchunk, (ls + 7) / 8);
    na_forward<R><<<grid, 256, 0, st>>>(n, ls, nchunk, static_cast<const T*>(V), ldv, static_cast<const T*>(x), partial);
  }
  na_coupling<R><<<1, 256, 0, st>>>(lt, ls, ls > 0 ? nchunk : 0, static_cast<const T*>(S), lds, partial, yhat);
  na_backward<R><<<static_cast<unsigned>((m + 255) / 256), 256, 0, st>>>(m, lt, static_cast<const T*>(U), ldu, yhat,
                                                                           static_cast<T*>(y));
  return cudaGetLastError();
}

// Device address of the scratch array for the current device, looked up once per device.
int scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return uh::set_error(UH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kNaMaxDevices) return uh::set_error(UH_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return uh::set_error(UH_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return UH_OK;
}

}  // namespace

extern "C" int uh_block_apply_noalloc(int64_t m, int64_t n, int32_t lt, int32_t ls, const void* U, int64_t ldu,
                                      const void* S, int64_t lds, const void* V, int64_t ldv, const void* x,
                                      void* y, int32_t precision, void* stream) {
  if (precision != UH_PREC_C128 && precision != UH_PREC_C64)
    return uh::set_error(UH_EINVAL, "uh_block_apply_noalloc: precision %d not supported", precision);
  if (m < 1 || n < 1) return uh::set_error(UH_EINVAL, "uh_block_apply_noalloc: m = %lld, n = %lld must be >= 1",
                                           (long long)m, (long long)n);
  if (m > kNaMaxRows || n > kNaMaxRows)
    return uh::set_error(UH_EINVAL, "uh_block_apply_noalloc: m = %lld, n = %lld above the limit %lld",
                         (long long)m, (long long)n, (long long)kNaMaxRows);
  if (lt < 0 || ls < 0 || lt > kNaMaxRank || ls > kNaMaxRank)
    return uh::set_error(UH_EINVAL,
                         "uh_block_apply_noalloc: ranks l_tau = %d, l_sigma = %d outside [0, %d], the limit of the "
                         "fixed scratch array",
                         lt, ls, kNaMaxRank);
  if (lt > m || ls > n) return uh::set_error(UH_EINVAL, "uh_block_apply_noalloc: rank larger than block size");
  if ((lt > 0 && (!U || ldu < m)) || (lt > 0 && ls > 0 && (!S || lds < lt)) || (ls > 0 && (!V || ldv < n)) || !x || !y)
    return uh::set_error(UH_EINVAL, "uh_block_apply_noalloc: missing pointer or leading dimension too small");
  void* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != UH_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = precision == UH_PREC_C128
                      ? na_run<double>(m, n, lt, ls, U, ldu, S, lds, V, ldv, x, y, scratch, st)
                      : na_run<float>(m, n, lt, ls, U, ldu, S, lds, V, ldv, x, y, scratch, st);
  if (e != cudaSuccess) return uh::set_error(UH_ECUDA, "uh_block_apply_noalloc launch: %s", cudaGetErrorString(e));
  return UH_OK;
}

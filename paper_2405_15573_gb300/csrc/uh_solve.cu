// FP64 vector kernels of the GMRES solves run by the serving runtime (uh_serve.cpp): conversions
// to and from the complex64 vectors of the UH product, the residual, the block dot products and
// updates of classical Gram-Schmidt (applied twice), norms and scaling. Every reduction has a
// fixed grid and a fixed order (partials per block, then one block sums them in block order), so
// a solve's arithmetic does not depend on anything else running on the GPU.
#include <cuda_runtime.h>

#include "uh.h"
#include "uh_internal.h"
#include "uh_solve.h"

namespace uh {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void d2f_kernel(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b[i] = make_float2(static_cast<float>(a[i].x), static_cast<float>(a[i].y));
}

__global__ void f2d_kernel(const float2* __restrict__ a, double2* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    b[i] = make_double2(a[i].x, a[i].y);
}

// r = b - y, y complex64 (c64 != 0) or complex128.
__global__ void residual_kernel(const double2* __restrict__ b, const void* __restrict__ y, int c64,
                                double2* __restrict__ r, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double2 v;
    if (c64) {
      const float2 f = static_cast<const float2*>(y)[i];
      v = make_double2(f.x, f.y);
    } else {
      v = static_cast<const double2*>(y)[i];
    }
    r[i] = make_double2(b[i].x - v.x, b[i].y - v.y);
  }
}

template <typename T>
__device__ T block_sum(T v, T* sh) {
  // fixed-order tree over the block (blockDim.x == kThreads)
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// part[i * nb + blk] = sum over block blk's slice of conj(V_i[k]) w[k], for i < cnt (grid nb x cnt).
__global__ void dots_kernel(const double2* __restrict__ V, int64_t n, int cnt, const double2* __restrict__ w,
                            double2* __restrict__ part) {
  __shared__ double2 sh[kThreads];
  const int i = blockIdx.y;
  const int nb = gridDim.x;
  const int64_t per = (n + nb - 1) / nb;
  const int64_t k0 = blockIdx.x * per, k1 = k0 + per < n ? k0 + per : n;
  const double2* v = V + static_cast<int64_t>(i) * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kThreads) acc = acc + cmul_conj(v[k], w[k]);
  const double2 s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[static_cast<int64_t>(i) * nb + blockIdx.x] = s;
  (void)cnt;
}

// h[i] (+)= sum_blk part[i * nb + blk], block order; one thread per i.
__global__ void dots_finish_kernel(const double2* __restrict__ part, int nb, int cnt, double2* __restrict__ h,
                                   int accumulate) {
  const int i = threadIdx.x;
  if (i >= cnt) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) s = s + part[static_cast<int64_t>(i) * nb + b];
  h[i] = accumulate ? h[i] + s : s;
}

// w[k] -= sum_{i < cnt} V_i[k] c[i]   (c on the device), or, with sign +1, x[k] += sum V_i[k] c[i].
__global__ void combine_kernel(const double2* __restrict__ V, int64_t n, int cnt, const double2* __restrict__ c,
                               double sign, double2* __restrict__ w) {
  __shared__ double2 cs[64];
  if (threadIdx.x < cnt) cs[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < cnt; ++i) {
      const double2 v = V[static_cast<int64_t>(i) * n + k];
      s = make_double2(s.x + v.x * cs[i].x - v.y * cs[i].y, s.y + v.x * cs[i].y + v.y * cs[i].x);
    }
    w[k] = make_double2(w[k].x + sign * s.x, w[k].y + sign * s.y);
  }
}

// part[blk] = sum over block blk's slice of |w[k]|^2.
__global__ void norm_kernel(const double2* __restrict__ w, int64_t n, double* __restrict__ part) {
  __shared__ double sh[kThreads];
  const int nb = gridDim.x;
  const int64_t per = (n + nb - 1) / nb;
  const int64_t k0 = blockIdx.x * per, k1 = k0 + per < n ? k0 + per : n;
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kThreads) acc += w[k].x * w[k].x + w[k].y * w[k].y;
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[0] = sqrt(sum part) (block order), out[1] = 1 / out[0] (0 if the norm is 0); optionally
// also written as a complex value to hcol (the subdiagonal entry of the Hessenberg column).
__global__ void norm_finish_kernel(const double* __restrict__ part, int nb, double* __restrict__ out,
                                   double2* __restrict__ hcol) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  const double nrm = sqrt(s);
  out[0] = nrm;
  out[1] = nrm > 0.0 ? 1.0 / nrm : 0.0;
  if (hcol) *hcol = make_double2(nrm, 0.0);
}

// v = w * scale[1] and, if v32 is not null, v32 = complex64(v) (the next product's input).
__global__ void scale_f_kernel(const double2* __restrict__ w, const double* __restrict__ scale, double2* __restrict__ v,
                               float2* __restrict__ v32, int64_t n) {
  const double f = scale[1];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double2 r = make_double2(w[k].x * f, w[k].y * f);
    v[k] = r;
    if (v32) v32[k] = make_float2(static_cast<float>(r.x), static_cast<float>(r.y));
  }
}

// Like dots_kernel, with w given as complex64 y; blocks of row 0 also write w = complex128(y).
__global__ void dots_f_kernel(const double2* __restrict__ V, int64_t n, const float2* __restrict__ y,
                              double2* __restrict__ w, double2* __restrict__ part) {
  __shared__ double2 sh[kThreads];
  const int i = blockIdx.y;
  const int nb = gridDim.x;
  const int64_t per = (n + nb - 1) / nb;
  const int64_t k0 = blockIdx.x * per, k1 = k0 + per < n ? k0 + per : n;
  const double2* v = V + static_cast<int64_t>(i) * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kThreads) {
    const double2 wk = make_double2(y[k].x, y[k].y);
    if (i == 0) w[k] = wk;
    acc = acc + cmul_conj(v[k], wk);
  }
  const double2 s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[static_cast<int64_t>(i) * nb + blockIdx.x] = s;
}

// v = w * scale[1] (the inverse norm on the device).
__global__ void scale_kernel(const double2* __restrict__ w, const double* __restrict__ scale, double2* __restrict__ v,
                             int64_t n) {
  const double f = scale[1];
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    v[k] = make_double2(w[k].x * f, w[k].y * f);
}

int grid_for(int64_t n) {
  const int64_t g = (n + kThreads - 1) / kThreads;
  return static_cast<int>(g < 1216 ? (g < 1 ? 1 : g) : 1216);
}

int launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? UH_OK : set_error(UH_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

int solve_partials(int64_t n) {
  const int64_t nb = (n + 4095) / 4096;
  return static_cast<int>(nb < 1 ? 1 : (nb > 152 ? 152 : nb));
}

int vec_d2f(const void* a, void* b, int64_t n, cudaStream_t s) {
  d2f_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double2*>(a), static_cast<float2*>(b), n);
  return launched("vector conversion");
}

int vec_f2d(const void* a, void* b, int64_t n, cudaStream_t s) {
  f2d_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const float2*>(a), static_cast<double2*>(b), n);
  return launched("vector conversion");
}

int vec_residual(const void* b, const void* y, bool y_c64, void* r, int64_t n, cudaStream_t s) {
  residual_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double2*>(b), y, y_c64 ? 1 : 0,
                                                   static_cast<double2*>(r), n);
  return launched("residual");
}

int vec_dots(const void* V, int64_t n, int cnt, const void* w, void* part, void* h, bool accumulate, cudaStream_t s) {
  const int nb = solve_partials(n);
  dots_kernel<<<dim3(nb, cnt), kThreads, 0, s>>>(static_cast<const double2*>(V), n, cnt,
                                                  static_cast<const double2*>(w), static_cast<double2*>(part));
  int rc = launched("block dot products");
  if (rc) return rc;
  dots_finish_kernel<<<1, 64, 0, s>>>(static_cast<const double2*>(part), nb, cnt, static_cast<double2*>(h),
                                      accumulate ? 1 : 0);
  return launched("block dot products");
}

int vec_combine(const void* V, int64_t n, int cnt, const void* c, double sign, void* w, cudaStream_t s) {
  combine_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double2*>(V), n, cnt,
                                                  static_cast<const double2*>(c), sign, static_cast<double2*>(w));
  return launched("block update");
}

int vec_norm(const void* w, int64_t n, void* part, double* out, void* hcol, cudaStream_t s) {
  const int nb = solve_partials(n);
  norm_kernel<<<nb, kThreads, 0, s>>>(static_cast<const double2*>(w), n, static_cast<double*>(part));
  int rc = launched("norm");
  if (rc) return rc;
  norm_finish_kernel<<<1, 32, 0, s>>>(static_cast<const double*>(part), nb, out, static_cast<double2*>(hcol));
  return launched("norm");
}

int vec_scale_f(const void* w, const double* scale, void* v, void* v32, int64_t n, cudaStream_t s) {
  scale_f_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double2*>(w), scale, static_cast<double2*>(v),
                                                  static_cast<float2*>(v32), n);
  return launched("scaling");
}

int vec_dots_f(const void* V, int64_t n, int cnt, const void* y, void* w, void* part, void* h, cudaStream_t s) {
  const int nb = solve_partials(n);
  dots_f_kernel<<<dim3(nb, cnt), kThreads, 0, s>>>(static_cast<const double2*>(V), n, static_cast<const float2*>(y),
                                                    static_cast<double2*>(w), static_cast<double2*>(part));
  int rc = launched("block dot products");
  if (rc) return rc;
  dots_finish_kernel<<<1, 64, 0, s>>>(static_cast<const double2*>(part), nb, cnt, static_cast<double2*>(h), 0);
  return launched("block dot products");
}

int vec_scale(const void* w, const double* scale, void* v, int64_t n, cudaStream_t s) {
  scale_kernel<<<grid_for(n), kThreads, 0, s>>>(static_cast<const double2*>(w), scale, static_cast<double2*>(v), n);
  return launched("scaling");
}

}  // namespace uh

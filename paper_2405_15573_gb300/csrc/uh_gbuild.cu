// Construction of the synthetic Helmholtz operators on the GPU (uh_build.h, uhb_build_helmholtz_gpu):
// the direct UH construction of Section 4.3 (Algorithms 3 and 4) with the admissible blocks from
// partially pivoted ACA and algebraic recompression (Section 2.3), all in FP64 on the device.
// The host builds the cluster and block trees (uh_build_internal.h); then, one CTA per unit of
// work (block or cluster), five kinds of kernels:
//   aca_kernel        per admissible block: ACA at tol_aca, factors U (m x k), V (n x k) with
//                     A|_b ~ U V^T, in the block's scratch (kcap columns each);
//   recompress_kernel per block: Householder QR of U and of conj(V), the small R1 R2^* by
//                     one-sided Jacobi, singular values > tol_aca * sigma_1 kept: U_b (orthonormal)
//                     and Y_b (orthonormal) in place, singular values s_b;
//   basis_kernel      per row (column) cluster: the stacked matrix [U_b s_b] ([Y_b s_b]) of its
//                     blocks (Algorithm 3's X_tau), column-pivoted Householder QR stopped once the
//                     rest is below 1e-3 eps of the largest column, one-sided Jacobi of the small
//                     triangular factor (after one more QR: r x r rotations), the rank-revealing
//                     route of Remark 4.2; basis = left singular vectors with sigma > eps sigma_1;
//   coupling_kernel   per block: S_b = (U_tau^* U_b s_b)(V_sigma^* Y_b)^*, the projection of the
//                     block onto the two bases (Section 4.1);
//   dense_kernel      the near-field blocks' entries;
// plus gathers into the compact arrays of the H form (X_b = U_b s_b, Y_b, blocks truncated at
// eps) and of the bases. These are the steps of the host builder (uh_build.cpp), so both build
// the same operator up to rounding and the ordering of equal pivots.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "uh.h"
#include "uh_build.h"
#include "uh_build_internal.h"
#include "uh_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = 64;  // largest ACA rank per block (the build fails with UH_EINVAL beyond it)

// ------------------------------------------------------------------------- complex FP64 helpers

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = cabs2(b);
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Sum over the CTA (every thread gets it); sh holds kWarps values. Fixed order.
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < kWarps; ++w) s += sh[w];
  return s;
}
// Largest value over the CTA and its index, the lowest index among equal values (-1, -1 when
// every value is negative, i.e. no candidate).
struct ArgMax {
  double v;
  int i;
};
__device__ __forceinline__ ArgMax better(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i >= 0 && (a.i < 0 || b.i < a.i))) return b;
  return a;
}
__device__ ArgMax block_argmax(ArgMax a, ArgMax* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax b{__shfl_xor_sync(0xffffffffu, a.v, o), __shfl_xor_sync(0xffffffffu, a.i, o)};
    a = better(a, b);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  ArgMax r{-1.0, -1};
  for (int w = 0; w < kWarps; ++w) r = better(r, sh[w]);
  return r;
}

// ------------------------------------------------------------------------- matrix entries

struct Points {
  const double* x;  // coordinates in cluster order (position p = original index perm[p])
  const double* y;
  const double* z;
  double wavenumber;
  double inv_n;     // (4 pi / N) / (4 pi) = 1 / N
};

// A at cluster positions (p, q): delta/2 + exp(i k r) / (N r), the kernel term 0 for r = 0.
__device__ __forceinline__ double2 entry(const Points& P, int64_t p, int64_t q) {
  const double dx = P.x[p] - P.x[q], dy = P.y[p] - P.y[q], dz = P.z[p] - P.z[q];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  double2 a = make_double2(p == q ? 0.5 : 0.0, 0.0);
  if (r > 0.0) {
    double s, c;
    sincos(P.wavenumber * r, &s, &c);
    const double w = P.inv_n / r;
    a.x += c * w;
    a.y += s * w;
  }
  return a;
}

// ------------------------------------------------------------------------- ACA (Section 2.3)

struct BlockTab {
  const int64_t* r0;   // first row position
  const int32_t* m;    // rows
  const int64_t* c0;   // first column position
  const int32_t* n;    // columns
  const int64_t* uoff; // U scratch (m x kCap, column-major)
  const int64_t* voff; // V scratch (n x kCap)
};

// Partially pivoted ACA of one block per CTA (grid-stride): A|_b ~ sum_q u_q v_q^T, the first
// row first, the next row the unused one where |u_k| is largest, stop at |u_k||v_k| <=
// tol |S_k|_F with |S_k|_F^2 updated with the cross terms. rank[b] = terms, or -1 when kCap
// terms did not reach the tolerance (and fewer than min(m, n)).
__global__ void __launch_bounds__(kThreads) aca_kernel(Points P, BlockTab T, int64_t nblocks, double tol, double2* U,
                                                       double2* V, int32_t* rank) {
  extern __shared__ unsigned char dyn[];
  unsigned char* used = dyn;  // [m]
  __shared__ double shd[kWarps];
  __shared__ ArgMax sha[kWarps];
  __shared__ double2 dots[2 * kCap];
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int64_t r0 = T.r0[b], c0 = T.c0[b];
    const int m = T.m[b], n = T.n[b];
    double2* Ub = U + T.uoff[b];
    double2* Vb = V + T.voff[b];
    for (int t = threadIdx.x; t < m; t += kThreads) used[t] = 0;
    __syncthreads();
    const int kmax = min(min(m, n), kCap);
    int k = 0, i = 0;
    double norm2 = 0.0;
    bool converged = false;
    while (k < kmax) {
      // residual row i into column k of V
      double2* vk = Vb + static_cast<int64_t>(k) * n;
      for (int j = threadIdx.x; j < n; j += kThreads) {
        double2 a = entry(P, r0 + i, c0 + j);
        for (int q = 0; q < k; ++q) a = csub(a, cmul(Ub[i + static_cast<int64_t>(q) * m], Vb[j + static_cast<int64_t>(q) * n]));
        vk[j] = a;
      }
      if (threadIdx.x == 0) used[i] = 1;
      __syncthreads();
      ArgMax best{-1.0, -1};
      for (int j = threadIdx.x; j < n; j += kThreads) best = better(best, ArgMax{cabs2(vk[j]), j});
      best = block_argmax(best, sha);
      if (best.v <= 0.0) {
        // a zero row: the next unused row in order
        ArgMax f{-1.0, -1};
        for (int t = threadIdx.x; t < m; t += kThreads)
          if (!used[t]) f = better(f, ArgMax{1.0, t});
        f = block_argmax(f, sha);
        if (f.i < 0) {
          converged = true;
          break;
        }
        i = f.i;
        continue;
      }
      const int jp = best.i;
      const double2 piv = vk[jp];
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += kThreads) vk[j] = cdiv(vk[j], piv);
      // residual column jp into column k of U
      double2* uk = Ub + static_cast<int64_t>(k) * m;
      for (int t = threadIdx.x; t < m; t += kThreads) {
        double2 a = entry(P, r0 + t, c0 + jp);
        for (int q = 0; q < k; ++q) a = csub(a, cmul(Vb[jp + static_cast<int64_t>(q) * n], Ub[t + static_cast<int64_t>(q) * m]));
        uk[t] = a;
      }
      __syncthreads();
      // cross terms (u_q^* u_k)(v_q^* v_k) for q < k: one warp per q; then the norms
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int q = warp; q < k; q += kWarps) {
        double2 a = make_double2(0.0, 0.0), c = make_double2(0.0, 0.0);
        const double2* uq = Ub + static_cast<int64_t>(q) * m;
        const double2* vq = Vb + static_cast<int64_t>(q) * n;
        for (int t = lane; t < m; t += 32) a = cadd(a, cmulc(uq[t], uk[t]));
        for (int t = lane; t < n; t += 32) c = cadd(c, cmulc(vq[t], vk[t]));
        a = warp_sum(a);
        c = warp_sum(c);
        if (lane == 0) {
          dots[2 * q] = a;
          dots[2 * q + 1] = c;
        }
      }
      double pu = 0.0, pv = 0.0;
      for (int t = threadIdx.x; t < m; t += kThreads) pu += cabs2(uk[t]);
      for (int t = threadIdx.x; t < n; t += kThreads) pv += cabs2(vk[t]);
      const double nu2 = block_sum(pu, shd);
      const double nv2 = block_sum(pv, shd);  // (its barriers also publish dots)
      double cross = 0.0;
      for (int q = 0; q < k; ++q) cross += cmul(dots[2 * q], dots[2 * q + 1]).x;
      norm2 += 2.0 * cross + nu2 * nv2;
      ++k;
      if (sqrt(nu2 * nv2) <= tol * sqrt(fmax(norm2, 0.0))) {
        converged = true;
        break;
      }
      // next row: the unused one with the largest |u_k|
      ArgMax nx{-1.0, -1};
      for (int t = threadIdx.x; t < m; t += kThreads)
        if (!used[t]) nx = better(nx, ArgMax{cabs2(uk[t]), t});
      nx = block_argmax(nx, sha);
      if (nx.i < 0) {
        converged = true;
        break;
      }
      i = nx.i;
    }
    if (!converged && k == kmax && kmax == min(m, n)) converged = true;  // full rank reached
    if (threadIdx.x == 0) rank[b] = converged ? k : -1;
    __syncthreads();
  }
}


// ------------------------------------------------------------------------- CTA-level dense kernels
// Column-major complex matrices in global memory, one CTA (256 threads) working on one matrix.

// Householder QR of A (m x k, lda) in place, LAPACK convention: A = H_0 ... H_{k-1} R with
// H_j = I - tau_j v_j v_j^*, v_j = (0..0, 1, A[j+1.., j]); R in the upper triangle. tau[] in shared
// memory (k entries). Columns of the trailing update are spread over the warps.
__device__ void cta_qr(double2* A, int m, int k, int64_t lda, double2* tau, double* shd) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = min(m, k);
  for (int j = 0; j < p; ++j) {
    double2* a = A + static_cast<int64_t>(j) * lda;
    double part = 0.0;
    for (int t = j + 1 + threadIdx.x; t < m; t += kThreads) part += cabs2(a[t]);
    const double xnorm2 = block_sum(part, shd);
    const double2 alpha = a[j];
    double2 tj = make_double2(0.0, 0.0);
    double beta = alpha.x;
    if (xnorm2 > 0.0 || alpha.y != 0.0) {
      const double nrm = sqrt(cabs2(alpha) + xnorm2);
      beta = alpha.x >= 0.0 ? -nrm : nrm;
      tj = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
      const double2 sc = cdiv(make_double2(1.0, 0.0), csub(alpha, make_double2(beta, 0.0)));
      for (int t = j + 1 + threadIdx.x; t < m; t += kThreads) a[t] = cmul(a[t], sc);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a[j] = make_double2(beta, 0.0);
      tau[j] = tj;
    }
    __syncthreads();
    // columns c > j: A[j:, c] -= conj(tau) v (v^* A[j:, c])
    const double2 ctj = cconj(tj);
    for (int c = j + 1 + warp; c < k; c += kWarps) {
      double2* x = A + static_cast<int64_t>(c) * lda;
      double2 w = make_double2(0.0, 0.0);
      for (int t = j + lane; t < m; t += 32) w = cadd(w, cmulc(t == j ? make_double2(1.0, 0.0) : a[t], x[t]));
      w = warp_sum(w);
      const double2 f = cmul(ctj, w);
      for (int t = j + lane; t < m; t += 32) x[t] = csub(x[t], cmul(t == j ? make_double2(1.0, 0.0) : a[t], f));
    }
    __syncthreads();
  }
}

// Q = H_0 ... H_{p-1} applied to the first p columns of the identity, in place over the
// reflectors that cta_qr left in A (p = min(m, k) columns).
__device__ void cta_form_q(double2* A, int m, int p, int64_t lda, const double2* tau) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = p - 1; j >= 0; --j) {
    double2* a = A + static_cast<int64_t>(j) * lda;
    const double2 tj = tau[j];
    for (int c = j + 1 + warp; c < p; c += kWarps) {
      double2* x = A + static_cast<int64_t>(c) * lda;
      double2 w = make_double2(0.0, 0.0);
      for (int t = j + lane; t < m; t += 32) w = cadd(w, cmulc(t == j ? make_double2(1.0, 0.0) : a[t], x[t]));
      w = warp_sum(w);
      const double2 f = cmul(tj, w);
      for (int t = j + lane; t < m; t += 32) x[t] = csub(x[t], cmul(t == j ? make_double2(1.0, 0.0) : a[t], f));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m; t += kThreads) {
      if (t < j) a[t] = make_double2(0.0, 0.0);
      else if (t == j) a[t] = make_double2(1.0 - tj.x, -tj.y);
      else a[t] = cmul(make_double2(-tj.x, -tj.y), a[t]);
    }
    __syncthreads();
  }
}

// One-sided (Hestenes) Jacobi: B (rows x cols, ldb) <- B J with mutually orthogonal columns, J
// (cols x cols, ldj) unitary, accumulated from the identity. Pairs of columns in the round-robin
// order (cols/2 disjoint pairs per round, one warp per pair), sweeps until a sweep rotates
// nothing (at most 60). A pair is rotated unless |b_p^* b_q| <= 1e-15 |b_p| |b_q|.
__device__ void cta_jacobi(double2* B, int rows, int cols, int64_t ldb, double2* J, int64_t ldj, int* flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < cols * cols; e += kThreads) {
    const int i = e % cols, j = e / cols;
    J[i + static_cast<int64_t>(j) * ldj] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  const int cp = cols + (cols & 1);  // even number of positions; position cols (if odd) is idle
  __syncthreads();
  for (int sweep = 0; sweep < 60 && cols > 1; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int r = 0; r < cp - 1; ++r) {
      for (int i = warp; i < cp / 2; i += kWarps) {
        int pp, qq;
        if (i == 0) {
          pp = cp - 1;
          qq = r;
        } else {
          pp = (r + i) % (cp - 1);
          qq = (r - i + cp - 1) % (cp - 1);
        }
        if (pp >= cols || qq >= cols) continue;
        double2* bp = B + static_cast<int64_t>(pp) * ldb;
        double2* bq = B + static_cast<int64_t>(qq) * ldb;
        double a = 0.0, b = 0.0;
        double2 g = make_double2(0.0, 0.0);
        for (int t = lane; t < rows; t += 32) {
          a += cabs2(bp[t]);
          b += cabs2(bq[t]);
          g = cadd(g, cmulc(bp[t], bq[t]));
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        const double ag = sqrt(cabs2(g));
        if (ag == 0.0 || ag <= 1e-15 * sqrt(a * b)) continue;
        if (lane == 0) *flag = 1;
        const double2 ph = cscale(g, 1.0 / ag);
        const double zeta = (b - a) / (2.0 * ag);
        const double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
        const double2 phc = cconj(ph);
        for (int t = lane; t < rows; t += 32) {
          const double2 x = bp[t], y = cmul(bq[t], phc);
          bp[t] = csub(cscale(x, c), cscale(y, s));
          bq[t] = cadd(cscale(x, s), cscale(y, c));
        }
        double2* jp = J + static_cast<int64_t>(pp) * ldj;
        double2* jq = J + static_cast<int64_t>(qq) * ldj;
        for (int t = lane; t < cols; t += 32) {
          const double2 x = jp[t], y = cmul(jq[t], phc);
          jp[t] = csub(cscale(x, c), cscale(y, s));
          jq[t] = cadd(cscale(x, s), cscale(y, c));
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
  __syncthreads();
}

// Column norms of B (rows x cols), their order (descending, stable) and the number kept above
// rel * the largest: sv[] and ord[] in shared memory (cols <= kRowMax). Returns the kept count.
__device__ int cta_order(const double2* B, int rows, int cols, int64_t ldb, double rel, double* sv, int* ord) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = warp; c < cols; c += kWarps) {
    double a = 0.0;
    for (int t = lane; t < rows; t += 32) a += cabs2(B[t + static_cast<int64_t>(c) * ldb]);
    a = warp_sum(a);
    if (lane == 0) sv[c] = sqrt(a);
  }
  __syncthreads();
  __shared__ int keep;
  if (threadIdx.x == 0) {
    for (int c = 0; c < cols; ++c) ord[c] = c;
    for (int x = 1; x < cols; ++x) {  // insertion sort, stable, descending
      const int v = ord[x];
      int y = x - 1;
      while (y >= 0 && sv[ord[y]] < sv[v]) {
        ord[y + 1] = ord[y];
        --y;
      }
      ord[y + 1] = v;
    }
    int kp = 0;
    if (cols > 0 && sv[ord[0]] > 0.0)
      while (kp < cols && sv[ord[kp]] > rel * sv[ord[0]]) ++kp;
    keep = kp;
  }
  __syncthreads();
  return keep;
}

// A (m x p) <- A (m x p) W (p x q), q <= p, in place row by row (W in shared or global memory,
// ldw). p <= P.
constexpr int kRowMax = 256;  // largest numerical rank of a cluster's stacked matrix
template <int P>
__device__ void cta_rows_times(double2* A, int m, int p, int64_t lda, const double2* W, int64_t ldw, int q) {
  for (int t = threadIdx.x; t < m; t += kThreads) {
    double2 row[P];
    for (int a = 0; a < p; ++a) row[a] = A[t + static_cast<int64_t>(a) * lda];
    for (int c = 0; c < q; ++c) {
      double2 s = make_double2(0.0, 0.0);
      for (int a = 0; a < p; ++a) s = cadd(s, cmul(row[a], W[a + static_cast<int64_t>(c) * ldw]));
      A[t + static_cast<int64_t>(c) * lda] = s;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------------- recompression (Section 2.3)

// Per block (grid-stride): A|_b ~ U V^T = X Y^* with X = U, Y = conj(V); X = Q1 R1, Y = Q2 R2;
// R1 R2^* = W diag(s) Z^* by one-sided Jacobi; keep s > tol s_1: U_b = Q1 W (in U), Y_b = Q2 Z
// (in V), s_b; kb[b] = the kept rank. small: per-CTA scratch of 3 kCap x kCap matrices.
__global__ void __launch_bounds__(kThreads) recompress_kernel(BlockTab T, int64_t nblocks, const int32_t* rank,
                                                              double tol, double2* U, double2* V, double2* small,
                                                              double* sv_out, int32_t* kb) {
  __shared__ double shd[kWarps];
  __shared__ double2 tau[kCap];
  __shared__ double sv[kCap];
  __shared__ int ord[kCap];
  __shared__ int flag;
  double2* R1 = small + static_cast<int64_t>(blockIdx.x) * 3 * kCap * kCap;
  double2* M = R1 + kCap * kCap;
  double2* J = M + kCap * kCap;
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int m = T.m[b], n = T.n[b], k = rank[b];
    double2* X = U + T.uoff[b];
    double2* Y = V + T.voff[b];
    if (k <= 0) {
      if (threadIdx.x == 0) kb[b] = 0;
      continue;
    }
    const int p1 = min(m, k), p2 = min(n, k);
    // X = Q1 R1: R1 (p1 x k) kept
    cta_qr(X, m, k, m, tau, shd);
    for (int e = threadIdx.x; e < p1 * k; e += kThreads) {
      const int i = e % p1, c = e / p1;
      R1[i + c * kCap] = i <= c ? X[i + static_cast<int64_t>(c) * m] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    cta_form_q(X, m, p1, m, tau);
    // Y = conj(V) = Q2 R2; M = R1 R2^* (p1 x p2) built column by column while R2 is in Y
    for (int e = threadIdx.x; e < n * k; e += kThreads) Y[e] = cconj(Y[e]);
    __syncthreads();
    cta_qr(Y, n, k, n, tau, shd);
    for (int e = threadIdx.x; e < p1 * p2; e += kThreads) {
      const int i = e % p1, c = e / p1;
      double2 s = make_double2(0.0, 0.0);
      for (int q = c; q < k; ++q)  // R2[c][q] nonzero for q >= c
        s = cadd(s, cmul(R1[i + q * kCap], cconj(Y[c + static_cast<int64_t>(q) * n])));
      M[i + c * kCap] = s;
    }
    __syncthreads();
    cta_form_q(Y, n, p2, n, tau);
    cta_jacobi(M, p1, p2, kCap, J, kCap, &flag);
    const int keep = cta_order(M, p1, p2, kCap, tol, sv, ord);
    // W[:, c] = M[:, ord[c]] / s, Z[:, c] = J[:, ord[c]], placed in R1 (W) and the front of M
    // (Z): M's columns are read before they are overwritten (ord is a permutation, copied first)
    for (int e = threadIdx.x; e < p1 * keep; e += kThreads) {
      const int i = e % p1, c = e / p1;
      R1[i + c * kCap] = cscale(M[i + ord[c] * kCap], 1.0 / sv[ord[c]]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p2 * keep; e += kThreads) {
      const int i = e % p2, c = e / p2;
      M[i + c * kCap] = J[i + ord[c] * kCap];
    }
    __syncthreads();
    cta_rows_times<kCap>(X, m, p1, m, R1, kCap, keep);
    cta_rows_times<kCap>(Y, n, p2, n, M, kCap, keep);
    for (int c = threadIdx.x; c < keep; c += kThreads) sv_out[b * kCap + c] = sv[ord[c]];
    if (threadIdx.x == 0) kb[b] = keep;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------- cluster bases (Algorithm 3)

struct BasisWork {
  int64_t xoff;     // X scratch (m x K): the stacked factors, then the basis in its first l columns
  int64_t boff;     // B scratch (K x rcap): Rt^* for the Jacobi step
  int64_t joff;     // J scratch (rcap x rcap)
  int64_t first;    // blocks of the cluster: members[first .. first + count)
  int32_t count;
  int32_t m;        // cluster size
  int32_t K;        // columns of X (sum of the blocks' ranks)
  int32_t side;     // 0: row cluster (U_b s_b), 1: column cluster (Y_b s_b)
};

// One cluster per CTA (grid-stride over the work list, largest first): X = [F_b s_b]_b, then the
// column-pivoted Householder QR of X stopped once the Frobenius norm of the untreated part is
// <= 1e-3 eps max_c |X_c| (rank r), X = Q R P^T; Rt = R P^T (r x K); one-sided Jacobi of
// B = Rt^* (K x r): B J = Z diag(s); the left singular vectors of X are Q J; keep s > eps s_1.
// ell[w] = kept rank (-1: r above kRowMax); the basis is left in X's first ell columns.
__global__ void __launch_bounds__(kThreads) basis_kernel(const BasisWork* work, int64_t nwork, const int64_t* members,
                                                         BlockTab T, const double2* U, const double2* V,
                                                         const double* sv_in, const int32_t* kb, double eps,
                                                         double2* Xs, double2* Bs, double2* Js, int32_t* ell) {
  extern __shared__ unsigned char dyn[];
  double* nrm = reinterpret_cast<double*>(dyn);          // [K] column norms of the untreated part
  int* piv = reinterpret_cast<int*>(nrm + 0) + 0;        // placed after nrm below
  __shared__ double shd[kWarps];
  __shared__ ArgMax sha[kWarps];
  __shared__ double2 tau[kRowMax];
  __shared__ double sv[kRowMax];
  __shared__ int ord[kRowMax];
  __shared__ int flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
    const BasisWork W = work[w];
    const int m = W.m, K = W.K;
    piv = reinterpret_cast<int*>(nrm + K);
    double2* X = Xs + W.xoff;
    // stacked factors, scaled by their singular values
    int64_t col = 0;
    for (int32_t e = 0; e < W.count; ++e) {
      const int64_t b = members[W.first + e];
      const int k = kb[b];
      const double2* F = W.side == 0 ? U + T.uoff[b] : V + T.voff[b];
      for (int64_t t = threadIdx.x; t < static_cast<int64_t>(m) * k; t += kThreads) {
        const int j = static_cast<int>(t / m);
        X[col * m + t] = cscale(F[t], sv_in[b * kCap + j]);
      }
      col += k;
    }
    for (int c = threadIdx.x; c < K; c += kThreads) piv[c] = c;
    __syncthreads();
    // largest column norm
    double mx = 0.0;
    for (int c = warp; c < K; c += kWarps) {
      double a = 0.0;
      for (int t = lane; t < m; t += 32) a += cabs2(X[t + static_cast<int64_t>(c) * m]);
      a = warp_sum(a);
      if (lane == 0) nrm[c] = a;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += kThreads) mx = fmax(mx, nrm[c]);
    {
      ArgMax a = block_argmax(ArgMax{mx, 0}, sha);
      mx = sqrt(fmax(a.v, 0.0));
    }
    const double abs_tol = 1e-3 * eps * mx;
    const int p = min(m, K);
    int r = 0;
    bool too_big = false;
    for (int j = 0; j < p && mx > 0.0; ++j) {
      // norms of the untreated part of the remaining columns; the largest one and their sum
      for (int c = j + warp; c < K; c += kWarps) {
        double a = 0.0;
        const double2* x = X + static_cast<int64_t>(c) * m;
        for (int t = j + lane; t < m; t += 32) a += cabs2(x[t]);
        a = warp_sum(a);
        if (lane == 0) nrm[c] = a;
      }
      __syncthreads();
      ArgMax best{-1.0, -1};
      double rest = 0.0;
      for (int c = j + threadIdx.x; c < K; c += kThreads) {
        best = better(best, ArgMax{nrm[c], c});
        rest += nrm[c];
      }
      rest = block_sum(rest, shd);
      best = block_argmax(best, sha);
      if (sqrt(rest) <= abs_tol) break;
      if (j >= kRowMax) {
        too_big = true;
        break;
      }
      if (best.i != j) {
        double2* a = X + static_cast<int64_t>(j) * m;
        double2* bcol = X + static_cast<int64_t>(best.i) * m;
        for (int t = threadIdx.x; t < m; t += kThreads) {
          const double2 v = a[t];
          a[t] = bcol[t];
          bcol[t] = v;
        }
        if (threadIdx.x == 0) {
          const int v = piv[j];
          piv[j] = piv[best.i];
          piv[best.i] = v;
        }
      }
      __syncthreads();
      // Householder step j on the remaining columns (as in cta_qr, one column)
      double2* a = X + static_cast<int64_t>(j) * m;
      double part = 0.0;
      for (int t = j + 1 + threadIdx.x; t < m; t += kThreads) part += cabs2(a[t]);
      const double xnorm2 = block_sum(part, shd);
      const double2 alpha = a[j];
      double2 tj = make_double2(0.0, 0.0);
      double beta = alpha.x;
      if (xnorm2 > 0.0 || alpha.y != 0.0) {
        const double nn = sqrt(cabs2(alpha) + xnorm2);
        beta = alpha.x >= 0.0 ? -nn : nn;
        tj = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        const double2 sc = cdiv(make_double2(1.0, 0.0), csub(alpha, make_double2(beta, 0.0)));
        for (int t = j + 1 + threadIdx.x; t < m; t += kThreads) a[t] = cmul(a[t], sc);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        a[j] = make_double2(beta, 0.0);
        tau[j] = tj;
      }
      __syncthreads();
      const double2 ctj = cconj(tj);
      for (int c = j + 1 + warp; c < K; c += kWarps) {
        double2* x = X + static_cast<int64_t>(c) * m;
        double2 wv = make_double2(0.0, 0.0);
        for (int t = j + lane; t < m; t += 32) wv = cadd(wv, cmulc(t == j ? make_double2(1.0, 0.0) : a[t], x[t]));
        wv = warp_sum(wv);
        const double2 f = cmul(ctj, wv);
        for (int t = j + lane; t < m; t += 32) x[t] = csub(x[t], cmul(t == j ? make_double2(1.0, 0.0) : a[t], f));
      }
      __syncthreads();
      r = j + 1;
    }
    if (too_big) {
      if (threadIdx.x == 0) ell[w] = -1;
      __syncthreads();
      continue;
    }
    // B = Rt^* (K x r): B[c][i] = conj(R[i][c']) with c = piv[c'] (original column order)
    double2* B = Bs + W.boff;
    double2* Jm = Js + W.joff;
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(K) * r; e += kThreads) {
      const int cp = static_cast<int>(e % K), i = static_cast<int>(e / K);
      const double2 v = i <= cp ? X[i + static_cast<int64_t>(cp) * m] : make_double2(0.0, 0.0);
      B[piv[cp] + static_cast<int64_t>(i) * K] = cconj(v);
    }
    __syncthreads();
    cta_form_q(X, m, r, m, tau);
    // B = Q_B R_B (Householder): R_B J = Z' diag(s) gives the same J and s as B J = Z diag(s), and
    // the rotations run on r x r instead of K x r entries.
    cta_qr(B, K, r, K, tau, shd);
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(r) * r; e += kThreads) {
      const int i = static_cast<int>(e % r), c = static_cast<int>(e / r);
      if (i > c) B[i + static_cast<int64_t>(c) * K] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    cta_jacobi(B, r, r, K, Jm, r, &flag);
    const int keep = cta_order(B, r, r, K, eps, sv, ord);
    // the kept columns of J, in order, at the front of B's first column block (r x keep, ld r)
    double2* Jsel = B;  // B is no longer needed
    for (int e = threadIdx.x; e < r * keep; e += kThreads) {
      const int i = e % r, c = e / r;
      Jsel[i + static_cast<int64_t>(c) * r] = Jm[i + static_cast<int64_t>(ord[c]) * r];
    }
    __syncthreads();
    cta_rows_times<kRowMax>(X, m, r, m, Jsel, r, keep);
    if (threadIdx.x == 0) ell[w] = keep;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------- coupling matrices

struct CouplingWork {
  int64_t urow;   // X scratch offset of the row basis (|tau| x l_tau, ld |tau|)
  int64_t vcol;   // X scratch offset of the column basis (|sigma| x l_sigma)
  int64_t soff;   // S_b (l_tau x l_sigma, column-major) in the compact S
  int64_t poff;   // the pair (factored option): P at Pg + poff (l_tau x kCap), conj(R) at Rg + roff
  int64_t roff;   // (l_sigma x kCap)
  int32_t lt, ls;
};

// S_b = (U_tau^* U_b s_b)(V_sigma^* Y_b)^* per block (grid-stride); P (lt x k) and R (ls x k)
// in per-CTA scratch (kRowMax x kCap each). With Pg != nullptr the pair is also stored, P and
// conj(R) column-major with leading dimensions lt and ls, for its recompression (Section 2.3).
__global__ void __launch_bounds__(kThreads) coupling_kernel(const CouplingWork* work, BlockTab T, int64_t nblocks,
                                                            const double2* Xs, const double2* U, const double2* V,
                                                            const double* sv_in, const int32_t* kb, double2* small,
                                                            double2* S, double2* Pg, double2* Rg) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2* P = small + static_cast<int64_t>(blockIdx.x) * 2 * kRowMax * kCap;
  double2* R = P + kRowMax * kCap;
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const CouplingWork W = work[b];
    const int m = T.m[b], n = T.n[b], k = kb[b], lt = W.lt, ls = W.ls;
    if (lt == 0 || ls == 0) continue;
    if (k == 0) {
      for (int e = threadIdx.x; e < lt * ls; e += kThreads) S[W.soff + e] = make_double2(0.0, 0.0);
      continue;
    }
    const double2* Ut = Xs + W.urow;
    const double2* Vs = Xs + W.vcol;
    const double2* Ub = U + T.uoff[b];
    const double2* Yb = V + T.voff[b];
    for (int e = warp; e < lt * k; e += kWarps) {
      const int i = e % lt, j = e / lt;
      double2 a = make_double2(0.0, 0.0);
      for (int t = lane; t < m; t += 32)
        a = cadd(a, cmulc(Ut[t + static_cast<int64_t>(i) * m], Ub[t + static_cast<int64_t>(j) * m]));
      a = warp_sum(a);
      if (lane == 0) P[i + j * kRowMax] = cscale(a, sv_in[b * kCap + j]);
    }
    for (int e = warp; e < ls * k; e += kWarps) {
      const int i = e % ls, j = e / ls;
      double2 a = make_double2(0.0, 0.0);
      for (int t = lane; t < n; t += 32)
        a = cadd(a, cmulc(Vs[t + static_cast<int64_t>(i) * n], Yb[t + static_cast<int64_t>(j) * n]));
      a = warp_sum(a);
      if (lane == 0) R[i + j * kRowMax] = a;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < lt * ls; e += kThreads) {
      const int i = e % lt, c = e / lt;
      double2 s = make_double2(0.0, 0.0);
      for (int j = 0; j < k; ++j) s = cadd(s, cmul(P[i + j * kRowMax], cconj(R[c + j * kRowMax])));
      S[W.soff + e] = s;
    }
    if (Pg) {
      for (int e = threadIdx.x; e < lt * k; e += kThreads) Pg[W.poff + e] = P[e % lt + (e / lt) * kRowMax];
      for (int e = threadIdx.x; e < ls * k; e += kThreads) Rg[W.roff + e] = cconj(R[e % ls + (e / ls) * kRowMax]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------- near field and gathers

// Dense block d (grid-stride over blocks): D[doff + j * m + i] = A(r0 + i, c0 + j).
__global__ void __launch_bounds__(kThreads) dense_kernel(Points P, const int64_t* r0, const int32_t* mm,
                                                         const int64_t* c0, const int32_t* nn, const int64_t* doff,
                                                         int64_t nblocks, double2* D) {
  for (int64_t d = blockIdx.x; d < nblocks; d += gridDim.x) {
    const int m = mm[d], n = nn[d];
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(m) * n; e += kThreads) {
      const int i = static_cast<int>(e % m), j = static_cast<int>(e / m);
      D[doff[d] + e] = entry(P, r0[d] + i, c0[d] + j);
    }
  }
}

// H form of block b: X_b = U_b s_b and Y_b, their first h[b] columns, at xoff / yoff.
__global__ void __launch_bounds__(kThreads) hform_kernel(BlockTab T, int64_t nblocks, const double2* U,
                                                         const double2* V, const double* sv_in, const int32_t* h,
                                                         const int64_t* xoff, const int64_t* yoff, double2* Xh,
                                                         double2* Yh) {
  for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
    const int m = T.m[b], n = T.n[b], k = h[b];
    const double2* Ub = U + T.uoff[b];
    const double2* Yb = V + T.voff[b];
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(m) * k; e += kThreads)
      Xh[xoff[b] + e] = cscale(Ub[e], sv_in[b * kCap + e / m]);
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(n) * k; e += kThreads) Yh[yoff[b] + e] = Yb[e];
  }
}

// Bases into the compact arrays: dst[off[w] + e] = Xs[xoff[w] + e] for e < m * ell.
__global__ void __launch_bounds__(kThreads) gather_kernel(const int64_t* xoff, const int64_t* off, const int64_t* len,
                                                          int64_t nwork, const double2* Xs, double2* dst) {
  for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x)
    for (int64_t e = threadIdx.x; e < len[w]; e += kThreads) dst[off[w] + e] = Xs[xoff[w] + e];
}
}  // namespace

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Device allocations of one build, freed together.
struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    *p = nullptr;
    const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  template <typename T>
  cudaError_t upload(T** p, const std::vector<T>& v) {
    cudaError_t e = alloc(p, v.size());
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
  }
};

template <typename T>
cudaError_t download(std::vector<T>& v, const T* d, size_t count) {
  v.resize(count);
  return count ? cudaMemcpy(v.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost) : cudaSuccess;
}

}  // namespace

#define GTRY(call)                                                                              \
  do {                                                                                          \
    const cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                                    \
      delete M;                                                                                 \
      return uh::set_error(e_ == cudaErrorMemoryAllocation ? UH_ENOMEM : UH_ECUDA, "%s: %s", #call, \
                           cudaGetErrorString(e_));                                             \
    }                                                                                           \
  } while (0)

extern "C" int uhb_build_helmholtz_gpu(int64_t n, const double* points, const uhb_params* prm, uh_model** out) {
  using uhb::cd;
  int rc;
  if ((rc = uhb::check_build_args(n, points, prm, out))) return rc;
  auto* M = new (std::nothrow) uh_model();
  if (!M) return uh::set_error(UH_ENOMEM, "host allocation");
  const double t0 = now_s();
  uhb::Builder B;
  B.n = n;
  B.pts = points;
  B.prm = *prm;
  uhb::BlockList adm, dense;
  uhb::make_trees(B, &adm, &dense);
  const int32_t ncl = static_cast<int32_t>(B.cl.size());
  uhb::fill_model_tree(M, B, adm, dense);
  const double t1 = now_s();
  M->info.seconds_tree = t1 - t0;

  DevMem mem;
  int dev = 0, sms = 0;
  GTRY(cudaGetDevice(&dev));
  GTRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 2 * sms;
  // points in cluster order
  std::vector<double> px(n), py(n), pz(n);
  for (int64_t p = 0; p < n; ++p) {
    const int64_t i = B.perm[p];
    px[p] = points[3 * i];
    py[p] = points[3 * i + 1];
    pz[p] = points[3 * i + 2];
  }
  double *dx, *dy, *dz;
  GTRY(mem.upload(&dx, px));
  GTRY(mem.upload(&dy, py));
  GTRY(mem.upload(&dz, pz));
  const Points P{dx, dy, dz, prm->wavenumber, 1.0 / static_cast<double>(n)};

  // ---- admissible blocks: ACA + recompression
  const int64_t na = static_cast<int64_t>(adm.size());
  std::vector<int64_t> r0(na), c0(na), uoff(na), voff(na);
  std::vector<int32_t> mm(na), nn(na);
  int64_t su = 0, svv = 0;
  int32_t maxm = 1;
  for (int64_t b = 0; b < na; ++b) {
    const uhb::Cluster& a = B.cl[adm[b].first];
    const uhb::Cluster& c = B.cl[adm[b].second];
    r0[b] = a.begin;
    mm[b] = static_cast<int32_t>(a.size);
    c0[b] = c.begin;
    nn[b] = static_cast<int32_t>(c.size);
    uoff[b] = su;
    voff[b] = svv;
    su += a.size * kCap;
    svv += c.size * kCap;
    maxm = std::max(maxm, mm[b]);
  }
  int64_t *d_r0, *d_c0, *d_uoff, *d_voff;
  int32_t *d_m, *d_n, *d_rank, *d_kb;
  double2 *dU, *dV, *d_small;
  double* d_sv;
  GTRY(mem.upload(&d_r0, r0));
  GTRY(mem.upload(&d_c0, c0));
  GTRY(mem.upload(&d_uoff, uoff));
  GTRY(mem.upload(&d_voff, voff));
  GTRY(mem.upload(&d_m, mm));
  GTRY(mem.upload(&d_n, nn));
  GTRY(mem.alloc(&d_rank, na));
  GTRY(mem.alloc(&d_kb, na));
  GTRY(mem.alloc(&dU, su));
  GTRY(mem.alloc(&dV, svv));
  GTRY(mem.alloc(&d_sv, na * kCap));
  GTRY(mem.alloc(&d_small, static_cast<size_t>(grid) * std::max(3 * kCap * kCap, 2 * kRowMax * kCap)));
  const BlockTab T{d_r0, d_m, d_c0, d_n, d_uoff, d_voff};
  if (na > 0) {
    GTRY(cudaFuncSetAttribute(aca_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxm));
    aca_kernel<<<grid, kThreads, maxm>>>(P, T, na, prm->tol_aca, dU, dV, d_rank);
    GTRY(cudaGetLastError());
    recompress_kernel<<<grid, kThreads>>>(T, na, d_rank, prm->tol_aca, dU, dV, d_small, d_sv, d_kb);
    GTRY(cudaGetLastError());
  }
  std::vector<int32_t> rank, kb;
  std::vector<double> sv;
  GTRY(download(rank, d_rank, na));
  GTRY(download(kb, d_kb, na));
  GTRY(download(sv, d_sv, na * kCap));
  for (int64_t b = 0; b < na; ++b)
    if (rank[b] < 0) {
      delete M;
      return uh::set_error(UH_EINVAL, "device build: ACA of block %lld (%d x %d) did not reach tol_aca in %d terms",
                           (long long)b, mm[b], nn[b], kCap);
    }
  const double t2 = now_s();
  M->info.seconds_aca = t2 - t1;

  // ---- H form: each block's singular values > eps s_1
  M->adm_row.resize(na);
  M->adm_col.resize(na);
  M->h_rank.resize(na);
  M->X_off.resize(na);
  M->Y_off.resize(na);
  int64_t px_len = 0, py_len = 0;
  int32_t kmax_aca = 0, kmax_h = 0;
  for (int64_t b = 0; b < na; ++b) {
    M->adm_row[b] = adm[b].first;
    M->adm_col[b] = adm[b].second;
    int32_t k = 0;
    while (k < kb[b] && sv[b * kCap + k] > prm->eps * sv[b * kCap]) ++k;
    M->h_rank[b] = k;
    M->X_off[b] = px_len;
    M->Y_off[b] = py_len;
    px_len += static_cast<int64_t>(mm[b]) * k;
    py_len += static_cast<int64_t>(nn[b]) * k;
    kmax_aca = std::max(kmax_aca, kb[b]);
    kmax_h = std::max(kmax_h, k);
  }
  {
    double2 *dXh, *dYh;
    int32_t* d_h;
    int64_t *d_xo, *d_yo;
    GTRY(mem.alloc(&dXh, px_len));
    GTRY(mem.alloc(&dYh, py_len));
    GTRY(mem.upload(&d_h, M->h_rank));
    GTRY(mem.upload(&d_xo, M->X_off));
    GTRY(mem.upload(&d_yo, M->Y_off));
    if (na > 0) {
      hform_kernel<<<grid, kThreads>>>(T, na, dU, dV, d_sv, d_h, d_xo, d_yo, dXh, dYh);
      GTRY(cudaGetLastError());
    }
    GTRY(download(M->X, reinterpret_cast<const cd*>(dXh), px_len));
    GTRY(download(M->Y, reinterpret_cast<const cd*>(dYh), py_len));
  }

  // ---- cluster bases: one work item per row cluster and per column cluster with blocks
  std::vector<std::vector<int64_t>> rows_of(ncl), cols_of(ncl);
  for (int64_t b = 0; b < na; ++b) {
    rows_of[adm[b].first].push_back(b);   // sorted by sigma: adm is sorted
    cols_of[adm[b].second].push_back(b);  // sorted by tau
  }
  std::vector<BasisWork> work;
  std::vector<int64_t> members;
  std::vector<int32_t> wcl;  // cluster of each work item
  for (int32_t c = 0; c < ncl; ++c)
    for (int side = 0; side < 2; ++side) {
      const auto& bl = side == 0 ? rows_of[c] : cols_of[c];
      if (bl.empty()) continue;
      BasisWork w{};
      w.first = static_cast<int64_t>(members.size());
      w.count = static_cast<int32_t>(bl.size());
      w.m = static_cast<int32_t>(B.cl[c].size);
      w.side = side;
      int64_t K = 0;
      for (int64_t b : bl) {
        members.push_back(b);
        K += kb[b];
      }
      w.K = static_cast<int32_t>(K);
      work.push_back(w);
      wcl.push_back(c);
    }
  // largest clusters first (balance), offsets of the scratch in that order
  std::vector<size_t> order(work.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a].m > work[b].m; });
  std::vector<BasisWork> sorted;
  std::vector<int32_t> scl;
  int64_t xs_len = 0, bs_len = 0, js_len = 0;
  int32_t maxK = 1;
  for (size_t i : order) {
    BasisWork w = work[i];
    const int64_t rcap = std::min<int64_t>(std::min<int64_t>(w.m, w.K), kRowMax);
    w.xoff = xs_len;
    w.boff = bs_len;
    w.joff = js_len;
    xs_len += static_cast<int64_t>(w.m) * w.K;
    bs_len += static_cast<int64_t>(w.K) * rcap;
    js_len += rcap * rcap;
    maxK = std::max(maxK, w.K);
    sorted.push_back(w);
    scl.push_back(wcl[i]);
  }
  const int64_t nw = static_cast<int64_t>(sorted.size());
  BasisWork* d_work;
  int64_t* d_members;
  double2 *dXs, *dBs, *dJs;
  int32_t* d_ell;
  GTRY(mem.upload(&d_work, sorted));
  GTRY(mem.upload(&d_members, members));
  GTRY(mem.alloc(&dXs, xs_len));
  GTRY(mem.alloc(&dBs, bs_len));
  GTRY(mem.alloc(&dJs, js_len));
  GTRY(mem.alloc(&d_ell, nw));
  const int basis_smem = maxK * 12;
  if (nw > 0) {
    GTRY(cudaFuncSetAttribute(basis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, basis_smem));
    basis_kernel<<<grid, kThreads, basis_smem>>>(d_work, nw, d_members, T, dU, dV, d_sv, d_kb, prm->eps, dXs, dBs, dJs,
                                                 d_ell);
    GTRY(cudaGetLastError());
  }
  std::vector<int32_t> ell;
  GTRY(download(ell, d_ell, nw));
  std::vector<int32_t> lrow(ncl, 0), lcol(ncl, 0);
  std::vector<int64_t> xrow(ncl, -1), xcol(ncl, -1);
  for (int64_t w = 0; w < nw; ++w) {
    if (ell[w] < 0) {
      delete M;
      return uh::set_error(UH_EINVAL, "device build: numerical rank of cluster %d above %d", scl[w], kRowMax);
    }
    (sorted[w].side == 0 ? lrow : lcol)[scl[w]] = ell[w];
    (sorted[w].side == 0 ? xrow : xcol)[scl[w]] = sorted[w].xoff;
  }
  // compact bases, in cluster order as the host builder lays them out
  M->row_rank.assign(ncl, 0);
  M->col_rank.assign(ncl, 0);
  M->row_off.assign(ncl, 0);
  M->col_off.assign(ncl, 0);
  int64_t pu = 0, pv = 0;
  int32_t lmax = 0;
  for (int32_t c = 0; c < ncl; ++c) {
    M->row_rank[c] = lrow[c];
    M->col_rank[c] = lcol[c];
    M->row_off[c] = pu;
    M->col_off[c] = pv;
    pu += B.cl[c].size * lrow[c];
    pv += B.cl[c].size * lcol[c];
    lmax = std::max(lmax, std::max(lrow[c], lcol[c]));
  }
  for (int side = 0; side < 2; ++side) {
    std::vector<int64_t> gx, go, gl;
    for (int32_t c = 0; c < ncl; ++c) {
      const int32_t l = side == 0 ? lrow[c] : lcol[c];
      if (l == 0) continue;
      gx.push_back(side == 0 ? xrow[c] : xcol[c]);
      go.push_back(side == 0 ? M->row_off[c] : M->col_off[c]);
      gl.push_back(B.cl[c].size * l);
    }
    const int64_t total = side == 0 ? pu : pv;
    double2* dst;
    int64_t *d_gx, *d_go, *d_gl;
    GTRY(mem.alloc(&dst, total));
    GTRY(mem.upload(&d_gx, gx));
    GTRY(mem.upload(&d_go, go));
    GTRY(mem.upload(&d_gl, gl));
    if (!gx.empty()) {
      gather_kernel<<<grid, kThreads>>>(d_gx, d_go, d_gl, static_cast<int64_t>(gx.size()), dXs, dst);
      GTRY(cudaGetLastError());
    }
    GTRY(download(side == 0 ? M->U : M->V, reinterpret_cast<const cd*>(dst), total));
  }
  // coupling matrices, in block order; with the factored option the pairs too, recompressed at
  // eps, and each block keeps the smaller form
  const bool factored = prm->factored != 0;
  std::vector<CouplingWork> cw(na);
  std::vector<int64_t> dense_off(na);
  std::vector<int32_t> plt(na), pls(na);
  int64_t ps = 0, pp = 0, pr = 0;
  for (int64_t b = 0; b < na; ++b) {
    const int32_t a = adm[b].first, c = adm[b].second;
    dense_off[b] = ps;
    plt[b] = lrow[a];
    pls[b] = lcol[c];
    cw[b] = CouplingWork{std::max<int64_t>(xrow[a], 0), std::max<int64_t>(xcol[c], 0), ps, pp, pr, lrow[a], lcol[c]};
    ps += static_cast<int64_t>(lrow[a]) * lcol[c];
    if (factored) {
      pp += static_cast<int64_t>(lrow[a]) * kCap;
      pr += static_cast<int64_t>(lcol[c]) * kCap;
    }
  }
  std::vector<cd> Sdense, Pf, Rf;
  std::vector<int32_t> kf;
  std::vector<double> sf;
  {
    CouplingWork* d_cw;
    double2 *dS, *dP = nullptr, *dR = nullptr;
    GTRY(mem.upload(&d_cw, cw));
    GTRY(mem.alloc(&dS, ps));
    if (factored) {
      GTRY(mem.alloc(&dP, pp));
      GTRY(mem.alloc(&dR, pr));
    }
    if (na > 0) {
      coupling_kernel<<<grid, kThreads>>>(d_cw, T, na, dXs, dU, dV, d_sv, d_kb, d_small, dS, dP, dR);
      GTRY(cudaGetLastError());
    }
    GTRY(download(Sdense, reinterpret_cast<const cd*>(dS), ps));
    if (factored && na > 0) {
      std::vector<int64_t> poff(na), roff(na);
      std::vector<int32_t> kp(na);  // the pair's inner rank (0 where a basis is empty: no pair)
      for (int64_t b = 0; b < na; ++b) {
        poff[b] = cw[b].poff;
        roff[b] = cw[b].roff;
        kp[b] = plt[b] > 0 && pls[b] > 0 ? kb[b] : 0;
      }
      int64_t *d_poff, *d_roff;
      int32_t *d_lt, *d_ls, *d_kf, *d_kp;
      GTRY(mem.upload(&d_kp, kp));
      double* d_sf;
      GTRY(mem.upload(&d_poff, poff));
      GTRY(mem.upload(&d_roff, roff));
      GTRY(mem.upload(&d_lt, plt));
      GTRY(mem.upload(&d_ls, pls));
      GTRY(mem.alloc(&d_kf, na));
      GTRY(mem.alloc(&d_sf, na * kCap));
      const BlockTab TP{nullptr, d_lt, nullptr, d_ls, d_poff, d_roff};
      recompress_kernel<<<grid, kThreads>>>(TP, na, d_kp, prm->eps, dP, dR, d_small, d_sf, d_kf);
      GTRY(cudaGetLastError());
      GTRY(download(kf, d_kf, na));
      GTRY(download(sf, d_sf, na * kCap));
      GTRY(download(Pf, reinterpret_cast<const cd*>(dP), pp));
      GTRY(download(Rf, reinterpret_cast<const cd*>(dR), pr));
    }
  }
  M->S_off.resize(na);
  if (factored) M->S_rank.assign(na, -1);
  int64_t fs = 0;
  for (int64_t b = 0; b < na; ++b) {
    M->S_off[b] = fs;
    const int64_t lt = plt[b], ls = pls[b];
    if (factored && lt > 0 && ls > 0 && static_cast<int64_t>(kf[b]) * (lt + ls) < lt * ls) {
      M->S_rank[b] = kf[b];
      fs += static_cast<int64_t>(kf[b]) * (lt + ls);
    } else {
      fs += lt * ls;
    }
  }
  M->S.resize(fs);
  for (int64_t b = 0; b < na; ++b) {
    const int64_t lt = plt[b], ls = pls[b];
    cd* out = M->S.data() + M->S_off[b];
    if (factored && M->S_rank[b] >= 0) {
      // S_X = Q1 W diag(s) (in P's place), S_Y = Q2 Z (in conj(R)'s place)
      for (int j = 0; j < M->S_rank[b]; ++j) {
        for (int64_t i = 0; i < lt; ++i) out[j * lt + i] = Pf[cw[b].poff + j * lt + i] * sf[b * kCap + j];
        for (int64_t i = 0; i < ls; ++i) out[lt * M->S_rank[b] + j * ls + i] = Rf[cw[b].roff + j * ls + i];
      }
    } else {
      std::copy(Sdense.begin() + dense_off[b], Sdense.begin() + dense_off[b] + lt * ls, out);
    }
  }
  const double t3 = now_s();
  M->info.seconds_bases = t3 - t2;

  // ---- near field
  const int64_t nd = static_cast<int64_t>(dense.size());
  M->dense_row.resize(nd);
  M->dense_col.resize(nd);
  M->D_off.resize(nd);
  std::vector<int64_t> dr0(nd), dc0(nd);
  std::vector<int32_t> dm(nd), dn(nd);
  int64_t pd = 0;
  for (int64_t q = 0; q < nd; ++q) {
    const uhb::Cluster& a = B.cl[dense[q].first];
    const uhb::Cluster& c = B.cl[dense[q].second];
    M->dense_row[q] = dense[q].first;
    M->dense_col[q] = dense[q].second;
    M->D_off[q] = pd;
    dr0[q] = a.begin;
    dc0[q] = c.begin;
    dm[q] = static_cast<int32_t>(a.size);
    dn[q] = static_cast<int32_t>(c.size);
    pd += a.size * c.size;
  }
  {
    int64_t *d_dr0, *d_dc0, *d_doff;
    int32_t *d_dm, *d_dn;
    double2* dD;
    GTRY(mem.upload(&d_dr0, dr0));
    GTRY(mem.upload(&d_dc0, dc0));
    GTRY(mem.upload(&d_doff, M->D_off));
    GTRY(mem.upload(&d_dm, dm));
    GTRY(mem.upload(&d_dn, dn));
    GTRY(mem.alloc(&dD, pd));
    if (nd > 0) {
      dense_kernel<<<grid, kThreads>>>(P, d_dr0, d_dm, d_dc0, d_dn, d_doff, nd, dD);
      GTRY(cudaGetLastError());
    }
    GTRY(download(M->D, reinterpret_cast<const cd*>(dD), pd));
  }
  M->info.seconds_dense = now_s() - t3;
  M->info.kmax_aca = kmax_aca;
  M->info.kmax_h = kmax_h;
  M->info.lmax = lmax;
  *out = M;
  return UH_OK;
}

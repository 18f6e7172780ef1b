// Host-side construction of the synthetic Helmholtz operators in UH and H form (uh_build.h).
// Independent of the products: it only fills the descriptors that uh_create / h_create take.
#include "uh_build.h"

#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <numeric>
#include <vector>

#include "uh_build_internal.h"
#include "uh_internal.h"

using cd = std::complex<double>;
using uhb::Builder;
using uhb::Cluster;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------------- dense kernels
// Column-major matrices as flat std::vector<cd>.

double colnorm2(int m, const cd* a) {
  double s = 0;
  for (int i = 0; i < m; ++i) s += std::norm(a[i]);
  return s;
}

// Householder vector for x (length L): v (normalised, L entries) with (I - 2 v v^*) x = beta e_1.
// Returns false if x = 0 (no reflection).
bool householder(int L, const cd* x, cd* v, cd* beta) {
  const double alpha = std::sqrt(colnorm2(L, x));
  if (alpha == 0.0) {
    *beta = 0.0;
    return false;
  }
  const double ax0 = std::abs(x[0]);
  const cd phase = ax0 > 0 ? x[0] / ax0 : cd(1.0, 0.0);
  *beta = -phase * alpha;
  for (int i = 0; i < L; ++i) v[i] = x[i];
  v[0] -= *beta;
  const double nv = std::sqrt(colnorm2(L, v));
  for (int i = 0; i < L; ++i) v[i] /= nv;
  return true;
}

// y <- (I - 2 v v^*) y, length L.
void reflect(int L, const cd* v, cd* y) {
  cd d = 0;
  for (int i = 0; i < L; ++i) d += std::conj(v[i]) * y[i];
  d *= 2.0;
  for (int i = 0; i < L; ++i) y[i] -= v[i] * d;
}

// Column-pivoted Householder QR of A (m x n), stopped when the Frobenius norm of the
// untreated block is <= abs_tol (or all min(m, n) steps are done). Returns the rank r and
// Q (m x r, orthonormal columns) and Rt (r x n) with A ~ Q Rt, Rt in the ORIGINAL column order.
int rrqr(int m, int n, const cd* A, double abs_tol, std::vector<cd>& Q, std::vector<cd>& Rt) {
  std::vector<cd> W(A, A + static_cast<size_t>(m) * n);
  std::vector<int> piv(n);
  std::iota(piv.begin(), piv.end(), 0);
  std::vector<double> nrm(n);
  const int p = std::min(m, n);
  std::vector<std::vector<cd>> vs;
  std::vector<cd> v(m);
  int r = 0;
  for (int j = 0; j < p; ++j) {
    double rest = 0;
    int best = j;
    for (int c = j; c < n; ++c) {
      nrm[c] = colnorm2(m - j, &W[static_cast<size_t>(c) * m + j]);
      rest += nrm[c];
      if (nrm[c] > nrm[best]) best = c;
    }
    if (std::sqrt(rest) <= abs_tol) break;
    if (best != j) {
      std::swap_ranges(&W[static_cast<size_t>(j) * m], &W[static_cast<size_t>(j) * m] + m, &W[static_cast<size_t>(best) * m]);
      std::swap(piv[j], piv[best]);
    }
    cd beta;
    const int L = m - j;
    householder(L, &W[static_cast<size_t>(j) * m + j], v.data(), &beta);
    for (int c = j + 1; c < n; ++c) reflect(L, v.data(), &W[static_cast<size_t>(c) * m + j]);
    W[static_cast<size_t>(j) * m + j] = beta;
    for (int i = j + 1; i < m; ++i) W[static_cast<size_t>(j) * m + i] = 0.0;
    vs.emplace_back(v.begin(), v.begin() + L);
    r = j + 1;
  }
  Q.assign(static_cast<size_t>(m) * r, 0.0);
  for (int j = 0; j < r; ++j) Q[static_cast<size_t>(j) * m + j] = 1.0;
  for (int j = r - 1; j >= 0; --j)
    for (int c = 0; c < r; ++c) reflect(m - j, vs[j].data(), &Q[static_cast<size_t>(c) * m + j]);
  Rt.assign(static_cast<size_t>(r) * n, 0.0);
  for (int c = 0; c < n; ++c)
    for (int i = 0; i < r && i <= c; ++i) Rt[static_cast<size_t>(piv[c]) * r + i] = W[static_cast<size_t>(c) * m + i];
  return r;
}

// One-sided (Hestenes) Jacobi: B (m x n) <- B J with mutually orthogonal columns, J unitary
// (n x n, accumulated if J != nullptr, initialised to I here).
void jacobi(int m, int n, cd* B, cd* J) {
  if (J) {
    std::fill(J, J + static_cast<size_t>(n) * n, cd(0.0));
    for (int i = 0; i < n; ++i) J[static_cast<size_t>(i) * n + i] = 1.0;
  }
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int i = 0; i < n - 1; ++i) {
      for (int j = i + 1; j < n; ++j) {
        cd* bi = B + static_cast<size_t>(i) * m;
        cd* bj = B + static_cast<size_t>(j) * m;
        double a = 0, b = 0;
        cd g = 0;
        for (int k = 0; k < m; ++k) {
          a += std::norm(bi[k]);
          b += std::norm(bj[k]);
          g += std::conj(bi[k]) * bj[k];
        }
        const double ag = std::abs(g);
        if (ag == 0.0 || ag <= 1e-15 * std::sqrt(a * b)) continue;
        rotated = true;
        // Rotate (b_i, e^{-i phi} b_j) by the real Jacobi angle that zeroes their inner product.
        const cd ph = g / ag;  // e^{i phi}
        const double zeta = (b - a) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::abs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        const cd phc = std::conj(ph);
        for (int k = 0; k < m; ++k) {
          const cd x = bi[k], y = bj[k] * phc;
          bi[k] = c * x - s * y;
          bj[k] = s * x + c * y;
        }
        if (J) {
          cd* ji = J + static_cast<size_t>(i) * n;
          cd* jj = J + static_cast<size_t>(j) * n;
          for (int k = 0; k < n; ++k) {
            const cd x = ji[k], y = jj[k] * phc;
            ji[k] = c * x - s * y;
            jj[k] = s * x + c * y;
          }
        }
      }
    }
    if (!rotated) break;
  }
}

// Left singular vectors of X (m x K) with singular value > rel * sigma_1: U (m x l), l.
void left_basis(int m, int K, const cd* X, double rel, std::vector<cd>& U, int* l) {
  double maxc = 0;
  for (int c = 0; c < K; ++c) maxc = std::max(maxc, std::sqrt(colnorm2(m, X + static_cast<size_t>(c) * m)));
  *l = 0;
  U.clear();
  if (maxc == 0.0) return;
  std::vector<cd> Q, Rt;
  const int r = rrqr(m, K, X, 1e-3 * rel * maxc, Q, Rt);
  // Rt (r x K) = W Sigma Z^*: one-sided Jacobi on B = Rt^* (K x r) gives B J = Z Sigma, so
  // Rt = J Sigma Z^* and the left vectors of X are Q J.
  std::vector<cd> B(static_cast<size_t>(K) * r), J(static_cast<size_t>(r) * r);
  for (int i = 0; i < r; ++i)
    for (int c = 0; c < K; ++c) B[static_cast<size_t>(i) * K + c] = std::conj(Rt[static_cast<size_t>(c) * r + i]);
  jacobi(K, r, B.data(), J.data());
  std::vector<double> sv(r);
  for (int i = 0; i < r; ++i) sv[i] = std::sqrt(colnorm2(K, &B[static_cast<size_t>(i) * K]));
  std::vector<int> ord(r);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  if (r == 0 || sv[ord[0]] == 0.0) return;
  int keep = 0;
  while (keep < r && sv[ord[keep]] > rel * sv[ord[0]]) ++keep;
  U.assign(static_cast<size_t>(m) * keep, 0.0);
  for (int q = 0; q < keep; ++q) {
    const cd* jc = &J[static_cast<size_t>(ord[q]) * r];
    cd* uc = &U[static_cast<size_t>(q) * m];
    for (int i = 0; i < r; ++i) {
      const cd w = jc[i];
      const cd* qc = &Q[static_cast<size_t>(i) * m];
      for (int k = 0; k < m; ++k) uc[k] += qc[k] * w;
    }
  }
  *l = keep;
}

// Thin Householder QR of A (m x k): Q (m x p), R (p x k), p = min(m, k).
void qr_thin(int m, int k, const cd* A, std::vector<cd>& Q, std::vector<cd>& R) {
  std::vector<cd> W(A, A + static_cast<size_t>(m) * k);
  const int p = std::min(m, k);
  std::vector<std::vector<cd>> vs(p);
  std::vector<cd> v(m);
  for (int j = 0; j < p; ++j) {
    cd beta;
    const int L = m - j;
    if (householder(L, &W[static_cast<size_t>(j) * m + j], v.data(), &beta)) {
      for (int c = j + 1; c < k; ++c) reflect(L, v.data(), &W[static_cast<size_t>(c) * m + j]);
      vs[j].assign(v.begin(), v.begin() + L);
    }
    W[static_cast<size_t>(j) * m + j] = beta;
  }
  R.assign(static_cast<size_t>(p) * k, 0.0);
  for (int c = 0; c < k; ++c)
    for (int i = 0; i <= std::min(c, p - 1); ++i) R[static_cast<size_t>(c) * p + i] = W[static_cast<size_t>(c) * m + i];
  Q.assign(static_cast<size_t>(m) * p, 0.0);
  for (int j = 0; j < p; ++j) Q[static_cast<size_t>(j) * m + j] = 1.0;
  for (int j = p - 1; j >= 0; --j)
    if (!vs[j].empty())
      for (int c = 0; c < p; ++c) reflect(m - j, vs[j].data(), &Q[static_cast<size_t>(c) * m + j]);
}

// ------------------------------------------------------------------------- geometry

struct LowRank {
  int32_t k = 0;              // rank after recompression at tol_aca
  std::vector<cd> Ub, Yb;     // |tau| x k and |sigma| x k, orthonormal columns
  std::vector<double> s;      // singular values, descending
};

// Algebraic recompression (Section 2.3) of X Y^* (X m x k, Y nn x k): QR of both factors, SVD of
// R1 R2^* by one-sided Jacobi, keep the singular values > tol * s_1. Returns U_b = Q1 W, Y_b = Q2 Z
// and s with X Y^* ~ U_b diag(s) Y_b^*.
LowRank recompress_pair(int m, int nn, int k, const cd* X, const cd* Y, double tol) {
  LowRank out;
  if (k == 0) return out;
  std::vector<cd> Q1, R1, Q2, R2;
  qr_thin(m, k, X, Q1, R1);
  qr_thin(nn, k, Y, Q2, R2);
  const int p1 = std::min(m, k), p2 = std::min(nn, k);
  std::vector<cd> Mx(static_cast<size_t>(p1) * p2, 0.0);  // R1 R2^*
  for (int b = 0; b < p2; ++b)
    for (int q = 0; q < k; ++q) {
      const cd w = std::conj(R2[static_cast<size_t>(q) * p2 + b]);
      if (w == 0.0) continue;
      for (int a = 0; a < p1; ++a) Mx[static_cast<size_t>(b) * p1 + a] += R1[static_cast<size_t>(q) * p1 + a] * w;
    }
  std::vector<cd> J(static_cast<size_t>(p2) * p2);
  jacobi(p1, p2, Mx.data(), J.data());  // Mx J = W Sigma
  std::vector<double> sv(p2);
  for (int q = 0; q < p2; ++q) sv[q] = std::sqrt(colnorm2(p1, &Mx[static_cast<size_t>(q) * p1]));
  std::vector<int> ord(p2);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  if (sv[ord[0]] == 0.0) return out;
  int keep = 0;
  while (keep < p2 && sv[ord[keep]] > tol * sv[ord[0]]) ++keep;
  out.k = keep;
  out.s.resize(keep);
  out.Ub.assign(static_cast<size_t>(m) * keep, 0.0);
  out.Yb.assign(static_cast<size_t>(nn) * keep, 0.0);
  for (int q = 0; q < keep; ++q) {
    const int col = ord[q];
    out.s[q] = sv[col];
    // left vector w = Mx[:, col] / sigma; U_b = Q1 w
    for (int a = 0; a < p1; ++a) {
      const cd w = Mx[static_cast<size_t>(col) * p1 + a] / sv[col];
      for (int t = 0; t < m; ++t) out.Ub[static_cast<size_t>(q) * m + t] += Q1[static_cast<size_t>(a) * m + t] * w;
    }
    // right vector = J[:, col]; Y_b = Q2 J[:, col]
    for (int b = 0; b < p2; ++b) {
      const cd w = J[static_cast<size_t>(col) * p2 + b];
      for (int t = 0; t < nn; ++t) out.Yb[static_cast<size_t>(q) * nn + t] += Q2[static_cast<size_t>(b) * nn + t] * w;
    }
  }
  return out;
}

// Partially pivoted ACA of block (rows, cols) followed by recompression (Section 2.3).
LowRank aca_block(const Builder& B, const int64_t* rows, int m, const int64_t* cols, int nn, double tol) {
  std::vector<std::vector<cd>> us, vs;
  std::vector<char> used(m, 0);
  double norm2 = 0;
  int i = 0;
  const int kmax = std::min(m, nn);
  std::vector<cd> r(nn), c(m);
  while (static_cast<int>(us.size()) < kmax) {
    for (int j = 0; j < nn; ++j) r[j] = B.entry(rows[i], cols[j]);
    for (size_t q = 0; q < us.size(); ++q) {
      const cd ui = us[q][i];
      for (int j = 0; j < nn; ++j) r[j] -= ui * vs[q][j];
    }
    used[i] = 1;
    int jp = 0;
    for (int j = 1; j < nn; ++j)
      if (std::abs(r[j]) > std::abs(r[jp])) jp = j;
    if (std::abs(r[jp]) == 0.0) {
      int f = -1;
      for (int q = 0; q < m; ++q)
        if (!used[q]) { f = q; break; }
      if (f < 0) break;
      i = f;
      continue;
    }
    const cd piv = r[jp];
    std::vector<cd> v(nn), u(m);
    for (int j = 0; j < nn; ++j) v[j] = r[j] / piv;
    for (int q = 0; q < m; ++q) u[q] = B.entry(rows[q], cols[jp]);
    for (size_t q = 0; q < us.size(); ++q) {
      const cd vj = vs[q][jp];
      for (int t = 0; t < m; ++t) u[t] -= vj * us[q][t];
    }
    double cross = 0;
    for (size_t q = 0; q < us.size(); ++q) {
      cd a = 0, b = 0;
      for (int t = 0; t < m; ++t) a += std::conj(us[q][t]) * u[t];
      for (int t = 0; t < nn; ++t) b += std::conj(vs[q][t]) * v[t];
      cross += (a * b).real();
    }
    const double nu = std::sqrt(colnorm2(m, u.data())), nv = std::sqrt(colnorm2(nn, v.data()));
    norm2 += 2.0 * cross + nu * nu * nv * nv;
    us.push_back(std::move(u));
    vs.push_back(std::move(v));
    if (nu * nv <= tol * std::sqrt(std::max(norm2, 0.0))) break;
    int nxt = -1;
    double best = -1;
    for (int t = 0; t < m; ++t)
      if (!used[t] && std::abs(us.back()[t]) > best) { best = std::abs(us.back()[t]); nxt = t; }
    if (nxt < 0) break;
    i = nxt;
  }
  const int k = static_cast<int>(us.size());
  if (k == 0) return LowRank();
  // A ~ U V^T = X Y^* with X = U, Y = conj(V).
  std::vector<cd> X(static_cast<size_t>(m) * k), Y(static_cast<size_t>(nn) * k);
  for (int q = 0; q < k; ++q) {
    std::copy(us[q].begin(), us[q].end(), &X[static_cast<size_t>(q) * m]);
    for (int t = 0; t < nn; ++t) Y[static_cast<size_t>(q) * nn + t] = std::conj(vs[q][t]);
  }
  return recompress_pair(m, nn, k, X.data(), Y.data(), tol);
}

}  // namespace

namespace {

void fill_tree(const uh_model* m, uh_tree_desc* t) {
  t->n = m->info.n;
  t->perm = m->perm.data();
  t->n_clusters = static_cast<int32_t>(m->cl_begin.size());
  t->cl_begin = m->cl_begin.data();
  t->cl_size = m->cl_size.data();
}

void fill_dense(const uh_model* m, uh_dense_desc* d) {
  d->n_dense = static_cast<int64_t>(m->dense_row.size());
  d->row_cl = m->dense_row.data();
  d->col_cl = m->dense_col.data();
  d->off = m->D_off.data();
  d->data = m->D.data();
  d->len = static_cast<int64_t>(m->D.size());
}

}  // namespace

int uhb::check_build_args(int64_t n, const double* points, const uhb_params* prm, uh_model** out) {
  if (!points || !prm || !out) return uh::set_error(UH_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1 || n > INT32_MAX) return uh::set_error(UH_EINVAL, "n = %lld out of range", (long long)n);
  if (prm->leaf < 1 || !(prm->eta > 0) || !(prm->eps >= 0 && prm->eps < 1) || !(prm->tol_aca > 0 && prm->tol_aca < 1))
    return uh::set_error(UH_EINVAL, "invalid parameters (leaf %d, eta %g, eps %g, tol_aca %g)", prm->leaf, prm->eta,
                         prm->eps, prm->tol_aca);
  if (prm->strong != 0 && prm->strong != 1) return uh::set_error(UH_EINVAL, "strong = %d (0 or 1)", prm->strong);
  if (prm->factored != 0 && prm->factored != 1)
    return uh::set_error(UH_EINVAL, "factored = %d (0 or 1)", prm->factored);
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(points[i])) return uh::set_error(UH_EINVAL, "point coordinate %lld is not finite", (long long)i);
  return UH_OK;
}

void uhb::fill_model_tree(uh_model* M, const Builder& B, const BlockList& adm, const BlockList& dense) {
  const int32_t ncl = static_cast<int32_t>(B.cl.size());
  M->perm = B.perm;
  M->cl_begin.resize(ncl);
  M->cl_size.resize(ncl);
  int32_t depth = 0;
  for (int32_t c = 0; c < ncl; ++c) {
    M->cl_begin[c] = B.cl[c].begin;
    M->cl_size[c] = B.cl[c].size;
    depth = std::max(depth, B.cl[c].level + 1);
  }
  std::vector<int32_t> rc(ncl, 0), cc(ncl, 0);
  int32_t csp = 0;
  for (auto& pr : adm) {
    csp = std::max(csp, ++rc[pr.first]);
    csp = std::max(csp, ++cc[pr.second]);
  }
  M->info.n = B.n;
  M->info.n_clusters = ncl;
  M->info.n_adm = static_cast<int64_t>(adm.size());
  M->info.n_dense = static_cast<int64_t>(dense.size());
  M->info.depth = depth;
  M->info.csp = csp;
}

extern "C" {

int uhb_build_helmholtz(int64_t n, const double* points, const uhb_params* prm, uh_model** out) {
  int rc;
  if ((rc = uhb::check_build_args(n, points, prm, out))) return rc;
  if (prm->nthreads > 0) omp_set_num_threads(prm->nthreads);
  auto* M = new (std::nothrow) uh_model();
  if (!M) return uh::set_error(UH_ENOMEM, "host allocation");
  double t0 = now_s();
  Builder B;
  B.n = n;
  B.pts = points;
  B.prm = *prm;
  uhb::BlockList adm, dense;
  uhb::make_trees(B, &adm, &dense);
  const int32_t ncl = static_cast<int32_t>(B.cl.size());
  uhb::fill_model_tree(M, B, adm, dense);
  double t1 = now_s();
  M->info.seconds_tree = t1 - t0;

  // ACA + recompression per admissible block.
  const int64_t na = static_cast<int64_t>(adm.size());
  std::vector<LowRank> lr(na);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < na; ++q) {
    const Cluster& a = B.cl[adm[q].first];
    const Cluster& b = B.cl[adm[q].second];
    lr[q] = aca_block(B, &B.perm[a.begin], static_cast<int>(a.size), &B.perm[b.begin], static_cast<int>(b.size),
                      prm->tol_aca);
  }
  double t2 = now_s();
  M->info.seconds_aca = t2 - t1;

  // H operator: blocks truncated at eps.
  M->adm_row.resize(na);
  M->adm_col.resize(na);
  M->h_rank.resize(na);
  M->X_off.resize(na);
  M->Y_off.resize(na);
  int64_t px = 0, py = 0;
  int32_t kmax_aca = 0, kmax_h = 0;
  for (int64_t q = 0; q < na; ++q) {
    M->adm_row[q] = adm[q].first;
    M->adm_col[q] = adm[q].second;
    const LowRank& L = lr[q];
    int32_t k = 0;
    while (k < L.k && L.s[k] > prm->eps * L.s[0]) ++k;
    M->h_rank[q] = k;
    M->X_off[q] = px;
    M->Y_off[q] = py;
    px += B.cl[adm[q].first].size * k;
    py += B.cl[adm[q].second].size * k;
    kmax_aca = std::max(kmax_aca, L.k);
    kmax_h = std::max(kmax_h, k);
  }
  M->X.resize(px);
  M->Y.resize(py);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < na; ++q) {
    const LowRank& L = lr[q];
    const int64_t m = B.cl[adm[q].first].size, nn = B.cl[adm[q].second].size;
    for (int j = 0; j < M->h_rank[q]; ++j) {
      for (int64_t t = 0; t < m; ++t) M->X[M->X_off[q] + j * m + t] = L.Ub[j * m + t] * L.s[j];
      for (int64_t t = 0; t < nn; ++t) M->Y[M->Y_off[q] + j * nn + t] = L.Yb[j * nn + t];
    }
  }

  // UH operator: bases from the stacked scaled factors, then S_b by projection.
  std::vector<std::vector<int64_t>> rows_of(ncl), cols_of(ncl);
  for (int64_t q = 0; q < na; ++q) {
    rows_of[adm[q].first].push_back(q);   // sorted by sigma since adm is sorted
    cols_of[adm[q].second].push_back(q);  // sorted by tau
  }
  std::vector<std::vector<cd>> Ub(ncl), Vb(ncl);
  std::vector<int32_t> lrow(ncl, 0), lcol(ncl, 0);
  std::vector<std::pair<int32_t, int>> work;
  for (int32_t c = 0; c < ncl; ++c) {
    if (!rows_of[c].empty()) work.push_back({c, 0});
    if (!cols_of[c].empty()) work.push_back({c, 1});
  }
  std::sort(work.begin(), work.end(), [&](auto& a, auto& b) { return B.cl[a.first].size > B.cl[b.first].size; });
#pragma omp parallel for schedule(dynamic, 1)
  for (size_t w = 0; w < work.size(); ++w) {
    const int32_t c = work[w].first;
    const bool row = work[w].second == 0;
    const int64_t m = B.cl[c].size;
    const auto& blocks = row ? rows_of[c] : cols_of[c];
    int64_t K = 0;
    for (int64_t q : blocks) K += lr[q].k;
    std::vector<cd> Xs(static_cast<size_t>(m) * K);
    int64_t col = 0;
    for (int64_t q : blocks) {
      const LowRank& L = lr[q];
      const std::vector<cd>& F = row ? L.Ub : L.Yb;
      for (int j = 0; j < L.k; ++j, ++col)
        for (int64_t t = 0; t < m; ++t) Xs[col * m + t] = F[j * m + t] * L.s[j];
    }
    int l = 0;
    if (K > 0) left_basis(static_cast<int>(m), static_cast<int>(K), Xs.data(), prm->eps, row ? Ub[c] : Vb[c], &l);
    (row ? lrow : lcol)[c] = l;
  }
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
  M->U.resize(pu);
  M->V.resize(pv);
  for (int32_t c = 0; c < ncl; ++c) {
    std::copy(Ub[c].begin(), Ub[c].end(), M->U.begin() + M->row_off[c]);
    std::copy(Vb[c].begin(), Vb[c].end(), M->V.begin() + M->col_off[c]);
  }
  // Coupling matrices by projection: P = U_tau^* U_b Sigma_b, R = V_sigma^* V_b, S_b = P R^*. With
  // prm->factored the pair (P, R) is recompressed at eps (Section 2.3) and, where
  // k (l_tau + l_sigma) < l_tau l_sigma, stored as S_X = Q1 W diag(s), S_Y = Q2 Z (Section 4.2).
  std::vector<std::vector<cd>> Sq(na);
  M->S_rank.assign(prm->factored ? na : 0, -1);
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t q = 0; q < na; ++q) {
    const int32_t a = adm[q].first, b = adm[q].second;
    const int64_t m = B.cl[a].size, nn = B.cl[b].size;
    const int la = lrow[a], lb = lcol[b], k = lr[q].k;
    if (la == 0 || lb == 0) continue;
    const LowRank& L = lr[q];
    std::vector<cd> P(static_cast<size_t>(la) * k, 0.0), R(static_cast<size_t>(lb) * k, 0.0);
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < la; ++i) {  // P = U_tau^* U_b Sigma_b
        cd s = 0;
        const cd* u = &Ub[a][static_cast<size_t>(i) * m];
        const cd* f = &L.Ub[static_cast<size_t>(j) * m];
        for (int64_t t = 0; t < m; ++t) s += std::conj(u[t]) * f[t];
        P[static_cast<size_t>(j) * la + i] = s * L.s[j];
      }
      for (int i = 0; i < lb; ++i) {  // R = V_sigma^* V_b
        cd s = 0;
        const cd* v = &Vb[b][static_cast<size_t>(i) * nn];
        const cd* f = &L.Yb[static_cast<size_t>(j) * nn];
        for (int64_t t = 0; t < nn; ++t) s += std::conj(v[t]) * f[t];
        R[static_cast<size_t>(j) * lb + i] = s;
      }
    }
    if (prm->factored) {
      const LowRank f = recompress_pair(la, lb, k, P.data(), R.data(), prm->eps);
      if (static_cast<int64_t>(f.k) * (la + lb) < static_cast<int64_t>(la) * lb) {
        std::vector<cd>& out = Sq[q];
        out.assign(static_cast<size_t>(f.k) * (la + lb), 0.0);
        for (int j = 0; j < f.k; ++j) {
          for (int i = 0; i < la; ++i) out[static_cast<size_t>(j) * la + i] = f.Ub[static_cast<size_t>(j) * la + i] * f.s[j];
          for (int i = 0; i < lb; ++i)
            out[static_cast<size_t>(la) * f.k + static_cast<size_t>(j) * lb + i] = f.Yb[static_cast<size_t>(j) * lb + i];
        }
        M->S_rank[q] = f.k;
        continue;
      }
    }
    std::vector<cd>& S = Sq[q];  // S = P R^*  (la x lb)
    S.assign(static_cast<size_t>(la) * lb, 0.0);
    for (int jb = 0; jb < lb; ++jb)
      for (int j = 0; j < k; ++j) {
        const cd w = std::conj(R[static_cast<size_t>(j) * lb + jb]);
        for (int i = 0; i < la; ++i) S[static_cast<size_t>(jb) * la + i] += P[static_cast<size_t>(j) * la + i] * w;
      }
  }
  M->S_off.resize(na);
  int64_t ps = 0;
  for (int64_t q = 0; q < na; ++q) {
    M->S_off[q] = ps;
    ps += static_cast<int64_t>(Sq[q].size());
  }
  M->S.resize(ps);
  for (int64_t q = 0; q < na; ++q) {
    std::copy(Sq[q].begin(), Sq[q].end(), M->S.begin() + M->S_off[q]);
    std::vector<cd>().swap(Sq[q]);
  }
  double t3 = now_s();
  M->info.seconds_bases = t3 - t2;

  // Near field.
  const int64_t nd = static_cast<int64_t>(dense.size());
  M->dense_row.resize(nd);
  M->dense_col.resize(nd);
  M->D_off.resize(nd);
  int64_t pd = 0;
  for (int64_t q = 0; q < nd; ++q) {
    M->dense_row[q] = dense[q].first;
    M->dense_col[q] = dense[q].second;
    M->D_off[q] = pd;
    pd += B.cl[dense[q].first].size * B.cl[dense[q].second].size;
  }
  M->D.resize(pd);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < nd; ++q) {
    const Cluster& a = B.cl[dense[q].first];
    const Cluster& b = B.cl[dense[q].second];
    cd* D = &M->D[M->D_off[q]];
    for (int64_t j = 0; j < b.size; ++j)
      for (int64_t i = 0; i < a.size; ++i) D[j * a.size + i] = B.entry(B.perm[a.begin + i], B.perm[b.begin + j]);
  }
  M->info.seconds_dense = now_s() - t3;

  M->info.kmax_aca = kmax_aca;
  M->info.kmax_h = kmax_h;
  M->info.lmax = lmax;
  *out = M;
  return UH_OK;
}

int uhb_uh_desc(const uh_model* m, uh_desc* d) {
  if (!m || !d) return uh::set_error(UH_EINVAL, "null argument");
  std::memset(d, 0, sizeof *d);
  fill_tree(m, &d->tree);
  d->data_type = UH_DATA_C128;
  d->row_rank = m->row_rank.data();
  d->row_off = m->row_off.data();
  d->U_data = m->U.data();
  d->U_len = static_cast<int64_t>(m->U.size());
  d->col_rank = m->col_rank.data();
  d->col_off = m->col_off.data();
  d->V_data = m->V.data();
  d->V_len = static_cast<int64_t>(m->V.size());
  d->n_adm = static_cast<int64_t>(m->adm_row.size());
  d->adm_row = m->adm_row.data();
  d->adm_col = m->adm_col.data();
  d->S_off = m->S_off.data();
  d->S_data = m->S.data();
  d->S_len = static_cast<int64_t>(m->S.size());
  d->S_rank = m->S_rank.empty() ? nullptr : m->S_rank.data();
  fill_dense(m, &d->dense);
  return UH_OK;
}

int uhb_h_desc(const uh_model* m, h_desc* d) {
  if (!m || !d) return uh::set_error(UH_EINVAL, "null argument");
  std::memset(d, 0, sizeof *d);
  fill_tree(m, &d->tree);
  d->data_type = UH_DATA_C128;
  d->n_adm = static_cast<int64_t>(m->adm_row.size());
  d->adm_row = m->adm_row.data();
  d->adm_col = m->adm_col.data();
  d->adm_rank = m->h_rank.data();
  d->X_off = m->X_off.data();
  d->X_data = m->X.data();
  d->X_len = static_cast<int64_t>(m->X.size());
  d->Y_off = m->Y_off.data();
  d->Y_data = m->Y.data();
  d->Y_len = static_cast<int64_t>(m->Y.size());
  fill_dense(m, &d->dense);
  return UH_OK;
}

int uhb_info(const uh_model* m, uhb_info_t* out) {
  if (!m || !out) return uh::set_error(UH_EINVAL, "null argument");
  *out = m->info;
  return UH_OK;
}

int uhb_free(uh_model* m) {
  delete m;
  return UH_OK;
}

}  // extern "C"

// Internal to the host and device builders (uh_build.cpp, uh_gbuild.cu): the cluster tree and
// block cluster tree of the synthetic workloads (Defs. 2.1, 2.2), and the model that owns the
// descriptor arrays the builders fill.
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <numeric>
#include <utility>
#include <vector>

#include "uh_build.h"

namespace uhb {

using cd = std::complex<double>;
using BlockList = std::vector<std::pair<int32_t, int32_t>>;

struct Cluster {
  int64_t begin, size;
  int32_t level, parent, child0 = -1, child1 = -1;
  double lo[3], hi[3];
};

struct Builder {
  int64_t n = 0;
  const double* pts = nullptr;
  uhb_params prm{};
  std::vector<Cluster> cl;
  std::vector<int64_t> perm;  // position -> original index

  void split(int64_t begin, std::vector<int64_t>& idx, int32_t level, int32_t parent) {
    const int32_t id = static_cast<int32_t>(cl.size());
    Cluster c{};
    c.begin = begin;
    c.size = static_cast<int64_t>(idx.size());
    c.level = level;
    c.parent = parent;
    for (int d = 0; d < 3; ++d) { c.lo[d] = INFINITY; c.hi[d] = -INFINITY; }
    for (int64_t i : idx)
      for (int d = 0; d < 3; ++d) {
        c.lo[d] = std::min(c.lo[d], pts[3 * i + d]);
        c.hi[d] = std::max(c.hi[d], pts[3 * i + d]);
      }
    cl.push_back(c);
    if (c.size > prm.leaf) {
      int ax = 0;
      for (int d = 1; d < 3; ++d)
        if (c.hi[d] - c.lo[d] > c.hi[ax] - c.lo[ax]) ax = d;
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
        const double pa = pts[3 * a + ax], pb = pts[3 * b + ax];
        return pa < pb || (pa == pb && a < b);
      });
      const int64_t half = c.size / 2;
      std::vector<int64_t> left(idx.begin(), idx.begin() + half), right(idx.begin() + half, idx.end());
      idx.clear();
      idx.shrink_to_fit();
      const int32_t c0 = static_cast<int32_t>(cl.size());
      split(begin, left, level + 1, id);
      const int32_t c1 = static_cast<int32_t>(cl.size());
      split(begin + half, right, level + 1, id);
      cl[id].child0 = c0;
      cl[id].child1 = c1;
    } else {
      for (int64_t q = 0; q < c.size; ++q) perm[begin + q] = idx[q];
    }
  }

  double diam(int32_t c) const {
    double s = 0;
    for (int d = 0; d < 3; ++d) s += (cl[c].hi[d] - cl[c].lo[d]) * (cl[c].hi[d] - cl[c].lo[d]);
    return std::sqrt(s);
  }
  double dist(int32_t a, int32_t b) const {
    double s = 0;
    for (int d = 0; d < 3; ++d) {
      const double g = std::max(0.0, std::max(cl[b].lo[d] - cl[a].hi[d], cl[a].lo[d] - cl[b].hi[d]));
      s += g * g;
    }
    return std::sqrt(s);
  }

  // A_ij for original indices i, j.
  cd entry(int64_t i, int64_t j) const {
    const double dx = pts[3 * i] - pts[3 * j], dy = pts[3 * i + 1] - pts[3 * j + 1], dz = pts[3 * i + 2] - pts[3 * j + 2];
    const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    cd a = (i == j) ? cd(0.5, 0.0) : cd(0.0, 0.0);
    if (r > 0) {
      const double kr = prm.wavenumber * r;
      a += cd(std::cos(kr), std::sin(kr)) / (static_cast<double>(n) * r);
    }
    return a;
  }
};

// The cluster tree of B's points (split of the root) and the leaves of the level-conserving block
// cluster tree: admissible iff the boxes are at positive distance and min (weak, eq. (3.3)) or
// max (strong, eq. (3.2)) of the diameters <= eta * dist; dense if not admissible and a cluster
// is a leaf; subdivided otherwise. Both lists sorted.
inline void make_trees(Builder& B, BlockList* adm, BlockList* dense) {
  B.perm.assign(B.n, 0);
  {
    std::vector<int64_t> idx(B.n);
    std::iota(idx.begin(), idx.end(), 0);
    B.split(0, idx, 0, -1);
  }
  BlockList stack = {{0, 0}};
  while (!stack.empty()) {
    auto [a, b] = stack.back();
    stack.pop_back();
    const double d = B.dist(a, b);
    const double dm = B.prm.strong ? std::max(B.diam(a), B.diam(b)) : std::min(B.diam(a), B.diam(b));
    if (d > 0 && dm <= B.prm.eta * d) {
      adm->push_back({a, b});
    } else if (B.cl[a].child0 < 0 || B.cl[b].child0 < 0) {
      dense->push_back({a, b});
    } else {
      for (int32_t ca : {B.cl[a].child0, B.cl[a].child1})
        for (int32_t cb : {B.cl[b].child0, B.cl[b].child1}) stack.push_back({ca, cb});
    }
  }
  std::sort(adm->begin(), adm->end());
  std::sort(dense->begin(), dense->end());
}

}  // namespace uhb

struct uh_model {
  uhb_info_t info{};
  std::vector<int64_t> perm, cl_begin, cl_size;
  // UH
  std::vector<int32_t> row_rank, col_rank;
  std::vector<int64_t> row_off, col_off;
  std::vector<uhb::cd> U, V, S;
  std::vector<int32_t> adm_row, adm_col;
  std::vector<int64_t> S_off;
  std::vector<int32_t> S_rank;  // inner rank of each factored S_b (-1: dense); empty: all dense
  // H
  std::vector<int32_t> h_rank;
  std::vector<int64_t> X_off, Y_off;
  std::vector<uhb::cd> X, Y;
  // near field
  std::vector<int32_t> dense_row, dense_col;
  std::vector<int64_t> D_off;
  std::vector<uhb::cd> D;
};

namespace uhb {

// Checks of the builders' arguments; UH_OK or UH_EINVAL with a message.
int check_build_args(int64_t n, const double* points, const uhb_params* prm, uh_model** out);
// The tree part of the model (perm, clusters) and its statistics (counts, c_sp, depth).
void fill_model_tree(uh_model* M, const Builder& B, const BlockList& adm, const BlockList& dense);

}  // namespace uhb

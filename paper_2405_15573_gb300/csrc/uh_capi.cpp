// C ABI of the UH / H matrix-vector library: descriptor validation, packing of every product
// phase into segmented-GEMV work items (see uh_internal.h), device upload, and the launches.
//
// UH matvec (Algorithm 6, Section 4.4) = three launches of the segmented GEMV:
//   launch 0: forward transform xhat_sigma = V_sigma^* x|_sigma   (chunks of xhat)
//             + near field y|_tile += A|_b x|_sigma               (chunks of y row tiles)
//   launch 1: coupling yhat_tau = sum_{sigma in row(tau)} S_b xhat_sigma
//   launch 2: backward transform y|_tile += U_tau|_tile yhat_tau  (same y chunks as the near field)
// H matvec (Algorithm 5) = two launches: t_b = Y_b^* x|_sigma (+ near field), then
// y|_tile += X_b|_tile t_b. Row tiles are the segments between consecutive row-cluster
// boundaries of all blocks, cut to at most kHpMax rows, so each tile lies inside every row
// cluster it meets and every y element is written by exactly one chunk.
#include <algorithm>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "uh.h"
#include "uh_internal.h"

using cd = std::complex<double>;
using cf = std::complex<float>;

namespace {

thread_local std::string g_err;

}  // namespace

int uh::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

namespace {

#define fail uh::set_error

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(UH_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Reads complex elements of either data type as complex<double>.
struct Src {
  const void* p = nullptr;
  int type = UH_DATA_C128;
  cd at(int64_t i) const {
    if (type == UH_DATA_C128) return static_cast<const cd*>(p)[i];
    const cf f = static_cast<const cf*>(p)[i];
    return cd(f.real(), f.imag());
  }
};

struct Tile {
  int64_t p0;
  int32_t h;
};

// A source column: rows i = 0..h-1 are src[off + i*step] (conjugated if conj).
struct ColRef {
  int64_t off;
  int64_t step;
  int32_t idx;
};

struct Launch {
  int32_t first, count;
  int in0;   // 0: none, 1: z1, 2: z2
  int out;   // 0: none, 1: z1, 2: z2
};

// Host-side program under construction: chunks, items and packed tiles (in complex<double>,
// converted to the op's element type at upload).
struct Program {
  std::vector<uh::Chunk> chunks;
  std::vector<int> chunk_launch;  // launch whose items complete the chunk's inputs' consumers
  std::vector<uh::Item> items;
  std::vector<int> item_launch;
  std::vector<cd> M;
  std::vector<int32_t> colidx;
  int epl = 1;                   // complex values per 16-byte load (2 for c64, 1 for c128)
  int64_t target_bytes = 32768;  // bytes of one item's tile
  int elem_bytes = 16;

  int add_chunk(int kind, int64_t dst, int h, int launch) {
    uh::Chunk c{};
    c.dst = dst;
    c.h = h;
    c.kind = kind;
    chunks.push_back(c);
    chunk_launch.push_back(launch);
    return static_cast<int>(chunks.size()) - 1;
  }

  // Emit the columns `cols` (each read from `src`) as items for chunk `chunk` in `launch`.
  void add_columns(int chunk, int launch, const Src& src, bool conj, const std::vector<ColRef>& cols) {
    const int h = chunks[chunk].h;
    const int hp = (h + epl - 1) / epl * epl;
    const int64_t ncols = static_cast<int64_t>(cols.size());
    if (ncols == 0) return;
    int64_t per = target_bytes / (static_cast<int64_t>(hp) * elem_bytes);
    per = std::max<int64_t>(8, std::min<int64_t>(per, uh::kMaxCols));
    const int64_t nitems = (ncols + per - 1) / per;
    for (int64_t q = 0; q < nitems; ++q) {
      const int64_t c0 = ncols * q / nitems, c1 = ncols * (q + 1) / nitems;
      uh::Item it{};
      it.data_off = static_cast<int64_t>(M.size());
      it.hp = hp;
      it.ncols = static_cast<int32_t>(c1 - c0);
      it.idx_off = static_cast<int32_t>(colidx.size());
      it.chunk = chunk;
      it.part = -1;
      M.resize(M.size() + static_cast<size_t>((c1 - c0) * hp), cd(0, 0));
      cd* dst = M.data() + it.data_off;
      for (int64_t c = c0; c < c1; ++c) {
        const ColRef& r = cols[c];
        for (int i = 0; i < h; ++i) {
          const cd v = src.at(r.off + i * r.step);
          dst[(c - c0) * hp + i] = conj ? std::conj(v) : v;
        }
        colidx.push_back(r.idx);
      }
      items.push_back(it);
      item_launch.push_back(launch);
    }
  }

  // Chunks that received no item (possible when all their blocks have rank 0) get one empty
  // item, in the chunk's own launch, which writes zeros.
  void add_empty_items() {
    std::vector<int> cnt(chunks.size(), 0);
    for (const auto& it : items) cnt[it.chunk]++;
    for (size_t c = 0; c < chunks.size(); ++c) {
      if (cnt[c]) continue;
      uh::Item it{};
      it.data_off = static_cast<int64_t>(M.size());
      it.hp = (chunks[c].h + epl - 1) / epl * epl;
      it.ncols = 0;
      it.idx_off = static_cast<int32_t>(colidx.size());
      it.chunk = static_cast<int32_t>(c);
      it.part = -1;
      items.push_back(it);
      item_launch.push_back(chunk_launch[c]);
    }
  }

  // Assign partial slots (creation order within each chunk) and order each launch's items
  // largest first. Returns the launch table.
  std::vector<Launch> finalize(int nlaunch, int32_t* nslots) {
    std::vector<int> cnt(chunks.size(), 0);
    for (const auto& it : items) cnt[it.chunk]++;
    int32_t slot = 0;
    for (size_t c = 0; c < chunks.size(); ++c) {
      chunks[c].nparts = cnt[c];
      chunks[c].part_base = cnt[c] > 1 ? slot : -1;
      if (cnt[c] > 1) slot += cnt[c];
    }
    std::vector<int> seen(chunks.size(), 0);
    for (auto& it : items) {
      const auto& ch = chunks[it.chunk];
      it.part = ch.nparts > 1 ? ch.part_base + seen[it.chunk] : -1;
      seen[it.chunk]++;
    }
    *nslots = slot;
    std::vector<size_t> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      if (item_launch[a] != item_launch[b]) return item_launch[a] < item_launch[b];
      return static_cast<int64_t>(items[a].hp) * items[a].ncols >
             static_cast<int64_t>(items[b].hp) * items[b].ncols;
    });
    std::vector<uh::Item> sorted;
    sorted.reserve(items.size());
    std::vector<Launch> launches(nlaunch, Launch{0, 0, 0, 0});
    for (int l = 0; l < nlaunch; ++l) launches[l].first = -1;
    for (size_t k = 0; k < order.size(); ++k) {
      const int l = item_launch[order[k]];
      if (launches[l].first < 0) launches[l].first = static_cast<int32_t>(k);
      launches[l].count++;
      sorted.push_back(items[order[k]]);
    }
    for (int l = 0; l < nlaunch; ++l)
      if (launches[l].first < 0) launches[l].first = 0;
    items.swap(sorted);
    return launches;
  }
};

// ------------------------------------------------------------------------- validation

struct Tree {
  int64_t n = 0;
  int32_t ncl = 0;
  std::vector<int64_t> begin, size;
  std::vector<int32_t> perm;  // position -> original index
};

int check_tree(const uh_tree_desc& t, Tree* out) {
  if (t.n < 1 || t.n > INT32_MAX) return fail(UH_EINVAL, "n = %lld out of range", (long long)t.n);
  if (t.n_clusters < 1 || !t.cl_begin || !t.cl_size)
    return fail(UH_EINVAL, "cluster table missing");
  out->n = t.n;
  out->ncl = t.n_clusters;
  out->begin.assign(t.cl_begin, t.cl_begin + t.n_clusters);
  out->size.assign(t.cl_size, t.cl_size + t.n_clusters);
  for (int32_t c = 0; c < t.n_clusters; ++c) {
    if (out->begin[c] < 0 || out->size[c] < 1 || out->begin[c] + out->size[c] > t.n)
      return fail(UH_EINVAL, "cluster %d = [%lld, +%lld) outside [0, %lld)", c,
                  (long long)out->begin[c], (long long)out->size[c], (long long)t.n);
  }
  out->perm.resize(t.n);
  if (t.perm) {
    std::vector<char> seen(t.n, 0);
    for (int64_t p = 0; p < t.n; ++p) {
      const int64_t o = t.perm[p];
      if (o < 0 || o >= t.n || seen[o]) return fail(UH_EINVAL, "perm is not a permutation (position %lld)", (long long)p);
      seen[o] = 1;
      out->perm[p] = static_cast<int32_t>(o);
    }
  } else {
    for (int64_t p = 0; p < t.n; ++p) out->perm[p] = static_cast<int32_t>(p);
  }
  return UH_OK;
}

// Row tiles from the row-cluster boundaries of all blocks; then checks that, for every tile,
// the column clusters of the blocks covering it tile [0, n) exactly (Def. 2.2).
int make_tiles_and_check(const Tree& T, const std::vector<int32_t>& brow, const std::vector<int32_t>& bcol,
                         std::vector<Tile>* tiles) {
  std::vector<int64_t> bp = {0, T.n};
  for (size_t b = 0; b < brow.size(); ++b) {
    bp.push_back(T.begin[brow[b]]);
    bp.push_back(T.begin[brow[b]] + T.size[brow[b]]);
  }
  std::sort(bp.begin(), bp.end());
  bp.erase(std::unique(bp.begin(), bp.end()), bp.end());
  tiles->clear();
  for (size_t i = 0; i + 1 < bp.size(); ++i) {
    const int64_t len = bp[i + 1] - bp[i];
    const int64_t k = (len + uh::kHpMax - 1) / uh::kHpMax;
    for (int64_t q = 0; q < k; ++q) {
      const int64_t a = bp[i] + len * q / k, e = bp[i] + len * (q + 1) / k;
      tiles->push_back(Tile{a, static_cast<int32_t>(e - a)});
    }
  }
  std::vector<std::vector<std::pair<int64_t, int64_t>>> iv(tiles->size());
  for (size_t b = 0; b < brow.size(); ++b) {
    const int64_t r0 = T.begin[brow[b]], r1 = r0 + T.size[brow[b]];
    const int64_t c0 = T.begin[bcol[b]], c1 = c0 + T.size[bcol[b]];
    auto it = std::lower_bound(tiles->begin(), tiles->end(), r0,
                               [](const Tile& t, int64_t v) { return t.p0 < v; });
    for (; it != tiles->end() && it->p0 < r1; ++it) iv[it - tiles->begin()].push_back({c0, c1});
  }
  for (size_t t = 0; t < tiles->size(); ++t) {
    auto& v = iv[t];
    std::sort(v.begin(), v.end());
    int64_t pos = 0;
    for (auto& pr : v) {
      if (pr.first != pos)
        return fail(UH_EINVAL, "blocks do not tile the index square: rows from %lld, column %lld %s",
                    (long long)(*tiles)[t].p0, (long long)pos, pr.first < pos ? "covered twice" : "not covered");
      pos = pr.second;
    }
    if (pos != T.n)
      return fail(UH_EINVAL, "blocks do not tile the index square: rows from %lld, columns from %lld not covered",
                  (long long)(*tiles)[t].p0, (long long)pos);
  }
  return UH_OK;
}

int check_cluster_index(const Tree& T, int32_t c, const char* what, int64_t i) {
  if (c < 0 || c >= T.ncl) return fail(UH_EINVAL, "%s[%lld] = %d is not a cluster", what, (long long)i, c);
  return UH_OK;
}

int check_range(int64_t off, int64_t count, int64_t len, const char* what, int64_t i) {
  if (off < 0 || count < 0 || off + count > len)
    return fail(UH_EINVAL, "%s %lld: elements [%lld, +%lld) outside data of length %lld", what, (long long)i,
                (long long)off, (long long)count, (long long)len);
  return UH_OK;
}

int check_dense(const Tree& T, const uh_dense_desc& d) {
  if (d.n_dense < 0) return fail(UH_EINVAL, "n_dense < 0");
  if (d.n_dense > 0 && (!d.row_cl || !d.col_cl || !d.off || !d.data)) return fail(UH_EINVAL, "dense list incomplete");
  for (int64_t i = 0; i < d.n_dense; ++i) {
    int rc;
    if ((rc = check_cluster_index(T, d.row_cl[i], "dense.row_cl", i))) return rc;
    if ((rc = check_cluster_index(T, d.col_cl[i], "dense.col_cl", i))) return rc;
    if ((rc = check_range(d.off[i], T.size[d.row_cl[i]] * T.size[d.col_cl[i]], d.len, "dense block", i))) return rc;
  }
  return UH_OK;
}

// ------------------------------------------------------------------------- op

struct OpBase {
  int device = 0;
  bool c128 = true;
  int64_t n = 0;
  void* d_M = nullptr;
  int32_t* d_colidx = nullptr;
  uh::Item* d_items = nullptr;
  uh::Chunk* d_chunks = nullptr;
  int32_t* d_perm = nullptr;
  void* d_z1 = nullptr;
  void* d_z2 = nullptr;
  void* d_partials = nullptr;
  uint32_t* d_cnt = nullptr;
  uint32_t* d_sched = nullptr;
  std::vector<Launch> launches;
  int grid = 1;
  uh_stats_t st{};
};

void free_op(OpBase* o) {
  if (!o) return;
  void* ptrs[] = {o->d_M, o->d_colidx, o->d_items, o->d_chunks, o->d_perm, o->d_z1,
                  o->d_z2, o->d_partials, o->d_cnt, o->d_sched};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
int upload(const void* host, size_t bytes, T** dev) {
  *dev = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dev), bytes);
  if (e != cudaSuccess) {
    *dev = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? UH_ENOMEM : UH_ECUDA, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  if (host) CUDA_TRY(cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice));
  else CUDA_TRY(cudaMemset(*dev, 0, bytes));
  return UH_OK;
}

// Checks every address the GEMV kernel derives from the program against the buffer it reads
// or writes, before anything is uploaded: tiles inside M, column lists inside colidx, input
// indices inside the launch's input vectors, destinations inside their outputs, partial slots
// inside the partial buffer, heights within the kernel's limits.
int self_check(const Program& P, const std::vector<Launch>& L, int64_t n, int64_t z1len, int64_t z2len,
               int32_t nslots) {
  const int64_t zlen[3] = {0, z1len, z2len};
  const int64_t msize = static_cast<int64_t>(P.M.size());
  const int64_t csize = static_cast<int64_t>(P.colidx.size());
  for (size_t l = 0; l < L.size(); ++l) {
    for (int32_t k = L[l].first; k < L[l].first + L[l].count; ++k) {
      const uh::Item& it = P.items[k];
      if (it.hp < P.epl || it.hp > uh::kHpMax || it.hp % P.epl || it.ncols < 0 || it.ncols > uh::kMaxCols ||
          it.data_off < 0 || it.data_off + static_cast<int64_t>(it.ncols) * it.hp > msize ||
          (it.data_off * P.elem_bytes) % 16 != 0 || it.idx_off < 0 ||
          static_cast<int64_t>(it.idx_off) + it.ncols > csize || it.chunk < 0 ||
          it.chunk >= static_cast<int32_t>(P.chunks.size()) || it.part >= nslots || it.part < -1)
        return fail(UH_EINVAL, "internal packing error: item %d of launch %zu", k, l);
      for (int32_t c = 0; c < it.ncols; ++c) {
        const int32_t ix = P.colidx[it.idx_off + c];
        if (ix >= 0 ? (L[l].in0 == 0 || ix >= zlen[L[l].in0]) : (-static_cast<int64_t>(ix) - 1 >= n))
          return fail(UH_EINVAL, "internal packing error: input index %d of item %d, launch %zu", ix, k, l);
      }
      const uh::Chunk& ch = P.chunks[it.chunk];
      if (ch.h < 1 || ch.h > it.hp || ch.dst < 0 ||
          (ch.kind == 0 ? (L[l].out == 0 || ch.dst + ch.h > zlen[L[l].out]) : (ch.kind != 1 || ch.dst + ch.h > n)))
        return fail(UH_EINVAL, "internal packing error: chunk %d of item %d, launch %zu", it.chunk, k, l);
      if ((ch.nparts > 1) != (it.part >= 0) || (ch.nparts > 1 && ch.part_base + ch.nparts > nslots))
        return fail(UH_EINVAL, "internal packing error: partial slots of chunk %d", it.chunk);
    }
  }
  return UH_OK;
}

// Uploads a finished program and allocates scratch. z1/z2 lengths in complex elements.
int upload_program(OpBase* o, Program& P, const Tree& T, int nlaunch, int64_t z1len, int64_t z2len,
                   const int* in0, const int* out) {
  int32_t nslots = 0;
  P.add_empty_items();
  o->launches = P.finalize(nlaunch, &nslots);
  for (int l = 0; l < nlaunch; ++l) {
    o->launches[l].in0 = in0[l];
    o->launches[l].out = out[l];
  }
  int rc;
  if ((rc = self_check(P, o->launches, T.n, z1len, z2len, nslots))) return rc;
  CUDA_TRY(cudaGetDevice(&o->device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o->device));
  o->grid = std::max(1, sms * 8);
  const size_t eb = o->c128 ? 16 : 8;
  if (o->c128) {
    if ((rc = upload(P.M.data(), P.M.size() * sizeof(cd), &o->d_M))) return rc;
  } else {
    std::vector<cf> m32(P.M.size());
    for (size_t i = 0; i < P.M.size(); ++i) m32[i] = cf(static_cast<float>(P.M[i].real()), static_cast<float>(P.M[i].imag()));
    if ((rc = upload(m32.data(), m32.size() * sizeof(cf), &o->d_M))) return rc;
  }
  if ((rc = upload(P.colidx.data(), P.colidx.size() * sizeof(int32_t), &o->d_colidx))) return rc;
  if ((rc = upload(P.items.data(), P.items.size() * sizeof(uh::Item), &o->d_items))) return rc;
  if ((rc = upload(P.chunks.data(), P.chunks.size() * sizeof(uh::Chunk), &o->d_chunks))) return rc;
  if ((rc = upload(T.perm.data(), T.perm.size() * sizeof(int32_t), &o->d_perm))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), std::max<int64_t>(z1len, 1) * eb, &o->d_z1))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), std::max<int64_t>(z2len, 1) * eb, &o->d_z2))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(std::max(nslots, 1)) * uh::kHpMax * eb, &o->d_partials))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), std::max<size_t>(P.chunks.size(), 1) * sizeof(uint32_t), &o->d_cnt))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), 4 * sizeof(uint32_t), &o->d_sched))) return rc;
  o->st.packed_bytes = static_cast<int64_t>(P.M.size() * eb + P.colidx.size() * sizeof(int32_t));
  o->st.device_bytes = o->st.packed_bytes + static_cast<int64_t>(P.items.size() * sizeof(uh::Item) +
                       P.chunks.size() * sizeof(uh::Chunk) + T.n * 4 + (z1len + z2len) * eb +
                       static_cast<int64_t>(std::max(nslots, 1)) * uh::kHpMax * eb);
  o->st.n_launches = nlaunch;
  o->st.n_items = static_cast<int64_t>(P.items.size());
  return UH_OK;
}

int run_matvec(OpBase* o, const void* x, void* y, void* stream) {
  if (!x || !y) return fail(UH_EINVAL, "x and y must be device pointers");
  const size_t eb = o->c128 ? 16 : 8;
  const char* xa = static_cast<const char*>(x);
  const char* ya = static_cast<const char*>(y);
  if (xa < ya + o->n * eb && ya < xa + o->n * eb) return fail(UH_EINVAL, "x and y overlap");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const Launch& L : o->launches) {
    uh::SegGemvParams p{};
    p.items = o->d_items + L.first;
    p.item_count = L.count;
    p.chunks = o->d_chunks;
    p.M = o->d_M;
    p.colidx = o->d_colidx;
    p.in0 = L.in0 == 1 ? o->d_z1 : (L.in0 == 2 ? o->d_z2 : nullptr);
    p.in1 = x;
    p.out_lin = L.out == 1 ? o->d_z1 : (L.out == 2 ? o->d_z2 : nullptr);
    p.out_perm = y;
    p.perm = o->d_perm;
    p.partials = o->d_partials;
    p.chunk_cnt = o->d_cnt;
    p.sched = o->d_sched;
    cudaError_t e = uh::launch_seg_gemv(o->c128, p, o->grid, s);
    if (e != cudaSuccess) return fail(UH_ECUDA, "segmented GEMV launch: %s", cudaGetErrorString(e));
  }
  return UH_OK;
}

int check_precision(int32_t precision) {
  if (precision != UH_PREC_C128 && precision != UH_PREC_C64)
    return fail(UH_EINVAL, "precision %d not supported", precision);
  return UH_OK;
}

void init_program(Program& P, bool c128) {
  P.elem_bytes = c128 ? 16 : 8;
  P.epl = c128 ? 1 : 2;
}

// Near-field items (launch `launch`): for every dense block and every row tile inside its row
// cluster, the columns D_b[tile rows, :] with inputs x at the column cluster's positions.
void add_near_field(Program& P, const Tree& T, const uh_dense_desc& d, int data_type,
                    const std::vector<Tile>& tiles, const std::vector<int>& tile_chunk, int launch) {
  Src src{d.data, data_type};
  // Group dense blocks by tile so that each tile's columns form one stream.
  std::vector<std::vector<int64_t>> per_tile(tiles.size());
  for (int64_t i = 0; i < d.n_dense; ++i) {
    const int64_t r0 = T.begin[d.row_cl[i]], r1 = r0 + T.size[d.row_cl[i]];
    auto it = std::lower_bound(tiles.begin(), tiles.end(), r0, [](const Tile& t, int64_t v) { return t.p0 < v; });
    for (; it != tiles.end() && it->p0 < r1; ++it) per_tile[it - tiles.begin()].push_back(i);
  }
  std::vector<ColRef> cols;
  for (size_t t = 0; t < tiles.size(); ++t) {
    cols.clear();
    for (int64_t i : per_tile[t]) {
      const int32_t tau = d.row_cl[i], sg = d.col_cl[i];
      const int64_t m = T.size[tau];
      const int64_t roff = tiles[t].p0 - T.begin[tau];
      for (int64_t c = 0; c < T.size[sg]; ++c)
        cols.push_back(ColRef{d.off[i] + c * m + roff, 1, -(T.perm[T.begin[sg] + c]) - 1});
    }
    P.add_columns(tile_chunk[t], launch, src, false, cols);
  }
}

void fill_common_stats(OpBase* o, const Tree& T, const uh_dense_desc& d, int32_t precision) {
  o->st.n = T.n;
  o->st.precision = precision;
  o->st.elem_bytes = o->c128 ? 16 : 8;
  o->st.n_dense = d.n_dense;
  int64_t ed = 0;
  for (int64_t i = 0; i < d.n_dense; ++i) ed += T.size[d.row_cl[i]] * T.size[d.col_cl[i]];
  o->st.E_D = ed;
}

}  // namespace

struct uh_op : OpBase {};
struct h_op : OpBase {};

extern "C" {

const char* uh_last_error(void) { return g_err.c_str(); }
const char* uh_version(void) { return "uh-gb300 0.1 (sm_103a)"; }

int uh_create(const uh_desc* d, int32_t precision, uh_op** out) {
  g_err.clear();
  if (!d || !out) return fail(UH_EINVAL, "null argument");
  *out = nullptr;
  int rc;
  if ((rc = check_precision(precision))) return rc;
  if (d->data_type != UH_DATA_C128 && d->data_type != UH_DATA_C64) return fail(UH_EINVAL, "data_type %d", d->data_type);
  Tree T;
  if ((rc = check_tree(d->tree, &T))) return rc;
  if (d->n_adm < 0) return fail(UH_EINVAL, "n_adm < 0");
  if (d->n_adm > 0 && (!d->adm_row || !d->adm_col || !d->S_off || !d->S_data || !d->row_rank || !d->row_off ||
                       !d->col_rank || !d->col_off || !d->U_data || !d->V_data))
    return fail(UH_EINVAL, "admissible part incomplete");
  if ((rc = check_dense(T, d->dense))) return rc;
  std::vector<char> is_row(T.ncl, 0), is_col(T.ncl, 0);
  for (int64_t i = 0; i < d->n_adm; ++i) {
    if ((rc = check_cluster_index(T, d->adm_row[i], "adm_row", i))) return rc;
    if ((rc = check_cluster_index(T, d->adm_col[i], "adm_col", i))) return rc;
    is_row[d->adm_row[i]] = 1;
    is_col[d->adm_col[i]] = 1;
  }
  for (int32_t c = 0; c < T.ncl; ++c) {
    if (is_row[c]) {
      const int32_t l = d->row_rank[c];
      if (l < 0 || l > T.size[c]) return fail(UH_EINVAL, "row_rank[%d] = %d outside [0, %lld]", c, l, (long long)T.size[c]);
      if ((rc = check_range(d->row_off[c], T.size[c] * l, d->U_len, "row basis", c))) return rc;
    }
    if (is_col[c]) {
      const int32_t l = d->col_rank[c];
      if (l < 0 || l > T.size[c]) return fail(UH_EINVAL, "col_rank[%d] = %d outside [0, %lld]", c, l, (long long)T.size[c]);
      if ((rc = check_range(d->col_off[c], T.size[c] * l, d->V_len, "column basis", c))) return rc;
    }
  }
  for (int64_t i = 0; i < d->n_adm; ++i) {
    const int64_t cnt = static_cast<int64_t>(d->row_rank[d->adm_row[i]]) * d->col_rank[d->adm_col[i]];
    if ((rc = check_range(d->S_off[i], cnt, d->S_len, "coupling matrix", i))) return rc;
  }
  std::vector<int32_t> brow, bcol;
  for (int64_t i = 0; i < d->n_adm; ++i) { brow.push_back(d->adm_row[i]); bcol.push_back(d->adm_col[i]); }
  for (int64_t i = 0; i < d->dense.n_dense; ++i) { brow.push_back(d->dense.row_cl[i]); bcol.push_back(d->dense.col_cl[i]); }
  std::vector<Tile> tiles;
  if ((rc = make_tiles_and_check(T, brow, bcol, &tiles))) return rc;

  auto* o = new (std::nothrow) uh_op();
  if (!o) return fail(UH_ENOMEM, "host allocation");
  o->c128 = precision == UH_PREC_C128;
  o->n = T.n;
  Program P;
  init_program(P, o->c128);

  // xhat / yhat offsets (clusters in increasing number).
  std::vector<int64_t> xoff(T.ncl, -1), yoff(T.ncl, -1);
  int64_t nx = 0, ny = 0;
  for (int32_t c = 0; c < T.ncl; ++c) {
    if (is_col[c] && d->col_rank[c] > 0) { xoff[c] = nx; nx += d->col_rank[c]; }
    if (is_row[c] && d->row_rank[c] > 0) { yoff[c] = ny; ny += d->row_rank[c]; }
  }
  // y tile chunks.
  std::vector<int> tile_chunk(tiles.size());
  for (size_t t = 0; t < tiles.size(); ++t) tile_chunk[t] = P.add_chunk(1, tiles[t].p0, tiles[t].h, 0);

  // Launch 0: forward transform, chunks of at most kHpMax rows of V_sigma^*.
  Src vs{d->V_data, d->data_type};
  std::vector<ColRef> cols;
  for (int32_t s = 0; s < T.ncl; ++s) {
    if (xoff[s] < 0) continue;
    const int32_t l = d->col_rank[s];
    const int64_t m = T.size[s];
    const int k = (l + uh::kHpMax - 1) / uh::kHpMax;
    for (int q = 0; q < k; ++q) {
      const int j0 = l * q / k, j1 = l * (q + 1) / k;
      const int ch = P.add_chunk(0, xoff[s] + j0, j1 - j0, 0);
      cols.clear();
      // column r of V_sigma^*[j0:j1, :] = conj(V_sigma[r, j0:j1]), input x at position begin+r
      for (int64_t r = 0; r < m; ++r)
        cols.push_back(ColRef{d->col_off[s] + r + j0 * m, m, -(T.perm[T.begin[s] + r]) - 1});
      P.add_columns(ch, 0, vs, true, cols);
    }
  }
  // Launch 0 (continued): near field.
  add_near_field(P, T, d->dense, d->data_type, tiles, tile_chunk, 0);
  // Launch 1: coupling, per row cluster tau, columns of [S_b]_{sigma in row(tau)}.
  std::vector<std::vector<int64_t>> row_blocks(T.ncl);
  for (int64_t i = 0; i < d->n_adm; ++i) row_blocks[d->adm_row[i]].push_back(i);
  Src ss{d->S_data, d->data_type};
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (yoff[t] < 0) continue;
    auto& bl = row_blocks[t];
    std::stable_sort(bl.begin(), bl.end(), [&](int64_t a, int64_t b) { return d->adm_col[a] < d->adm_col[b]; });
    const int32_t l = d->row_rank[t];
    const int k = (l + uh::kHpMax - 1) / uh::kHpMax;
    for (int q = 0; q < k; ++q) {
      const int i0 = l * q / k, i1 = l * (q + 1) / k;
      const int ch = P.add_chunk(0, yoff[t] + i0, i1 - i0, 1);
      cols.clear();
      for (int64_t b : bl) {
        const int32_t s = d->adm_col[b];
        const int32_t ls = d->col_rank[s];
        for (int j = 0; j < ls; ++j) cols.push_back(ColRef{d->S_off[b] + static_cast<int64_t>(j) * l + i0, 1, static_cast<int32_t>(xoff[s] + j)});
      }
      P.add_columns(ch, 1, ss, false, cols);
    }
  }
  // Launch 2: backward transform, per y tile, columns U_tau[tile rows, :] of every row
  // cluster tau that contains the tile, inputs yhat_tau.
  std::vector<std::vector<int32_t>> tile_rows(tiles.size());
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (yoff[t] < 0) continue;
    const int64_t r0 = T.begin[t], r1 = r0 + T.size[t];
    auto it = std::lower_bound(tiles.begin(), tiles.end(), r0, [](const Tile& a, int64_t v) { return a.p0 < v; });
    for (; it != tiles.end() && it->p0 < r1; ++it) tile_rows[it - tiles.begin()].push_back(t);
  }
  Src us{d->U_data, d->data_type};
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    cols.clear();
    for (int32_t t : tile_rows[ti]) {
      const int64_t m = T.size[t];
      const int64_t roff = tiles[ti].p0 - T.begin[t];
      for (int j = 0; j < d->row_rank[t]; ++j)
        cols.push_back(ColRef{d->row_off[t] + j * m + roff, 1, static_cast<int32_t>(yoff[t] + j)});
    }
    P.add_columns(tile_chunk[ti], 2, us, false, cols);
  }
  const int in0[3] = {0, 1, 2}, outsel[3] = {1, 2, 0};
  if ((rc = upload_program(o, P, T, 3, nx, ny, in0, outsel))) { free_op(o); delete o; return rc; }

  // Statistics.
  fill_common_stats(o, T, d->dense, precision);
  int64_t eu = 0, ev = 0, es = 0, nrb = 0, ncb = 0, srr = 0, scr = 0;
  int32_t rmin = INT32_MAX, rmax = 0;
  int64_t rsum = 0, rcnt = 0;
  std::vector<int32_t> rowc(T.ncl, 0), colc(T.ncl, 0);
  for (int64_t i = 0; i < d->n_adm; ++i) {
    rowc[d->adm_row[i]]++;
    colc[d->adm_col[i]]++;
    es += static_cast<int64_t>(d->row_rank[d->adm_row[i]]) * d->col_rank[d->adm_col[i]];
  }
  int32_t csp = 0;
  for (int32_t c = 0; c < T.ncl; ++c) {
    csp = std::max(csp, std::max(rowc[c], colc[c]));
    if (is_row[c]) {
      nrb++; eu += T.size[c] * d->row_rank[c]; srr += d->row_rank[c];
      if (d->row_rank[c] > 0) { rmin = std::min(rmin, d->row_rank[c]); rmax = std::max(rmax, d->row_rank[c]); rsum += d->row_rank[c]; rcnt++; }
    }
    if (is_col[c]) {
      ncb++; ev += T.size[c] * d->col_rank[c]; scr += d->col_rank[c];
      if (d->col_rank[c] > 0) { rmin = std::min(rmin, d->col_rank[c]); rmax = std::max(rmax, d->col_rank[c]); rsum += d->col_rank[c]; rcnt++; }
    }
  }
  o->st.n_row_bases = nrb;
  o->st.n_col_bases = ncb;
  o->st.n_adm = d->n_adm;
  o->st.E_U = eu;
  o->st.E_V = ev;
  o->st.E_S = es;
  o->st.sum_row_rank = srr;
  o->st.sum_col_rank = scr;
  o->st.rank_min = rcnt ? rmin : 0;
  o->st.rank_max = rmax;
  o->st.rank_mean = rcnt ? static_cast<double>(rsum) / rcnt : 0.0;
  o->st.csp = csp;
  o->st.algo_bytes_matvec = o->st.elem_bytes * (eu + ev + es + o->st.E_D + 2 * T.n + 2 * (srr + scr));
  *out = o;
  return UH_OK;
}

int uh_destroy(uh_op* op) {
  if (!op) return UH_OK;
  cudaDeviceSynchronize();
  free_op(op);
  delete op;
  return UH_OK;
}

int uh_matvec(uh_op* op, const void* x, void* y, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  return run_matvec(op, x, y, stream);
}

int uh_stats(const uh_op* op, uh_stats_t* out) {
  if (!op || !out) return fail(UH_EINVAL, "null argument");
  *out = op->st;
  return UH_OK;
}

int h_create(const h_desc* d, int32_t precision, h_op** out) {
  g_err.clear();
  if (!d || !out) return fail(UH_EINVAL, "null argument");
  *out = nullptr;
  int rc;
  if ((rc = check_precision(precision))) return rc;
  if (d->data_type != UH_DATA_C128 && d->data_type != UH_DATA_C64) return fail(UH_EINVAL, "data_type %d", d->data_type);
  Tree T;
  if ((rc = check_tree(d->tree, &T))) return rc;
  if (d->n_adm < 0) return fail(UH_EINVAL, "n_adm < 0");
  if (d->n_adm > 0 && (!d->adm_row || !d->adm_col || !d->adm_rank || !d->X_off || !d->Y_off || !d->X_data || !d->Y_data))
    return fail(UH_EINVAL, "admissible part incomplete");
  if ((rc = check_dense(T, d->dense))) return rc;
  for (int64_t i = 0; i < d->n_adm; ++i) {
    if ((rc = check_cluster_index(T, d->adm_row[i], "adm_row", i))) return rc;
    if ((rc = check_cluster_index(T, d->adm_col[i], "adm_col", i))) return rc;
    const int32_t k = d->adm_rank[i];
    const int64_t m = T.size[d->adm_row[i]], nn = T.size[d->adm_col[i]];
    if (k < 0 || k > std::min(m, nn)) return fail(UH_EINVAL, "adm_rank[%lld] = %d out of range", (long long)i, k);
    if ((rc = check_range(d->X_off[i], m * k, d->X_len, "X factor", i))) return rc;
    if ((rc = check_range(d->Y_off[i], nn * k, d->Y_len, "Y factor", i))) return rc;
  }
  std::vector<int32_t> brow, bcol;
  for (int64_t i = 0; i < d->n_adm; ++i) { brow.push_back(d->adm_row[i]); bcol.push_back(d->adm_col[i]); }
  for (int64_t i = 0; i < d->dense.n_dense; ++i) { brow.push_back(d->dense.row_cl[i]); bcol.push_back(d->dense.col_cl[i]); }
  std::vector<Tile> tiles;
  if ((rc = make_tiles_and_check(T, brow, bcol, &tiles))) return rc;

  auto* o = new (std::nothrow) h_op();
  if (!o) return fail(UH_ENOMEM, "host allocation");
  o->c128 = precision == UH_PREC_C128;
  o->n = T.n;
  Program P;
  init_program(P, o->c128);
  std::vector<int> tile_chunk(tiles.size());
  for (size_t t = 0; t < tiles.size(); ++t) tile_chunk[t] = P.add_chunk(1, tiles[t].p0, tiles[t].h, 0);
  // Launch 0: t_b = Y_b^* x|_sigma per block (chunks of at most kHpMax), plus the near field.
  std::vector<int64_t> toff(d->n_adm, -1);
  int64_t nt = 0;
  Src ys{d->Y_data, d->data_type};
  std::vector<ColRef> cols;
  for (int64_t b = 0; b < d->n_adm; ++b) {
    const int32_t k = d->adm_rank[b];
    if (k == 0) continue;
    toff[b] = nt;
    nt += k;
    const int32_t s = d->adm_col[b];
    const int64_t m = T.size[s];
    const int nq = (k + uh::kHpMax - 1) / uh::kHpMax;
    for (int q = 0; q < nq; ++q) {
      const int j0 = k * q / nq, j1 = k * (q + 1) / nq;
      const int ch = P.add_chunk(0, toff[b] + j0, j1 - j0, 0);
      cols.clear();
      for (int64_t r = 0; r < m; ++r)
        cols.push_back(ColRef{d->Y_off[b] + r + j0 * m, m, -(T.perm[T.begin[s] + r]) - 1});
      P.add_columns(ch, 0, ys, true, cols);
    }
  }
  add_near_field(P, T, d->dense, d->data_type, tiles, tile_chunk, 0);
  // Launch 1: y|_tile += X_b|_tile t_b for every block whose row cluster contains the tile.
  std::vector<std::vector<int64_t>> tile_blocks(tiles.size());
  for (int64_t b = 0; b < d->n_adm; ++b) {
    if (toff[b] < 0) continue;
    const int64_t r0 = T.begin[d->adm_row[b]], r1 = r0 + T.size[d->adm_row[b]];
    auto it = std::lower_bound(tiles.begin(), tiles.end(), r0, [](const Tile& a, int64_t v) { return a.p0 < v; });
    for (; it != tiles.end() && it->p0 < r1; ++it) tile_blocks[it - tiles.begin()].push_back(b);
  }
  Src xs{d->X_data, d->data_type};
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    cols.clear();
    for (int64_t b : tile_blocks[ti]) {
      const int32_t t = d->adm_row[b];
      const int64_t m = T.size[t];
      const int64_t roff = tiles[ti].p0 - T.begin[t];
      for (int j = 0; j < d->adm_rank[b]; ++j)
        cols.push_back(ColRef{d->X_off[b] + j * m + roff, 1, static_cast<int32_t>(toff[b] + j)});
    }
    P.add_columns(tile_chunk[ti], 1, xs, false, cols);
  }
  const int in0[2] = {0, 1}, outsel[2] = {1, 0};
  if ((rc = upload_program(o, P, T, 2, nt, 1, in0, outsel))) { free_op(o); delete o; return rc; }
  fill_common_stats(o, T, d->dense, precision);
  int64_t ex = 0, ey = 0, sk = 0;
  for (int64_t b = 0; b < d->n_adm; ++b) {
    ex += T.size[d->adm_row[b]] * d->adm_rank[b];
    ey += T.size[d->adm_col[b]] * d->adm_rank[b];
    sk += d->adm_rank[b];
  }
  o->st.n_adm = d->n_adm;
  o->st.E_U = ex;
  o->st.E_V = ey;
  o->st.E_S = 0;
  o->st.algo_bytes_matvec = o->st.elem_bytes * (ex + ey + o->st.E_D + 2 * T.n + 2 * sk);
  *out = o;
  return UH_OK;
}

int h_destroy(h_op* op) {
  if (!op) return UH_OK;
  cudaDeviceSynchronize();
  free_op(op);
  delete op;
  return UH_OK;
}

int h_matvec(h_op* op, const void* x, void* y, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  return run_matvec(op, x, y, stream);
}

int h_stats(const h_op* op, uh_stats_t* out) {
  if (!op || !out) return fail(UH_EINVAL, "null argument");
  *out = op->st;
  return UH_OK;
}

int uh_matmat(uh_op*, int32_t, const void*, int64_t, void*, int64_t, void*) {
  return fail(UH_EINVAL, "uh_matmat: not available in this build");
}
int uh_reserve(uh_op*, int32_t) { return fail(UH_EINVAL, "uh_reserve: not available in this build"); }
int h_matmat(h_op*, int32_t, const void*, int64_t, void*, int64_t, void*) {
  return fail(UH_EINVAL, "h_matmat: not available in this build");
}
int h_reserve(h_op*, int32_t) { return fail(UH_EINVAL, "h_reserve: not available in this build"); }

}  // extern "C"

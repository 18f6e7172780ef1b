// C ABI of the UH / H matrix-vector library: descriptor validation, packing of a product into the
// streaming kernel's device program (uh_program.h), device upload, and the launch.
//
// UH matvec (Algorithm 6, Section 4.4) as chunks of outputs, in the schedule groups every CTA runs
// in order (uh_program.h):
//   permutation  xp = x in cluster order, one slice per CTA;
//   forward      xhat_sigma = V_sigma^* xp|_sigma                 (chunks of xhat, z1);
//   near field   z3|_tile = sum_b A|_b|_tile xp|_sigma            (row tiles with a backward part),
//                or y|_tile directly (row tiles without one); split into two groups around the
//                coupling so that each CTA has independent work while the coupling's inputs finish;
//   coupling     yhat_tau = sum_{sigma in row(tau)} S_b xhat_sigma  (chunks of yhat, z2);
//   backward     y|_tile = z3|_tile + sum_{tau > tile} U_tau|_tile yhat_tau.
// UH ops made with a tensor-core precision also hold the multi-RHS program of uh_panel.h (three
// launches per pass of 64 right-hand sides, compact xhat / yhat panels, no scatter).
// H matvec (Algorithm 5): permutation; t_b = Y_b^* xp|_sigma (z1); near field; then
// y|_tile = z3|_tile + sum_b X_b|_tile t_b. Row tiles are the segments between consecutive
// row-cluster boundaries of all blocks, cut to at most 64 rows, so each tile lies inside every row
// cluster it meets and each y entry is written by exactly one chunk.
#include <algorithm>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "uh.h"
#include "uh_debug.h"
#include "uh_internal.h"
#include "uh_panel.h"
#include "uh_panel_pack.h"
#include "uh_program.h"

using cd = std::complex<double>;
using cf = std::complex<float>;

namespace uh {
cudaError_t stream_prepare(int variant);
cudaError_t stream_occupancy(int variant, int* blocks_per_sm);
cudaError_t stream_launch(int variant, const StreamParams& p, int grid, cudaStream_t stream);
}  // namespace uh

namespace {

thread_local std::string g_err;
// > 0 while uh_pack_check / h_pack_check run: pack for this many CTAs, check, make no CUDA call.
thread_local int g_pack_only_ncta = 0;

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

using uh::Src;
using uh::ColSpec;
using uh::ProgramBuilder;

struct Tile {
  int64_t p0;
  int32_t h;
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
    const int64_t k = (len + uh::kStreamHpMax - 1) / uh::kStreamHpMax;
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

// Device wait bound: about two seconds at the GB300's maximum SM clock.
constexpr long long kTimeoutCycles = 4000000000LL;

struct OpBase {
  int device = 0;
  bool c128 = true;
  int64_t n = 0;
  int ncta = 1;
  uint64_t epoch = 0;  // products launched since creation (or since the last reported timeout)
  void* d_M = nullptr;
  uh::WorkItem* d_items = nullptr;
  int32_t* d_cta = nullptr;
  unsigned long long* d_done = nullptr;  // group counters, the pool ticket, the flags
  int64_t done_len = 0;
  uh::Scatter* d_scatter = nullptr;
  uh::PoolRange* d_pool = nullptr;
  int64_t pool_chunks = 0;
  int64_t perm_n = 0;  // positions of x permuted at the start of a product
  bool dual = false;   // program packed for two CTAs per SM (uh::kGeomDual)
  int64_t counter_total[uh::kNumCounters] = {};
  uint32_t* d_status = nullptr;
  int32_t* d_perm = nullptr;
  void* d_xp = nullptr;
  void* d_z1 = nullptr;
  void* d_z2 = nullptr;
  void* d_z3 = nullptr;
  void* d_z4 = nullptr;
  // uh_matvec_mixed (complex64 UH ops): xp, z1, z2, z3, z4 at 16 bytes per value
  void* d_xm[uh::kNumSources] = {};
  // CUDA-core multi-RHS product (complex64 UH ops, after uh_reserve): the same vectors with
  // multi_r values per position
  int multi_r = 0;
  void* d_xr[uh::kNumSources] = {};
  int64_t src_len[uh::kNumSources] = {};
  // tensor-core uh_matmat (UH_PREC_C64_TF32 / UH_PREC_C64_BF16X3 ops)
  int mm_mode = -1;       // UH_MM_TF32 or UH_MM_BF16X3
  int panel_mode = 0;     // uh::kPanelTF32 or uh::kPanelBF16X3
  int panel_ncta = 0;
  int64_t panel_xp_rows = 0;  // rows of XP, its zero block included
  unsigned long long* d_pdone = nullptr;  // [2] Z1 / Z2 chunk counters of the passes, monotonic
  int64_t panel_zchunks[2] = {0, 0};
  unsigned long long panel_epoch = 0;     // passes launched since the counters were last reset
  unsigned char* d_ptiles = nullptr;
  uh::PanelItem* d_pitems = nullptr;
  int32_t* d_pbegin = nullptr;
  void* d_pxp = nullptr;
  void* d_pz1 = nullptr;
  void* d_pz2 = nullptr;
  uh_stats_t st{};
  // Calls on one op run in the order they are made, from any streams and host threads: they
  // share the op's scratch and its per-call counters, and two products of one op could not run
  // at the same time anyway (each fills the GPU). `mu` serialises the host side; every call
  // records `order_ev` on its stream after its work, and a call on another stream than the
  // previous one first waits for that event.
  std::mutex mu;
  bool called = false;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t order_ev = nullptr;
};

void free_op(OpBase* o) {
  if (!o) return;
  void* ptrs[] = {o->d_M, o->d_items, o->d_cta, o->d_done, o->d_scatter, o->d_pool, o->d_status,
                  o->d_perm, o->d_xp, o->d_z1, o->d_z2, o->d_z3, o->d_z4, o->d_xm[4],
                  o->d_ptiles, o->d_pitems, o->d_pbegin, o->d_pxp, o->d_pz1, o->d_pz2,
                  o->d_xm[0], o->d_xm[1], o->d_xm[2], o->d_xm[3], o->d_pdone,
                  o->d_xr[0], o->d_xr[1], o->d_xr[2], o->d_xr[3], o->d_xr[4]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (o->order_ev) cudaEventDestroy(o->order_ev);
}

// Orders a call on stream s after the op's previous call (the caller holds o->mu).
int order_call(OpBase* o, cudaStream_t s) {
  if (!o->order_ev) CUDA_TRY(cudaEventCreateWithFlags(&o->order_ev, cudaEventDisableTiming));
  if (o->called && s != o->last_stream) CUDA_TRY(cudaStreamWaitEvent(s, o->order_ev, 0));
  return UH_OK;
}

// Marks the end of a call's work on stream s (the caller holds o->mu).
int call_done(OpBase* o, cudaStream_t s) {
  CUDA_TRY(cudaEventRecord(o->order_ev, s));
  o->called = true;
  o->last_stream = s;
  return UH_OK;
}

template <typename T>
int upload(const void* host, size_t bytes, T** dev) {
  *dev = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dev), bytes);
  if (e != cudaSuccess) {
    *dev = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? UH_ENOMEM : UH_ECUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  if (host) CUDA_TRY(cudaMemcpy(*dev, host, bytes, cudaMemcpyHostToDevice));
  else CUDA_TRY(cudaMemset(*dev, 0, bytes));
  return UH_OK;
}

// Number of CTAs of the persistent launch (one per SM when the kernel fits once per SM).
// Grid of the streaming kernel: SMs x CTAs per SM (dual: the two-CTA variants).
int query_ncta(bool c128, int* ncta, int* device, bool dual = false) {
  CUDA_TRY(cudaGetDevice(device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, *device));
  const int variant = c128 ? (dual ? uh::kVarC128Dual : uh::kVarC128) : dual ? uh::kVarC64Dual : uh::kVarC64;
  CUDA_TRY(uh::stream_prepare(variant));
  int per = 0;
  CUDA_TRY(uh::stream_occupancy(variant, &per));
  if (per < (dual ? 2 : 1)) return fail(UH_ECUDA, "streaming kernel does not fit %d CTAs on an SM", dual ? 2 : 1);
  per = dual ? 2 : 1;
  *ncta = sms * per;
  if (!c128) {
    // the extended-precision variant runs the same program on the same grid
    const int vm = dual ? uh::kVarMixedDual : uh::kVarMixed;
    CUDA_TRY(uh::stream_prepare(vm));
    int pm = 0;
    CUDA_TRY(uh::stream_occupancy(vm, &pm));
    if (pm < per) return fail(UH_ECUDA, "extended-precision streaming kernel does not fit the grid");
  }
  return UH_OK;
}

// Packing parameters from the C struct (zeros: the defaults), checked.
int pack_params_from(const uh_pack_params* params, bool c128, uh::PackParams* pp) {
  if (!params) return UH_OK;
  if (params->tile_bytes) pp->tile_bytes = params->tile_bytes;
  if (params->item_cost) pp->item_cost = params->item_cost;
  if (params->chunk_cost) pp->chunk_cost = params->chunk_cost;
  if (params->pool_unit) pp->pool_unit = params->pool_unit;
  pp->ctas_per_sm = params->ctas_per_sm;
  if (pp->tile_bytes < 4096 || pp->tile_bytes > uh::kTileBytes || pp->item_cost < 0 || pp->chunk_cost < 0 ||
      pp->pool_unit < 0)
    return fail(UH_EINVAL, "pack parameters: tile_bytes %lld (4096..%d), costs >= 0", (long long)pp->tile_bytes,
                uh::kTileBytes);
  if (pp->ctas_per_sm < 0 || pp->ctas_per_sm > 2)
    return fail(UH_EINVAL, "pack parameters: ctas_per_sm %lld (0: automatic, 1 or 2)", (long long)pp->ctas_per_sm);
  return UH_OK;
}

// The automatic choice of CTAs per SM (ctas_per_sm 0): two for programs that stream at least
// kDualMinBytes per product (measured on GB300: complex64 products 10-23% faster for operators of
// 300-720 MB with ranks of 20-60, about neutral at the N = 32768 sphere, 17% slower at 168 MB, where
// the per-CTA start and phase waits dominate; complex128 2% faster at the N = 32768 sphere), else one.
constexpr int64_t kDualMinBytes = int64_t{256} << 20;
void resolve_ctas(uh::PackParams* pp, int64_t algo_bytes) {
  if (pp->ctas_per_sm == 0) pp->ctas_per_sm = algo_bytes >= kDualMinBytes ? 2 : 1;
}

void fill_pack_stats(const uh::PackParams& pp, const uh::StreamGeometry& g, uh_stats_t* st) {
  st->pack_tile_bytes = std::min<int64_t>(pp.tile_bytes, g.tile_bytes);
  st->pack_item_cost = pp.item_cost;
  st->pack_chunk_cost = pp.chunk_cost;
  st->pack_pool_unit = pp.pool_unit;
  st->pack_ctas_per_sm = g.ctas_per_sm;
}

// Finalize, self-check and upload the program; allocate the scratch vectors.
int upload_program(OpBase* o, ProgramBuilder& P, const Tree& T, bool mixed_vectors = false) {
  if (const char* e = P.finalize()) return fail(UH_EINVAL, "packing: %s", e);
  if (const char* e = P.self_check()) return fail(UH_EINVAL, "internal packing error: %s", e);
  int rc;
  const size_t eb = o->c128 ? 16 : 8;
  if (o->c128) {
    if ((rc = upload(P.M.data(), P.M.size() * sizeof(cd), &o->d_M))) return rc;
  } else {
    std::vector<cf> m32(P.M.size());
    for (size_t i = 0; i < P.M.size(); ++i)
      m32[i] = cf(static_cast<float>(P.M[i].real()), static_cast<float>(P.M[i].imag()));
    if ((rc = upload(m32.data(), m32.size() * sizeof(cf), &o->d_M))) return rc;
  }
  if ((rc = upload(P.items.data(), P.items.size() * sizeof(uh::WorkItem), &o->d_items))) return rc;
  if ((rc = upload(P.cta_begin.data(), P.cta_begin.size() * sizeof(int32_t), &o->d_cta))) return rc;
  if ((rc = upload(P.scatter.data(), P.scatter.size() * sizeof(uh::Scatter), &o->d_scatter))) return rc;
  if ((rc = upload(P.pool.data(), P.pool.size() * sizeof(uh::PoolRange), &o->d_pool))) return rc;
  o->pool_chunks = static_cast<int64_t>(P.pool.size());
  o->perm_n = P.permutation_length();
  o->done_len = uh::kFlagBase + P.flag_count();
  if ((rc = upload(static_cast<const void*>(nullptr), o->done_len * sizeof(unsigned long long), &o->d_done)))
    return rc;
  for (int c = 0; c < uh::kNumCounters; ++c) o->counter_total[c] = P.counter_total(c);
  if ((rc = upload(static_cast<const void*>(nullptr), sizeof(uint32_t), &o->d_status))) return rc;
  if ((rc = upload(T.perm.data(), T.perm.size() * sizeof(int32_t), &o->d_perm))) return rc;
  void** z[uh::kNumSources] = {&o->d_xp, &o->d_z1, &o->d_z2, &o->d_z3, &o->d_z4};
  int64_t vec_len = 0;
  for (int k = 0; k < uh::kNumSources; ++k) vec_len += P.src_len_[k];
  for (int k = 0; k < uh::kNumSources; ++k) o->src_len[k] = P.src_len_[k];
  for (int k = 0; k < uh::kNumSources; ++k)
    if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(std::max<int64_t>(P.src_len_[k], 2)) * eb, z[k])))
      return rc;
  if (mixed_vectors)
    for (int k = 0; k < uh::kNumSources; ++k)
      if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(std::max<int64_t>(P.src_len_[k], 2)) * 16,
                       &o->d_xm[k])))
        return rc;
  o->st.packed_bytes = P.tile_bytes_total + P.input_bytes_total;
  o->st.device_bytes = static_cast<int64_t>(P.M.size() * eb + P.items.size() * sizeof(uh::WorkItem) +
                                            P.chunks.size() * (sizeof(uh::OutChunk) + 4) + T.n * 4) +
                       vec_len * static_cast<int64_t>(eb);
  if (mixed_vectors) o->st.device_bytes += vec_len * int64_t{16};
  o->st.n_launches = 1;
  o->st.n_items = static_cast<int64_t>(P.items.size());
  return UH_OK;
}

// One product (nr = 1), or nr = 2 or 4 right-hand sides in one pass over the operator (complex64 UH
// ops with reserved multi-RHS scratch): x = xs[0], y = ys[0], right-hand side r at xs[r] / ys[r]
// (n values each; the caller checks that no output overlaps an input or another output).
int run_matvec(OpBase* o, const void* x, void* y, void* stream, long long timeout = kTimeoutCycles,
               bool stall = false, bool mixed = false, int nr = 1, const void* const* xs = nullptr,
               void* const* ys = nullptr) {
  if (!x || !y) return fail(UH_EINVAL, "x and y must be device pointers");
  if (mixed && (o->c128 || !o->d_xm[0]))
    return fail(UH_EINVAL, "the extended-precision product needs a complex64 UH op");
  const size_t eb = o->c128 || mixed ? 16 : 8;
  const char* xa = static_cast<const char*>(x);
  const char* ya = static_cast<const char*>(y);
  if (nr > 1 && (o->c128 || mixed || nr > o->multi_r || (nr != 2 && nr != 4) || (o->dual && nr > 2)))
    return fail(UH_EINVAL, "%d right-hand sides per pass need reserved scratch (uh_reserve)", nr);
  if (nr > 1 && (!xs || !ys)) return fail(UH_EINVAL, "right-hand side pointers missing");
  if (nr == 1 && xa < ya + o->n * static_cast<int64_t>(eb) && ya < xa + o->n * static_cast<int64_t>(eb))
    return fail(UH_EINVAL, "x and y overlap");
  std::lock_guard<std::mutex> lock(o->mu);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  if ((rc = order_call(o, s))) return rc;
  ++o->epoch;
  uh::StreamParams p{};
  p.items = o->d_items;
  p.cta_begin = o->d_cta;
  p.pool = o->d_pool;
  p.pool_chunks = o->pool_chunks;
  p.group_done = o->d_done;
  // every call takes pool_chunks + ncta tickets (each CTA stops after one past the end)
  p.ticket_base = (o->epoch - 1u) * static_cast<unsigned long long>(o->pool_chunks + o->ncta);
  p.flag_need = stall ? o->epoch + 1u : o->epoch;
  // A group is complete in call number `epoch` when its counter reaches epoch * (its chunks);
  // the stall test asks for one call more, which no chunk ever delivers.
  for (int c = 0; c < uh::kNumCounters; ++c)
    p.need[c] = static_cast<unsigned long long>(stall ? o->epoch + 1u : o->epoch) *
                static_cast<unsigned long long>(o->counter_total[c]);
  p.M = o->d_M;
  p.x = x;
  p.n = o->perm_n;
  p.y = y;
  p.perm = o->d_perm;
  p.scatter = o->d_scatter;
  void* const* vec = mixed ? o->d_xm : nr > 1 ? o->d_xr : nullptr;
  p.xp = vec ? vec[0] : o->d_xp;
  p.z1 = vec ? vec[1] : o->d_z1;
  p.z2 = vec ? vec[2] : o->d_z2;
  p.z3 = vec ? vec[3] : o->d_z3;
  p.z4 = vec ? vec[4] : o->d_z4;
  for (int r = 0; r < nr && nr > 1; ++r) {
    p.xr[r] = xs[r];
    p.yr[r] = ys[r];
  }
  p.status = o->d_status;
  p.timeout_cycles = timeout;
  const int variant = mixed ? (o->dual ? uh::kVarMixedDual : uh::kVarMixed)
                      : o->c128 ? (o->dual ? uh::kVarC128Dual : uh::kVarC128)
                      : nr == 4 ? uh::kVarC64R4
                      : nr == 2 ? (o->dual ? uh::kVarC64DualR2 : uh::kVarC64R2)
                      : o->dual ? uh::kVarC64Dual : uh::kVarC64;
  cudaError_t e = uh::stream_launch(variant, p, o->ncta, s);
  if (e != cudaSuccess) {
    --o->epoch;  // nothing launched: the counters did not move
    return fail(UH_ECUDA, "streaming kernel launch: %s", cudaGetErrorString(e));
  }
  return call_done(o, s);
}

int check_status(OpBase* o, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(o->mu);
  int rc;
  if ((rc = order_call(o, s))) return rc;
  uint32_t v = 0;
  CUDA_TRY(cudaMemcpyAsync(&v, o->d_status, sizeof v, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (v) {
    // A call that ran out left its group counters short: restart the counting.
    CUDA_TRY(cudaMemsetAsync(o->d_status, 0, sizeof(uint32_t), s));
    CUDA_TRY(cudaMemsetAsync(o->d_done, 0, o->done_len * sizeof(unsigned long long), s));
    if (o->d_pdone) CUDA_TRY(cudaMemsetAsync(o->d_pdone, 0, 2 * sizeof(unsigned long long), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    o->epoch = 0;
    o->panel_epoch = 0;
    return fail(UH_ETIMEOUT, "a bounded device-side wait ran out (code %u)", v);
  }
  return UH_OK;
}

int check_precision(int32_t precision, bool tensor_ok) {
  if (precision == UH_PREC_C128 || precision == UH_PREC_C64) return UH_OK;
  if (tensor_ok && (precision == UH_PREC_C64_TF32 || precision == UH_PREC_C64_BF16X3)) return UH_OK;
  return fail(UH_EINVAL, "precision %d not supported%s", precision,
              tensor_ok ? "" : " here (UH_PREC_C128 or UH_PREC_C64 only)");
}


// Row tiles covered by [r0, r1).
template <class F>
void for_tiles(const std::vector<Tile>& tiles, int64_t r0, int64_t r1, F f) {
  auto it = std::lower_bound(tiles.begin(), tiles.end(), r0, [](const Tile& t, int64_t v) { return t.p0 < v; });
  for (; it != tiles.end() && it->p0 < r1; ++it) f(static_cast<size_t>(it - tiles.begin()));
}

// Checks of a matmat call shared by the UH and H forms.
int check_matmat_args(const OpBase* o, int32_t nrhs, const void* X, int64_t ldx, const void* Y, int64_t ldy) {
  if (nrhs < 1) return fail(UH_EINVAL, "nrhs = %d", nrhs);
  if (!X || !Y) return fail(UH_EINVAL, "X and Y must be device pointers");
  if (ldx < o->n || ldy < o->n) return fail(UH_EINVAL, "leading dimensions %lld, %lld below n = %lld", (long long)ldx,
                                            (long long)ldy, (long long)o->n);
  const size_t eb = o->c128 ? 16 : 8;
  const char* xa = static_cast<const char*>(X);
  const char* ya = static_cast<const char*>(Y);
  const size_t xl = (static_cast<size_t>(ldx) * (nrhs - 1) + o->n) * eb;
  const size_t yl = (static_cast<size_t>(ldy) * (nrhs - 1) + o->n) * eb;
  if (xa < ya + yl && ya < xa + xl) return fail(UH_EINVAL, "X and Y overlap");
  return UH_OK;
}

// The tensor-core multi-RHS program of a UH op (uh_panel.h): xhat and yhat as compact panels
// (xhat_sigma at rows xo[sigma], yhat_tau at rows yo[tau]); phase 0 forward chunks, phase 1
// coupling chunks, phase 2 one chunk per row tile (near-field blocks, then the row bases of the
// tile's row clusters). Packs, self-checks and, unless only packing, uploads it.
int build_panel(OpBase* o, const uh_desc* d, const Tree& T, const std::vector<Tile>& tiles,
                const std::vector<std::vector<int32_t>>& tile_rows, const std::vector<char>& is_row,
                const std::vector<char>& is_col, const std::vector<std::vector<int64_t>>& row_blocks,
                const std::vector<std::vector<int64_t>>& col_blocks, int mm_mode, int ncta) {
  const int mode = mm_mode == UH_MM_BF16X3 ? uh::kPanelBF16X3 : uh::kPanelTF32;
  // Panels in operand-A layout: whole blocks of C rows; XP has one more, always zero, block.
  const int64_t C = uh::panel_block_rows(mode);
  auto up = [&](int64_t v) { return (v + C - 1) / C * C; };
  const int64_t xp_rows = up(T.n) + C;
  uh::PanelBuilder B(mode, ncta, up(T.n));
  auto live = [&](int64_t b) {
    return d->row_rank[d->adm_row[b]] > 0 && d->col_rank[d->adm_col[b]] > 0 && !(d->S_rank && d->S_rank[b] == 0);
  };
  // xhat_sigma and yhat_tau each start a block
  std::vector<int64_t> xo(T.ncl, -1), yo(T.ncl, -1);
  int64_t nx = 0, ny = 0;
  for (int32_t c = 0; c < T.ncl; ++c) {
    if (is_col[c] && d->col_rank[c] > 0) { xo[c] = nx; nx += up(d->col_rank[c]); }
    if (is_row[c] && d->row_rank[c] > 0) { yo[c] = ny; ny += up(d->row_rank[c]); }
  }
  // Splits l outputs into chunks of at most kPanelMaxH rows that start on block boundaries.
  auto pieces = [&](int32_t l) {
    std::vector<int32_t> cut;
    const int32_t k = static_cast<int32_t>((l + (uh::kPanelMaxH - C) - 1) / (uh::kPanelMaxH - C));
    for (int32_t q = 0; q <= k; ++q) cut.push_back(q == k ? l : static_cast<int32_t>(up(static_cast<int64_t>(l) * q / k)));
    return cut;
  };
  const Src V{d->V_data, d->data_type}, S{d->S_data, d->data_type}, U{d->U_data, d->data_type};
  const Src D{d->dense.data, d->data_type};
  // Coefficient matrices stored factored are assembled here, S_b = S_X,b S_Y,b^* in FP64 from the
  // stored factors, and packed like the dense ones.
  std::vector<std::complex<double>> sfull;
  std::vector<int64_t> sfull_off(d->n_adm, -1);
  for (int64_t b = 0; b < d->n_adm; ++b) {
    const int32_t k = d->S_rank ? d->S_rank[b] : -1;
    if (k <= 0 || !live(b)) continue;
    const int64_t lt = d->row_rank[d->adm_row[b]], ls = d->col_rank[d->adm_col[b]];
    sfull_off[b] = static_cast<int64_t>(sfull.size());
    sfull.resize(sfull.size() + static_cast<size_t>(lt * ls));
    std::complex<double>* out = sfull.data() + sfull_off[b];
    const int64_t x0 = d->S_off[b], y0 = d->S_off[b] + lt * k;
    for (int64_t j = 0; j < ls; ++j)
      for (int64_t i = 0; i < lt; ++i) {
        std::complex<double> v = 0;
        for (int64_t r = 0; r < k; ++r) v += S.at(x0 + r * lt + i) * std::conj(S.at(y0 + r * ls + j));
        out[j * lt + i] = v;
      }
  }
  const Src SF{sfull.data(), UH_DATA_C128};
  for (int32_t s = 0; s < T.ncl; ++s) {
    if (xo[s] < 0) continue;
    bool used = false;
    for (int64_t b : col_blocks[s]) used = used || live(b);
    if (!used) continue;
    const int32_t l = d->col_rank[s];
    const int64_t m = T.size[s];
    const std::vector<int32_t> cut = pieces(l);
    for (size_t q = 0; q + 1 < cut.size(); ++q) {
      const int j0 = cut[q], j1 = cut[q + 1];
      B.add_chunk(0, uh::kPOutZ1, xo[s] + j0, j1 - j0,
                  {ColSpec{uh::kPSrcXP, T.begin[s], m, &V, true, d->col_off[s] + j0 * m, 1, m}});
    }
  }
  std::vector<ColSpec> cols;
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (yo[t] < 0) continue;
    const int32_t l = d->row_rank[t];
    const std::vector<int32_t> cut = pieces(l);
    for (size_t q = 0; q + 1 < cut.size(); ++q) {
      const int i0 = cut[q], i1 = cut[q + 1];
      cols.clear();
      for (int64_t b : row_blocks[t]) {
        if (!live(b)) continue;
        const int32_t s = d->adm_col[b];
        if (sfull_off[b] >= 0)
          cols.push_back(ColSpec{uh::kPSrcZ1, xo[s], d->col_rank[s], &SF, false, sfull_off[b] + i0, l, 1});
        else
          cols.push_back(ColSpec{uh::kPSrcZ1, xo[s], d->col_rank[s], &S, false, d->S_off[b] + i0, l, 1});
      }
      B.add_chunk(1, uh::kPOutZ2, yo[t] + i0, i1 - i0, cols);
    }
  }
  std::vector<std::vector<int64_t>> near(tiles.size());
  for (int64_t i = 0; i < d->dense.n_dense; ++i)
    for_tiles(tiles, T.begin[d->dense.row_cl[i]], T.begin[d->dense.row_cl[i]] + T.size[d->dense.row_cl[i]],
              [&](size_t t) { near[t].push_back(i); });
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    const int64_t p0 = tiles[ti].p0;
    cols.clear();
    for (int64_t i : near[ti]) {
      const int32_t tau = d->dense.row_cl[i], sg = d->dense.col_cl[i];
      cols.push_back(ColSpec{uh::kPSrcXP, T.begin[sg], T.size[sg], &D, false, d->dense.off[i] + p0 - T.begin[tau],
                             T.size[tau], 1});
    }
    for (int32_t t : tile_rows[ti])
      cols.push_back(ColSpec{uh::kPSrcZ2, yo[t], d->row_rank[t], &U, false, d->row_off[t] + p0 - T.begin[t],
                             T.size[t], 1});
    B.add_chunk(2, uh::kPOutY, p0, static_cast<int>(tiles[ti].h), cols);
  }
  if (const char* e = B.finalize()) return fail(UH_EINVAL, "multi-RHS packing: %s", e);
  const int64_t src_rows[3] = {xp_rows, std::max<int64_t>(nx, C), std::max<int64_t>(ny, C)},
                out_rows[3] = {nx, ny, T.n};
  if (const char* e = B.self_check(src_rows, out_rows)) return fail(UH_EINVAL, "internal multi-RHS packing error: %s", e);
  if (!o) return UH_OK;
  int rc;
  if ((rc = uh::panel_prepare())) return rc;
  if ((rc = upload(B.tiles.data(), B.tiles.size(), &o->d_ptiles))) return rc;
  if ((rc = upload(B.items.data(), B.items.size() * sizeof(uh::PanelItem), &o->d_pitems))) return rc;
  if ((rc = upload(B.begin.data(), B.begin.size() * sizeof(int32_t), &o->d_pbegin))) return rc;
  const size_t row = uh::kPanelRowBytes;
  // zero-filled: the padding rows of every block stay zero (the epilogues write whole blocks of
  // zeros past a chunk's rows, the gather zeros past n)
  if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(src_rows[0]) * row, &o->d_pxp))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(src_rows[1]) * row, &o->d_pz1))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), static_cast<size_t>(src_rows[2]) * row, &o->d_pz2))) return rc;
  if ((rc = upload(static_cast<const void*>(nullptr), 2 * sizeof(unsigned long long), &o->d_pdone))) return rc;
  o->mm_mode = mm_mode;
  o->panel_mode = mode;
  o->panel_ncta = ncta;
  o->panel_xp_rows = xp_rows;
  o->panel_zchunks[0] = B.z_chunks[0];
  o->panel_zchunks[1] = B.z_chunks[1];
  o->st.matmat_mode = mm_mode;
  o->st.panel_bytes = B.streamed_bytes;
  o->st.panel_mma_flops = B.mma_flops;
  o->st.panel_items = static_cast<int64_t>(B.items.size());
  o->st.device_bytes += static_cast<int64_t>(B.tiles.size() + B.items.size() * sizeof(uh::PanelItem)) +
                        (src_rows[0] + src_rows[1] + src_rows[2]) * static_cast<int64_t>(row);
  return UH_OK;
}

// Number of CTAs of the multi-RHS launches: one per SM.
int panel_ncta(int* ncta) {
  int device = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&device));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  *ncta = sms;
  return UH_OK;
}

// The CUDA-core multi-RHS product: passes of multi_r right-hand sides (then 2), then one product
// per remaining column (X and Y do not overlap: checked by the caller).
int matmat_by_columns(OpBase* o, int32_t nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy, void* stream) {
  const size_t eb = o->c128 ? 16 : 8;
  for (int32_t r = 0; r < nrhs;) {
    const int left = nrhs - r;
    const int nr = o->multi_r >= 4 && left >= 4 ? 4 : o->multi_r >= 2 && left >= 2 ? 2 : 1;
    const void* xs[4];
    void* ys[4];
    for (int q = 0; q < nr; ++q) {
      xs[q] = static_cast<const char*>(X) + static_cast<size_t>(r + q) * ldx * eb;
      ys[q] = static_cast<char*>(Y) + static_cast<size_t>(r + q) * ldy * eb;
    }
    const int rc = run_matvec(o, xs[0], ys[0], stream, kTimeoutCycles, false, false, nr, xs, ys);
    if (rc) return rc;
    r += nr;
  }
  return UH_OK;
}


// Near-field chunks of the row tiles, alternating between the two near-field groups (static,
// before the coupling; and the first part of the pool); with `split`, the static half is itself
// shared between the group before the t_b chunks and the group after them. A tile with a backward part writes its z3
// slot (the backward chunk adds it), otherwise y directly. Returns, per tile, the near-field chunk
// writing z3 (or -1).
// offN: position of the operator's first point in the program's vectors; z3pos: next free z3 slot
// (advanced; when null the slots start at 0 and the z3 length is set here).
std::vector<int> add_near_field(ProgramBuilder& P, const Tree& T, const uh_dense_desc& d, const Src& D,
                                const std::vector<Tile>& tiles, const std::vector<char>& has_back,
                                std::vector<char>* has_near, int64_t offN = 0, int64_t* z3pos = nullptr,
                                bool split = false) {
  const int64_t A = P.align();
  std::vector<std::vector<int64_t>> per_tile(tiles.size());
  for (int64_t i = 0; i < d.n_dense; ++i)
    for_tiles(tiles, T.begin[d.row_cl[i]], T.begin[d.row_cl[i]] + T.size[d.row_cl[i]],
              [&](size_t t) { per_tile[t].push_back(i); });
  std::vector<int> zchunk(tiles.size(), -1);
  has_near->assign(tiles.size(), 0);
  int64_t pos = z3pos ? *z3pos : 0;
  std::vector<int64_t> slot(tiles.size(), -1);
  for (size_t t = 0; t < tiles.size(); ++t) {
    (*has_near)[t] = !per_tile[t].empty();
    if (per_tile[t].empty() || !has_back[t]) continue;
    slot[t] = pos;
    pos += ProgramBuilder::round_up(tiles[t].h, A);
  }
  if (z3pos) *z3pos = pos;
  else P.set_source_len(uh::kSrcZ3, pos);
  int parity = 0;
  std::vector<ColSpec> cols;
  for (size_t t = 0; t < tiles.size(); ++t) {
    if (per_tile[t].empty()) continue;
    const int par = parity++;
    const int group = (par & 1) ? uh::kGroupNearB : (split && (par & 2)) ? uh::kGroupNearA2 : uh::kGroupNearA;
    const int c = slot[t] >= 0 ? P.add_chunk(uh::kToZ3, slot[t], tiles[t].h, group)
                               : P.add_chunk(uh::kToY, offN + tiles[t].p0, tiles[t].h, group);
    if (slot[t] >= 0) zchunk[t] = c;
    cols.clear();
    for (int64_t i : per_tile[t]) {
      const int32_t tau = d.row_cl[i], sg = d.col_cl[i];
      cols.push_back(ColSpec{uh::kSrcXp, offN + T.begin[sg], T.size[sg], &D, false,
                             d.off[i] + tiles[t].p0 - T.begin[tau], T.size[tau], 1});
    }
    P.add_columns(c, cols);
  }
  return zchunk;
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


// A validated UH descriptor and the structure derived from it.
struct UHPrep {
  const uh_desc* d = nullptr;
  Tree T;
  std::vector<char> is_row, is_col;
  std::vector<Tile> tiles;
  std::vector<std::vector<int64_t>> row_blocks, col_blocks;  // sorted by column / row cluster
  std::vector<std::vector<int32_t>> tile_rows;               // row clusters with a basis containing each tile
};

int prepare_uh(const uh_desc* d, UHPrep* u) {
  int rc;
  if (d->data_type != UH_DATA_C128 && d->data_type != UH_DATA_C64) return fail(UH_EINVAL, "data_type %d", d->data_type);
  u->d = d;
  Tree& T = u->T;
  if ((rc = check_tree(d->tree, &T))) return rc;
  if (d->n_adm < 0) return fail(UH_EINVAL, "n_adm < 0");
  if (d->n_adm > 0 && (!d->adm_row || !d->adm_col || !d->S_off || !d->S_data || !d->row_rank || !d->row_off ||
                       !d->col_rank || !d->col_off || !d->U_data || !d->V_data))
    return fail(UH_EINVAL, "admissible part incomplete");
  if ((rc = check_dense(T, d->dense))) return rc;
  u->is_row.assign(T.ncl, 0);
  u->is_col.assign(T.ncl, 0);
  for (int64_t i = 0; i < d->n_adm; ++i) {
    if ((rc = check_cluster_index(T, d->adm_row[i], "adm_row", i))) return rc;
    if ((rc = check_cluster_index(T, d->adm_col[i], "adm_col", i))) return rc;
    u->is_row[d->adm_row[i]] = 1;
    u->is_col[d->adm_col[i]] = 1;
  }
  for (int32_t c = 0; c < T.ncl; ++c) {
    if (u->is_row[c]) {
      const int32_t l = d->row_rank[c];
      if (l < 0 || l > T.size[c]) return fail(UH_EINVAL, "row_rank[%d] = %d outside [0, %lld]", c, l, (long long)T.size[c]);
      if ((rc = check_range(d->row_off[c], T.size[c] * l, d->U_len, "row basis", c))) return rc;
    }
    if (u->is_col[c]) {
      const int32_t l = d->col_rank[c];
      if (l < 0 || l > T.size[c]) return fail(UH_EINVAL, "col_rank[%d] = %d outside [0, %lld]", c, l, (long long)T.size[c]);
      if ((rc = check_range(d->col_off[c], T.size[c] * l, d->V_len, "column basis", c))) return rc;
    }
  }
  for (int64_t i = 0; i < d->n_adm; ++i) {
    const int32_t lt = d->row_rank[d->adm_row[i]], ls = d->col_rank[d->adm_col[i]];
    const int32_t k = d->S_rank ? d->S_rank[i] : -1;
    if (k < -1 || k > std::min(lt, ls))
      return fail(UH_EINVAL, "S_rank[%lld] = %d outside [-1, %d]", (long long)i, k, std::min(lt, ls));
    const int64_t cnt = k < 0 ? static_cast<int64_t>(lt) * ls : static_cast<int64_t>(k) * (lt + ls);
    if ((rc = check_range(d->S_off[i], cnt, d->S_len, "coupling matrix", i))) return rc;
  }
  std::vector<int32_t> brow, bcol;
  for (int64_t i = 0; i < d->n_adm; ++i) { brow.push_back(d->adm_row[i]); bcol.push_back(d->adm_col[i]); }
  for (int64_t i = 0; i < d->dense.n_dense; ++i) { brow.push_back(d->dense.row_cl[i]); bcol.push_back(d->dense.col_cl[i]); }
  if ((rc = make_tiles_and_check(T, brow, bcol, &u->tiles))) return rc;
  u->row_blocks.assign(T.ncl, {});
  u->col_blocks.assign(T.ncl, {});
  for (int64_t i = 0; i < d->n_adm; ++i) {
    u->row_blocks[d->adm_row[i]].push_back(i);
    u->col_blocks[d->adm_col[i]].push_back(i);
  }
  for (int32_t c = 0; c < T.ncl; ++c) {
    std::stable_sort(u->row_blocks[c].begin(), u->row_blocks[c].end(),
                     [&](int64_t a, int64_t b) { return d->adm_col[a] < d->adm_col[b]; });
    std::stable_sort(u->col_blocks[c].begin(), u->col_blocks[c].end(),
                     [&](int64_t a, int64_t b) { return d->adm_row[a] < d->adm_row[b]; });
  }
  u->tile_rows.assign(u->tiles.size(), {});
  for (int32_t t = 0; t < T.ncl; ++t)
    if (u->is_row[t] && d->row_rank[t] > 0)
      for_tiles(u->tiles, T.begin[t], T.begin[t] + T.size[t], [&](size_t i) { u->tile_rows[i].push_back(t); });
  return UH_OK;
}

// Vector offsets of one operator inside a program that may hold several (a batch): its points
// start at position n in xp and y; its z1, z2, z3 and z4 parts start at x, y, z3, t (all advanced
// past what the operator uses).
struct Offsets {
  int64_t n = 0, x = 0, y = 0, z3 = 0, t = 0;
};

// The forward, near-field, coupling and backward chunks of one UH operator (Algorithm 6), with
// the scatter layout of z1 / z2 (see the file comment), and for coefficient matrices stored
// factored the t_b chunks into z4. The permutation chunks and the source lengths are the caller's.
void add_uh_program(ProgramBuilder& P, const UHPrep& u, Offsets* off) {
  const uh_desc* d = u.d;
  const Tree& T = u.T;
  const int64_t A = P.align();
  const auto& tiles = u.tiles;
  const auto& row_blocks = u.row_blocks;
  const auto& col_blocks = u.col_blocks;
  const auto& tile_rows = u.tile_rows;
  const int64_t on = off->n;
  // inner rank k_b of a coefficient matrix stored factored (Section 4.2), -1 for a dense S_b
  auto frank = [&](int64_t b) { return d->S_rank ? d->S_rank[b] : -1; };
  auto live = [&](int64_t b) {
    return d->row_rank[d->adm_row[b]] > 0 && d->col_rank[d->adm_col[b]] > 0 && frank(b) != 0;
  };
  auto dense_s = [&](int64_t b) { return live(b) && frank(b) < 0; };
  auto fact_s = [&](int64_t b) { return live(b) && frank(b) > 0; };
  // z1: per row cluster tau, the coupling inputs [xhat_sigma] of its dense-S blocks back to back
  // (the forward chunks scatter each xhat_sigma into every segment that uses it); then, per column
  // cluster sigma with factored blocks, one more copy of xhat_sigma at xs[sigma], the input of t_b.
  std::vector<int64_t> xin(T.ncl, -1), xpos(d->n_adm, -1), xs(T.ncl, -1);
  int64_t nx = off->x;
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (!u.is_row[t] || d->row_rank[t] == 0) continue;
    xin[t] = nx;
    int64_t pos = 0;
    for (int64_t b : row_blocks[t])
      if (dense_s(b)) { xpos[b] = pos; pos += d->col_rank[d->adm_col[b]]; }
    nx += ProgramBuilder::round_up(std::max<int64_t>(pos, 1), A);
  }
  for (int32_t s = 0; s < T.ncl; ++s) {
    if (!u.is_col[s] || d->col_rank[s] == 0) continue;
    bool f = false;
    for (int64_t b : col_blocks[s]) f = f || fact_s(b);
    if (f) { xs[s] = nx; nx += ProgramBuilder::round_up(d->col_rank[s], A); }
  }
  // z4: per row cluster tau, [t_b] of its factored blocks back to back (the t_b chunks scatter
  // each block's rows there), so the coupling chunk of tau reads them as one run.
  std::vector<int64_t> tin(T.ncl, -1), tpos(d->n_adm, -1);
  int64_t nt = off->t;
  bool any_factored = false;
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (!u.is_row[t] || d->row_rank[t] == 0) continue;
    int64_t pos = 0;
    for (int64_t b : row_blocks[t])
      if (fact_s(b)) { tpos[b] = pos; pos += frank(b); }
    if (pos == 0) continue;
    tin[t] = nt;
    nt += ProgramBuilder::round_up(pos, A);
    any_factored = true;
  }
  std::vector<char> has_back(tiles.size(), 0);
  // z2: per row tile, the backward inputs [yhat_tau]_{tau contains the tile} back to back (the
  // coupling chunks scatter each yhat_tau into every tile inside tau).
  std::vector<int64_t> yin(tiles.size(), -1);
  std::vector<std::vector<int64_t>> ypos(tiles.size());
  int64_t ny = off->y;
  for (size_t i = 0; i < tiles.size(); ++i) {
    has_back[i] = !tile_rows[i].empty();
    if (!has_back[i]) continue;
    yin[i] = ny;
    int64_t pos = 0;
    for (int32_t t : tile_rows[i]) { ypos[i].push_back(pos); pos += d->row_rank[t]; }
    ny += ProgramBuilder::round_up(pos, A);
  }
  const Src V{d->V_data, d->data_type}, S{d->S_data, d->data_type}, U{d->U_data, d->data_type};
  const Src D{d->dense.data, d->data_type};
  // Forward transform: chunks of at most 64 rows of V_sigma^*; column r = conj(V_sigma[r, rows]).
  for (int32_t s = 0; s < T.ncl; ++s) {
    if (!u.is_col[s] || d->col_rank[s] == 0) continue;
    std::vector<int64_t> users;
    for (int64_t b : col_blocks[s])
      if (dense_s(b)) users.push_back(b);
    if (users.empty() && xs[s] < 0) continue;
    const int32_t l = d->col_rank[s];
    const int64_t m = T.size[s];
    const int k = (l + uh::kStreamHpMax - 1) / uh::kStreamHpMax;
    for (int q = 0; q < k; ++q) {
      const int j0 = l * q / k, j1 = l * (q + 1) / k;
      const int c = P.add_chunk(uh::kScatterZ1, 0, j1 - j0, uh::kGroupForward, uh::kCounterForward);
      for (int64_t b : users) P.add_scatter(c, xin[d->adm_row[b]] + xpos[b] + j0, 0, j1 - j0);
      if (xs[s] >= 0) P.add_scatter(c, xs[s] + j0, 0, j1 - j0);
      P.add_columns(c, {ColSpec{uh::kSrcXp, on + T.begin[s], m, &V, true, d->col_off[s] + j0 * m, 1, m}});
    }
  }
  std::vector<char> has_near;
  const std::vector<int> zchunk =
      add_near_field(P, T, d->dense, D, tiles, has_back, &has_near, on, &off->z3, any_factored);
  // t_b = S_Y,b^* xhat_sigma: per column cluster sigma, the rows conj(S_Y,b[:, j]) of its factored
  // blocks stacked (blocks in increasing row cluster) and cut into tall chunks of at most
  // kStreamHpTall rows, input
  // the copy of xhat_sigma at xs[sigma]; each block's rows are scattered to its place in z4.
  std::vector<int64_t> rowoff;
  std::vector<std::pair<int64_t, int32_t>> rowblk;  // (block, j) of each stacked row
  for (int32_t s = 0; s < T.ncl; ++s) {
    if (xs[s] < 0) continue;
    const int32_t ls = d->col_rank[s];
    rowoff.clear();
    rowblk.clear();
    for (int64_t b : col_blocks[s]) {
      if (!fact_s(b)) continue;
      const int64_t lt = d->row_rank[d->adm_row[b]];
      const int32_t k = frank(b);
      for (int32_t j = 0; j < k; ++j) {
        rowoff.push_back(d->S_off[b] + lt * k + static_cast<int64_t>(j) * ls);
        rowblk.emplace_back(b, j);
      }
    }
    const int64_t rows = static_cast<int64_t>(rowoff.size());
    const int64_t nq = (rows + uh::kStreamHpTall - 1) / uh::kStreamHpTall;
    for (int64_t q = 0; q < nq; ++q) {
      const int64_t r0 = rows * q / nq, r1 = rows * (q + 1) / nq;
      const int c = P.add_chunk(uh::kScatterZ4, 0, static_cast<int>(r1 - r0), uh::kGroupCouplingY, uh::kCounterCouplingY);
      for (int64_t r = r0; r < r1;) {
        const int64_t b = rowblk[r].first;
        int64_t e = r;
        while (e < r1 && rowblk[e].first == b) ++e;
        P.add_scatter(c, tin[d->adm_row[b]] + tpos[b] + rowblk[r].second, static_cast<int>(r - r0),
                      static_cast<int>(e - r0));
        r = e;
      }
      ColSpec cs{uh::kSrcZ1, xs[s], ls, &S, true, 0, 1, 0};
      cs.rowoff = rowoff.data() + r0;
      P.add_columns(c, {cs});
    }
  }
  // Coupling: per row cluster tau (chunks of at most 64 rows), columns [S_b] of its dense-S blocks
  // (inputs one run of z1), then [S_X,b] of its factored blocks (inputs one run of z4); outputs
  // scattered to the tiles inside tau.
  std::vector<ColSpec> cols;
  for (int32_t t = 0; t < T.ncl; ++t) {
    if (!u.is_row[t] || d->row_rank[t] == 0) continue;
    const int32_t l = d->row_rank[t];
    const int k = (l + uh::kStreamHpMax - 1) / uh::kStreamHpMax;
    for (int q = 0; q < k; ++q) {
      const int i0 = l * q / k, i1 = l * (q + 1) / k;
      const int c = P.add_chunk(uh::kScatterZ2, 0, i1 - i0, uh::kGroupCoupling, uh::kCounterCoupling);
      for_tiles(tiles, T.begin[t], T.begin[t] + T.size[t], [&](size_t ti) {
        const auto& tr = tile_rows[ti];
        const size_t w = std::find(tr.begin(), tr.end(), t) - tr.begin();
        P.add_scatter(c, yin[ti] + ypos[ti][w] + i0, 0, i1 - i0);
      });
      cols.clear();
      for (int64_t b : row_blocks[t]) {
        if (!dense_s(b)) continue;
        const int32_t s = d->adm_col[b];
        cols.push_back(ColSpec{uh::kSrcZ1, xin[t] + xpos[b], d->col_rank[s], &S, false, d->S_off[b] + i0, l, 1});
      }
      for (int64_t b : row_blocks[t])
        if (fact_s(b)) cols.push_back(ColSpec{uh::kSrcZ4, tin[t] + tpos[b], frank(b), &S, false, d->S_off[b] + i0, l, 1});
      P.add_columns(c, cols);
    }
  }
  // Backward transform (+ near-field base): per row tile, columns U_tau[tile rows, :] of every
  // row cluster tau containing the tile, inputs one run of z2.
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    if (!has_back[ti]) {
      // the near-field chunk writes y; a tile whose blocks all have rank 0 and no near field
      // gets an empty chunk, which writes zeros
      if (!has_near[ti]) P.add_columns(P.add_chunk(uh::kToY, on + tiles[ti].p0, tiles[ti].h, uh::kGroupBackward), {});
      continue;
    }
    const int c = P.add_chunk(uh::kToY, on + tiles[ti].p0, tiles[ti].h, uh::kGroupBackward);
    cols.clear();
    for (size_t w = 0; w < tile_rows[ti].size(); ++w) {
      const int32_t t = tile_rows[ti][w];
      const int64_t m = T.size[t];
      cols.push_back(ColSpec{uh::kSrcZ2, yin[ti] + ypos[ti][w], d->row_rank[t], &U, false,
                             d->row_off[t] + tiles[ti].p0 - T.begin[t], m, 1});
    }
    P.add_columns(c, cols, zchunk[ti]);
  }
  off->n += T.n;
  off->x = nx;
  off->y = ny;
  off->t = nt;
}

// Sizes of one UH operator and of its product (uh_stats_t); elem_bytes s.
void uh_fill_stats(const UHPrep& u, int32_t precision, int s, uh_stats_t* st) {
  const uh_desc* d = u.d;
  const Tree& T = u.T;
  st->n = T.n;
  st->precision = precision;
  st->elem_bytes = s;
  st->n_dense = d->dense.n_dense;
  int64_t ed = 0;
  for (int64_t i = 0; i < d->dense.n_dense; ++i) ed += T.size[d->dense.row_cl[i]] * T.size[d->dense.col_cl[i]];
  st->E_D = ed;
  int64_t eu = 0, ev = 0, es = 0, nrb = 0, ncb = 0, srr = 0, scr = 0;
  int32_t rmin = INT32_MAX, rmax = 0;
  int64_t rsum = 0, rcnt = 0;
  std::vector<int32_t> rowc(T.ncl, 0), colc(T.ncl, 0);
  int64_t nf = 0, kf = 0;
  for (int64_t i = 0; i < d->n_adm; ++i) {
    rowc[d->adm_row[i]]++;
    colc[d->adm_col[i]]++;
    const int64_t lt = d->row_rank[d->adm_row[i]], ls = d->col_rank[d->adm_col[i]];
    const int32_t k = d->S_rank ? d->S_rank[i] : -1;
    if (k < 0) {
      es += lt * ls;
    } else {
      es += k * (lt + ls);
      nf++;
      kf += k;
    }
  }
  int32_t csp = 0;
  for (int32_t c = 0; c < T.ncl; ++c) {
    csp = std::max(csp, std::max(rowc[c], colc[c]));
    if (u.is_row[c]) {
      nrb++; eu += T.size[c] * d->row_rank[c]; srr += d->row_rank[c];
      if (d->row_rank[c] > 0) { rmin = std::min(rmin, d->row_rank[c]); rmax = std::max(rmax, d->row_rank[c]); rsum += d->row_rank[c]; rcnt++; }
    }
    if (u.is_col[c]) {
      ncb++; ev += T.size[c] * d->col_rank[c]; scr += d->col_rank[c];
      if (d->col_rank[c] > 0) { rmin = std::min(rmin, d->col_rank[c]); rmax = std::max(rmax, d->col_rank[c]); rsum += d->col_rank[c]; rcnt++; }
    }
  }
  st->n_row_bases = nrb;
  st->n_col_bases = ncb;
  st->n_adm = d->n_adm;
  st->E_U = eu;
  st->E_V = ev;
  st->E_S = es;
  st->sum_row_rank = srr;
  st->sum_col_rank = scr;
  st->rank_min = rcnt ? rmin : 0;
  st->rank_max = rmax;
  st->rank_mean = rcnt ? static_cast<double>(rsum) / rcnt : 0.0;
  st->csp = csp;
  st->n_factored = nf;
  st->sum_factored_rank = kf;
  st->algo_bytes_matvec = s * (eu + ev + es + ed + 2 * T.n + 2 * (srr + scr) + 2 * kf);
  st->matmat_mode = -1;
}

// Scratch of the CUDA-core multi-RHS product (uh_reserve / h_reserve).
int reserve_multi(OpBase* op, int32_t max_nrhs) {
  if (!op) return fail(UH_EINVAL, "null op");
  if (max_nrhs < 1) return fail(UH_EINVAL, "max_nrhs = %d", max_nrhs);
  if (op->c128) return UH_OK;
  // right-hand sides per pass: 4 (one CTA per SM), 2 (two CTAs per SM: the shared memory of the
  // four-wide stages does not fit twice)
  const int want = max_nrhs >= 4 && !op->dual ? 4 : max_nrhs >= 2 ? 2 : 1;
  if (want <= op->multi_r || want < 2) return UH_OK;
  std::lock_guard<std::mutex> lock(op->mu);
  CUDA_TRY(cudaDeviceSynchronize());  // no pass may use the old scratch while it is replaced
  const int variants[] = {op->dual ? uh::kVarC64DualR2 : uh::kVarC64R2, uh::kVarC64R4};
  const int need = op->dual ? 2 : 1;
  for (int v = 0; v < (want == 4 ? 2 : 1); ++v) {
    CUDA_TRY(uh::stream_prepare(variants[v]));
    int per = 0;
    CUDA_TRY(uh::stream_occupancy(variants[v], &per));
    if (per < need) return fail(UH_ECUDA, "multi-RHS streaming kernel does not fit %d CTAs per SM", need);
  }
  for (int k = 0; k < uh::kNumSources; ++k) {
    if (op->d_xr[k]) cudaFree(op->d_xr[k]);
    op->d_xr[k] = nullptr;
  }
  op->multi_r = 0;
  for (int k = 0; k < uh::kNumSources; ++k) {
    int rc = upload(static_cast<const void*>(nullptr),
                    static_cast<size_t>(std::max<int64_t>(op->src_len[k], 2)) * 8 * want, &op->d_xr[k]);
    if (rc) return rc;
  }
  op->multi_r = want;
  op->st.device_bytes += (op->src_len[0] + op->src_len[1] + op->src_len[2] + op->src_len[3] + op->src_len[4]) * 8 * want;
  return UH_OK;
}

}  // namespace

struct uh_op : OpBase {};
struct h_op : OpBase {};
struct uh_batch : OpBase {
  std::vector<int64_t> offsets;  // count + 1
};

extern "C" {

const char* uh_last_error(void) { return g_err.c_str(); }
const char* uh_version(void) { return "uh-gb300 0.2 (sm_103a)"; }

int uh_create(const uh_desc* d, int32_t precision, uh_op** out) { return uh_create_ex(d, precision, nullptr, out); }

int uh_create_ex(const uh_desc* d, int32_t precision, const uh_pack_params* params, uh_op** out) {
  g_err.clear();
  if (!d || !out) return fail(UH_EINVAL, "null argument");
  *out = nullptr;
  int rc;
  if ((rc = check_precision(precision, true))) return rc;
  const bool c128 = precision == UH_PREC_C128;
  uh::PackParams pp;
  if ((rc = pack_params_from(params, c128, &pp))) return rc;
  UHPrep u;
  if ((rc = prepare_uh(d, &u))) return rc;
  const Tree& T = u.T;
  {
    uh_stats_t est{};
    uh_fill_stats(u, precision, c128 ? 16 : 8, &est);
    resolve_ctas(&pp, est.algo_bytes_matvec);
  }

  const bool dual = pp.ctas_per_sm == 2;
  int ncta = g_pack_only_ncta, device = 0;
  if (!ncta && (rc = query_ncta(c128, &ncta, &device, dual))) return rc;
  ProgramBuilder P(c128, T.n, ncta, pp);
  const int64_t A = P.align();
  P.set_permutation(T.n);
  Offsets off;
  add_uh_program(P, u, &off);
  P.set_source_len(uh::kSrcXp, ProgramBuilder::round_up(T.n, A));
  P.set_source_len(uh::kSrcZ1, off.x);
  P.set_source_len(uh::kSrcZ2, off.y);
  P.set_source_len(uh::kSrcZ3, off.z3);
  P.set_source_len(uh::kSrcZ4, off.t);

  const int mm_mode = precision == UH_PREC_C64_TF32 ? UH_MM_TF32 : precision == UH_PREC_C64_BF16X3 ? UH_MM_BF16X3 : -1;
  if (g_pack_only_ncta) {
    if (const char* e = P.finalize()) return fail(UH_EINVAL, "packing: %s", e);
    if (const char* e = P.self_check()) return fail(UH_EINVAL, "internal packing error: %s", e);
    if (mm_mode >= 0)
      return build_panel(nullptr, d, T, u.tiles, u.tile_rows, u.is_row, u.is_col, u.row_blocks, u.col_blocks, mm_mode,
                         g_pack_only_ncta);
    return UH_OK;
  }
  auto* o = new (std::nothrow) uh_op();
  if (!o) return fail(UH_ENOMEM, "host allocation");
  o->c128 = c128;
  o->n = T.n;
  o->ncta = ncta;
  o->device = device;
  o->dual = dual;
  if ((rc = upload_program(o, P, T, !c128))) { free_op(o); delete o; return rc; }
  const uh_stats_t packed = o->st;  // packing figures filled by the upload
  uh_fill_stats(u, precision, c128 ? 16 : 8, &o->st);
  o->st.packed_bytes = packed.packed_bytes;
  o->st.device_bytes = packed.device_bytes;
  o->st.n_launches = packed.n_launches;
  o->st.n_items = packed.n_items;
  fill_pack_stats(pp, P.geometry(), &o->st);
  if (mm_mode >= 0) {
    int pn = 0;
    if ((rc = panel_ncta(&pn)) ||
        (rc = build_panel(o, d, T, u.tiles, u.tile_rows, u.is_row, u.is_col, u.row_blocks, u.col_blocks, mm_mode, pn))) {
      free_op(o);
      delete o;
      return rc;
    }
  }
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

int uh_matvec_mixed(uh_op* op, const void* x, void* y, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  return run_matvec(op, x, y, stream, kTimeoutCycles, false, true);
}

int uh_check(uh_op* op, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  return check_status(op, stream);
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
  if ((rc = check_precision(precision, false))) return rc;
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

  const bool c128 = precision == UH_PREC_C128;
  int ncta = g_pack_only_ncta, device = 0;
  if (!ncta && (rc = query_ncta(c128, &ncta, &device))) return rc;
  ProgramBuilder P(c128, T.n, ncta);
  const int64_t A = P.align();
  P.set_source_len(uh::kSrcXp, ProgramBuilder::round_up(T.n, A));
  P.set_source_len(uh::kSrcZ2, 0);
  P.set_permutation(T.n);
  // t_b = Y_b^* x|_sigma. The blocks of one column cluster sigma share their input x|_sigma, so
  // their rows Y_b^* are stacked (blocks in increasing row cluster) and cut into chunks of at most
  // 64 rows; t holds each sigma's t_b consecutively.
  std::vector<int64_t> toff(d->n_adm, -1);
  std::vector<std::vector<int64_t>> col_blocks(T.ncl);
  for (int64_t b = 0; b < d->n_adm; ++b)
    if (d->adm_rank[b] > 0) col_blocks[d->adm_col[b]].push_back(b);
  int64_t nt = 0;
  std::vector<int64_t> sbase(T.ncl, -1);
  for (int32_t s = 0; s < T.ncl; ++s) {
    auto& bl = col_blocks[s];
    if (bl.empty()) continue;
    std::stable_sort(bl.begin(), bl.end(), [&](int64_t a, int64_t b) { return d->adm_row[a] < d->adm_row[b]; });
    sbase[s] = nt;
    for (int64_t b : bl) { toff[b] = nt; nt += d->adm_rank[b]; }
    nt = ProgramBuilder::round_up(nt, A);
  }
  P.set_source_len(uh::kSrcZ1, nt);
  const Src Y{d->Y_data, d->data_type}, X{d->X_data, d->data_type}, D{d->dense.data, d->data_type};
  std::vector<int64_t> rowoff;
  for (int32_t s = 0; s < T.ncl; ++s) {
    const auto& bl = col_blocks[s];
    if (bl.empty()) continue;
    const int64_t m = T.size[s];
    rowoff.clear();  // row (b, j) of the stack: conj(Y_b[:, j]) starts at Y_off[b] + j * |sigma|
    for (int64_t b : bl)
      for (int j = 0; j < d->adm_rank[b]; ++j) rowoff.push_back(d->Y_off[b] + j * m);
    const int64_t rows = static_cast<int64_t>(rowoff.size());
    const int64_t nq = (rows + uh::kStreamHpMax - 1) / uh::kStreamHpMax;
    for (int64_t q = 0; q < nq; ++q) {
      const int64_t r0 = rows * q / nq, r1 = rows * (q + 1) / nq;
      const int c = P.add_chunk(uh::kToZ1, sbase[s] + r0, static_cast<int>(r1 - r0), uh::kGroupForward, uh::kCounterForward);
      ColSpec cs{uh::kSrcXp, T.begin[s], m, &Y, true, 0, 1, 0};
      cs.rowoff = rowoff.data() + r0;
      P.add_columns(c, {cs});
    }
  }
  std::vector<std::vector<int64_t>> tile_blocks(tiles.size());
  for (int64_t b = 0; b < d->n_adm; ++b)
    if (toff[b] >= 0)
      for_tiles(tiles, T.begin[d->adm_row[b]], T.begin[d->adm_row[b]] + T.size[d->adm_row[b]],
                [&](size_t i) { tile_blocks[i].push_back(b); });
  std::vector<char> has_back(tiles.size(), 0);
  for (size_t i = 0; i < tiles.size(); ++i) has_back[i] = !tile_blocks[i].empty();
  std::vector<char> has_near;
  const std::vector<int> zchunk = add_near_field(P, T, d->dense, D, tiles, has_back, &has_near);
  std::vector<ColSpec> cols;
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    if (!has_back[ti]) {
      if (!has_near[ti]) P.add_columns(P.add_chunk(uh::kToY, tiles[ti].p0, tiles[ti].h, uh::kGroupBackward), {});
      continue;
    }
    const int c = P.add_chunk(uh::kToY, tiles[ti].p0, tiles[ti].h, uh::kGroupBackward);
    cols.clear();
    for (int64_t b : tile_blocks[ti]) {
      const int32_t t = d->adm_row[b];
      const int64_t m = T.size[t];
      cols.push_back(ColSpec{uh::kSrcZ1, toff[b], d->adm_rank[b], &X, false, d->X_off[b] + tiles[ti].p0 - T.begin[t], m, 1});
    }
    P.add_columns(c, cols, zchunk[ti]);
  }

  if (g_pack_only_ncta) {
    if (const char* e = P.finalize()) return fail(UH_EINVAL, "packing: %s", e);
    if (const char* e = P.self_check()) return fail(UH_EINVAL, "internal packing error: %s", e);
    return UH_OK;
  }
  auto* o = new (std::nothrow) h_op();
  if (!o) return fail(UH_ENOMEM, "host allocation");
  o->c128 = c128;
  o->n = T.n;
  o->ncta = ncta;
  o->device = device;
  if ((rc = upload_program(o, P, T))) { free_op(o); delete o; return rc; }
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
  o->st.matmat_mode = -1;
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

int h_check(h_op* op, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  return check_status(op, stream);
}

int h_stats(const h_op* op, uh_stats_t* out) {
  if (!op || !out) return fail(UH_EINVAL, "null argument");
  *out = op->st;
  return UH_OK;
}

int uh_batch_create(const uh_desc* const* descs, int32_t count, int32_t precision, uh_batch** out) {
  return uh_batch_create_ex(descs, count, precision, nullptr, out);
}

int uh_batch_create_ex(const uh_desc* const* descs, int32_t count, int32_t precision, const uh_pack_params* params,
                       uh_batch** out) {
  g_err.clear();
  if (!descs || !out) return fail(UH_EINVAL, "null argument");
  *out = nullptr;
  if (count < 1) return fail(UH_EINVAL, "count = %d", count);
  int rc;
  if ((rc = check_precision(precision, false))) return rc;
  uh::PackParams pp;
  if ((rc = pack_params_from(params, precision == UH_PREC_C128, &pp))) return rc;
  std::vector<UHPrep> preps(count);
  int64_t total = 0;
  for (int32_t k = 0; k < count; ++k) {
    if (!descs[k]) return fail(UH_EINVAL, "operator %d: null descriptor", k);
    if ((rc = prepare_uh(descs[k], &preps[k]))) {
      const std::string msg = g_err;
      return fail(rc, "operator %d: %s", k, msg.c_str());
    }
    total += preps[k].T.n;
    if (total > INT32_MAX) return fail(UH_EINVAL, "the batch holds more than 2^31 - 1 points");
  }
  const bool c128 = precision == UH_PREC_C128;
  {
    int64_t bytes = 0;
    for (int32_t k = 0; k < count; ++k) {
      uh_stats_t est{};
      uh_fill_stats(preps[k], precision, c128 ? 16 : 8, &est);
      bytes += est.algo_bytes_matvec;
    }
    resolve_ctas(&pp, bytes);
  }
  const bool dual = pp.ctas_per_sm == 2;
  int ncta = g_pack_only_ncta, device = 0;
  if (!ncta && (rc = query_ncta(c128, &ncta, &device, dual))) return rc;
  ProgramBuilder P(c128, total, ncta, pp);
  const int64_t A = P.align();
  P.set_permutation(total);
  // The batch as one operator on the concatenated vectors: position offsets[k] + i of the
  // cluster order is point perm_k[i] of operator k, i.e. entry offsets[k] + perm_k[i].
  Tree all;
  all.n = total;
  all.perm.resize(static_cast<size_t>(total));
  std::vector<int64_t> offsets(count + 1, 0);
  Offsets off;
  for (int32_t k = 0; k < count; ++k) {
    offsets[k] = off.n;
    for (int64_t i = 0; i < preps[k].T.n; ++i)
      all.perm[off.n + i] = static_cast<int32_t>(off.n + preps[k].T.perm[i]);
    add_uh_program(P, preps[k], &off);
  }
  offsets[count] = off.n;
  P.set_source_len(uh::kSrcXp, ProgramBuilder::round_up(total, A));
  P.set_source_len(uh::kSrcZ1, off.x);
  P.set_source_len(uh::kSrcZ2, off.y);
  P.set_source_len(uh::kSrcZ3, off.z3);
  P.set_source_len(uh::kSrcZ4, off.t);
  if (g_pack_only_ncta) {
    if (const char* e = P.finalize()) return fail(UH_EINVAL, "packing: %s", e);
    if (const char* e = P.self_check()) return fail(UH_EINVAL, "internal packing error: %s", e);
    return UH_OK;
  }
  auto* o = new (std::nothrow) uh_batch();
  if (!o) return fail(UH_ENOMEM, "host allocation");
  o->c128 = c128;
  o->n = total;
  o->ncta = ncta;
  o->device = device;
  o->offsets = offsets;
  o->dual = dual;
  if ((rc = upload_program(o, P, all))) { free_op(o); delete o; return rc; }
  const uh_stats_t packed = o->st;
  uh_stats_t sum{};
  double rank_total = 0.0;
  int64_t rank_count = 0;
  sum.rank_min = INT32_MAX;
  for (int32_t k = 0; k < count; ++k) {
    uh_stats_t st{};
    uh_fill_stats(preps[k], precision, c128 ? 16 : 8, &st);
    sum.n_row_bases += st.n_row_bases;
    sum.n_col_bases += st.n_col_bases;
    sum.n_adm += st.n_adm;
    sum.n_dense += st.n_dense;
    sum.E_U += st.E_U;
    sum.E_V += st.E_V;
    sum.E_S += st.E_S;
    sum.E_D += st.E_D;
    sum.n_factored += st.n_factored;
    sum.sum_factored_rank += st.sum_factored_rank;
    sum.sum_row_rank += st.sum_row_rank;
    sum.sum_col_rank += st.sum_col_rank;
    if (st.rank_max > 0) sum.rank_min = std::min(sum.rank_min, st.rank_min);
    sum.rank_max = std::max(sum.rank_max, st.rank_max);
    const int64_t nb = st.n_row_bases + st.n_col_bases;
    rank_total += st.rank_mean * static_cast<double>(nb);
    rank_count += nb;
    sum.csp = std::max(sum.csp, st.csp);
    sum.algo_bytes_matvec += st.algo_bytes_matvec;
  }
  if (sum.rank_max == 0) sum.rank_min = 0;
  sum.rank_mean = rank_count ? rank_total / static_cast<double>(rank_count) : 0.0;
  sum.n = total;
  sum.precision = precision;
  sum.elem_bytes = c128 ? 16 : 8;
  sum.packed_bytes = packed.packed_bytes;
  sum.device_bytes = packed.device_bytes;
  sum.n_launches = packed.n_launches;
  sum.n_items = packed.n_items;
  sum.matmat_mode = -1;
  fill_pack_stats(pp, P.geometry(), &sum);
  o->st = sum;
  *out = o;
  return UH_OK;
}

int uh_batch_tune(const uh_desc* const* descs, int32_t count, int32_t precision, int32_t sample, int32_t reps,
                  uh_pack_params* best, double* best_ms, double* default_ms, void* stream) {
  g_err.clear();
  if (!descs || !best || count < 1 || reps < 1) return fail(UH_EINVAL, "uh_batch_tune: invalid argument");
  // an evenly spaced sample of the operators
  std::vector<const uh_desc*> sub;
  const int32_t ns = sample > 0 && sample < count ? sample : count;
  for (int32_t i = 0; i < ns; ++i) sub.push_back(descs[static_cast<int64_t>(i) * count / ns]);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *x = nullptr, *y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int rc = UH_OK;
  int64_t cap = 0;
  // Mean time of `reps` back-to-back products of the sample packed with p (ms), or < 0 on error.
  auto timed = [&](const uh_pack_params& p, double* ms) -> int {
    uh_batch* b = nullptr;
    int r = uh_batch_create_ex(sub.data(), ns, precision, &p, &b);
    if (r) return r;
    const int64_t need = b->n * (b->c128 ? 16 : 8);
    if (need > cap) {
      if (x) cudaFree(x);
      if (y) cudaFree(y);
      x = y = nullptr;
      if (cudaMalloc(&x, need) != cudaSuccess || cudaMalloc(&y, need) != cudaSuccess ||
          cudaMemsetAsync(x, 0, need, st) != cudaSuccess) {
        uh_batch_destroy(b);
        return fail(UH_ENOMEM, "uh_batch_tune: vectors of %lld bytes", (long long)need);
      }
      cap = need;
    }
    for (int i = 0; i < 3 && !r; ++i) r = uh_batch_matvec(b, x, y, stream);
    if (!r && cudaEventRecord(e0, st) != cudaSuccess) r = fail(UH_ECUDA, "event");
    for (int i = 0; i < reps && !r; ++i) r = uh_batch_matvec(b, x, y, stream);
    if (!r && cudaEventRecord(e1, st) != cudaSuccess) r = fail(UH_ECUDA, "event");
    float t = 0.0f;
    if (!r && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      r = fail(UH_ECUDA, "event timing");
    if (!r) r = uh_batch_check(b, stream);
    uh_batch_destroy(b);
    *ms = t / reps;
    return r;
  };
  uh_pack_params cur{};  // zeros: the defaults
  uh::PackParams d;
  cur.tile_bytes = static_cast<int32_t>(d.tile_bytes);
  cur.item_cost = static_cast<int32_t>(d.item_cost);
  cur.chunk_cost = static_cast<int32_t>(d.chunk_cost);
  cur.pool_unit = static_cast<int32_t>(d.pool_unit);
  cur.ctas_per_sm = static_cast<int32_t>(d.ctas_per_sm);
  double cur_ms = 0.0;
  rc = timed(cur, &cur_ms);
  if (default_ms) *default_ms = cur_ms;
  // coordinate descent over the knobs, one pass; a change is kept if at least 1% faster (the CTAs
  // per SM first: complex64 only; the tile sizes above the two-CTA geometry's cap pack alike)
  const int32_t ctas[] = {1, 2}, tiles[] = {16384, 32768, 65536}, items[] = {1024, 4096, 16384},
                chunks[] = {12288, 49152, 196608}, pools[] = {32768, 131072, 524288};
  int32_t* knob[] = {&cur.ctas_per_sm, &cur.tile_bytes, &cur.item_cost, &cur.chunk_cost, &cur.pool_unit};
  const int32_t* vals[] = {ctas, tiles, items, chunks, pools};
  const int nvals[] = {precision == UH_PREC_C128 ? 1 : 2, 3, 3, 3, 3};
  for (int k = 0; k < 5 && !rc; ++k) {
    const int32_t keep = *knob[k];
    int32_t pick = keep;
    for (int v = 0; v < nvals[k] && !rc; ++v) {
      if (vals[k][v] == keep) continue;
      *knob[k] = vals[k][v];
      double ms = 0.0;
      rc = timed(cur, &ms);
      if (!rc && ms < 0.99 * cur_ms) {
        cur_ms = ms;
        pick = vals[k][v];
      }
      *knob[k] = keep;
    }
    *knob[k] = pick;
  }
  if (x) cudaFree(x);
  if (y) cudaFree(y);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return UH_OK;
}

int uh_batch_destroy(uh_batch* batch) {
  if (!batch) return UH_OK;
  cudaDeviceSynchronize();
  free_op(batch);
  delete batch;
  return UH_OK;
}

int uh_batch_offsets(const uh_batch* batch, int64_t* offsets) {
  if (!batch || !offsets) return fail(UH_EINVAL, "null argument");
  std::copy(batch->offsets.begin(), batch->offsets.end(), offsets);
  return UH_OK;
}

int uh_batch_matvec(uh_batch* batch, const void* x, void* y, void* stream) {
  if (!batch) return fail(UH_EINVAL, "null batch");
  return run_matvec(batch, x, y, stream);
}

int uh_batch_check(uh_batch* batch, void* stream) {
  if (!batch) return fail(UH_EINVAL, "null batch");
  return check_status(batch, stream);
}

int uh_batch_stats(const uh_batch* batch, uh_stats_t* out) {
  if (!batch || !out) return fail(UH_EINVAL, "null argument");
  *out = batch->st;
  return UH_OK;
}

int uh_batch_pack_check(const uh_desc* const* descs, int32_t count, int32_t precision, int32_t ncta) {
  return uh_batch_pack_check_ex(descs, count, precision, nullptr, ncta);
}

int uh_batch_pack_check_ex(const uh_desc* const* descs, int32_t count, int32_t precision,
                           const uh_pack_params* params, int32_t ncta) {
  if (ncta < 1) return fail(UH_EINVAL, "ncta = %d", ncta);
  g_pack_only_ncta = ncta;
  uh_batch* o = nullptr;
  const int rc = uh_batch_create_ex(descs, count, precision, params, &o);
  g_pack_only_ncta = 0;
  return rc;
}

int uh_pack_check(const uh_desc* desc, int32_t precision, int32_t ncta) {
  if (ncta < 1) return fail(UH_EINVAL, "ncta = %d", ncta);
  g_pack_only_ncta = ncta;
  uh_op* o = nullptr;
  const int rc = uh_create(desc, precision, &o);
  g_pack_only_ncta = 0;
  return rc;
}

int h_pack_check(const h_desc* desc, int32_t precision, int32_t ncta) {
  if (ncta < 1) return fail(UH_EINVAL, "ncta = %d", ncta);
  g_pack_only_ncta = ncta;
  h_op* o = nullptr;
  const int rc = h_create(desc, precision, &o);
  g_pack_only_ncta = 0;
  return rc;
}

int uh_debug_stalled_matvec(uh_op* op, const void* x, void* y, long long timeout_cycles, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  if (timeout_cycles < 1000 || timeout_cycles > kTimeoutCycles)
    return fail(UH_EINVAL, "timeout_cycles %lld outside [1000, %lld]", timeout_cycles, kTimeoutCycles);
  return run_matvec(op, x, y, stream, timeout_cycles, true);
}

int uh_matmat(uh_op* op, int32_t nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t mode,
              void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  int rc;
  if ((rc = check_matmat_args(op, nrhs, X, ldx, Y, ldy))) return rc;
  if (mode == UH_MM_SIMT) return matmat_by_columns(op, nrhs, X, ldx, Y, ldy, stream);
  if (mode != UH_MM_TF32 && mode != UH_MM_BF16X3) return fail(UH_EINVAL, "matmat mode %d", mode);
  if (op->mm_mode != mode)
    return fail(UH_EINVAL, "matmat mode %d needs an op created with precision %s", mode,
                mode == UH_MM_TF32 ? "UH_PREC_C64_TF32" : "UH_PREC_C64_BF16X3");
  std::lock_guard<std::mutex> lock(op->mu);
  if ((rc = order_call(op, static_cast<cudaStream_t>(stream)))) return rc;
  for (int32_t rhs0 = 0; rhs0 < nrhs; rhs0 += uh::kPanelR) {
    const int32_t nb = std::min<int32_t>(uh::kPanelR, nrhs - rhs0);
    // at most 32 right-hand sides: MMAs of M = 64 on the compact panel layout
    const int32_t m64 = nb <= uh::kPanelR / 2 ? 1 : 0;
    // on a failed launch, still mark the call's end so that the next call is ordered after the
    // panels already queued (they share the op's panel scratch)
    if ((rc = uh::panel_gather(X, ldx, op->n, op->panel_xp_rows, op->d_perm, rhs0, nb, op->panel_mode, m64,
                               op->d_pxp, stream))) {
      call_done(op, static_cast<cudaStream_t>(stream));
      return rc;
    }
    {
      uh::PanelParams p{};
      ++op->panel_epoch;
      for (int k = 0; k < 2; ++k)
        p.need[k] = op->panel_epoch * static_cast<unsigned long long>(op->panel_zchunks[k]);
      p.done = op->d_pdone;
      p.items = op->d_pitems;
      p.cta_begin = op->d_pbegin;
      p.tiles = op->d_ptiles;
      p.src[0] = op->d_pxp;
      p.src[1] = op->d_pz1;
      p.src[2] = op->d_pz2;
      p.zout[0] = op->d_pz1;
      p.zout[1] = op->d_pz2;
      p.y = Y;
      p.ldy = ldy;
      p.perm = op->d_perm;
      p.rhs0 = rhs0;
      p.nb = nb;
      p.m64 = m64;
      p.mode = op->panel_mode;
      p.status = op->d_status;
      p.timeout_cycles = kTimeoutCycles;
      if ((rc = uh::panel_launch(p, op->panel_ncta, stream))) {
        --op->panel_epoch;  // nothing launched: the counters did not move
        call_done(op, static_cast<cudaStream_t>(stream));
        return rc;
      }
    }
  }
  return call_done(op, static_cast<cudaStream_t>(stream));
}
int uh_reserve(uh_op* op, int32_t max_nrhs) { return reserve_multi(op, max_nrhs); }
int h_matmat(h_op* op, int32_t nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t mode, void* stream) {
  if (!op) return fail(UH_EINVAL, "null op");
  int rc;
  if ((rc = check_matmat_args(op, nrhs, X, ldx, Y, ldy))) return rc;
  if (mode != UH_MM_SIMT) return fail(UH_EINVAL, "h_matmat: only UH_MM_SIMT (mode %d)", mode);
  return matmat_by_columns(op, nrhs, X, ldx, Y, ldy, stream);
}
int h_reserve(h_op* op, int32_t max_nrhs) { return reserve_multi(op, max_nrhs); }

}  // extern "C"

extern "C" int uh_pack_check_ex(const uh_desc* desc, int32_t precision, const uh_pack_params* params, int32_t ncta) {
  if (ncta < 1) return fail(UH_EINVAL, "ncta = %d", ncta);
  g_pack_only_ncta = ncta;
  uh_op* o = nullptr;
  const int rc = uh_create_ex(desc, precision, params, &o);
  g_pack_only_ncta = 0;
  return rc;
}

namespace uh {

int multi_rhs_width(const uh_op* op) { return op && !op->c128 ? op->multi_r : 0; }

int matvec_group(uh_op* op, int nr, const void* const* xs, void* const* ys, void* stream) {
  if (!op || !xs || !ys) return fail(UH_EINVAL, "null argument");
  if (op->c128 || (nr != 2 && nr != 4) || nr > op->multi_r)
    return fail(UH_EINVAL, "%d products in one pass need a complex64 op with uh_reserve(op, %d)", nr, nr);
  const int64_t bytes = op->n * 8;
  for (int a = 0; a < nr; ++a) {
    if (!xs[a] || !ys[a]) return fail(UH_EINVAL, "null vector");
    const char* ya = static_cast<const char*>(ys[a]);
    // no output overlaps an input or another output
    for (int b = 0; b < nr; ++b) {
      const char* xb = static_cast<const char*>(xs[b]);
      const char* yb = static_cast<const char*>(ys[b]);
      if (ya < xb + bytes && xb < ya + bytes) return fail(UH_EINVAL, "grouped vectors overlap");
      if (b != a && ya < yb + bytes && yb < ya + bytes) return fail(UH_EINVAL, "grouped outputs overlap");
    }
  }
  return run_matvec(op, xs[0], ys[0], stream, kTimeoutCycles, false, false, nr, xs, ys);
}

}  // namespace uh

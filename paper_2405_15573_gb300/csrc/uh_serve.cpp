// Serving runtime: GMRES(m) solves A x = b with resident UH operators, admitted by device-memory
// footprint and advanced together in rounds (continuous batching).
//
// One worker thread owns one CUDA stream and one completion event per running solve. It admits
// queued solves while the admitted footprint stays within the budget and fewer than max_active
// are running, and keeps every running solve's next step queued on the GPU: a solve's step (its
// product and vector kernels, asynchronous on its own stream, then a small device-to-host copy
// and its completion event) is issued as soon as the worker sees that solve's previous step
// complete (event query) and has updated the solve's small host-side state (Givens rotations of
// the Hessenberg matrix, convergence), independently of the other solves. So the GPU always has
// the other solves' steps queued while the host handles one, and a slow step holds back only its
// own solve. The products of one operator are chained across streams by an event in launch
// order: they share the operator's scratch and its per-call group counters. A solve
// is restarted GMRES with its matrix-vector products in the operator's precision (complex64
// storage, FP32 accumulation for UH_PREC_C64 ops) and everything else in FP64 on the GPU: the
// true residual r = b - A x at every restart (its product in extended precision on the
// complex128 x for complex64 ops, uh_matvec_mixed), classical Gram-Schmidt applied twice for the
// Arnoldi basis, the norms and the solution update x += V y. The restarts with the recomputed
// residual are the mixed-precision refinement: a solve only stops as converged when the true
// residual of the returned x against the stored operator is below the tolerance. The kernel sequence of a solve depends only on its own
// data, so its result is the same whether it runs alone or among other solves.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "uh.h"
#include "uh_internal.h"
#include "uh_solve.h"

using cd = std::complex<double>;

namespace {

#define fail uh::set_error

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum Phase { kStart, kArnoldi, kUpdate, kFinish, kDone };

// Device and pinned host buffers of one solve; kept after the solve for reuse by the next solve of
// the same shape.
struct Workspace {
  int64_t n = 0;
  int m = 0;
  void *V = nullptr, *x = nullptr, *db = nullptr, *w = nullptr, *v32 = nullptr, *y32 = nullptr;
  void *y = nullptr, *part = nullptr, *small = nullptr;  // small: h1 [m+2], h2 [m+2], scal [2 doubles]
  cd *hy = nullptr, *hx = nullptr, *hsmall = nullptr;
};

struct Solve {
  uint64_t ticket = 0;
  uh_op* op = nullptr;
  int64_t n = 0;
  bool c64 = true;
  double tol = 1e-6;
  int m = 30, maxit = 300;
  std::vector<cd> b;
  double bnorm = 0.0;
  int64_t footprint = 0;
  // workspace (device, pinned host) and views into it
  Workspace ws;
  bool has_ws = false;
  void *V = nullptr, *x = nullptr, *db = nullptr, *w = nullptr, *v32 = nullptr, *y32 = nullptr;
  void *h1 = nullptr, *h2 = nullptr, *y = nullptr, *part = nullptr;
  double* scal = nullptr;
  cd *hh1 = nullptr, *hh2 = nullptr, *hy = nullptr, *hx = nullptr;
  double* hscal = nullptr;
  bool v32_ready = false;  // v32 holds complex64(V_j) for the next Arnoldi step
  int slot = -1;           // index of the solve's stream and event
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;  // recorded after each issued step
  bool inflight = false;     // a step is issued and its event not yet seen complete
  bool held = false;         // ready for an Arnoldi step, waiting for a partner of the same op
  int paired_steps = 0;      // Arnoldi steps whose product shared a pass with another solve's
  // GMRES state
  Phase phase = kStart;
  bool x_zero = true;
  int j = 0, iters = 0, restarts = 0;
  std::vector<cd> H, g, sn;
  std::vector<double> cs;
  double resid = 0.0;
  int status = UH_OK;
  bool converged = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
  std::vector<cd> result;
};

int64_t footprint_of(int64_t n, int m) {
  const int64_t nb = uh::solve_partials(n);
  return (m + 1 + 3) * n * 16 + 2 * n * 8 + 3 * (m + 2) * 16 + (m + 1) * nb * 16 + 64;
}

}  // namespace

struct uh_server {
  int device = 0;
  int max_active = 8;
  int64_t budget = 0, used = 0;
  int queue_cap = 64;
  std::vector<cudaStream_t> streams;          // one per running solve (slots)
  std::vector<cudaEvent_t> events;            // completion of the slot's last issued step
  std::vector<char> slot_used;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Solve*> pending;
  std::vector<Solve*> active;
  std::map<uint64_t, std::unique_ptr<Solve>> all;  // every solve not yet collected by poll
  std::vector<Workspace> spare;                    // workspaces of finished solves
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
};

namespace {

void free_workspace(Workspace& w) {
  void* dev[] = {w.V, w.x, w.db, w.w, w.v32, w.y32, w.y, w.part, w.small};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {w.hy, w.hx, w.hsmall};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  w = Workspace{};
}

int alloc_workspace(Workspace& w, int64_t n, int m) {
  const int64_t nb = uh::solve_partials(n);
  const size_t small = static_cast<size_t>(2 * (m + 2) + 1) * 16;
  w.n = n;
  w.m = m;
  auto dev = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
  auto host = [&](void** p, size_t bytes) { return cudaMallocHost(p, bytes) == cudaSuccess; };
  const bool ok = dev(&w.V, static_cast<size_t>((m + 1) * n) * 16) && dev(&w.x, n * 16) && dev(&w.db, n * 16) &&
                  dev(&w.w, n * 16) && dev(&w.v32, n * 8) && dev(&w.y32, n * 8) && dev(&w.y, (m + 2) * 16) &&
                  dev(&w.part, static_cast<size_t>((m + 1) * nb) * 16) && dev(&w.small, small) &&
                  host(reinterpret_cast<void**>(&w.hy), (m + 2) * 16) &&
                  host(reinterpret_cast<void**>(&w.hx), n * 16) &&
                  host(reinterpret_cast<void**>(&w.hsmall), small);
  if (!ok) {
    cudaGetLastError();
    free_workspace(w);
    return UH_ENOMEM;
  }
  return UH_OK;
}

void bind_workspace(Solve* s) {
  Workspace& w = s->ws;
  const int m = s->m;
  s->V = w.V; s->x = w.x; s->db = w.db; s->w = w.w; s->v32 = w.v32; s->y32 = w.y32; s->y = w.y; s->part = w.part;
  s->h1 = w.small;
  s->h2 = static_cast<char*>(w.small) + (m + 2) * 16;
  s->scal = reinterpret_cast<double*>(static_cast<char*>(w.small) + 2 * (m + 2) * 16);
  s->hy = w.hy; s->hx = w.hx;
  s->hh1 = w.hsmall;
  s->hh2 = w.hsmall + (m + 2);
  s->hscal = reinterpret_cast<double*>(w.hsmall + 2 * (m + 2));
}

// A workspace for solve s: a spare one of its shape, else a new one (spares are freed first if
// the allocation fails).
int take_workspace(uh_server* sv, Solve* s) {
  for (size_t i = 0; i < sv->spare.size(); ++i)
    if (sv->spare[i].n == s->n && sv->spare[i].m == s->m) {
      s->ws = sv->spare[i];
      sv->spare.erase(sv->spare.begin() + static_cast<std::ptrdiff_t>(i));
      s->has_ws = true;
      bind_workspace(s);
      return UH_OK;
    }
  int rc = alloc_workspace(s->ws, s->n, s->m);
  if (rc) {
    for (Workspace& w : sv->spare) free_workspace(w);
    sv->spare.clear();
    rc = alloc_workspace(s->ws, s->n, s->m);
    if (rc) return rc;
  }
  s->has_ws = true;
  bind_workspace(s);
  return UH_OK;
}

// Workspace back to the spares (at most max_active of them are kept).
void release_workspace(uh_server* sv, Solve* s) {
  if (!s->has_ws) return;
  if (static_cast<int>(sv->spare.size()) < sv->max_active) sv->spare.push_back(s->ws);
  else free_workspace(s->ws);
  s->ws = Workspace{};
  s->has_ws = false;
}

int start_solve(uh_server* sv, Solve* s, cudaStream_t st) {
  const int rc = take_workspace(sv, s);
  if (rc) return rc;
  const int m = s->m;
  if (cudaMemcpyAsync(s->db, s->b.data(), s->n * 16, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(s->x, 0, s->n * 16, st) != cudaSuccess)
    return UH_ECUDA;
  s->H.assign(static_cast<size_t>((m + 1) * m), cd(0, 0));
  s->g.assign(m + 1, cd(0, 0));
  s->cs.assign(m, 0.0);
  s->sn.assign(m, cd(0, 0));
  return UH_OK;
}

// out = A v (complex128 out; for complex64 ops through v32 / y32). With out null, a complex64 op
// leaves its product in y32 for the caller to widen; v32_ready: v32 already holds complex64(v).
// Products of one op issued from different solves' streams run in call order: uh_matvec orders
// the calls on an op.
int apply_op(Solve* s, const void* v, void* out, cudaStream_t st, bool v32_ready = false) {
  int rc;
  if (s->c64) {
    if (!v32_ready && (rc = uh::vec_d2f(v, s->v32, s->n, st))) return rc;
    if ((rc = uh_matvec(s->op, s->v32, s->y32, st))) return rc;
    return out ? uh::vec_f2d(s->y32, out, s->n, st) : UH_OK;
  }
  return uh_matvec(s->op, v, out, st);
}

// Kernels of the start of a cycle: V_0 = (b - A x) / ||b - A x|| (and its complex64 copy for the
// next product), the norm copied to the host.
int issue_start(Solve* s, cudaStream_t st) {
  int rc;
  if (s->x_zero) {
    if (cudaMemcpyAsync(s->V, s->db, s->n * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess) return UH_ECUDA;
  } else {
    // The true residual of the current x against the stored operator: for complex64 ops the
    // product runs in extended precision on the complex128 x (uh_matvec_mixed), so the restart
    // sees b - A x to about 1e-13, not the FP32-accumulated product of the Arnoldi steps.
    if (s->c64) {
      if ((rc = uh_matvec_mixed(s->op, s->x, s->w, st))) return rc;
    } else if ((rc = apply_op(s, s->x, s->w, st))) {
      return rc;
    }
    if ((rc = uh::vec_residual(s->db, s->w, false, s->V, s->n, st))) return rc;
  }
  if ((rc = uh::vec_norm(s->V, s->n, s->part, s->scal, nullptr, st))) return rc;
  if ((rc = uh::vec_scale_f(s->V, s->scal, s->V, s->c64 ? s->v32 : nullptr, s->n, st))) return rc;
  s->v32_ready = s->c64;
  return cudaMemcpyAsync(s->hscal, s->scal, 16, cudaMemcpyDeviceToHost, st) == cudaSuccess ? UH_OK : UH_ECUDA;
}

// One Arnoldi step j: w = A V_j, two passes of classical Gram-Schmidt against V_0..V_j,
// V_{j+1} = w / ||w|| (and its complex64 copy); both coefficient passes and the norm copied to
// the host in one copy. With product = false the product A V_j is already in y32 (a paired
// product).
int issue_arnoldi(Solve* s, cudaStream_t st, bool product = true) {
  int rc;
  const int64_t n = s->n;
  const int cnt = s->j + 1;
  const char* Vj = static_cast<const char*>(s->V) + static_cast<size_t>(s->j) * n * 16;
  if (s->c64) {
    if (product && (rc = apply_op(s, Vj, nullptr, st, s->v32_ready))) return rc;
    if ((rc = uh::vec_dots_f(s->V, n, cnt, s->y32, s->w, s->part, s->h1, st))) return rc;
  } else {
    if ((rc = apply_op(s, Vj, s->w, st))) return rc;
    if ((rc = uh::vec_dots(s->V, n, cnt, s->w, s->part, s->h1, false, st))) return rc;
  }
  if ((rc = uh::vec_combine(s->V, n, cnt, s->h1, -1.0, s->w, st))) return rc;
  if ((rc = uh::vec_dots(s->V, n, cnt, s->w, s->part, s->h2, false, st))) return rc;
  if ((rc = uh::vec_combine(s->V, n, cnt, s->h2, -1.0, s->w, st))) return rc;
  if ((rc = uh::vec_norm(s->w, n, s->part, s->scal, nullptr, st))) return rc;
  char* Vn = static_cast<char*>(s->V) + static_cast<size_t>(cnt) * n * 16;
  if ((rc = uh::vec_scale_f(s->w, s->scal, Vn, s->c64 ? s->v32 : nullptr, n, st))) return rc;
  s->v32_ready = s->c64;
  const size_t small = static_cast<size_t>(2 * (s->m + 2) + 1) * 16;
  return cudaMemcpyAsync(s->hh1, s->h1, small, cudaMemcpyDeviceToHost, st) == cudaSuccess ? UH_OK : UH_ECUDA;
}

// x += V_0..V_{cnt-1} y (y from the host), then the next cycle's start.
int issue_update(Solve* s, int cnt, cudaStream_t st) {
  int rc;
  if (cudaMemcpyAsync(s->y, s->hy, cnt * 16, cudaMemcpyHostToDevice, st) != cudaSuccess) return UH_ECUDA;
  if ((rc = uh::vec_combine(s->V, s->n, cnt, s->y, 1.0, s->x, st))) return rc;
  s->x_zero = false;
  return issue_start(s, st);
}

int issue_finish(Solve* s, cudaStream_t st) {
  return cudaMemcpyAsync(s->hx, s->x, s->n * 16, cudaMemcpyDeviceToHost, st) == cudaSuccess ? UH_OK : UH_ECUDA;
}

int issue(Solve* s, cudaStream_t st) {
  switch (s->phase) {
    case kStart: return issue_start(s, st);
    case kArnoldi: return issue_arnoldi(s, st);
    case kUpdate: return issue_update(s, s->j + 1, st);
    case kFinish: return issue_finish(s, st);
    default: return UH_OK;
  }
}

// After the start of a cycle (or an update followed by a start): the true residual decides.
void after_start(Solve* s) {
  s->resid = s->hscal[0];
  const double rel = s->bnorm > 0 ? s->resid / s->bnorm : 0.0;
  if (rel <= s->tol || s->iters >= s->maxit || s->resid == 0.0) {
    s->converged = rel <= s->tol;
    s->phase = kFinish;
    return;
  }
  std::fill(s->g.begin(), s->g.end(), cd(0, 0));
  s->g[0] = cd(s->resid, 0);
  s->j = 0;
  s->phase = kArnoldi;
}

// After Arnoldi step j: rotate the new Hessenberg column, update the residual estimate.
void after_arnoldi(Solve* s) {
  const int j = s->j, m = s->m;
  cd* col = &s->H[static_cast<size_t>(j) * (m + 1)];
  for (int i = 0; i <= j; ++i) col[i] = s->hh1[i] + s->hh2[i];
  const double hnext = s->hscal[0];
  col[j + 1] = cd(hnext, 0);
  for (int i = 0; i < j; ++i) {
    const cd a = col[i], b = col[i + 1];
    col[i] = s->cs[i] * a + s->sn[i] * b;
    col[i + 1] = -std::conj(s->sn[i]) * a + s->cs[i] * b;
  }
  const cd a = col[j], b = col[j + 1];
  const double rho = std::sqrt(std::norm(a) + std::norm(b));
  if (std::abs(a) == 0.0) {
    s->cs[j] = 0.0;
    s->sn[j] = cd(1, 0);
    col[j] = b;
  } else {
    const cd ph = a / std::abs(a);
    s->cs[j] = std::abs(a) / rho;
    s->sn[j] = ph * std::conj(b) / rho;
    col[j] = ph * rho;
  }
  col[j + 1] = cd(0, 0);
  s->g[j + 1] = -std::conj(s->sn[j]) * s->g[j];
  s->g[j] = s->cs[j] * s->g[j];
  s->iters++;
  const double est = std::abs(s->g[j + 1]) / (s->bnorm > 0 ? s->bnorm : 1.0);
  if (est <= s->tol || j + 1 == m || s->iters >= s->maxit || hnext == 0.0) {
    // y = R^{-1} g, R the rotated (j+1) x (j+1) upper triangle.
    for (int i = j; i >= 0; --i) {
      cd v = s->g[i];
      for (int k = i + 1; k <= j; ++k) v -= s->H[static_cast<size_t>(k) * (m + 1) + i] * s->hy[k];
      const cd d = s->H[static_cast<size_t>(i) * (m + 1) + i];
      s->hy[i] = d != cd(0, 0) ? v / d : cd(0, 0);
    }
    s->restarts++;
    s->phase = kUpdate;
  } else {
    s->j = j + 1;
  }
}

void after(Solve* s) {
  switch (s->phase) {
    case kStart:
    case kUpdate: after_start(s); break;
    case kArnoldi: after_arnoldi(s); break;
    case kFinish:
      s->result.assign(s->hx, s->hx + s->n);
      s->phase = kDone;
      break;
    default: break;
  }
}

// Issues solve s's next step and records its completion event; a failure ends the solve.
void issue_step(uh_server* sv, Solve* s) {
  int rc = UH_OK;
  if (!s->has_ws) rc = start_solve(sv, s, s->st);
  if (!rc) rc = issue(s, s->st);
  if (!rc && cudaEventRecord(s->ev, s->st) != cudaSuccess) rc = UH_ECUDA;
  if (rc) {
    s->status = rc;
    s->phase = kDone;
    s->inflight = false;
    return;
  }
  s->inflight = true;
}

// Whether solve s's next step is an Arnoldi step whose product can share a pass with another's:
// complex64 op with two-wide scratch, x in complex64 already (v32).
bool pairable(const Solve* s) {
  return s->phase == kArnoldi && s->c64 && s->v32_ready && uh::multi_rhs_width(s->op) >= 2;
}

void issue_group(uh_server* sv, const std::vector<Solve*>& g);

// The Arnoldi steps of the solves in g (2 or 4, one op) with one product of that many right-hand
// sides, on the first solve's stream; the others' streams wait for it, then each runs its
// Gram-Schmidt on its own stream. Each result is bitwise that of its own product, so a solve's
// arithmetic does not depend on its partners.
void issue_group(uh_server* sv, const std::vector<Solve*>& g) {
  const int nr = static_cast<int>(g.size());
  Solve* a = g[0];
  const void* xs[4];
  void* ys[4];
  for (int r = 0; r < nr; ++r) {
    xs[r] = g[r]->v32;
    ys[r] = g[r]->y32;
  }
  int rc = uh::matvec_group(a->op, nr, xs, ys, a->st);
  if (!rc && cudaEventRecord(a->ev, a->st) != cudaSuccess) rc = UH_ECUDA;
  for (int r = 1; r < nr && !rc; ++r)
    if (cudaStreamWaitEvent(g[r]->st, a->ev, 0) != cudaSuccess) rc = UH_ECUDA;
  if (rc) {  // not issued together: each on its own
    for (Solve* s : g) issue_step(sv, s);
    return;
  }
  for (Solve* s : g) {
    int r = issue_arnoldi(s, s->st, false);
    if (!r && cudaEventRecord(s->ev, s->st) != cudaSuccess) r = UH_ECUDA;
    if (r) {
      s->status = r;
      s->phase = kDone;
      s->inflight = false;
    } else {
      s->inflight = true;
      s->paired_steps++;
    }
  }
}

// Ends the solves still running when the server stops (after their streams drain).
void abort_active(uh_server* sv) {
  for (Solve* s : sv->active) {
    if (s->st) cudaStreamSynchronize(s->st);
    release_workspace(sv, s);
    if (s->phase != kDone) s->status = UH_ECUDA;
    s->phase = kDone;
    s->inflight = false;
  }
  sv->active.clear();
  for (Workspace& w : sv->spare) free_workspace(w);
  sv->spare.clear();
}

void worker_main(uh_server* sv) {
  cudaSetDevice(sv->device);
  std::vector<Solve*> running, fresh;
  int idle = 0;
  for (;;) {
    fresh.clear();
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      while (!sv->pending.empty() && static_cast<int>(sv->active.size()) < sv->max_active &&
             sv->used + sv->pending.front()->footprint <= sv->budget) {
        Solve* s = sv->pending.front();
        sv->pending.pop_front();
        sv->used += s->footprint;
        s->t_admit = now_s();
        for (int k = 0; k < static_cast<int>(sv->slot_used.size()); ++k)
          if (!sv->slot_used[k]) {
            sv->slot_used[k] = 1;
            s->slot = k;
            s->st = sv->streams[k];
            s->ev = sv->events[k];
            break;
          }
        sv->active.push_back(s);
        fresh.push_back(s);
      }
      if (sv->stop) {
        abort_active(sv);
        return;
      }
      if (sv->active.empty()) {
        sv->cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      running = sv->active;
    }
    bool progress = !fresh.empty();
    // newly admitted solves: workspace, then their first step
    for (Solve* s : fresh) issue_step(sv, s);
    // every solve whose step has completed: host-side update; its next step is issued at once,
    // or held while another solve of the same op has a step in flight and both can share their
    // next product (one pass of two right-hand sides)
    for (Solve* s : running) {
      if (s->phase == kDone || !s->inflight) continue;
      const cudaError_t q = cudaEventQuery(s->ev);
      if (q == cudaErrorNotReady) continue;
      progress = true;
      s->inflight = false;
      if (q != cudaSuccess) {
        s->status = UH_ECUDA;
        s->phase = kDone;
        continue;
      }
      after(s);
      if (s->phase == kDone) {
        // did a bounded wait of one of the op's products run out meanwhile (a GPU that could not
        // run a product's CTAs together)?
        if (s->status == UH_OK && uh_check(s->op, s->st) != UH_OK) s->status = UH_ETIMEOUT;
        continue;
      }
      if (pairable(s)) {
        s->held = true;
        continue;
      }
      issue_step(sv, s);
    }
    // held solves, per op: as soon as as many are held as one pass takes (2 or 4), or when no
    // other solve of the op has a step in flight (that step ends, so every hold ends), they go in
    // groups of 4, 2, then alone
    for (size_t i = 0; i < running.size(); ++i) {
      Solve* a = running[i];
      if (!a->held) continue;
      std::vector<Solve*> held = {a};
      bool busy = false;
      for (size_t k = 0; k < running.size(); ++k) {
        Solve* c = running[k];
        if (c == a || c->op != a->op || c->phase == kDone) continue;
        if (c->held) held.push_back(c);
        if (c->inflight) busy = true;
      }
      const int width = uh::multi_rhs_width(a->op);
      if (busy && static_cast<int>(held.size()) < width) continue;
      size_t at = 0;
      while (at < held.size()) {
        const size_t left = held.size() - at;
        const size_t nr = width >= 4 && left >= 4 ? 4 : left >= 2 ? 2 : 1;
        std::vector<Solve*> g(held.begin() + static_cast<std::ptrdiff_t>(at),
                              held.begin() + static_cast<std::ptrdiff_t>(at + nr));
        for (Solve* c : g) c->held = false;
        if (nr == 1) issue_step(sv, g[0]);
        else issue_group(sv, g);
        at += nr;
      }
      progress = true;
    }
    bool finished = false;
    for (Solve* s : running) finished = finished || s->phase == kDone;
    if (finished) {
      std::lock_guard<std::mutex> lk(sv->mu);
      std::vector<Solve*> still;
      for (Solve* s : sv->active) {
        if (s->phase == kDone) {
          s->t_done = now_s();
          release_workspace(sv, s);
          sv->used -= s->footprint;
          if (s->slot >= 0) sv->slot_used[s->slot] = 0;
        } else {
          still.push_back(s);
        }
      }
      sv->active.swap(still);
    }
    // Nothing completed: let the GPU work (yield; after a long idle stretch, a short sleep).
    if (progress) {
      idle = 0;
    } else if (++idle < 2000) {
      std::this_thread::yield();
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
}

}  // namespace

extern "C" {

int uh_server_create(int32_t max_active, int64_t hbm_budget_bytes, int32_t queue_capacity, uh_server** out) {
  if (!out) return fail(UH_EINVAL, "null argument");
  *out = nullptr;
  if (max_active < 1 || hbm_budget_bytes < 1 || queue_capacity < 1)
    return fail(UH_EINVAL, "max_active %d, budget %lld, queue capacity %d must be >= 1", max_active,
                (long long)hbm_budget_bytes, queue_capacity);
  auto* sv = new (std::nothrow) uh_server();
  if (!sv) return fail(UH_ENOMEM, "host allocation");
  sv->max_active = max_active;
  sv->budget = hbm_budget_bytes;
  sv->queue_cap = queue_capacity;
  bool ok = cudaGetDevice(&sv->device) == cudaSuccess;
  sv->streams.assign(max_active, nullptr);
  sv->events.assign(max_active, nullptr);
  sv->slot_used.assign(max_active, 0);
  for (int k = 0; ok && k < max_active; ++k)
    ok = cudaStreamCreateWithFlags(&sv->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&sv->events[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    for (cudaStream_t st : sv->streams)
      if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : sv->events)
      if (ev) cudaEventDestroy(ev);
    delete sv;
    return fail(UH_ECUDA, "stream or event creation failed");
  }
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return UH_OK;
}

int uh_server_destroy(uh_server* sv) {
  if (!sv) return UH_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->pending.clear();
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : sv->events) cudaEventDestroy(ev);
  delete sv;
  return UH_OK;
}

int uh_solve_submit(uh_server* sv, uh_op* op, const void* b, double tol, int32_t restart, int32_t maxit,
                    uint64_t* ticket) {
  if (!sv || !op || !b || !ticket) return fail(UH_EINVAL, "null argument");
  if (!(tol > 0.0) || restart < 1 || restart > 60 || maxit < 1)
    return fail(UH_EINVAL, "tol %g, restart %d (1..60), maxit %d", tol, restart, maxit);
  uh_stats_t st{};
  int rc;
  if ((rc = uh_stats(op, &st))) return rc;
  auto s = std::make_unique<Solve>();
  s->op = op;
  s->n = st.n;
  s->c64 = st.precision != UH_PREC_C128;
  s->tol = tol;
  s->m = restart;
  s->maxit = maxit;
  s->b.assign(static_cast<const cd*>(b), static_cast<const cd*>(b) + st.n);
  double nb = 0.0;
  for (const cd& v : s->b) nb += std::norm(v);
  s->bnorm = std::sqrt(nb);
  s->footprint = footprint_of(st.n, restart);
  s->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  if (s->footprint > sv->budget)
    return fail(UH_EINVAL, "a solve of n = %lld needs %lld bytes, above the budget %lld", (long long)st.n,
                (long long)s->footprint, (long long)sv->budget);
  const bool fits_now = static_cast<int>(sv->active.size()) < sv->max_active && sv->pending.empty() &&
                        sv->used + s->footprint <= sv->budget;
  if (!fits_now && static_cast<int>(sv->pending.size()) >= sv->queue_cap)
    return fail(UH_EBUSY, "admission limit reached and %d solves queued", sv->queue_cap);
  s->ticket = sv->next_ticket++;
  *ticket = s->ticket;
  sv->pending.push_back(s.get());
  sv->all[s->ticket] = std::move(s);
  sv->cv.notify_all();
  return UH_OK;
}

int uh_solve_poll(uh_server* sv, uint64_t ticket, void* x, uh_solve_info* info) {
  if (!sv) return fail(UH_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return fail(UH_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  Solve* s = it->second.get();
  const bool queued = std::find(sv->pending.begin(), sv->pending.end(), s) != sv->pending.end();
  const bool running = std::find(sv->active.begin(), sv->active.end(), s) != sv->active.end();
  if (queued || running || s->phase != kDone) return UH_ENOTREADY;
  if (info) {
    info->status = s->status;
    info->converged = s->converged ? 1 : 0;
    info->iterations = s->iters;
    info->restarts = s->restarts;
    info->rel_residual = s->bnorm > 0 ? s->resid / s->bnorm : 0.0;
    info->queue_s = s->t_admit - s->t_submit;
    info->latency_s = s->t_done - s->t_submit;
    info->paired_steps = s->paired_steps;
  }
  if (x && s->status == UH_OK) std::memcpy(x, s->result.data(), s->result.size() * sizeof(cd));
  const int status = s->status;
  sv->all.erase(it);
  return status == UH_OK ? UH_OK : fail(status, "solve %llu failed", (unsigned long long)ticket);
}

}  // extern "C"

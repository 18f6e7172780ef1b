/*
 * uh.h - C ABI of the GB300 uniform H-matrix (UH) and H-matrix matrix-vector library.
 *
 * The operator is the uniform hierarchical matrix of Def. 2.4 of Bruyninckx, Huybrechs and
 * Meerbergen, "Uniform H-matrix compression with applications to boundary integral equations":
 *
 *     A|_b = U_tau S_b V_sigma^*   for every admissible leaf b = tau x sigma in P^+,
 *     A|_b  stored dense           for every inadmissible leaf b in P^-,
 *
 * with one row basis U_tau per row cluster and one column basis V_sigma per column cluster
 * (Section 2.2, eq. (2.1)). uh_matvec computes w = A v in the four steps of Algorithm 6
 * (Section 4.4): forward transform xhat_sigma = V_sigma^* x|_sigma, coupling
 * yhat_tau = sum_{sigma in row(tau)} S_b xhat_sigma, backward transform y|_tau += U_tau yhat_tau,
 * and the dense near field y|_tau += A|_b x|_sigma. h_* is the ordinary H-matrix of Def. 2.3,
 * A|_b = X_b Y_b^* per admissible block, applied as in Algorithm 5, kept beside it as the plain
 * form to compare with.
 *
 * Conventions (all entry points):
 *  - Every call returns an int status: UH_OK (0) or one of the UH_E* codes below. No C++
 *    exception crosses this boundary. uh_last_error() gives a message for the calling thread's
 *    most recent failure.
 *  - Complex numbers are stored interleaved (re, im), as C99 complex / std::complex.
 *  - Matrices are column-major with the leading dimension equal to the row count unless a
 *    leading dimension argument says otherwise.
 *  - Index sets: points carry two orderings. "Original" indices are the caller's; "positions"
 *    are the cluster ordering in which every cluster is a contiguous range [begin, begin+size).
 *    perm[p] is the original index stored at position p. Vectors passed to the products are in
 *    ORIGINAL ordering; the permutation is applied inside the kernels.
 *  - uh_create / h_create read HOST memory only, copy what they need to device memory that the
 *    op owns, and return; the caller keeps ownership of its arrays and may free them afterwards.
 *  - Product calls take DEVICE pointers owned by the caller and are asynchronous on the given
 *    cudaStream_t (passed as void*, NULL = legacy default stream). Scratch memory belongs to the
 *    op. Calls on one op may come from several streams and host threads: the library runs them
 *    in the order they are made (a call on another stream than the op's previous call waits,
 *    on the device, for that call's work), since they share the op's scratch and its per-call
 *    counters. Two products of one op could not overlap anyway: each one fills the GPU. Calls on
 *    different ops are independent. Inside a CUDA-graph stream capture, keep an op on one stream.
 */
#ifndef UH_H
#define UH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
enum {
  UH_OK = 0,
  UH_EINVAL = 1,     /* invalid argument or descriptor (message in uh_last_error) */
  UH_ENOMEM = 2,     /* a host or device allocation failed */
  UH_ECUDA = 3,      /* a CUDA call failed (message names it) */
  UH_ENOTREADY = 4,  /* result not available yet */
  UH_ETIMEOUT = 5,   /* a bounded device-side wait ran out */
  UH_EBUSY = 6       /* resource limit reached */
};

/* Message for the calling thread's most recent failed call ("" if none). Never NULL. */
const char* uh_last_error(void);

/* Library version string. */
const char* uh_version(void);

/* ---------------------------------------------------------------- element types */
/* Element type of the arrays a descriptor points to. */
enum { UH_DATA_C128 = 0, /* complex double, 16 bytes */
       UH_DATA_C64 = 1   /* complex float, 8 bytes */ };

/* Storage and arithmetic of a created op.
 *  UH_PREC_C128: operator stored complex128, products in FP64; x and y are complex128.
 *  UH_PREC_C64:  operator stored complex64, products accumulated in FP32; x and y complex64.
 *  UH_PREC_C64_TF32, UH_PREC_C64_BF16X3: as UH_PREC_C64, plus a second copy of the operator for
 *                the tensor-core uh_matmat: TF32 (rounded to nearest), or each FP32 value split
 *                into BF16 hi + lo (three products hi*hi + hi*lo + lo*hi, FP32 accumulation).
 *                Only for UH ops (h_create accepts UH_PREC_C128 and UH_PREC_C64). */
enum { UH_PREC_C128 = 0, UH_PREC_C64 = 1, UH_PREC_C64_TF32 = 2, UH_PREC_C64_BF16X3 = 3 };

/* Arithmetic of uh_matmat / h_matmat.
 *  UH_MM_SIMT:   the product on the CUDA cores in the precision of uh_matvec (any op): after
 *                uh_reserve / h_reserve(op, >= 2) on a complex64 op, 4 (or 2) right-hand sides per pass
 *                over the operator, each column bitwise equal to its uh_matvec; otherwise one
 *                product per column.
 *  UH_MM_TF32:   tensor cores, TF32 operands, FP32 accumulation (op made with UH_PREC_C64_TF32).
 *  UH_MM_BF16X3: tensor cores, BF16 hi/lo split of both operands, 3 products, FP32 accumulation
 *                (op made with UH_PREC_C64_BF16X3). */
enum { UH_MM_SIMT = 0, UH_MM_TF32 = 1, UH_MM_BF16X3 = 2 };

/* ---------------------------------------------------------------- shared structure */
/*
 * Cluster table (Def. 2.1). Cluster c covers positions [cl_begin[c], cl_begin[c]+cl_size[c]).
 * Only clusters named by a block need to be meaningful; the tree structure itself is not
 * needed, because the blocks must tile the index square exactly (checked by uh_create).
 */
typedef struct {
  int64_t n;               /* |I| = |J| = number of points, >= 1 */
  const int64_t* perm;     /* [n] position -> original index, a permutation; NULL = identity */
  int32_t n_clusters;      /* >= 1 */
  const int64_t* cl_begin; /* [n_clusters] first position of each cluster */
  const int64_t* cl_size;  /* [n_clusters] number of positions, >= 1 */
} uh_tree_desc;

/* Near field P^- (Def. 2.3): dense blocks A|_b, |tau| x |sigma| column-major at D_data+D_off[i]. */
typedef struct {
  int64_t n_dense;
  const int32_t* row_cl;   /* [n_dense] tau */
  const int32_t* col_cl;   /* [n_dense] sigma */
  const int64_t* off;      /* [n_dense] element offset into data */
  const void* data;        /* complex elements of type data_type */
  int64_t len;             /* number of complex elements in data (bounds check) */
} uh_dense_desc;

/* ---------------------------------------------------------------- UH operator */
/*
 * Uniform H-matrix (Def. 2.4):
 *  row bases  U_tau   = U_data + row_off[tau],   |tau| x row_rank[tau] column-major;
 *  col bases  V_sigma = V_data + col_off[sigma], |sigma| x col_rank[sigma] column-major;
 *  coupling   S_b     = S_data + S_off[i], row_rank[tau] x col_rank[sigma] column-major, for the
 *             admissible block b = (adm_row[i], adm_col[i]);
 *             or, where S_rank is not NULL and k = S_rank[i] >= 0, stored factored as
 *             S_b = S_X,b S_Y,b^* (Section 4.2): S_X,b = S_data + S_off[i], row_rank[tau] x k
 *             column-major, then S_Y,b = S_data + S_off[i] + row_rank[tau] * k, col_rank[sigma] x k
 *             column-major; k lies in [0, min(row_rank[tau], col_rank[sigma])]. S_rank[i] = -1
 *             (or S_rank NULL) is the dense form. The product then computes
 *             t_b = S_Y,b^* xhat_sigma and adds S_X,b t_b to yhat_tau (Algorithm 6 with the
 *             factored coefficients), streaming k (l_tau + l_sigma) elements instead of
 *             l_tau l_sigma; the tensor-core uh_matmat assembles S_b from its factors when it
 *             packs its operator;
 *  near field as in uh_dense_desc.
 * Ranks may be 0 (the block then contributes nothing). A cluster that is not the row cluster of
 * an admissible block may carry row_rank 0 and any offset (likewise for columns).
 */
typedef struct {
  uh_tree_desc tree;
  int32_t data_type;        /* UH_DATA_C128 or UH_DATA_C64, for every *_data array */
  const int32_t* row_rank;  /* [n_clusters] */
  const int64_t* row_off;   /* [n_clusters] */
  const void* U_data;
  int64_t U_len;
  const int32_t* col_rank;  /* [n_clusters] */
  const int64_t* col_off;   /* [n_clusters] */
  const void* V_data;
  int64_t V_len;
  int64_t n_adm;
  const int32_t* adm_row;   /* [n_adm] tau */
  const int32_t* adm_col;   /* [n_adm] sigma */
  const int64_t* S_off;     /* [n_adm] */
  const void* S_data;
  int64_t S_len;
  uh_dense_desc dense;
  const int32_t* S_rank;    /* [n_adm] inner rank k of a factored S_b, -1 = dense; NULL = all dense */
} uh_desc;

typedef struct uh_op uh_op;

/*
 * Validate the descriptor and create a device-resident op with storage `precision`
 * (UH_PREC_*). Checks: perm is a permutation; every cluster lies in [0, n); the admissible and
 * dense blocks together cover the n x n index square exactly once (Def. 2.2); ranks lie in
 * [0, cluster size]; every matrix lies inside its data array. Fails with UH_EINVAL (nothing
 * allocated) on the first violation, UH_ENOMEM / UH_ECUDA on allocation or copy failure.
 * Uses the current CUDA device; the op must be used and destroyed with that device current.
 */
int uh_create(const uh_desc* desc, int32_t precision, uh_op** out);
/* uh_create with packing parameters for the streaming program (uh_pack_params below; NULL: the
 * defaults, as uh_create). UH_EINVAL for parameters out of range, or two CTAs per SM with
 * UH_PREC_C128. */
int uh_create_ex(const uh_desc* desc, int32_t precision, const struct uh_pack_params_s* params, uh_op** out);

/* Free all device and host memory of the op. NULL is accepted. Synchronises the device. */
int uh_destroy(uh_op* op);

/*
 * y = A^UH x (overwrites y). x and y: device arrays of n complex values in ORIGINAL ordering,
 * complex128 for UH_PREC_C128 ops and complex64 for UH_PREC_C64 ops; they must not overlap.
 * Asynchronous on `stream` (cudaStream_t as void*). Algorithm 6 (Section 4.4).
 */
int uh_matvec(uh_op* op, const void* x, void* y, void* stream);

/*
 * y = A^UH x with the op's complex64 storage and extended-precision arithmetic: x and y are
 * complex128 device arrays of n values in ORIGINAL ordering (not overlapping); every product
 * and sum of Algorithm 6 (Section 4.4) is carried in pairs of FP32 values (hi + lo, exact
 * products by fma and Knuth's two-sum), about 48 significant bits, so y is the product of the
 * STORED complex64 operator with x to about 1e-13 relative, not the FP32-accumulated product of
 * uh_matvec. It is the residual product of mixed-precision iterative refinement (r = b - A x).
 * For ops created with UH_PREC_C64, UH_PREC_C64_TF32 or UH_PREC_C64_BF16X3 (whose scratch for
 * it is allocated by uh_create: 16 bytes per intermediate value); UH_EINVAL for complex128 ops.
 * Ordered with the op's other calls like uh_matvec; asynchronous on `stream`.
 */
int uh_matvec_mixed(uh_op* op, const void* x, void* y, void* stream);

/*
 * Waits for `stream` and reports whether a bounded device-side wait of this op's products ran
 * out since the last check (UH_ETIMEOUT, status then cleared) - which only happens if the GPU
 * could not run all of the product's CTAs at once. UH_OK otherwise.
 */
int uh_check(uh_op* op, void* stream);

/*
 * Y = A^UH X for nrhs right-hand sides (Algorithm 6 applied to each column): X is n x nrhs
 * column-major with leading dimension ldx (>= n), Y likewise with ldy, both device arrays in
 * ORIGINAL ordering, types as for uh_matvec; X and Y must not overlap. nrhs >= 1. `mode` is a
 * UH_MM_* value the op supports (else UH_EINVAL). The tensor-core modes run in passes of 64
 * right-hand sides: a gather of X into cluster order, then three launches (forward transform,
 * coupling, near field + backward transform), all on `stream`. No allocation: the scratch of
 * the tensor-core modes is allocated by uh_create.
 */
int uh_matmat(uh_op* op, int32_t nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy,
              int32_t mode, void* stream);

/* Scratch of the CUDA-core multi-RHS product (UH_MM_SIMT) for complex64 ops: with max_nrhs >= 2,
 * allocates the product's vectors for 4 right-hand sides per pass (2 for ops of two CTAs per SM,
 * uh_pack_params.ctas_per_sm), R times the bytes of uh_matvec's vectors. Synchronises the device
 * when it allocates. Complex128 ops and max_nrhs = 1: nothing to allocate. The tensor-core modes'
 * scratch exists from uh_create on. UH_EINVAL for max_nrhs < 1. */
int uh_reserve(uh_op* op, int32_t max_nrhs);

/* Sizes of the stored operator and of one product (Lemma 2.6, Def. 2.5). */
typedef struct {
  int64_t n;
  int32_t precision;
  int32_t elem_bytes;         /* 16 (C128) or 8 (C64) */
  int64_t n_row_bases, n_col_bases, n_adm, n_dense;
  int64_t E_U, E_V, E_S, E_D; /* stored complex element counts (E_S: l_tau l_sigma per dense S_b,
                                 k (l_tau + l_sigma) per factored one) */
  int64_t sum_row_rank, sum_col_rank;
  int32_t rank_min, rank_max; /* over all row and column bases with rank > 0 */
  double rank_mean;
  int32_t csp;                /* sparsity constant c_sp (Def. 2.5) */
  int64_t algo_bytes_matvec;  /* elem_bytes*(E_U+E_V+E_S+E_D + 2n + 2(sum ranks) + 2 K) */
  int64_t device_bytes;       /* device memory held by the op (packed operator, indices, scratch) */
  int64_t packed_bytes;       /* bytes streamed per matvec: packed matrices + column indices */
  int32_t n_launches;         /* kernel launches per uh_matvec */
  int64_t n_items;            /* work items per matvec, all launches */
  int32_t matmat_mode;        /* tensor-core uh_matmat mode of the op (UH_MM_TF32 / UH_MM_BF16X3), or -1 */
  int64_t panel_bytes;        /* its packed operator: bytes streamed per pass of 64 right-hand sides */
  int64_t panel_items;        /* its work items per pass */
  int64_t panel_mma_flops;    /* its tensor-core flops per pass of 33-64 right-hand sides (2 M N K of
                                 every MMA, M = 128); a pass of at most 32 issues them with M = 64,
                                 half the flops */
  int64_t pack_tile_bytes;    /* packing of the streaming program (uh_pack_params), as used */
  int64_t pack_item_cost;
  int64_t pack_chunk_cost;
  int64_t pack_pool_unit;
  int64_t pack_ctas_per_sm;   /* CTAs of the streaming kernel per SM */
  int64_t n_factored;         /* coupling matrices stored factored (uh_desc.S_rank >= 0) */
  int64_t sum_factored_rank;  /* K: sum of their inner ranks k */
} uh_stats_t;

int uh_stats(const uh_op* op, uh_stats_t* out);

/* ---------------------------------------------------------------- batched operators */
/*
 * Many independent UH operators applied together (Algorithm 6 for each; the operators share no
 * data). The batch packs all of them into ONE device program, so one launch of the streaming
 * kernel computes every operator's product: its work list is flattened across the operators
 * (each phase of Algorithm 6 over all operators, longest chunks first), instead of one launch
 * per operator. The paper has no batched product; its per-cluster independence (Section 4.4)
 * is what lets the chunks of different operators share one schedule.
 */
typedef struct uh_batch uh_batch;

/*
 * Validate descs[0..count-1] (each as uh_create does; the message names the failing operator)
 * and create the batch with storage `precision` (UH_PREC_C128 or UH_PREC_C64). The descriptors'
 * arrays are copied; the caller keeps them. count >= 1; the points of all operators together
 * must number at most 2^31 - 1.
 */
int uh_batch_create(const uh_desc* const* descs, int32_t count, int32_t precision, uh_batch** out);

/*
 * Packing and scheduling of the streaming program (not in the paper: how the products of
 * Algorithm 6 are cut into work items and spread over the CTAs). 0 selects the default.
 *  tile_bytes  largest tile of a work item, 4096 .. 65536 (default 65536)
 *  item_cost   schedule cost of a work item beyond its bytes (default 4096)
 *  chunk_cost  schedule cost of a chunk end (default 49152)
 *  pool_unit   consecutive chunks of the dynamic pool share a ticket until their cost reaches this
 *              (default 131072)
 * Costs are in bytes streamed in the same time.
 */
typedef struct uh_pack_params_s {
  int32_t tile_bytes, item_cost, chunk_cost, pool_unit;
  int32_t ctas_per_sm; /* 1 or 2 CTAs of the streaming kernel per SM (2: tiles up to 24 KB in
                          three 26 KB stages, so that the per-item and per-chunk latencies of two
                          CTAs overlap on an SM); 0: automatic, two for operators streaming
                          at least 256 MiB per product, else one */
} uh_pack_params;

/* uh_batch_create with packing parameters (NULL: the defaults). */
int uh_batch_create_ex(const uh_desc* const* descs, int32_t count, int32_t precision, const uh_pack_params* params,
                       uh_batch** out);

/*
 * Autotuner of the batched product: packs an evenly spaced sample of `sample` of the operators
 * (all of them for sample <= 0 or >= count) with candidate parameters, times `reps` back-to-back
 * products of each on `stream` (CUDA events, after 3 warm-up products; zero vectors), and returns
 * the fastest parameters in *best: one pass of coordinate descent over ctas_per_sm {1, 2}
 * (complex64), tile_bytes {16, 32, 64 KB}, item_cost {1, 4, 16 KB}, chunk_cost {12, 48, 192 KB} and
 * pool_unit {32, 128, 512 KB} from the defaults (ctas_per_sm automatic), a change kept when it is at
 * least 1% faster. *default_ms / *best_ms (optional): the
 * mean product time with the defaults / with *best. Allocates and frees its own batches and
 * vectors; blocks until done. Pass *best to uh_batch_create_ex for the whole set.
 */
int uh_batch_tune(const uh_desc* const* descs, int32_t count, int32_t precision, int32_t sample, int32_t reps,
                  uh_pack_params* best, double* best_ms, double* default_ms, void* stream);
int uh_batch_destroy(uh_batch* batch);

/* offsets[0..count]: operator k's points are positions [offsets[k], offsets[k+1]) of the batch
 * vectors; offsets[count] is the total. */
int uh_batch_offsets(const uh_batch* batch, int64_t* offsets);

/*
 * y_k = A_k x_k for every operator k, in one launch: x and y are device arrays of offsets[count]
 * complex values (the operators' vectors back to back, each in its ORIGINAL ordering), types as
 * for uh_matvec; they must not overlap. Asynchronous on `stream`.
 */
int uh_batch_matvec(uh_batch* batch, const void* x, void* y, void* stream);

/* As uh_check. */
int uh_batch_check(uh_batch* batch, void* stream);

/* Sums over the operators (counts, bytes; n = total points; rank_min / rank_max / csp over all
 * operators, rank_mean over all bases); the packing figures are those of the batch program. */
int uh_batch_stats(const uh_batch* batch, uh_stats_t* out);

/* ---------------------------------------------------------------- serving: GMRES solves */
/*
 * A server runs GMRES(restart) solves A x = b with resident UH ops (the paper's application of
 * the product: solving the boundary integral equation, Sections 1 and 7). Solves are admitted in
 * submission order while their device workspace ((restart + 4) n complex128 values and a little
 * more) fits in the budget and fewer than max_active run, and run together (continuous
 * batching): each running solve's next step is queued on the GPU as soon as its previous step
 * has completed, on a stream of its own, so the steps of different solves overlap and none waits
 * for another's. In a solve the operator's
 * products run in its precision (complex64 storage with FP32 accumulation for UH_PREC_C64 ops);
 * the residual r = b - A x recomputed at every restart, the Arnoldi orthogonalisation (classical
 * Gram-Schmidt, two passes), the norms and the update x += V y run in FP64 on the GPU. A solve
 * ends as converged only when the recomputed residual of the returned x satisfies
 * ||b - A x|| <= tol ||b||. Its arithmetic does not depend on the other solves running with it.
 * Solves of one complex64 op that has multi-RHS scratch (uh_reserve) share their Arnoldi
 * products: a solve ready for its next product waits while another solve of the same op has a
 * step in flight, and the waiting solves run their products as one pass of up to the reserved
 * width (4, or 2 for ops of two CTAs per SM) right-hand sides (each result bitwise that of its
 * own product, so the results do not change).
 * The server uses the device current at uh_server_create and streams of its own; the ops it is
 * given must live on that device and outlive their solves. Products the caller runs on the same
 * ops meanwhile are ordered with the solves' products, like any calls on one op.
 */
typedef struct uh_server uh_server;

typedef struct {
  int32_t status;       /* UH_OK, or the error that ended the solve */
  int32_t converged;    /* 1 if ||b - A x|| <= tol ||b|| for the returned x */
  int32_t iterations;   /* Arnoldi steps (one operator product each), all cycles */
  int32_t restarts;     /* cycles ended by an update x += V y */
  double rel_residual;  /* ||b - A x|| / ||b|| of the returned x (FP64 residual, product in the op's precision) */
  double queue_s;       /* submission -> admission, seconds */
  double latency_s;     /* submission -> completion, seconds */
  int32_t paired_steps; /* Arnoldi steps whose product shared a pass with another solve's */
} uh_solve_info;

/* max_active >= 1 solves at a time, hbm_budget_bytes for their workspaces, at most
 * queue_capacity solves waiting for admission. */
int uh_server_create(int32_t max_active, int64_t hbm_budget_bytes, int32_t queue_capacity, uh_server** out);
/* Stops the server: waiting solves are dropped, running ones end with UH_ECUDA; frees everything. */
int uh_server_destroy(uh_server* server);

/*
 * Submit the solve of op x = b; b: host array of n complex128 values (copied). tol > 0, restart in
 * [1, 60], maxit >= 1 (Arnoldi steps). Returns a ticket, or UH_EBUSY when the solve cannot be
 * admitted now and queue_capacity solves are already waiting, UH_EINVAL when its workspace alone
 * exceeds the budget.
 */
int uh_solve_submit(uh_server* server, uh_op* op, const void* b, double tol, int32_t restart, int32_t maxit,
                    uint64_t* ticket);

/*
 * UH_ENOTREADY while the solve waits or runs. When it has ended: fills info, copies x (host array
 * of n complex128, may be NULL) and forgets the ticket; returns UH_OK, or the solve's error.
 */
int uh_solve_poll(uh_server* server, uint64_t ticket, void* x, uh_solve_info* info);

/* ---------------------------------------------------------------- H operator (plain form) */
/*
 * H-matrix (Def. 2.3): admissible block i = (adm_row[i], adm_col[i]) with rank adm_rank[i] = k_b
 * holds X_b = X_data + X_off[i] (|tau| x k_b) and Y_b = Y_data + Y_off[i] (|sigma| x k_b), both
 * column-major, A|_b = X_b Y_b^*. Near field as for the UH operator.
 */
typedef struct {
  uh_tree_desc tree;
  int32_t data_type;
  int64_t n_adm;
  const int32_t* adm_row;
  const int32_t* adm_col;
  const int32_t* adm_rank;
  const int64_t* X_off;
  const void* X_data;
  int64_t X_len;
  const int64_t* Y_off;
  const void* Y_data;
  int64_t Y_len;
  uh_dense_desc dense;
} h_desc;

typedef struct h_op h_op;

/* Same conventions, checks and errors as uh_create. */
int h_create(const h_desc* desc, int32_t precision, h_op** out);
int h_destroy(h_op* op);
/* y = A^H x, Algorithm 5 (Section 4.4); arguments as for uh_matvec. */
int h_matvec(h_op* op, const void* x, void* y, void* stream);
/* Y = A^H X; arguments as for uh_matmat; only UH_MM_SIMT (in passes of 4 right-hand sides after
 * h_reserve(op, >= 4) on a complex64 op). */
int h_matmat(h_op* op, int32_t nrhs, const void* X, int64_t ldx, void* Y, int64_t ldy,
             int32_t mode, void* stream);
int h_reserve(h_op* op, int32_t max_nrhs);
/* As uh_check. */
int h_check(h_op* op, void* stream);
/* Fills the fields that apply: E_D, n_adm, n_dense, algo_bytes_matvec (elem_bytes*(E_H+2n+2 sum k_b)),
 * E_U = sum_b k_b |tau|, E_V = sum_b k_b |sigma|, E_S = 0. */
int h_stats(const h_op* op, uh_stats_t* out);

/* ---------------------------------------------------------------- allocation-free block product */
/*
 * y = U (S (V^* x)) for one admissible block tau x sigma of a UH-matrix (the block form of
 * Def. 2.4), computed in the forward, coupling and backward steps of the UH product. The paper has
 * no counterpart to this entry point: it is here for callers that cannot call cudaMalloc - code
 * running while a stream is being captured into a CUDA graph, or code that must keep to device
 * memory handed out by its own arena or a framework's allocator. It allocates nothing: the
 * intermediate vectors live in a fixed device array inside the library (266,240 bytes, held on
 * every GPU that loads the library until the process exits).
 *  m, n      block size |tau| x |sigma|, each in [1, (2^31 - 1) * 256]; UH_EINVAL outside
 *  lt, ls    ranks l_tau, l_sigma, each in [0, 256] (the limit set by the fixed array; larger
 *            ranks are rejected with UH_EINVAL) and lt <= m, ls <= n
 *  U         device, m x lt column-major, leading dimension ldu >= m
 *  S         device, lt x ls column-major, lds >= lt
 *  V         device, n x ls column-major, ldv >= n
 *  x         device, n values; y device, m values (overwritten); x, y must not overlap
 *  precision UH_PREC_C128 (complex128, FP64) or UH_PREC_C64 (complex64, FP32 accumulation);
 *            every array has that element type
 *  stream    cudaStream_t as void*; the call is asynchronous on it.
 * All calls share the fixed array, and each call overwrites it before reading it, so nothing
 * carries over between calls; but calls that overlap on the GPU (on different streams, or on
 * several host threads without ordering) race on it and give wrong results. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture begins.
 */
int uh_block_apply_noalloc(int64_t m, int64_t n, int32_t lt, int32_t ls, const void* U, int64_t ldu,
                           const void* S, int64_t lds, const void* V, int64_t ldv, const void* x,
                           void* y, int32_t precision, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* UH_H */

/*
 * uh_build.h - host-side construction of the synthetic Helmholtz workloads as UH and H operators.
 *
 * Produces the descriptors that uh_create / h_create take, for the collocation operator
 *     A_ij = delta_ij / 2 + (4 pi / N) exp(i k |p_i - p_j|) / (4 pi |p_i - p_j|)   (0 for i = j)
 * of the Helmholtz single-layer kernel (Section 6.1), following the construction of Sections 2-4:
 *  - cluster tree (Def. 2.1): split a cluster iff it has more than `leaf` points, along the
 *    longest axis of its bounding box, first floor(|tau|/2) points (stable order by coordinate,
 *    then original index) to the first child;
 *  - block cluster tree (Def. 2.2), level-conserving: a block is admissible iff the boxes are at
 *    positive distance and min(diam) <= eta * dist (eq. (3.3), box diagonal and box distance),
 *    dense if not admissible and one of its clusters is a leaf, subdivided otherwise;
 *  - admissible blocks by partially pivoted ACA at relative tolerance tol_aca, then algebraic
 *    recompression to A|_b = U_b Sigma_b V_b^* (Section 2.3);
 *  - H operator: each block truncated to its singular values > eps * sigma_1;
 *  - UH operator: row basis of tau from the stacked matrix [U_b Sigma_b]_{sigma in row(tau)}
 *    (the agglomeration matrix up to an orthonormal factor, eq. (4.2)), column basis likewise
 *    from [V_b Sigma_b]_{tau in col(sigma)}, each truncated to the singular values
 *    > eps * sigma_1; the singular vectors come from a column-pivoted QR stopped once the
 *    remainder is below 1e-3 * eps * (largest column norm), followed by a one-sided Jacobi SVD
 *    of the small triangular factor (the rank-revealing alternative of Remark 4.2);
 *    S_b = (U_tau^* U_b Sigma_b)(V_sigma^* V_b)^*, the optimal coefficient of Section 4.1, or
 *    with params.factored that pair recompressed at eps and stored factored where smaller.
 * All arithmetic is complex128 on the host, parallel over blocks and clusters with OpenMP.
 *
 * The model owns every array its descriptors point to; they stay valid until uhb_free.
 * Status codes and uh_last_error() as in uh.h.
 */
#ifndef UH_BUILD_H
#define UH_BUILD_H

#include "uh.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double wavenumber;  /* k */
  int32_t leaf;       /* largest leaf size, >= 1 */
  double eta;         /* admissibility parameter, > 0 */
  double eps;         /* relative truncation of bases and H blocks, in [0, 1) */
  double tol_aca;     /* relative ACA / recompression tolerance, in (0, 1) */
  int32_t nthreads;   /* OpenMP threads; <= 0: the OpenMP default */
  int32_t strong;     /* 0: weak admissibility min(diam) <= eta dist (eq. (3.3));
                         1: strong admissibility max(diam) <= eta dist (eq. (3.2)) */
  int32_t factored;   /* 0: every S_b dense; 1: the coefficient pair (U_tau^* U_b Sigma_b,
                         V_sigma^* V_b) recompressed at eps (Section 2.3) and S_b stored factored,
                         S_b = S_X,b S_Y,b^* (Section 4.2, uh_desc.S_rank), where its rank k gives
                         k (l_tau + l_sigma) < l_tau l_sigma */
} uhb_params;

typedef struct {
  int64_t n, n_clusters, n_adm, n_dense;
  int32_t depth;        /* L(T_I) */
  int32_t csp;          /* sparsity constant (Def. 2.5) */
  int32_t kmax_aca;     /* largest block rank after recompression at tol_aca */
  int32_t kmax_h;       /* largest block rank of the H operator (eps) */
  int32_t lmax;         /* largest cluster rank of the UH operator */
  double seconds_tree, seconds_aca, seconds_bases, seconds_dense;
} uhb_info_t;

typedef struct uh_model uh_model;

/* Build both operators for n points (row-major n x 3 doubles, host). */
int uhb_build_helmholtz(int64_t n, const double* points, const uhb_params* params, uh_model** out);
/*
 * The same construction on the current CUDA device (Section 4.3, Algorithms 3 and 4, with the
 * admissible blocks from ACA and recompression, Section 2.3): the host builds the two trees; the
 * device computes, one CTA per block or cluster and all in FP64, every block's ACA (at most 64
 * terms; UH_EINVAL if a block needs more) and recompression, every cluster basis (column-pivoted
 * QR stopped at 1e-3 eps of the largest column, then one-sided Jacobi; UH_EINVAL if a numerical
 * rank exceeds 256), the coupling matrices and the dense blocks; the results are copied into the
 * model's host arrays, laid out as uhb_build_helmholtz lays them out. nthreads is unused.
 * Synchronous; device memory is freed before it returns. UH_ENOMEM / UH_ECUDA on device errors.
 */
int uhb_build_helmholtz_gpu(int64_t n, const double* points, const uhb_params* params, uh_model** out);
/* Descriptors into the model's arrays (complex128, UH_DATA_C128). */
int uhb_uh_desc(const uh_model* m, uh_desc* out);
int uhb_h_desc(const uh_model* m, h_desc* out);
int uhb_info(const uh_model* m, uhb_info_t* out);
/* Free the model. NULL is accepted. */
int uhb_free(uh_model* m);

#ifdef __cplusplus
}
#endif

#endif /* UH_BUILD_H */

"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: closed forms worked by hand,
brute force on tiny inputs, invariants of the definitions (Defs. 2.1-2.4), the exactness of
Algorithm 2 at full rank, the projection identity of Section 4.2, the Frobenius identity and
the spectral bound of Section 5 (Theorem 5.1), and the storage bounds of Lemma 2.6.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I


# ---------------------------------------------------------------- inputs and matrix entries


def test_fibonacci_closed_form():
    p = I.fibonacci_sphere(4)
    assert np.allclose(p[:, 2], [0.75, 0.25, -0.25, -0.75], atol=0, rtol=0)
    assert np.allclose(np.linalg.norm(I.fibonacci_sphere(1000), axis=1), 1.0, atol=1e-15)
    # i = 0: theta = 0 -> (rho, 0, z) with z = 1 - 1/N
    q = I.fibonacci_sphere(8)[0]
    assert q[1] == 0.0 and abs(q[2] - 0.875) < 1e-16 and abs(q[0] - math.sqrt(1 - 0.875 ** 2)) < 1e-16
    # golden-angle increment between consecutive points
    ang = np.arctan2(p[1, 1], p[1, 0]) % (2 * math.pi)
    assert abs(ang - (math.pi * (3 - math.sqrt(5))) % (2 * math.pi)) < 1e-14


def test_ellipsoid_and_noise_bounds():
    p = I.ellipsoid_points(4096, (1.0, 0.7, 0.4), 0.01, seed=0)
    q = I.fibonacci_sphere(4096) * np.array([1.0, 0.7, 0.4])
    ratio = np.linalg.norm(p, axis=1) / np.linalg.norm(q, axis=1)
    assert ratio.min() >= 0.99 - 1e-15 and ratio.max() <= 1.01 + 1e-15
    assert np.abs(ratio - 1).max() > 0.009  # the noise is really applied


def test_entries_closed_form_by_hand():
    # Three points at distances 1 (0-1), 2 (0-2), sqrt(5) (1-2); N = 3, k = pi.
    pts = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 2, 0]])
    A = O.entries(pts, np.arange(3), np.arange(3), math.pi, 3)
    # (4 pi / 3) * exp(i pi r) / (4 pi r) = exp(i pi r) / (3 r)
    assert abs(A[0, 0] - 0.5) < 1e-16
    assert abs(A[0, 1] - (-1.0 / 3.0)) < 1e-15          # exp(i pi) / 3
    assert abs(A[0, 2] - (1.0 / 6.0)) < 1e-15           # exp(2 i pi) / 6
    r = math.sqrt(5.0)
    assert abs(A[1, 2] - cmath.exp(1j * math.pi * r) / (3 * r)) < 1e-15
    assert np.array_equal(A, A.T)  # complex symmetric, not Hermitian
    assert abs(A[1, 2].imag) > 0.01


def test_entries_modulus():
    pts = I.fibonacci_sphere(64)
    A = O.dense_matrix(pts, 7.0)
    d = np.linalg.norm(pts[:, None] - pts[None], axis=2)
    off = ~np.eye(64, dtype=bool)
    assert np.allclose(np.abs(A[off]), 1.0 / (64 * d[off]), rtol=1e-14)
    assert np.allclose(np.diag(A), 0.5)


def test_dense_rows_matvec():
    pts = I.fibonacci_sphere(300)
    A = O.dense_matrix(pts, 3.0)
    x = I.complex_normal(300, 5)
    rows = np.array([0, 17, 299])
    assert np.allclose(O.dense_rows_matvec(pts, 3.0, rows, x), (A @ x)[rows], rtol=1e-13)


# ---------------------------------------------------------------- cluster and block trees


@pytest.fixture(scope="module")
def tree1000():
    pts = I.ellipsoid_points(1000, (1.0, 0.6, 0.3), 0.02, seed=3)
    return pts, O.ClusterTree(pts, 32)


def test_cluster_tree_partition(tree1000):
    pts, t = tree1000
    assert sorted(t.perm.tolist()) == list(range(1000))
    for c in range(t.n_clusters):
        ch = t.children[c]
        if ch:
            a, b = ch
            assert t.size[c] > 32
            assert t.size[a] == t.size[c] // 2 and t.size[a] + t.size[b] == t.size[c]
            assert t.begin[a] == t.begin[c] and t.begin[b] == t.begin[c] + t.size[a]
            assert t.level[a] == t.level[c] + 1 and t.parent[a] == c
            # split along the longest box axis: left child lies below right child on it
            axis = int(np.argmax(t.hi[c] - t.lo[c]))
            assert pts[t.indices(a), axis].max() <= pts[t.indices(b), axis].min()
        else:
            assert t.size[c] <= 32
        idx = t.indices(c)
        assert np.allclose(t.lo[c], pts[idx].min(0)) and np.allclose(t.hi[c], pts[idx].max(0))


def test_cluster_tree_depth_power_of_two():
    t = O.ClusterTree(I.fibonacci_sphere(2048), 32)
    assert t.depth() == int(math.log2(2048 / 32)) + 1
    leaves = [c for c in range(t.n_clusters) if t.is_leaf(c)]
    assert all(t.size[c] == 32 for c in leaves) and len(leaves) == 64


def test_block_tree_partition_brute_force(tree1000):
    pts, t = tree1000
    adm, dense = O.block_tree(t, 1.0)
    cover = np.zeros((1000, 1000), dtype=np.int32)
    for (a, b) in adm + dense:
        cover[np.ix_(t.indices(a), t.indices(b))] += 1
    assert (cover == 1).all()  # every (i, j) in exactly one leaf block (Def. 2.2)
    for (a, b) in adm:
        assert O.admissible(t, a, b, 1.0)
        # parent pair was not admissible (blocks are maximal, level-conserving subdivision)
        pa, pb = t.parent[a], t.parent[b]
        assert pa >= 0 and pb >= 0 and not O.admissible(t, pa, pb, 1.0)
        assert t.level[a] == t.level[b]
    for (a, b) in dense:
        assert t.is_leaf(a) or t.is_leaf(b)
        assert not O.admissible(t, a, b, 1.0)


def test_strong_admissibility_partition(tree1000):
    """Strong admissibility (eq. (3.2), max of the diameters): still an exact partition of I x J,
    every admissible leaf satisfies the strong condition (hence the weak one), and the dense part
    contains the weak partition's dense part."""
    pts, t = tree1000
    adm, dense = O.block_tree(t, 1.0, strong=True)
    cover = np.zeros((1000, 1000), dtype=np.int32)
    for (a, b) in adm + dense:
        cover[np.ix_(t.indices(a), t.indices(b))] += 1
    assert (cover == 1).all()
    for (a, b) in adm:
        d = O.box_dist(t.lo[a], t.hi[a], t.lo[b], t.hi[b])
        assert max(O.box_diam(t.lo[a], t.hi[a]), O.box_diam(t.lo[b], t.hi[b])) <= d
        assert O.admissible(t, a, b, 1.0) and O.admissible(t, a, b, 1.0, strong=True)
        assert not O.admissible(t, t.parent[a], t.parent[b], 1.0, strong=True)
    for (a, b) in dense:
        assert not O.admissible(t, a, b, 1.0, strong=True)
    # A strongly admissible pair is weakly admissible, so the weak recursion stops at or above
    # every strong leaf: each weakly dense block is strongly dense as well.
    wadm, wdense = O.block_tree(t, 1.0)
    assert set(wdense) <= set(dense)
    e_strong = sum(t.size[a] * t.size[b] for a, b in dense)
    e_weak = sum(t.size[a] * t.size[b] for a, b in wdense)
    assert e_strong > e_weak
    # a pair that is weakly but not strongly admissible: one small cluster near a large one
    found = False
    for a in range(t.n_clusters):
        for b in range(t.n_clusters):
            if O.admissible(t, a, b, 1.0) and not O.admissible(t, a, b, 1.0, strong=True):
                found = True
                break
        if found:
            break
    assert found


def test_box_measures_bound_point_measures(tree1000):
    pts, t = tree1000
    rng = np.random.default_rng(0)
    for _ in range(30):
        a, b = rng.integers(0, t.n_clusters, 2)
        pa, pb = pts[t.indices(a)], pts[t.indices(b)]
        dmin = np.linalg.norm(pa[:, None] - pb[None], axis=2).min()
        assert O.box_dist(t.lo[a], t.hi[a], t.lo[b], t.hi[b]) <= dmin + 1e-15
        dmax = np.linalg.norm(pa[:, None] - pa[None], axis=2).max()
        assert O.box_diam(t.lo[a], t.hi[a]) >= dmax - 1e-15
    assert O.box_dist([0, 0, 0], [1, 1, 1], [4, 5, 1], [6, 6, 6]) == 5.0  # gap (3, 4, 0)
    assert O.box_diam([0, 0, 0], [2, 3, 6]) == 7.0


# ---------------------------------------------------------------- ACA and recompression


def test_aca_recovers_exact_low_rank():
    rng = np.random.default_rng(1)
    A = (rng.standard_normal((60, 5)) + 1j * rng.standard_normal((60, 5))) @ \
        (rng.standard_normal((5, 50)) + 1j * rng.standard_normal((5, 50)))
    U, V = O.aca_partial(lambda i: A[i], lambda j: A[:, j], 60, 50, 1e-12)
    assert U.shape[1] <= 6
    assert np.linalg.norm(A - U @ V.T) <= 1e-12 * np.linalg.norm(A)
    Ub, s, Vb = O.recompress(U, V, 1e-12)
    assert len(s) == 5
    assert np.allclose(Ub.conj().T @ Ub, np.eye(5), atol=1e-13)
    assert np.allclose(Vb.conj().T @ Vb, np.eye(5), atol=1e-13)
    assert np.linalg.norm(A - (Ub * s) @ Vb.conj().T) <= 1e-12 * np.linalg.norm(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False)[:5], rtol=1e-12)


def test_aca_on_helmholtz_block():
    pts = I.fibonacci_sphere(2048)
    t = O.ClusterTree(pts, 32)
    adm, _ = O.block_tree(t, 1.0)
    worst = 0.0
    for (a, b) in adm[::97]:
        Ab = O.entries(pts, t.indices(a), t.indices(b), 4.0, 2048)
        U, V = O.aca_partial(lambda i: Ab[i], lambda j: Ab[:, j], *Ab.shape, 1e-8)
        worst = max(worst, np.linalg.norm(Ab - U @ V.T) / np.linalg.norm(Ab))
    assert worst <= 1e-7  # heuristic stop at tol 1e-8 (Section 6.1 footnote)


# ---------------------------------------------------------------- uniform compression


@pytest.fixture(scope="module")
def ops512():
    pts = I.fibonacci_sphere(512)
    tree = O.ClusterTree(pts, 16)
    adm, dense = O.block_tree(tree, 1.0)
    hf, sv = O.build_h(pts, tree, adm, dense, 6.0, 1e-10)
    uh = O.uniform_compression(hf, 1e-4)
    uh_full = O.uniform_compression(hf, 0.0)
    return pts, tree, hf, sv, uh, uh_full


def test_full_rank_exactness(ops512):
    """eps = 0 keeps every nonzero singular value: A^UH equals A^H up to rounding."""
    pts, tree, hf, sv, uh, uh_full = ops512
    AH = O.h_to_dense(hf)
    AU = O.uh_to_dense(uh_full)
    assert np.linalg.norm(AH - AU) <= 1e-13 * np.linalg.norm(AH)
    x = I.complex_normal(512, 2)
    assert np.linalg.norm(O.uh_matvec(uh_full, x) - AH @ x) <= 1e-13 * np.linalg.norm(AH @ x)


def test_orthogonality_and_rank_rule(ops512):
    *_, uh, _ = ops512
    for t, U in uh.U.items():
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-13)
        s, ell = uh.row_sv[t], U.shape[1]
        assert s[ell - 1] > 1e-4 * s[0] and (ell == len(s) or s[ell] <= 1e-4 * s[0])
    for c, V in uh.V.items():
        assert np.allclose(V.conj().T @ V, np.eye(V.shape[1]), atol=1e-13)


def test_projection_identity(ops512):
    """S_b = S_{X,b} S_{Y,b}^* equals U_tau^* X_b Y_b^* V_sigma (Section 4.2)."""
    _, _, hf, _, uh, _ = ops512
    for b in uh.adm[::5]:
        X, Y = hf.lowrank[b]
        t, s = b
        ref = uh.U[t].conj().T @ X @ Y.conj().T @ uh.V[s]
        assert np.linalg.norm(uh.S[b] - ref) <= 1e-12 * np.linalg.norm(X @ Y.conj().T)


def test_agglomeration_svd_equals_stacked_svd(ops512):
    """eq. (4.2): the nonzero singular values of A_tau (explicit, Algorithm 1) are those of X_tau."""
    _, tree, hf, _, uh, _ = ops512
    row, _ = O.row_sets(hf.adm)
    for t in list(row)[::7]:
        At = np.concatenate([hf.lowrank[(t, s)][0] @ hf.lowrank[(t, s)][1].conj().T
                             for s in row[t]], axis=1)
        sa = np.linalg.svd(At, compute_uv=False)
        sx = uh.row_sv[t]
        k = min(len(sx), len(sa))
        assert np.allclose(sa[:k], sx[:k], rtol=1e-10, atol=1e-14 * sa[0])


def test_frobenius_identity_and_bound(ops512):
    """Section 5: |A - A^UH|_F^2 = sum_b |A_b - UU^*A_b|^2 + |UU^*(A_b - A_b VV^*)|^2
    <= sum_tau sum_{i>l} sigma_i(X_tau)^2 + sum_sigma sum_{i>l} sigma_i(Y_sigma)^2."""
    _, tree, hf, _, uh, _ = ops512
    lhs = np.linalg.norm(O.h_to_dense(hf) - O.uh_to_dense(uh)) ** 2
    mid = 0.0
    for (t, s) in hf.adm:
        X, Y = hf.lowrank[(t, s)]
        Ab = X @ Y.conj().T
        Pu = uh.U[t] @ uh.U[t].conj().T
        Pv = uh.V[s] @ uh.V[s].conj().T
        mid += np.linalg.norm(Ab - Pu @ Ab) ** 2 + np.linalg.norm(Pu @ (Ab - Ab @ Pv)) ** 2
    assert abs(lhs - mid) <= 1e-9 * lhs
    assert lhs <= O.frobenius_tail(uh) * (1 + 1e-9)
    assert lhs > 0


def test_theorem51_spectral_bound(ops512):
    _, tree, hf, _, uh, _ = ops512
    err = np.linalg.norm(O.h_to_dense(hf) - O.uh_to_dense(uh), 2)
    bound = O.theorem51_bound(uh)
    assert 0 < err <= bound


def test_uh_matvec_matches_block_assembly(ops512):
    _, tree, hf, _, uh, _ = ops512
    X = I.complex_normal(512, 9, nrhs=3)
    assert np.allclose(O.uh_matvec(uh, X), O.uh_to_dense(uh) @ X, rtol=0, atol=1e-13)
    assert np.allclose(O.h_matvec(hf, X), O.h_to_dense(hf) @ X, rtol=0, atol=1e-13)


def test_storage_bounds(ops512):
    _, tree, hf, _, uh, _ = ops512
    c = uh.counts()
    bnd = O.storage_bounds(hf, uh)
    e_h_adm = hf.elements() - c["E_D"]
    assert e_h_adm <= bnd["H"]
    assert c["E_U"] + c["E_V"] + c["E_S"] <= bnd["UH"]


def test_power_iteration_matches_exact_norm(ops512):
    pts, tree, hf, _, uh, _ = ops512
    B = O.h_to_dense(hf) - O.uh_to_dense(uh)
    est = O.power_iteration_norm(lambda v: B @ v, lambda v: B.conj().T @ v, 512, iters=200)
    assert abs(est - np.linalg.norm(B, 2)) <= 1e-3 * np.linalg.norm(B, 2)


def test_parity_case_against_dense():
    """N = 2048 sphere: A^UH x against the dense product, within Theorem 5.1 plus the ACA error,
    and within C * eps * |A| |x| with C = sqrt(2) sqrt(|L'_I| + |L'_J|)."""
    w = I.SPHERE_2048
    pts = w.points()
    tree, hf, h, uh = O.build_operators(pts, w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    x = w.x()
    A = O.dense_matrix(pts, w.wavenumber)
    yd = A @ x
    yu = O.uh_matvec(uh, x)
    e_aca = np.linalg.norm(A - O.h_to_dense(hf), 2)
    normA = np.linalg.norm(A, 2)
    err = np.linalg.norm(yu - yd)
    assert err <= (O.theorem51_bound(uh) + e_aca) * np.linalg.norm(x)
    C = math.sqrt(2.0) * math.sqrt(len(uh.U) + len(uh.V))
    assert err <= C * w.eps * normA * np.linalg.norm(x)
    assert err / np.linalg.norm(yd) < 1e-5
    yh = O.h_matvec(h, x)
    assert np.linalg.norm(yh - yd) / np.linalg.norm(yd) < 1e-5


def test_aca_running_norm_is_exact():
    """The incremental |S_k|_F of the stopping test equals the Frobenius norm of U V^T."""
    pts = I.fibonacci_sphere(1024)
    t = O.ClusterTree(pts, 32)
    adm, _ = O.block_tree(t, 1.0)
    for (a, b) in adm[::151]:
        Ab = O.entries(pts, t.indices(a), t.indices(b), 9.0, 1024)
        U, V, nrm = O.aca_partial(lambda i: Ab[i], lambda j: Ab[:, j], *Ab.shape, 1e-9,
                                  return_norm=True)
        assert U.shape[1] >= 3
        assert abs(nrm - np.linalg.norm(U @ V.T)) <= 1e-12 * nrm


def test_compression_invariant_under_refactorisation(ops512):
    """Algorithm 2 sees each block only through X_b Y_b^*: replacing (X_b, Y_b) by
    (X_b M, Y_b M^{-*}) for random complex invertible M must give the same A^UH and ranks."""
    _, tree, hf, _, uh, _ = ops512
    rng = np.random.default_rng(4)
    mixed = {}
    for b, (X, Y) in hf.lowrank.items():
        k = X.shape[1]
        M = np.eye(k) + 0.3 * (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
        mixed[b] = (X @ M, Y @ np.linalg.inv(M).conj().T)
    hm = O.HMatrix(tree, hf.adm, hf.dense, mixed, hf.near)
    uhm = O.uniform_compression(hm, 1e-4)
    assert uhm.ranks() == uh.ranks()
    A1, A2 = O.uh_to_dense(uh), O.uh_to_dense(uhm)
    assert np.linalg.norm(A1 - A2) <= 1e-10 * np.linalg.norm(A1)


# ---------------------------------------------------------------- two-sided pins (Def. 2.5,
# Section 2.3, Theorem 5.1, Lemma 2.6): each equality fails on a one-index or missing-factor slip


def test_sparsity_constant_hand_counted():
    """Def. 2.5 on block lists written out by hand. row(1) = {2, 3}, row(4) = {2, 5, 6},
    row(7) = {2}; col(2) = {1, 4, 7}, col(3) = {1}, col(5) = {4}, col(6) = {4}: c_sp = 3,
    reached by a row set and by a column set. The second list reaches its maximum only on the
    column side, the third only on the row side."""
    adm = [(1, 2), (1, 3), (4, 2), (4, 5), (4, 6), (7, 2)]
    assert O.sparsity_constant(adm) == 3
    # col(9) = {1, 2, 3, 4}, every row set has one or two members: c_sp = 4 (columns only)
    adm_c = [(1, 9), (2, 9), (3, 9), (4, 9), (1, 8)]
    assert O.sparsity_constant(adm_c) == 4
    # row(5) = {1, 2, 3, 4, 6}, every column set has one member: c_sp = 5 (rows only)
    adm_r = [(5, 1), (5, 2), (5, 3), (5, 4), (5, 6)]
    assert O.sparsity_constant(adm_r) == 5
    # a repeated cluster number on the two sides is still two different sets
    assert O.sparsity_constant([(1, 1), (2, 1), (1, 2)]) == 2
    assert O.sparsity_constant([]) == 0


def test_sparsity_constant_brute_force_on_block_tree(tree1000):
    """The same count taken from the exact cover of I x J: for every cluster, the number of
    distinct admissible blocks whose row (column) index set is exactly that cluster's."""
    _, t = tree1000
    adm, _ = O.block_tree(t, 1.0)
    per_row, per_col = {}, {}
    for (a, b) in adm:
        key_r = tuple(t.indices(a))
        key_c = tuple(t.indices(b))
        per_row[key_r] = per_row.get(key_r, 0) + 1
        per_col[key_c] = per_col.get(key_c, 0) + 1
    assert O.sparsity_constant(adm) == max(list(per_row.values()) + list(per_col.values()))


def test_truncate_h_error_is_first_dropped_singular_value(ops512):
    """Section 2.3: truncating a block to the singular values > eps sigma_1 leaves a spectral
    error of exactly sigma_{k+1}, and the kept rank k satisfies the rule on both sides."""
    _, tree, hf, sv, _, _ = ops512
    eps = 1e-4
    h = O.truncate_h(hf, sv, eps)
    checked = 0
    for b in hf.adm[::3]:
        X, Y = hf.lowrank[b]
        Xt, Yt = h.lowrank[b]
        full = X @ Y.conj().T
        s = np.linalg.svd(full, compute_uv=False)  # the block's own singular values
        k = Xt.shape[1]
        assert k >= 1 and s[k - 1] > eps * s[0]
        if k < len(s):
            assert s[k] <= eps * s[0]
        err = np.linalg.norm(full - Xt @ Yt.conj().T, 2)
        expect = s[k] if k < len(s) else 0.0
        assert abs(err - expect) <= 1e-9 * expect + 1e-13 * s[0]
        checked += 1
    assert checked > 20
    # some blocks really lose rank at this eps
    assert any(h.lowrank[b][0].shape[1] < hf.lowrank[b][0].shape[1] for b in hf.adm)


def _cluster_projection_errors(hf, uh):
    """e_tau = |A_tau - U_tau U_tau^* A_tau|_2 with A_tau = [X_b Y_b^*]_{sigma in row(tau)}
    assembled explicitly, and likewise e_sigma for the column blocks (proof of Theorem 5.1)."""
    row, col = O.row_sets(hf.adm)
    e_row, e_col = {}, {}
    for t in row:
        At = np.concatenate([hf.lowrank[(t, s)][0] @ hf.lowrank[(t, s)][1].conj().T
                             for s in row[t]], axis=1)
        U = uh.U[t]
        e_row[t] = np.linalg.norm(At - U @ (U.conj().T @ At), 2)
    for s in col:
        Bs = np.concatenate([(hf.lowrank[(t, s)][0] @ hf.lowrank[(t, s)][1].conj().T).conj().T
                             for t in col[s]], axis=1)
        V = uh.V[s]
        e_col[s] = np.linalg.norm(Bs - V @ (V.conj().T @ Bs), 2)
    return e_row, e_col


def test_theorem51_terms_are_next_singular_values(ops512):
    """Theorem 5.1's terms: e_tau equals sigma_{l_tau+1}(X_tau) (two-sided), and the bound is
    sqrt(2) sqrt(sum e_tau^2 + sum e_sigma^2) of the explicitly assembled projections."""
    _, tree, hf, _, uh, _ = ops512
    e_row, e_col = _cluster_projection_errors(hf, uh)
    for t, e in e_row.items():
        s, ell = uh.row_sv[t], uh.U[t].shape[1]
        expect = s[ell] if ell < len(s) else 0.0
        assert abs(e - expect) <= 1e-9 * expect + 1e-13 * s[0]
    for c, e in e_col.items():
        s, ell = uh.col_sv[c], uh.V[c].shape[1]
        expect = s[ell] if ell < len(s) else 0.0
        assert abs(e - expect) <= 1e-9 * expect + 1e-13 * s[0]
    explicit = math.sqrt(2.0) * math.sqrt(sum(e * e for e in e_row.values())
                                          + sum(e * e for e in e_col.values()))
    assert explicit > 0
    assert abs(O.theorem51_bound(uh) - explicit) <= 1e-9 * explicit


def test_theorem51_single_block_is_eckart_young():
    """One admissible block with distinct singular values: U_tau and V_sigma are its leading
    singular vectors, so A^UH|_b is the best rank-l approximation (Eckart-Young) with spectral
    error sigma_{l+1}, e_tau = e_sigma = sigma_{l+1}, and the bound of eq. (5.1) is exactly
    sqrt(2) * sqrt(2) * sigma_{l+1} = 2 sigma_{l+1}: attained up to the factor 2."""
    pts = np.stack([np.arange(40.0), np.zeros(40), np.zeros(40)], axis=1)
    tree = O.ClusterTree(pts, 20)  # root and two leaves of 20 points
    a, b = tree.children[0]
    rng = np.random.default_rng(11)
    P, _ = np.linalg.qr(rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20)))
    Q, _ = np.linalg.qr(rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20)))
    s = 10.0 ** (-0.5 * np.arange(20))  # 1, 0.316, 0.1, ... distinct
    Ab = (P * s) @ Q.conj().T
    for eps, ell in ((0.05, 3), (2e-4, 8), (0.0, 20)):
        h = O.HMatrix(tree, [(a, b)], [], {(a, b): (P * s, Q)}, {})
        uh = O.uniform_compression(h, eps)
        assert uh.U[a].shape[1] == ell and uh.V[b].shape[1] == ell
        blk = uh.U[a] @ uh.S[(a, b)] @ uh.V[b].conj().T
        best = (P[:, :ell] * s[:ell]) @ Q[:, :ell].conj().T
        assert np.linalg.norm(blk - best) <= 1e-13
        err = np.linalg.norm(Ab - blk, 2)
        nxt = s[ell] if ell < 20 else 0.0
        assert abs(err - nxt) <= 1e-12
        assert abs(O.theorem51_bound(uh) - 2.0 * nxt) <= 1e-12


def test_storage_bounds_formula_by_hand():
    """Lemma 2.6 evaluated by hand on a balanced tree: 64 points on a line, leaf 8, so
    L = 4 levels and n_min = 8. Blocks are listed by hand with c_sp = 3 (row(1) has three
    members), k_max = 5 and l_max = 7:
      (2.2a)  c_sp k_max (L|I| + L|J|)                      = 3 * 5 * (256 + 256) = 7680,
      (2.2b)  l_max (L|I| + L|J|) + l_max^2 2 c_sp |I|/n_min = 7 * 512 + 49 * 2 * 3 * 8 = 5936."""
    pts = np.stack([np.arange(64.0), np.zeros(64), np.zeros(64)], axis=1)
    tree = O.ClusterTree(pts, 8)
    assert tree.depth() == 4 and min(tree.size) == 8 and tree.n == 64
    adm = [(1, 2), (1, 3), (1, 4), (5, 2)]
    ranks = {(1, 2): 5, (1, 3): 2, (1, 4): 4, (5, 2): 1}
    low = {b: (np.zeros((tree.size[b[0]], k)), np.zeros((tree.size[b[1]], k)))
           for b, k in ranks.items()}
    h = O.HMatrix(tree, adm, [], low, {})
    U = {1: np.zeros((tree.size[1], 7)), 5: np.zeros((tree.size[5], 3))}
    V = {2: np.zeros((tree.size[2], 6)), 3: np.zeros((tree.size[3], 2)),
         4: np.zeros((tree.size[4], 1))}
    uh = O.UHMatrix(tree, adm, [], U, V, {}, {}, {}, {})
    bnd = O.storage_bounds(h, uh)
    assert (bnd["csp"], bnd["kmax"], bnd["lmax"], bnd["L"], bnd["nmin"]) == (3, 5, 7, 4, 8)
    assert bnd["H"] == 7680
    assert bnd["UH"] == 5936


def test_frobenius_tail_equals_explicit_projection_errors(ops512):
    """The Frobenius estimate of Section 5 term by term: for every cluster,
    |A_tau - U U^* A_tau|_F^2 equals the sum of the dropped sigma_i(X_tau)^2 (two-sided)."""
    _, tree, hf, _, uh, _ = ops512
    row, col = O.row_sets(hf.adm)
    tot = 0.0
    for t in row:
        At = np.concatenate([hf.lowrank[(t, s)][0] @ hf.lowrank[(t, s)][1].conj().T
                             for s in row[t]], axis=1)
        U = uh.U[t]
        tot += np.linalg.norm(At - U @ (U.conj().T @ At)) ** 2
    for s in col:
        Bs = np.concatenate([(hf.lowrank[(t, s)][0] @ hf.lowrank[(t, s)][1].conj().T).conj().T
                             for t in col[s]], axis=1)
        V = uh.V[s]
        tot += np.linalg.norm(Bs - V @ (V.conj().T @ Bs)) ** 2
    assert tot > 0
    assert abs(O.frobenius_tail(uh) - tot) <= 1e-8 * tot


# ---------------------------------------------------------------- factored coefficients (Section 4.2)


def test_factored_truncation_is_eckart_young(ops512):
    """Reading R11: each factored block keeps the singular values of S_b above eps * s_1 (checked
    both ways against a plain SVD of the dense S_b), and its error is exactly the first dropped
    singular value (Eckart-Young), so a wrong rank, a lost diag(s) or a factor left unconjugated
    fails."""
    *_, uh, _ = ops512
    for eps in (1e-2, 1e-3):
        f = O.factor_coupling(uh, eps, force=True)
        assert not f.S and set(f.F) == set(uh.S)
        nontrivial = 0
        for b, (X, Y) in f.F.items():
            Sb = uh.S[b]
            s = np.linalg.svd(Sb, compute_uv=False)
            k = X.shape[1]
            assert Y.shape == (Sb.shape[1], k) and X.shape == (Sb.shape[0], k)
            assert k >= 1 and s[k - 1] > eps * s[0]
            nxt = s[k] if k < len(s) else 0.0
            assert nxt <= eps * s[0]
            err = np.linalg.norm(Sb - X @ Y.conj().T, 2)
            assert abs(err - nxt) <= 1e-9 * s[0]
            nontrivial += nxt > 0
        assert nontrivial > len(f.F) // 2


def test_factored_storage_rule_both_ways(ops512):
    """A block is stored factored exactly when k_b (l_tau + l_sigma) < l_tau l_sigma, with k_b the
    rank rule of a plain SVD of S_b; E_S counts the elements of both forms."""
    *_, uh, _ = ops512
    eps = 3e-4  # between the bases' eps and the ranks of these small blocks: both forms occur
    f = O.factor_coupling(uh, eps)
    es = 0
    for b, Sb in uh.S.items():
        s = np.linalg.svd(Sb, compute_uv=False)
        k = int(np.sum(s > eps * s[0]))
        lt, ls = Sb.shape
        small = k * (lt + ls) < lt * ls
        assert (b in f.F) == small and (b in f.S) == (not small)
        es += k * (lt + ls) if small else lt * ls
    assert f.F and f.S
    c = f.counts()
    assert c["E_S"] == es and c["K"] == sum(X.shape[1] for X, _ in f.F.values())


def test_factored_product_exact_without_truncation(ops512):
    """With eps = 0 every nonzero singular value is kept: the factored product (t_b = S_Y^* xhat,
    yhat += S_X t_b) equals the dense-S product of Algorithm 6 up to rounding."""
    *_, uh, _ = ops512
    f = O.factor_coupling(uh, 0.0, force=True)
    X = I.complex_normal(512, 11, nrhs=2)
    y0 = O.uh_matvec(uh, X)
    assert np.linalg.norm(O.uh_matvec(f, X) - y0) <= 1e-13 * np.linalg.norm(y0)
    assert np.allclose(O.uh_to_dense(f), O.uh_to_dense(uh), rtol=0, atol=1e-13)


def test_factored_product_error_within_dropped_values(ops512):
    """|y_f - y| <= sum_b s_{k_b+1}(S_b) |x_sigma| (the bases are orthonormal), and the factored
    product agrees with its own block assembly."""
    _, tree, _, _, uh, _ = ops512
    eps = 1e-3
    f = O.factor_coupling(uh, eps, force=True)
    x = I.complex_normal(512, 12)
    d = O.uh_matvec(f, x) - O.uh_matvec(uh, x)
    xp = x[tree.perm]
    bound = 0.0
    for (t, s), (Xf, _) in f.F.items():
        sv = np.linalg.svd(uh.S[(t, s)], compute_uv=False)
        k = Xf.shape[1]
        if k < len(sv):
            bound += sv[k] * np.linalg.norm(xp[tree.begin[s]:tree.begin[s] + tree.size[s]])
    assert 0 < np.linalg.norm(d) <= bound * (1 + 1e-9)
    assert np.allclose(O.uh_matvec(f, x), O.uh_to_dense(f) @ x, rtol=0, atol=1e-13)


def test_factored_rank_one_coupling_closed_form():
    """A rank-one S_b = a c^* is stored as one column pair that reproduces it exactly, and a zero
    S_b as an empty pair (k_b = 0)."""
    a = np.array([1.0 + 2.0j, -0.5j, 3.0])
    c = np.array([2.0, 1.0 - 1.0j])
    Sb = np.outer(a, c.conj())
    tree = O.ClusterTree(I.fibonacci_sphere(8), 8)
    U = {0: np.eye(8, 3, dtype=np.complex128)}
    V = {0: np.eye(8, 2, dtype=np.complex128)}
    uh = O.UHMatrix(tree, [(0, 0)], [], U, V, {(0, 0): Sb}, {}, {}, {})
    f = O.factor_coupling(uh, 1e-12)
    X, Y = f.F[(0, 0)]
    assert X.shape == (3, 1) and Y.shape == (2, 1)
    assert np.allclose(X @ Y.conj().T, Sb, rtol=0, atol=1e-14)
    assert abs(np.linalg.norm(X) - np.linalg.norm(a) * np.linalg.norm(c)) <= 1e-13
    z = O.factor_coupling(O.UHMatrix(tree, [(0, 0)], [], U, V, {(0, 0): 0 * Sb}, {}, {}, {}), 1e-12)
    assert z.F[(0, 0)][0].shape == (3, 0)

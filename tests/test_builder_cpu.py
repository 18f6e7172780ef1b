"""The library's host-side operator builder (uh_build.h) against the oracle's construction.

Both follow the same readings of the paper (tree, admissibility, ACA, relative truncation), by
different routes (pivoted QR + Jacobi and direct projection in the builder; Algorithm 2 with
its triangular solves in the oracle), so cluster ranks and matvec results must agree."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr


@pytest.fixture(scope="module")
def U():
    from paper_2405_15573_gb300 import uh
    return uh


def _oracle_view(a):
    """The builder's UH arrays as oracle blocks (same structure as the oracle's UHMatrix)."""
    size = a["cl_size"]
    U = {int(c): a["U_data"][a["row_off"][c]:a["row_off"][c] + size[c] * a["row_rank"][c]]
         .reshape(a["row_rank"][c], size[c]).T for c in set(a["adm_row"].tolist())}
    V = {int(c): a["V_data"][a["col_off"][c]:a["col_off"][c] + size[c] * a["col_rank"][c]]
         .reshape(a["col_rank"][c], size[c]).T for c in set(a["adm_col"].tolist())}
    S = {}
    for t, s, o in zip(a["adm_row"], a["adm_col"], a["S_off"]):
        lt, ls = int(a["row_rank"][t]), int(a["col_rank"][s])
        S[(int(t), int(s))] = a["S_data"][o:o + lt * ls].reshape(ls, lt).T
    near = {}
    for t, s, o in zip(a["dense_row"], a["dense_col"], a["D_off"]):
        m, k = int(size[t]), int(size[s])
        near[(int(t), int(s))] = a["D_data"][o:o + m * k].reshape(k, m).T
    return U, V, S, near


@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6, (1.0, 1.0, 1.0), 0.0, False),
                                  (1000, 6.0, 24, 1e-5, (1.0, 0.7, 0.4), 0.01, False),
                                  (1000, 6.0, 24, 1e-5, (1.0, 0.7, 0.4), 0.01, True)],
                         ids=["sphere2048", "ellipsoid1000", "ellipsoid1000_strong"])
def test_builder_matches_oracle(U, case):
    n, k, leaf, eps, axes, noise, strong = case
    pts, tree, hf, h, uh = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise, strong=strong)
    m = U.HelmholtzModel(pts, k, leaf, 1.0, eps, 1e-8, nthreads=2, strong=strong)
    a = m.uh_arrays()
    # identical trees and block partitions
    assert np.array_equal(a["perm"], tree.perm)
    assert np.array_equal(a["cl_begin"], np.array(tree.begin)) and np.array_equal(a["cl_size"], np.array(tree.size))
    assert sorted(zip(a["adm_row"].tolist(), a["adm_col"].tolist())) == uh.adm
    assert sorted(zip(a["dense_row"].tolist(), a["dense_col"].tolist())) == uh.dense
    Ub, Vb, Sb, near = _oracle_view(a)
    # cluster ranks agree (a rank may differ by one where a singular value sits on eps)
    lu, lv = uh.ranks()
    diffs = [abs(Ub[t].shape[1] - lu[t]) for t in lu] + [abs(Vb[s].shape[1] - lv[s]) for s in lv]
    assert max(diffs) <= 1 and np.mean(diffs) < 0.05
    for t, B in Ub.items():
        assert np.allclose(B.conj().T @ B, np.eye(B.shape[1]), atol=1e-12)
    # the two operators apply alike
    built = O.UHMatrix(uh.tree, uh.adm, uh.dense, Ub, Vb, Sb, near, {}, {})
    x = I.complex_normal(n, 4)
    y_o = O.uh_matvec(uh, x)
    y_b = O.uh_matvec(built, x)
    assert relerr(y_b, y_o) < 10 * eps
    # and both approximate the dense operator to within Theorem 5.1 + ACA error
    A = O.dense_matrix(pts, k)
    e = np.linalg.norm(A - O.h_to_dense(hf), 2) + O.theorem51_bound(uh)
    assert np.linalg.norm(y_b - A @ x) <= 2 * e * np.linalg.norm(x)
    # the H form: blocks truncated at eps
    ha = m.h_arrays()
    assert len(ha["adm_rank"]) == len(uh.adm)
    ko = {b: X.shape[1] for b, (X, Y) in h.lowrank.items()}
    kb = dict(zip(zip(ha["adm_row"].tolist(), ha["adm_col"].tolist()), ha["adm_rank"].tolist()))
    assert max(abs(kb[b] - ko[b]) for b in ko) <= 1
    info = m.info()
    assert info["csp"] == O.sparsity_constant(uh.adm) and info["n_adm"] == len(uh.adm)


def test_builder_rejects_bad_parameters(U):
    with pytest.raises(U.UHError, match="invalid parameters"):
        U.HelmholtzModel(I.fibonacci_sphere(64), 1.0, 0, 1.0, 1e-6, 1e-8)
    pts = I.fibonacci_sphere(64)
    pts[3, 1] = np.nan
    with pytest.raises(U.UHError, match="not finite"):
        U.HelmholtzModel(pts, 1.0, 16, 1.0, 1e-6, 1e-8)


def _factored_view(a):
    """The factored blocks of a builder's UH arrays: {(tau, sigma): (S_X, S_Y)}."""
    F = {}
    for i in np.flatnonzero(a["S_rank"] >= 0):
        t, s, o, kb = int(a["adm_row"][i]), int(a["adm_col"][i]), int(a["S_off"][i]), int(a["S_rank"][i])
        lt, ls = int(a["row_rank"][t]), int(a["col_rank"][s])
        F[(t, s)] = (a["S_data"][o:o + lt * kb].reshape(kb, lt).T,
                     a["S_data"][o + lt * kb:o + kb * (lt + ls)].reshape(kb, ls).T)
    return F


@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6, (1.0, 1.0, 1.0), 0.0),
                                  (1000, 6.0, 24, 1e-5, (1.0, 0.7, 0.4), 0.01)],
                         ids=["sphere2048", "ellipsoid1000"])
def test_builder_factored_option(U, case):
    """uhb_params.factored (Section 4.2, reading R11): the same bases and partition as the dense
    build; each factored block keeps the rank rule of a plain SVD of the dense S_b at eps (within
    one, a value decided within rounding), has its spectral error within eps s_1 and is stored only
    where k (l_tau + l_sigma) < l_tau l_sigma; a dense-kept block would not have been smaller at a rank within one of the rule's;
    the factored operator applies within 10 eps of the oracle's."""
    n, k, leaf, eps, axes, noise = case
    pts, tree, hf, h, uh = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
    md = U.HelmholtzModel(pts, k, leaf, 1.0, eps, 1e-8, nthreads=2)
    mf = U.HelmholtzModel(pts, k, leaf, 1.0, eps, 1e-8, nthreads=2, factored=True)
    ad, af = md.uh_arrays(), mf.uh_arrays()
    assert ad.get("S_rank") is None and af["S_rank"] is not None
    for key in ("row_rank", "col_rank", "adm_row", "adm_col", "U_data", "V_data", "D_data"):
        assert np.array_equal(ad[key], af[key]), key
    Ub, Vb, Sd, near = _oracle_view(ad)
    F = _factored_view(af)
    assert len(F) > len(Sd) // 10
    for b, Sb in Sd.items():
        if Sb.size == 0:
            continue
        s = np.linalg.svd(Sb, compute_uv=False)
        kr = int(np.sum(s > eps * s[0])) if s[0] > 0 else 0
        lt, ls = Sb.shape
        if b in F:
            X, Y = F[b]
            assert abs(X.shape[1] - kr) <= 1 and X.shape[1] * (lt + ls) < lt * ls
            assert np.linalg.norm(Sb - X @ Y.conj().T, 2) <= 1.01 * eps * s[0] + 1e-15
        else:
            assert (kr + 1) * (lt + ls) >= lt * ls
    built = O.UHMatrix(uh.tree, uh.adm, uh.dense, Ub, Vb, {b: S for b, S in Sd.items() if b not in F}, near,
                       {}, {}, F=F)
    x = I.complex_normal(n, 7)
    assert relerr(O.uh_matvec(built, x), O.uh_matvec(uh, x)) < 10 * eps
    md.close()
    mf.close()


def test_builder_rejects_bad_factored_flag(U):
    import ctypes as C
    pts = np.ascontiguousarray(I.fibonacci_sphere(64))
    h = C.c_void_p()
    for strong, factored in ((0, 2), (3, 0)):
        prm = U.BuildParams(1.0, 16, 1.0, 1e-6, 1e-8, 0, strong, factored)
        assert U.lib.uhb_build_helmholtz(64, pts.ctypes.data, C.byref(prm), C.byref(h)) == U.UH_EINVAL
        assert h.value is None

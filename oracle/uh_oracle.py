"""FP64 CPU oracle for the uniform H-matrix (UH) matrix-vector product.

TEST INFRASTRUCTURE ONLY. This is the plain, slow and independently written reference that the
CUDA path is checked against. Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import or run it; the library never does, and it shares no code with the library.

Everything is complex128 / float64 and follows the paper (Bruyninckx, Huybrechs, Meerbergen,
"Uniform H-matrix compression with applications to boundary integral equations"):

  * entries of the operator: Helmholtz single-layer kernel of Section 6.1 in collocation form,
    A_ij = delta_ij/2 + (4 pi / N) g(p_i, p_j), g(x, y) = exp(i k |x-y|) / (4 pi |x-y|), with the
    kernel term 0 on the diagonal;
  * cluster tree (Def. 2.1), block cluster tree with level-conserving subdivision and the weak
    admissibility rule on bounding boxes (Def. 2.2, eq. (3.3), Section 6.1);
  * H-matrix blocks (Def. 2.3) from partially pivoted ACA followed by algebraic recompression
    (Section 2.3);
  * uniform compression of the H-matrix (Algorithm 2, built on eq. (4.2) and the coefficient
    formula S_b = S_{X,b} S_{Y,b}^* of Section 4.2);
  * the dense, H (Algorithm 5) and UH (Algorithm 6) matrix-vector products, run sequentially.

Readings where the paper is silent or garbled (each also listed in the design notes):
  R1 admissible iff dist > 0 and min(diam_tau, diam_sigma) <= eta * dist (eq. (3.3) with "<=");
  R2 diam = length of the bounding-box diagonal, dist = Euclidean distance between the boxes;
  R3 a cluster is split iff |tau| > leaf, along the longest box axis, left child = first
     floor(|tau|/2) points after a stable sort by (coordinate, original index);
  R4 ACA with partial pivoting, first row first, next row = argmax |u_k| over unused rows,
     stop when |u_k||v_k| <= tol |S_k|_F, then recompression truncated at sigma_j <= tol sigma_1;
  R5 "choose optimal rank according to eps_tau" (Algorithms 1-3) = smallest l with
     sigma_{l+1}(X_tau) <= eps * sigma_1(X_tau) (relative spectral, Remark 6.1);
  R6 the second inner loop of Algorithm 6 runs over sigma in row(tau);
  R7 the UH operator is the general (non-symmetric) form, with separate row and column bases and
     a dense coefficient matrix S_b = S_{X,b} S_{Y,b}^* per admissible block;
  R11 the factored storage option (Section 4.2 keeps S_{X,b}, S_{Y,b}, k_b (l_tau + l_sigma)
     elements): the pair of Algorithm 2 has the inner rank of the fine block, so it is first
     recompressed at eps like an admissible block (Section 2.3: QR of both factors, SVD of the
     product of the triangles, keep s_j > eps * s_1), and a block keeps the factored form only
     where k_b (l_tau + l_sigma) < l_tau l_sigma.
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------------------------
# Matrix entries (Section 6.1, collocation form with equal weights 4 pi / N)
# ----------------------------------------------------------------------------------------------


def helmholtz_green(r: np.ndarray, wavenumber: float) -> np.ndarray:
    """g = exp(i k r) / (4 pi r) for r > 0 and 0 for r = 0 (the excluded singular term)."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros(r.shape, dtype=np.complex128)
    pos = r > 0
    rp = r[pos]
    out[pos] = np.exp(1j * wavenumber * rp) / (4.0 * math.pi * rp)
    return out


def entries(points: np.ndarray, rows: np.ndarray, cols: np.ndarray, wavenumber: float,
            n_total: int) -> np.ndarray:
    """Submatrix A[rows][:, cols] (original indices) of A_ij = delta_ij/2 + (4 pi/N) g(p_i, p_j)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    diff = points[rows][:, None, :] - points[cols][None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    a = (4.0 * math.pi / n_total) * helmholtz_green(r, wavenumber)
    a = a + 0.5 * (rows[:, None] == cols[None, :])
    return a


def dense_matrix(points: np.ndarray, wavenumber: float) -> np.ndarray:
    n = len(points)
    idx = np.arange(n)
    return entries(points, idx, idx, wavenumber, n)


def dense_rows_matvec(points: np.ndarray, wavenumber: float, rows: np.ndarray,
                      x: np.ndarray) -> np.ndarray:
    """(A x)_i for the listed rows only, straight from the definition, O(N) per row."""
    n = len(points)
    x2 = x.reshape(n, -1)
    out = np.zeros((len(rows), x2.shape[1]), dtype=np.complex128)
    allc = np.arange(n)
    for q, i in enumerate(np.asarray(rows)):
        a = entries(points, np.array([i]), allc, wavenumber, n)[0]
        out[q] = a @ x2
    return out if x.ndim == 2 else out[:, 0]


# ----------------------------------------------------------------------------------------------
# Cluster tree (Def. 2.1) and block cluster tree (Def. 2.2)
# ----------------------------------------------------------------------------------------------


class ClusterTree:
    """Binary cluster tree over points. Cluster c owns positions [begin[c], begin[c]+size[c]) of
    the permuted ordering; perm[p] is the original index at position p. Clusters are numbered in
    depth-first pre-order (root = 0)."""

    def __init__(self, points: np.ndarray, leaf: int):
        n = len(points)
        self.n = n
        self.leaf = leaf
        self.perm = np.zeros(n, dtype=np.int64)
        self.begin: list[int] = []
        self.size: list[int] = []
        self.level: list[int] = []
        self.parent: list[int] = []
        self.children: list[list[int]] = []
        self.lo: list[np.ndarray] = []
        self.hi: list[np.ndarray] = []
        self._split(points, 0, np.arange(n, dtype=np.int64), 0, -1)
        self.lo = np.array(self.lo)
        self.hi = np.array(self.hi)

    def _split(self, points, begin, idx, level, parent):
        cid = len(self.begin)
        pts = points[idx]
        self.begin.append(begin)
        self.size.append(len(idx))
        self.level.append(level)
        self.parent.append(parent)
        self.children.append([])
        self.lo.append(pts.min(axis=0))
        self.hi.append(pts.max(axis=0))
        if len(idx) > self.leaf:
            axis = int(np.argmax(self.hi[cid] - self.lo[cid]))
            order = np.lexsort((idx, pts[:, axis]))  # primary: coordinate, then original index
            idx = idx[order]
            half = len(idx) // 2
            c0 = self._split(points, begin, idx[:half], level + 1, cid)
            c1 = self._split(points, begin + half, idx[half:], level + 1, cid)
            self.children[cid] = [c0, c1]
        else:
            self.perm[begin:begin + len(idx)] = idx
        return cid

    @property
    def n_clusters(self) -> int:
        return len(self.begin)

    def indices(self, c: int) -> np.ndarray:
        """Original indices of cluster c."""
        return self.perm[self.begin[c]:self.begin[c] + self.size[c]]

    def depth(self) -> int:
        """L(T_I) = max level + 1 (Def. 2.1)."""
        return max(self.level) + 1

    def is_leaf(self, c: int) -> bool:
        return not self.children[c]


def box_diam(lo, hi) -> float:
    return float(np.linalg.norm(np.asarray(hi) - np.asarray(lo)))


def box_dist(lo1, hi1, lo2, hi2) -> float:
    gap = np.maximum(0.0, np.maximum(np.asarray(lo2) - hi1, np.asarray(lo1) - hi2))
    return float(np.linalg.norm(gap))


def admissible(tree: ClusterTree, t: int, s: int, eta: float, strong: bool = False) -> bool:
    """Admissibility on bounding boxes (readings R1/R2): the weak condition of eq. (3.3),
    min(diam tau, diam sigma) <= eta dist, or with strong=True the strong condition of eq. (3.2),
    max(diam tau, diam sigma) <= eta dist; both need dist > 0."""
    dist = box_dist(tree.lo[t], tree.hi[t], tree.lo[s], tree.hi[s])
    if dist <= 0.0:
        return False
    dt, ds = box_diam(tree.lo[t], tree.hi[t]), box_diam(tree.lo[s], tree.hi[s])
    return (max(dt, ds) if strong else min(dt, ds)) <= eta * dist


def block_tree(tree: ClusterTree, eta: float, strong: bool = False):
    """Leaves of the level-conserving block cluster tree, s(b) = s(tau) x s(sigma), under the weak
    (default) or strong admissibility condition.

    Returns (P_plus, P_minus): lists of (tau, sigma) cluster pairs (admissible, dense)."""
    adm, dense = [], []
    stack = [(0, 0)]
    while stack:
        t, s = stack.pop()
        if admissible(tree, t, s, eta, strong):
            adm.append((t, s))
        elif tree.is_leaf(t) or tree.is_leaf(s):
            dense.append((t, s))
        else:
            for tc in reversed(tree.children[t]):
                for sc in reversed(tree.children[s]):
                    stack.append((tc, sc))
    adm.sort()
    dense.sort()
    return adm, dense


def row_sets(adm):
    """row(tau) and col(sigma) of Def. 2.5, each sorted by cluster number."""
    row, col = {}, {}
    for t, s in adm:
        row.setdefault(t, []).append(s)
        col.setdefault(s, []).append(t)
    for d in (row, col):
        for key in d:
            d[key].sort()
    return row, col


def sparsity_constant(adm) -> int:
    row, col = row_sets(adm)
    return max([len(v) for v in row.values()] + [len(v) for v in col.values()] + [0])


# ----------------------------------------------------------------------------------------------
# ACA with partial pivoting and algebraic recompression (Section 2.3)
# ----------------------------------------------------------------------------------------------


def aca_partial(row_fn, col_fn, m: int, n: int, tol: float, return_norm: bool = False):
    """Partially pivoted ACA (reading R4). A_b ~ sum_k u_k v_k^T.

    row_fn(i) returns row i of the block (length n), col_fn(j) column j (length m).
    Returns U (m x k), V (n x k) with A_b ~ U V^T (and, if asked, the running estimate of
    |U V^T|_F that the stopping test uses)."""
    us: list[np.ndarray] = []
    vs: list[np.ndarray] = []
    used = np.zeros(m, dtype=bool)
    norm2 = 0.0
    i = 0
    kmax = min(m, n)
    while len(us) < kmax:
        r = np.array(row_fn(i), dtype=np.complex128)
        for u, v in zip(us, vs):
            r -= u[i] * v
        used[i] = True
        j = int(np.argmax(np.abs(r)))
        if abs(r[j]) == 0.0:
            free = np.flatnonzero(~used)
            if free.size == 0:
                break
            i = int(free[0])
            continue
        v_new = r / r[j]
        c = np.array(col_fn(j), dtype=np.complex128)
        for u, v in zip(us, vs):
            c -= v[j] * u
        u_new = c
        # |S_k|_F^2 = |S_{k-1}|_F^2 + 2 Re sum_l (u_l^H u_k)(v_l^H v_k) + |u_k|^2 |v_k|^2
        cross = 0.0
        for u, v in zip(us, vs):
            cross += (np.vdot(u, u_new) * np.vdot(v, v_new)).real
        nu = np.linalg.norm(u_new)
        nv = np.linalg.norm(v_new)
        norm2 = norm2 + 2.0 * cross + (nu * nv) ** 2
        us.append(u_new)
        vs.append(v_new)
        if nu * nv <= tol * math.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u_new)
        cand[used] = -1.0
        if cand.max() < 0:
            break
        i = int(np.argmax(cand))
    if not us:
        U, V = np.zeros((m, 0), np.complex128), np.zeros((n, 0), np.complex128)
    else:
        U, V = np.stack(us, axis=1), np.stack(vs, axis=1)
    return (U, V, math.sqrt(max(norm2, 0.0))) if return_norm else (U, V)


def recompress(U: np.ndarray, V: np.ndarray, tol: float):
    """Truncated SVD of U V^T via QR of both factors (Section 2.3).

    With X = U and Y = conj(V) (so that U V^T = X Y^*): X = Q1 R1, Y = Q2 R2,
    R1 R2^* = W diag(s) Z^*, keep s_j > tol * s_1. Returns (Ub, sb, Vb) with
    U V^T ~ Ub diag(sb) Vb^*."""
    m, k = U.shape
    n = V.shape[0]
    if k == 0:
        return np.zeros((m, 0), np.complex128), np.zeros(0), np.zeros((n, 0), np.complex128)
    Q1, R1 = np.linalg.qr(U)
    Q2, R2 = np.linalg.qr(np.conj(V))
    W, s, Zh = np.linalg.svd(R1 @ R2.conj().T)
    if s[0] == 0.0:
        return np.zeros((m, 0), np.complex128), np.zeros(0), np.zeros((n, 0), np.complex128)
    keep = int(np.sum(s > tol * s[0]))
    return Q1 @ W[:, :keep], s[:keep], Q2 @ Zh.conj().T[:, :keep]


# ----------------------------------------------------------------------------------------------
# H-matrix (Def. 2.3)
# ----------------------------------------------------------------------------------------------


class HMatrix:
    """Admissible blocks as (X_b, Y_b) with A|_b ~ X_b Y_b^*, dense blocks as A|_b."""

    def __init__(self, tree, adm, dense, lowrank, near):
        self.tree = tree
        self.adm = adm
        self.dense = dense
        self.lowrank = lowrank  # {(t, s): (X, Y)}
        self.near = near  # {(t, s): D}

    def elements(self) -> int:
        """Stored element count: sum k_b (|tau| + |sigma|) + dense (Lemma 2.6 and remark)."""
        e = 0
        for (t, s), (X, Y) in self.lowrank.items():
            e += X.shape[1] * (X.shape[0] + Y.shape[0])
        for D in self.near.values():
            e += D.size
        return e


def build_h(points, tree: ClusterTree, adm, dense, wavenumber: float, tol_aca: float):
    """ACA + recompression for every admissible block at relative tolerance tol_aca; dense blocks
    evaluated in full. Returns (HMatrix, sv) where sv[b] holds the kept singular values."""
    n = tree.n
    lowrank, sv, near = {}, {}, {}
    for (t, s) in adm:
        rows, cols = tree.indices(t), tree.indices(s)
        Ua, Va = aca_partial(
            lambda i: entries(points, rows[i:i + 1], cols, wavenumber, n)[0],
            lambda j: entries(points, rows, cols[j:j + 1], wavenumber, n)[:, 0],
            len(rows), len(cols), tol_aca)
        Ub, sb, Vb = recompress(Ua, Va, tol_aca)
        lowrank[(t, s)] = (Ub * sb[None, :], Vb)
        sv[(t, s)] = sb
    for (t, s) in dense:
        near[(t, s)] = entries(points, tree.indices(t), tree.indices(s), wavenumber, n)
    return HMatrix(tree, adm, dense, lowrank, near), sv


def truncate_h(h: HMatrix, sv, eps: float) -> HMatrix:
    """H-matrix whose blocks keep only the singular values > eps * sigma_1 of each block."""
    low = {}
    for b, (X, Y) in h.lowrank.items():
        s = sv[b]
        keep = int(np.sum(s > eps * s[0])) if len(s) else 0
        low[b] = (X[:, :keep], Y[:, :keep])
    return HMatrix(h.tree, h.adm, h.dense, low, h.near)


def h_matvec(h: HMatrix, x: np.ndarray) -> np.ndarray:
    """Algorithm 5 run on one thread: w|_tau += X_b (Y_b^* v|_sigma), then the dense blocks.
    x and the result are in original ordering (vector or n x R matrix)."""
    tree = h.tree
    xp = x[tree.perm]
    yp = np.zeros(xp.shape, dtype=np.complex128)
    for (t, s), (X, Y) in h.lowrank.items():
        bt, bs = tree.begin[t], tree.begin[s]
        yp[bt:bt + tree.size[t]] += X @ (Y.conj().T @ xp[bs:bs + tree.size[s]])
    for (t, s), D in h.near.items():
        bt, bs = tree.begin[t], tree.begin[s]
        yp[bt:bt + tree.size[t]] += D @ xp[bs:bs + tree.size[s]]
    y = np.empty_like(yp)
    y[tree.perm] = yp
    return y


def h_to_dense(h: HMatrix) -> np.ndarray:
    """Explicit assembly of A^H in original ordering (tiny N only)."""
    tree = h.tree
    A = np.zeros((tree.n, tree.n), dtype=np.complex128)
    for (t, s), (X, Y) in h.lowrank.items():
        A[np.ix_(tree.indices(t), tree.indices(s))] = X @ Y.conj().T
    for (t, s), D in h.near.items():
        A[np.ix_(tree.indices(t), tree.indices(s))] = D
    return A


# ----------------------------------------------------------------------------------------------
# Uniform compression (Algorithm 2) and the UH-matrix (Def. 2.4)
# ----------------------------------------------------------------------------------------------


class UHMatrix:
    """Row bases U_tau, column bases V_sigma, coefficients S_b (l_tau x l_sigma) and dense blocks.

    Also keeps, per cluster, all singular values of the stacked matrix X_tau (rows) or Y_sigma
    (columns) and the chosen rank, which the error bounds of Section 5 are written in."""

    def __init__(self, tree, adm, dense, U, V, S, near, row_sv, col_sv, F=None, pairs=None):
        self.tree = tree
        self.adm = adm
        self.dense = dense
        self.U = U  # {tau: (|tau| x l_tau)}
        self.V = V  # {sigma: (|sigma| x l_sigma)}
        self.S = S  # {(tau, sigma): (l_tau x l_sigma)}, the blocks stored dense
        self.near = near  # {(tau, sigma): (|tau| x |sigma|)}
        self.row_sv = row_sv  # {tau: all singular values of X_tau}
        self.col_sv = col_sv  # {sigma: all singular values of Y_sigma}
        # blocks stored factored (Section 4.2): {(tau, sigma): (S_X (l_tau x k_b), S_Y (l_sigma x k_b))}
        self.F = F if F is not None else {}
        # the coefficient pairs (S_X, S_Y) of Algorithm 2 (inner rank k_b of the fine block)
        self.pairs = pairs if pairs is not None else {}

    def counts(self) -> dict:
        """Stored element counts E_V, E_U, E_S (dense l_tau l_sigma, factored k_b (l_tau + l_sigma)),
        E_D, and K = sum of the inner ranks k_b of the factored blocks."""
        return dict(
            E_U=sum(u.size for u in self.U.values()),
            E_V=sum(v.size for v in self.V.values()),
            E_S=sum(s.size for s in self.S.values()) + sum(x.size + y.size for x, y in self.F.values()),
            E_D=sum(d.size for d in self.near.values()),
            K=sum(x.shape[1] for x, _ in self.F.values()))

    def coupling(self, b) -> np.ndarray:
        """S_b as a dense l_tau x l_sigma matrix, whichever form it is stored in."""
        if b in self.F:
            X, Y = self.F[b]
            return X @ Y.conj().T
        return self.S[b]

    def ranks(self):
        return ({t: u.shape[1] for t, u in self.U.items()},
                {s: v.shape[1] for s, v in self.V.items()})


def _rank_rule(s: np.ndarray, eps: float) -> int:
    """Reading R5: smallest l with sigma_{l+1} <= eps * sigma_1."""
    if len(s) == 0 or s[0] == 0.0:
        return 0
    return int(np.sum(s > eps * s[0]))


def _cluster_basis(factors, eps):
    """Lines 2-20 of Algorithm 2 for one cluster.

    factors: list of (F_b, G_b) with A-part F_b G_b^* (for rows: F = X_b, G = Y_b; for columns
    F = Y_b, G = X_b). Builds the stacked matrix F_tau = [F_b R_{G,b}^*]_b (eq. (4.2)), its SVD,
    the truncated basis, and for each block the coefficient factor
    S_b = Sigma(1:l,1:l) W(i:i+k_b, 1:l)^* (R_{G,b}^*)^{-1}.
    Returns (basis, [S_b], all singular values)."""
    cols, Rs = [], []
    for F, G in factors:
        _, R = np.linalg.qr(G)
        Rs.append(R)
        cols.append(F @ R.conj().T)
    Xt = np.concatenate(cols, axis=1)
    Uf, s, Wh = np.linalg.svd(Xt, full_matrices=False)
    ell = _rank_rule(s, eps)
    basis = Uf[:, :ell]
    W = Wh.conj().T
    out, i = [], 0
    for (F, G), R in zip(factors, Rs):
        kb = F.shape[1]
        Sx = np.diag(s[:ell]) @ W[i:i + kb, :ell].conj().T  # l x k_b
        i += kb
        # S_x <- S_x (R^*)^{-1}  <=>  R S_x^* = (old S_x)^*  (R upper triangular)
        if kb:
            Sx = np.linalg.solve(R, Sx.conj().T).conj().T
        out.append(Sx)
    return basis, out, s


def uniform_compression(h: HMatrix, eps: float) -> UHMatrix:
    """Algorithm 2: row bases from the row blocks, column bases from the column blocks,
    S_b = S_{X,b} S_{Y,b}^* (dense), dense blocks copied."""
    row, col = row_sets(h.adm)
    U, V, SX, SY, row_sv, col_sv = {}, {}, {}, {}, {}, {}
    for t in sorted(row):
        facs = [h.lowrank[(t, s)] for s in row[t]]  # (X_b, Y_b)
        U[t], parts, row_sv[t] = _cluster_basis(facs, eps)
        for s, P in zip(row[t], parts):
            SX[(t, s)] = P
    for s in sorted(col):
        facs = [(h.lowrank[(t, s)][1], h.lowrank[(t, s)][0]) for t in col[s]]  # (Y_b, X_b)
        V[s], parts, col_sv[s] = _cluster_basis(facs, eps)
        for t, P in zip(col[s], parts):
            SY[(t, s)] = P
    S = {b: SX[b] @ SY[b].conj().T for b in h.adm}
    pairs = {b: (SX[b], SY[b]) for b in h.adm}
    return UHMatrix(h.tree, h.adm, h.dense, U, V, S, dict(h.near), row_sv, col_sv, pairs=pairs)


def factor_coupling(uh: UHMatrix, eps: float, force: bool = False) -> UHMatrix:
    """Factored coefficient storage S_b = S_{X,b} S_{Y,b}^* (Section 4.2), reading R11.

    For each admissible block, the pair (S_X, S_Y) of Algorithm 2 (or, when the operator carries
    no pairs, (S_b, I)) is recompressed at eps as in Section 2.3 (recompress: QR of both factors,
    SVD of R_X R_Y^*, keep s_j > eps * s_1), giving S_X = Q_X W_k diag(s_1..s_k) and
    S_Y = Q_Y Z_k. The block is stored factored when k_b (l_tau + l_sigma) < l_tau l_sigma (always
    with force), else its dense S_b is kept unchanged. Bases and dense blocks are shared."""
    S, F = {}, {}
    for b, Sb in uh.S.items():
        lt, ls = Sb.shape
        if b in uh.pairs:
            X, Y = uh.pairs[b]
        else:
            X, Y = Sb, np.eye(ls, dtype=np.complex128)
        Ub, sb, Vb = recompress(X, np.conj(Y), eps)
        k = len(sb)
        if force or k * (lt + ls) < lt * ls:
            F[b] = (Ub * sb[None, :], Vb)
        else:
            S[b] = Sb
    return UHMatrix(uh.tree, uh.adm, uh.dense, uh.U, uh.V, S, uh.near, uh.row_sv, uh.col_sv,
                    F=F, pairs=uh.pairs)


def uh_matvec(uh: UHMatrix, x: np.ndarray) -> np.ndarray:
    """Algorithm 6 run on one thread (reading R6), x and result in original ordering.

    Phase 1: xhat_sigma = V_sigma^* x|_sigma, and for a factored block t_b = S_{Y,b}^* xhat_sigma.
    Coupling: yhat_tau = sum_{sigma in row(tau)} S_b xhat_sigma (dense S_b) or S_{X,b} t_b
    (factored). Phase 2: w|_tau += U_tau yhat_tau. Then w|_tau += A|_b x|_sigma for dense b."""
    tree = uh.tree
    xp = x[tree.perm]
    xhat = {}
    for s, V in uh.V.items():
        b = tree.begin[s]
        xhat[s] = V.conj().T @ xp[b:b + tree.size[s]]
    tb = {b: Y.conj().T @ xhat[b[1]] for b, (_, Y) in uh.F.items()}
    yhat = {}
    for (t, s), S in uh.S.items():
        contrib = S @ xhat[s]
        yhat[t] = contrib if t not in yhat else yhat[t] + contrib
    for (t, s), (X, _) in uh.F.items():
        contrib = X @ tb[(t, s)]
        yhat[t] = contrib if t not in yhat else yhat[t] + contrib
    yp = np.zeros(xp.shape, dtype=np.complex128)
    for t, U in uh.U.items():
        b = tree.begin[t]
        yp[b:b + tree.size[t]] += U @ yhat[t]
    for (t, s), D in uh.near.items():
        bt, bs = tree.begin[t], tree.begin[s]
        yp[bt:bt + tree.size[t]] += D @ xp[bs:bs + tree.size[s]]
    y = np.empty_like(yp)
    y[tree.perm] = yp
    return y


def uh_to_dense(uh: UHMatrix) -> np.ndarray:
    """Explicit assembly of A^UH in original ordering, block by block (tiny N only)."""
    tree = uh.tree
    A = np.zeros((tree.n, tree.n), dtype=np.complex128)
    for (t, s), S in uh.S.items():
        A[np.ix_(tree.indices(t), tree.indices(s))] = uh.U[t] @ S @ uh.V[s].conj().T
    for (t, s), (X, Y) in uh.F.items():
        A[np.ix_(tree.indices(t), tree.indices(s))] = (uh.U[t] @ X) @ (uh.V[s] @ Y).conj().T
    for (t, s), D in uh.near.items():
        A[np.ix_(tree.indices(t), tree.indices(s))] = D
    return A


# ----------------------------------------------------------------------------------------------
# Error quantities of Section 5 and the storage bounds of Lemma 2.6
# ----------------------------------------------------------------------------------------------


def theorem51_bound(uh: UHMatrix) -> float:
    """Right-hand side of eq. (5.1): sqrt(2) * sqrt(sum_tau e_tau^2 + sum_sigma e_sigma^2), with
    e_tau = |A_tau - U U^* A_tau|_2 = sigma_{l_tau+1}(X_tau) (0 if the basis has full rank).

    Uses that A_tau = X_tau Q_tau^* with Q_tau orthonormal (eq. (4.2)), so the singular values
    of A_tau are those of X_tau."""
    tot = 0.0
    for t, s in uh.row_sv.items():
        ell = uh.U[t].shape[1]
        tot += s[ell] ** 2 if ell < len(s) else 0.0
    for c, s in uh.col_sv.items():
        ell = uh.V[c].shape[1]
        tot += s[ell] ** 2 if ell < len(s) else 0.0
    return math.sqrt(2.0) * math.sqrt(tot)


def frobenius_tail(uh: UHMatrix) -> float:
    """sum_tau sum_{i > l_tau} sigma_i(X_tau)^2 + sum_sigma sum_{i > l_sigma} sigma_i(Y_sigma)^2,
    the right-hand side of the Frobenius estimate at the start of Section 5."""
    tot = 0.0
    for t, s in uh.row_sv.items():
        tot += float(np.sum(s[uh.U[t].shape[1]:] ** 2))
    for c, s in uh.col_sv.items():
        tot += float(np.sum(s[uh.V[c].shape[1]:] ** 2))
    return tot


def storage_bounds(h: HMatrix, uh: UHMatrix) -> dict:
    """Lemma 2.6, eqs. (2.2a) and (2.2b), for the admissible part (with I = J, one tree)."""
    tree = h.tree
    csp = sparsity_constant(h.adm)
    kmax = max([X.shape[1] for X, _ in h.lowrank.values()] + [0])
    lu, lv = uh.ranks()
    lmax = max(list(lu.values()) + list(lv.values()) + [0])
    L = tree.depth()
    n = tree.n
    nmin = min(tree.size)
    return dict(
        H=csp * kmax * (L * n + L * n),
        UH=lmax * (L * n + L * n) + lmax ** 2 * 2 * csp * n / nmin,
        csp=csp, kmax=kmax, lmax=lmax, L=L, nmin=nmin)


def power_iteration_norm(apply, apply_adj, n: int, iters: int = 30, seed: int = 1) -> float:
    """Estimate |B|_2 by power iteration on B^* B (the accuracy check of Section 6)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        w = apply_adj(apply(v))
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        est = math.sqrt(nw)
        v = w / nw
    return est


# ----------------------------------------------------------------------------------------------
# Convenience: the whole construction for one workload
# ----------------------------------------------------------------------------------------------


def build_operators(points, wavenumber, leaf, eta, eps, tol_aca, strong: bool = False):
    """points -> cluster tree -> block tree -> ACA H-matrix at tol_aca -> (H at eps, UH at eps).

    The H form used for comparison keeps each block's singular values above eps * sigma_1; the UH
    form is Algorithm 2 applied to the tol_aca blocks. strong: strong admissibility (eq. (3.2))."""
    tree = ClusterTree(points, leaf)
    adm, dense = block_tree(tree, eta, strong)
    h_fine, sv = build_h(points, tree, adm, dense, wavenumber, tol_aca)
    uh = uniform_compression(h_fine, eps)
    h = truncate_h(h_fine, sv, eps)
    return tree, h_fine, h, uh

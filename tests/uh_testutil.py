"""Test helpers: flatten oracle operators into the arrays of the C descriptors, and cache
oracle-built operators per workload within one test session."""
from __future__ import annotations

import functools

import numpy as np

from oracle import uh_oracle as O


def _tree_arrays(tree):
    return dict(n=tree.n, perm=np.asarray(tree.perm, np.int64),
                cl_begin=np.asarray(tree.begin, np.int64), cl_size=np.asarray(tree.size, np.int64))


def _pack(mats: dict, ncl: int):
    rank = np.zeros(ncl, np.int32)
    off = np.zeros(ncl, np.int64)
    parts, pos = [], 0
    for c in sorted(mats):
        M = mats[c]
        rank[c] = M.shape[1]
        off[c] = pos
        parts.append(M.ravel(order="F"))
        pos += M.size
    data = np.concatenate(parts) if parts else np.zeros(0, np.complex128)
    return rank, off, data


def _dense_arrays(near: dict):
    keys = sorted(near)
    offs, parts, pos = [], [], 0
    for b in keys:
        offs.append(pos)
        parts.append(near[b].ravel(order="F"))
        pos += near[b].size
    return dict(dense_row=np.array([b[0] for b in keys], np.int32),
                dense_col=np.array([b[1] for b in keys], np.int32),
                D_off=np.array(offs, np.int64),
                D_data=np.concatenate(parts) if parts else np.zeros(0, np.complex128))


def uh_arrays(uh: O.UHMatrix, dtype=np.complex128) -> dict:
    tree = uh.tree
    a = _tree_arrays(tree)
    a["row_rank"], a["row_off"], a["U_data"] = _pack(uh.U, tree.n_clusters)
    a["col_rank"], a["col_off"], a["V_data"] = _pack(uh.V, tree.n_clusters)
    keys = sorted(list(uh.S) + list(uh.F))
    offs, parts, ranks, pos = [], [], [], 0
    for b in keys:
        offs.append(pos)
        if b in uh.F:  # factored: S_X then S_Y, both column-major
            X, Y = uh.F[b]
            parts += [X.ravel(order="F"), Y.ravel(order="F")]
            pos += X.size + Y.size
            ranks.append(X.shape[1])
        else:
            parts.append(uh.S[b].ravel(order="F"))
            pos += uh.S[b].size
            ranks.append(-1)
    a["adm_row"] = np.array([b[0] for b in keys], np.int32)
    a["adm_col"] = np.array([b[1] for b in keys], np.int32)
    a["S_off"] = np.array(offs, np.int64)
    a["S_data"] = np.concatenate(parts) if parts else np.zeros(0, np.complex128)
    a["S_rank"] = np.array(ranks, np.int32) if uh.F else None
    a.update(_dense_arrays(uh.near))
    for k in ("U_data", "V_data", "S_data", "D_data"):
        a[k] = a[k].astype(dtype)
    return a


def h_arrays(h: O.HMatrix, dtype=np.complex128) -> dict:
    tree = h.tree
    a = _tree_arrays(tree)
    keys = sorted(h.lowrank)
    xo, yo, xs, ys, ranks = [], [], [], [], []
    px = py = 0
    for b in keys:
        X, Y = h.lowrank[b]
        xo.append(px)
        yo.append(py)
        xs.append(X.ravel(order="F"))
        ys.append(Y.ravel(order="F"))
        px += X.size
        py += Y.size
        ranks.append(X.shape[1])
    a["adm_row"] = np.array([b[0] for b in keys], np.int32)
    a["adm_col"] = np.array([b[1] for b in keys], np.int32)
    a["adm_rank"] = np.array(ranks, np.int32)
    a["X_off"] = np.array(xo, np.int64)
    a["Y_off"] = np.array(yo, np.int64)
    a["X_data"] = (np.concatenate(xs) if xs else np.zeros(0)).astype(dtype)
    a["Y_data"] = (np.concatenate(ys) if ys else np.zeros(0)).astype(dtype)
    a.update(_dense_arrays(h.near))
    a["D_data"] = a["D_data"].astype(dtype)
    return a


@functools.lru_cache(maxsize=8)
def oracle_ops(n: int, wavenumber: float, leaf: int, eta: float, eps: float, tol_aca: float,
               axes=(1.0, 1.0, 1.0), noise: float = 0.0, seed: int = 0, strong: bool = False):
    """(points, tree, h_fine, h, uh) for a Fibonacci sphere/ellipsoid workload, built once."""
    from paper_2405_15573_gb300 import inputs as I
    if axes == (1.0, 1.0, 1.0) and not noise:
        pts = I.fibonacci_sphere(n)
    else:
        pts = I.ellipsoid_points(n, axes, noise, seed)
    tree, hf, h, uh = O.build_operators(pts, wavenumber, leaf, eta, eps, tol_aca, strong)
    return pts, tree, hf, h, uh


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stored_c64(uh: O.UHMatrix) -> O.UHMatrix:
    """The operator a complex64 op stores: every entry of U, V, S and the dense blocks rounded to
    complex64 (round to nearest), held in complex128 so the oracle applies it in FP64."""
    r = lambda d: {k: v.astype(np.complex64).astype(np.complex128) for k, v in d.items()}  # noqa: E731
    F = {b: tuple(m.astype(np.complex64).astype(np.complex128) for m in xy) for b, xy in uh.F.items()}
    return O.UHMatrix(uh.tree, uh.adm, uh.dense, r(uh.U), r(uh.V), r(uh.S), r(uh.near),
                      uh.row_sv, uh.col_sv, F=F)

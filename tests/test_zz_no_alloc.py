"""uh_block_apply_noalloc (the allocation-free block product) against uh_matvec.

Callers that cannot call cudaMalloc (code inside a CUDA-graph stream capture, or code held to its
own memory arena) use uh_block_apply_noalloc, whose intermediate vectors sit in a fixed device
array inside the library. This checks it against the ordinary entry point: a UH operator whose
only admissible block is tau x sigma = [0, m) x [m, m+n), with zero dense blocks elsewhere, so
that uh_matvec of [0; x] gives U S V^* x in its first m entries. Two calls in a row must both
agree, since every call reuses the same fixed array.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def _single_block_op(U, S, V, prec):
    from paper_2405_15573_gb300 import uh
    m, lt = U.shape
    n, ls = V.shape
    N = m + n
    a = dict(n=N, perm=np.arange(N, dtype=np.int64),
             cl_begin=np.array([0, 0, m], np.int64), cl_size=np.array([N, m, n], np.int64),
             row_rank=np.array([0, lt, 0], np.int32), row_off=np.zeros(3, np.int64),
             U_data=U.ravel(order="F"), col_rank=np.array([0, 0, ls], np.int32),
             col_off=np.zeros(3, np.int64), V_data=V.ravel(order="F"),
             adm_row=np.array([1], np.int32), adm_col=np.array([2], np.int32),
             S_off=np.zeros(1, np.int64), S_data=S.ravel(order="F"))
    blocks = [(1, 1), (2, 1), (2, 2)]
    sizes = {1: m, 2: n}
    offs, pos = [], 0
    for t, s in blocks:
        offs.append(pos)
        pos += sizes[t] * sizes[s]
    a.update(dense_row=np.array([b[0] for b in blocks], np.int32),
             dense_col=np.array([b[1] for b in blocks], np.int32),
             D_off=np.array(offs, np.int64), D_data=np.zeros(pos, np.complex128))
    return uh.UHOp.from_arrays(a, prec)


@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c64", 5e-6)])
def test_noalloc_matches_uh_matvec_twice(prec, tol):
    import torch
    from paper_2405_15573_gb300 import uh
    rng = np.random.default_rng(11)
    m, n, lt, ls = 300, 517, 37, 53
    U, S, V = _rand(rng, m, lt), _rand(rng, lt, ls), _rand(rng, n, ls)
    op = _single_block_op(U, S, V, prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64

    def colmajor(A, ld):
        t = torch.zeros((A.shape[1], ld), dtype=dt, device="cuda")
        t[:, :A.shape[0]] = torch.from_numpy(A.T.copy()).to(dt)
        return t.T[:A.shape[0]]  # column-major view with leading dimension ld

    Ud, Sd, Vd = colmajor(U, m + 5), colmajor(S, lt), colmajor(V, n + 3)
    for call in range(2):
        x = _rand(rng, n)
        xd = torch.from_numpy(x).to("cuda", dt)
        y = torch.full((m,), complex(float("nan"), float("nan")), dtype=dt, device="cuda")
        uh.block_apply_noalloc(Ud, Sd, Vd, xd, y)
        xfull = torch.zeros(m + n, dtype=dt, device="cuda")
        xfull[m:] = xd
        yfull = op.matvec(xfull)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.complex128)
        ref = yfull[:m].cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref), f"call {call}"
        assert np.linalg.norm(got - U @ (S @ (V.conj().T @ x))) <= 10 * tol * np.linalg.norm(ref)


def test_noalloc_rejects_ranks_beyond_the_fixed_array():
    import torch
    from paper_2405_15573_gb300 import uh
    m = n = 300
    z = torch.zeros(m, 257, dtype=torch.complex128, device="cuda")
    s = torch.zeros(257, 257, dtype=torch.complex128, device="cuda")
    x = torch.zeros(n, dtype=torch.complex128, device="cuda")
    y = torch.zeros(m, dtype=torch.complex128, device="cuda")
    rc = uh.lib.uh_block_apply_noalloc(m, n, 257, 257, z.data_ptr(), m, s.data_ptr(), 257, z.data_ptr(), n,
                                       x.data_ptr(), y.data_ptr(), uh.UH_PREC_C128, None)
    assert rc == uh.UH_EINVAL
    assert "256" in uh.lib.uh_last_error().decode()

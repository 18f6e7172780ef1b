"""GPU parity of the multi-RHS product uh_matmat against the FP64 oracle, through the C ABI.

The operator is built by the oracle and handed to uh_create with a tensor-core precision, so the
two sides apply the same operator; the GPU side stores it in complex64 and multiplies on the
tensor cores, either with TF32 operands (10-bit mantissa, rounded to nearest) or with each FP32
value split into BF16 hi + lo (3 products), accumulating in FP32. Each column is compared with
the oracle's Algorithm 6 product of that column. Tolerance per column (relative 2-norm): 1e-3
for both, the bound the multi-RHS path is held to; BF16x3 is also held to 1e-4, since its
operand error (about 2^-16 relative after the split) is far below TF32's 2^-11.
"""
import functools

import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr, uh_arrays

pytestmark = pytest.mark.gpu

WORKLOADS = {
    "sphere2048": (2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0),
    "ellipsoid1000": (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01),
}
TOL = {"tf32": 1e-3, "bf16x3": 1e-4}


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


def _X(n, nrhs, seed=0):
    return np.stack([I.complex_normal(n, seed + j) for j in range(nrhs)], axis=1)


@functools.lru_cache(maxsize=None)
def _reference(name, nrhs):
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    X = _X(tree.n, nrhs)
    return X, np.stack([O.uh_matvec(uh, X[:, j]) for j in range(nrhs)], axis=1)


@functools.lru_cache(maxsize=None)
def _op(U, name, precision):
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    return U.UHOp.from_arrays(uh_arrays(uh), precision)


def _colmajor(torch, X, ld=None, dtype=None):
    """n x nrhs column-major CUDA tensor (leading dimension ld >= n) holding X."""
    n, r = X.shape
    ld = ld or n
    buf = torch.full((r, ld), complex(float("nan"), float("nan")), dtype=dtype or torch.complex64, device="cuda")
    view = buf[:, :n].T
    view.copy_(torch.from_numpy(X).to(view.dtype))
    return view


def _poisoned(torch, n, r, ld=None, dtype=None):
    ld = ld or n
    return torch.full((r, ld), complex(float("nan"), float("nan")), dtype=dtype or torch.complex64,
                      device="cuda")[:, :n].T


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("mode", ["tf32", "bf16x3"])
@pytest.mark.parametrize("nrhs", [1, 7, 64, 70])
def test_matmat_tensor_parity(U, name, mode, nrhs):
    import torch
    X, Yref = _reference(name, nrhs)
    op = _op(U, name, "c64_" + mode)
    Xd = _colmajor(torch, X)
    Yd = _poisoned(torch, *X.shape)
    op.matmat(Xd, Yd, mode=mode)
    op.check()
    Y = Yd.cpu().numpy().astype(np.complex128)
    assert np.isfinite(Y).all()
    errs = [relerr(Y[:, j], Yref[:, j]) for j in range(nrhs)]
    assert max(errs) <= TOL[mode], (max(errs), errs[:4])
    assert max(errs) <= 1e-3


def test_matmat_leading_dimensions_and_repeat(U):
    """ldx, ldy > n (padding left untouched), two passes of 64, bitwise repeatable."""
    import torch
    X, Yref = _reference("ellipsoid1000", 70)
    op = _op(U, "ellipsoid1000", "c64_bf16x3")
    n = X.shape[0]
    Xd = _colmajor(torch, X, ld=n + 5)
    Yd = _poisoned(torch, n, 70, ld=n + 3)
    op.matmat(Xd, Yd, mode="bf16x3")
    Y1 = Yd.cpu().numpy().copy()
    op.matmat(Xd, Yd, mode="bf16x3")
    op.check()
    Y2 = Yd.cpu().numpy()
    assert np.array_equal(Y1, Y2)
    pad = Yd.T.contiguous()  # noqa: F841  (the view itself excludes the padding rows)
    base = Yd.as_strided((70, n + 3), (n + 3, 1)).cpu().numpy()
    assert np.isnan(base[:, n:]).all()  # padding rows of Y untouched
    assert max(relerr(Y2[:, j].astype(np.complex128), Yref[:, j]) for j in range(70)) <= TOL["bf16x3"]


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_matmat_simt_equals_matvec_columns(U, prec):
    import torch
    X, Yref = _reference("sphere2048", 3)
    op = _op(U, "sphere2048", prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    Xd = _colmajor(torch, X, dtype=dt)
    Yd = _poisoned(torch, X.shape[0], 3, dtype=dt)
    op.matmat(Xd, Yd, mode="simt")
    for j in range(3):
        yj = op.matvec(Xd[:, j].contiguous())
        assert torch.equal(yj, Yd[:, j])
    op.check()


def test_tensor_modes_agree_with_c64_matvec(U):
    """The tensor-core product and the CUDA-core complex64 product of one column agree to the
    TF32 rounding (the layouts of the two programs are independent)."""
    import torch
    X, Yref = _reference("sphere2048", 1)
    for mode in ("tf32", "bf16x3"):
        op = _op(U, "sphere2048", "c64_" + mode)
        Xd = _colmajor(torch, X)
        Yd = _poisoned(torch, X.shape[0], 1)
        op.matmat(Xd, Yd, mode=mode)
        y = op.matvec(Xd[:, 0].contiguous())
        op.check()
        assert relerr(Yd[:, 0].cpu().numpy().astype(np.complex128), y.cpu().numpy().astype(np.complex128)) <= TOL[mode]


def test_matmat_argument_errors(U):
    import torch
    X, _ = _reference("ellipsoid1000", 1)
    n = X.shape[0]
    op64 = _op(U, "ellipsoid1000", "c64")
    opt = _op(U, "ellipsoid1000", "c64_tf32")
    Xd = _colmajor(torch, X)
    Yd = _poisoned(torch, n, 1)
    with pytest.raises(U.UHError) as e:
        op64.matmat(Xd, Yd, mode="tf32")  # op without the tensor-core copy
    assert e.value.code == U.UH_EINVAL
    with pytest.raises(U.UHError) as e:
        opt.matmat(Xd, Yd, mode="bf16x3")  # the other tensor-core mode
    assert e.value.code == U.UH_EINVAL
    with pytest.raises(U.UHError) as e:
        opt.matmat(Xd, Xd, mode="tf32")  # X and Y overlap
    assert e.value.code == U.UH_EINVAL
    rc = U.lib.uh_matmat(opt.handle, 0, Xd.data_ptr(), n, Yd.data_ptr(), n, U.UH_MM_TF32, None)
    assert rc == U.UH_EINVAL
    rc = U.lib.uh_matmat(opt.handle, 1, Xd.data_ptr(), n - 1, Yd.data_ptr(), n, U.UH_MM_TF32, None)
    assert rc == U.UH_EINVAL
    st = opt.stats()
    assert st["matmat_mode"] == U.UH_MM_TF32 and st["panel_items"] > 0
    assert op64.stats()["matmat_mode"] == -1


@pytest.mark.parametrize("case", ["one_cta", "two_ctas", "factored"])
def test_multi_rhs_simt_product_equals_matvec_columns(U, case):
    """After uh_reserve, the CUDA-core multi-RHS product runs 4 (one CTA per SM) or 2 (two CTAs
    per SM) right-hand sides per pass over the operator. Each column's arithmetic is that of its
    single product, so every column equals uh_matvec bit for bit; leading dimensions above n."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["ellipsoid1000"])
    if case == "factored":
        uh = O.factor_coupling(uh, 3e-5)
    params = U.PackParams(0, 0, 0, 0, 2) if case == "two_ctas" else None
    op = U.UHOp.from_arrays(uh_arrays(uh), "c64", params)
    op.reserve(8)
    nrhs = 9  # passes of 4 + 4 + 1 (one CTA per SM) or 2 + 2 + 2 + 2 + 1 (two)
    X = _X(tree.n, nrhs, seed=50)
    Xd = _colmajor(torch, X, ld=tree.n + 3)
    Yd = _poisoned(torch, tree.n, nrhs, ld=tree.n + 5)
    op.matmat(Xd, Yd, mode="simt")
    for j in range(nrhs):
        yj = op.matvec(Xd[:, j].contiguous())
        assert torch.equal(yj, Yd[:, j]), j
    op.check()
    Y = Yd.cpu().numpy().astype(np.complex128)
    for j in range(nrhs):
        assert relerr(Y[:, j], O.uh_matvec(uh, X[:, j])) <= 5e-6
    st = op.stats()
    assert st["pack_ctas_per_sm"] == (2 if case == "two_ctas" else 1)
    op.close()


def test_h_form_multi_rhs_simt_product(U):
    """The H form (Algorithm 5) in passes of 4 right-hand sides after h_reserve: every column equals
    h_matvec bit for bit and the oracle's H product to the complex64 tolerance."""
    import torch
    from tests.uh_testutil import h_arrays
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.HOp.from_arrays(h_arrays(h), "c64")
    op.reserve(4)
    X = _X(tree.n, 6, seed=70)
    Xd = _colmajor(torch, X)
    Yd = _poisoned(torch, tree.n, 6)
    op.matmat(Xd, Yd, mode="simt")
    for j in range(6):
        assert torch.equal(op.matvec(Xd[:, j].contiguous()), Yd[:, j]), j
    op.check()
    Y = Yd.cpu().numpy().astype(np.complex128)
    for j in range(6):
        assert relerr(Y[:, j], O.h_matvec(h, X[:, j])) <= 5e-6
    op.close()

"""GPU parity of the extended-precision product uh_matvec_mixed: the complex64-stored operator
applied to a complex128 x with every product and sum carried in FP32 pairs (about 48 significant
bits). The oracle applies the same stored operator (its entries rounded to complex64) in FP64,
so only rounding in the kernel's arithmetic differs; the bound is 1e-11 relative 2-norm and
element-wise against the largest output, four to five orders of magnitude below the FP32
accumulation of uh_matvec."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.test_gpu_matvec import WORKLOADS
from tests.uh_testutil import oracle_ops, relerr, stored_c64, uh_arrays

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-11


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


def _mixed(op, x):
    import torch
    xt = torch.from_numpy(x).to("cuda", torch.complex128)
    y = torch.full_like(xt, complex(float("nan"), float("nan")))
    op.matvec_mixed(xt, y)
    op.check()
    return y.cpu().numpy()


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("prec", ["c64", "c64_bf16x3"])
def test_mixed_parity_with_stored_operator(U, name, prec):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    op = U.UHOp.from_arrays(uh_arrays(uh), prec)
    stored = stored_c64(uh)
    for seed in (0, 1):
        x = I.complex_normal(tree.n, seed)
        yref = O.uh_matvec(stored, x)
        y = _mixed(op, x)
        assert np.isfinite(y).all()
        err = relerr(y, yref)
        assert err <= TOL_MIXED, err
        assert np.max(np.abs(y - yref)) <= TOL_MIXED * np.max(np.abs(yref))
    # the FP32-accumulated product of the same op is far less accurate against the same truth
    y32 = op.matvec(torch.from_numpy(x).to("cuda", torch.complex64)).cpu().numpy()
    assert relerr(y32.astype(np.complex128), yref) > 1e3 * err


def test_mixed_small_ragged_and_all_dense(U):
    for n, leaf in ((1, 8), (40, 64), (97, 16)):
        pts = I.fibonacci_sphere(n)
        tree, hf, h, uh = O.build_operators(pts, 3.0, leaf, 1.0, 1e-6, 1e-8)
        op = U.UHOp.from_arrays(uh_arrays(uh), "c64")
        x = I.complex_normal(n, 2)
        assert relerr(_mixed(op, x), O.uh_matvec(stored_c64(uh), x)) <= TOL_MIXED


def test_mixed_rank_zero_bases(U):
    pts = I.fibonacci_sphere(512)
    tree = O.ClusterTree(pts, 16)
    adm, dense = O.block_tree(tree, 1.0)
    hf, _ = O.build_h(pts, tree, adm, dense, 2.0, 1e-8)
    uh = O.uniform_compression(hf, 1.0)
    op = U.UHOp.from_arrays(uh_arrays(uh), "c64")
    x = I.complex_normal(512, 0)
    assert relerr(_mixed(op, x), O.uh_matvec(stored_c64(uh), x)) <= TOL_MIXED


def test_mixed_deterministic_and_interleaved_with_matvec(U):
    """Repeated extended-precision products are bitwise equal, also when ordinary complex64
    products of the same op run in between (they share the op's counters, not its vectors)."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c64")
    x = torch.from_numpy(I.complex_normal(tree.n, 3)).to("cuda", torch.complex128)
    x32 = x.to(torch.complex64)
    ys, y32s = [], []
    for _ in range(4):
        ys.append(op.matvec_mixed(x).clone())
        y32s.append(op.matvec(x32).clone())
    torch.cuda.synchronize()
    op.check()
    for y in ys[1:]:
        assert torch.equal(y.view(torch.float64), ys[0].view(torch.float64))
    for y in y32s[1:]:
        assert torch.equal(y.view(torch.float32), y32s[0].view(torch.float32))


def test_mixed_rejects_complex128_op(U):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["ellipsoid1000"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128")
    x = torch.zeros(tree.n, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    rc = U.lib.uh_matvec_mixed(op.handle, x.data_ptr(), y.data_ptr(), None)
    assert rc == U.UH_EINVAL

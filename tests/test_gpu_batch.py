"""GPU parity of the batched product (uh_batch_*): several independent operators of uneven size in
one launch, each compared with the FP64 oracle's Algorithm 6 product of its own vector and with
the same operator applied alone (uh_matvec). Tolerances as for the single product: relative
2-norm 1e-12 (complex128) and 5e-6 (complex64) per operator."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr, uh_arrays

pytestmark = pytest.mark.gpu

CASES = [(512, 3.0, 16, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0),
         (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01),
         (97, 3.0, 16, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0),
         (40, 3.0, 64, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0),
         (2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0)]
TOL = {"c128": 1e-12, "c64": 5e-6}


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batch_matches_oracle_and_single(U, prec):
    import torch
    ops = [oracle_ops(*c)[4] for c in CASES]
    arrays = [uh_arrays(op) for op in ops]
    batch = U.UHBatch.from_arrays(arrays, prec)
    off = batch.offsets
    assert off[-1] == sum(op.tree.n for op in ops)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    xs = [I.complex_normal(op.tree.n, 10 + k) for k, op in enumerate(ops)]
    x = torch.from_numpy(np.concatenate(xs)).to("cuda", dt)
    y = torch.full_like(x, complex(float("nan"), float("nan")))
    batch.matvec(x, y)
    batch.check()
    yb = y.cpu().numpy().astype(np.complex128)
    y2 = batch.matvec(x).cpu().numpy().astype(np.complex128)
    assert np.array_equal(yb, y2)  # bitwise repeatable
    for k, op in enumerate(ops):
        part = yb[off[k]:off[k + 1]]
        assert np.isfinite(part).all()
        assert relerr(part, O.uh_matvec(op, xs[k])) <= TOL[prec], k
        single = U.UHOp.from_arrays(arrays[k], prec)
        ys = single.matvec(torch.from_numpy(xs[k]).to("cuda", dt)).cpu().numpy().astype(np.complex128)
        single.check()
        assert relerr(part, ys) <= TOL[prec], k
    st = batch.stats()
    assert st["n"] == off[-1]
    assert st["E_D"] == sum(op.counts()["E_D"] for op in ops)
    assert st["n_launches"] == 1
    batch.close()

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


TUNER_PARAMS = [(16384, 0, 0, 0, 0), (32768, 0, 0, 0, 0), (0, 1024, 0, 0, 0), (0, 16384, 0, 0, 0),
                (0, 0, 12288, 0, 0), (0, 0, 196608, 0, 0), (0, 0, 0, 32768, 0), (0, 0, 0, 524288, 0),
                (16384, 16384, 196608, 524288, 0), (0, 0, 0, 0, 2), (16384, 1024, 12288, 32768, 2)]


@pytest.mark.parametrize("params", TUNER_PARAMS)
def test_batch_with_every_tuner_choice(U, params):
    """Every packing the autotuner can choose gives the same per-operator products (complex64)."""
    import torch
    ops = [oracle_ops(*c)[4] for c in CASES]
    arrays = [uh_arrays(op) for op in ops]
    batch = U.UHBatch.from_arrays(arrays, "c64", U.PackParams(*params))
    st = batch.stats()
    expect = [v if v else d for v, d in zip(params, (65536, 4096, 49152, 131072, 1))]
    if expect[4] == 2:
        expect[0] = min(expect[0], 24576)  # the two-CTA geometry's largest tile
    assert [st["pack_tile_bytes"], st["pack_item_cost"], st["pack_chunk_cost"], st["pack_pool_unit"],
            st["pack_ctas_per_sm"]] == expect
    off = batch.offsets
    xs = [I.complex_normal(op.tree.n, 10 + k) for k, op in enumerate(ops)]
    x = torch.from_numpy(np.concatenate(xs)).to("cuda", torch.complex64)
    y = batch.matvec(x)
    batch.check()
    yb = y.cpu().numpy().astype(np.complex128)
    for k, op in enumerate(ops):
        assert relerr(yb[off[k]:off[k + 1]], O.uh_matvec(op, xs[k])) <= TOL["c64"], k
    batch.close()


def test_autotuner_picks_a_candidate_and_stays_correct(U):
    """uh_batch_tune times candidate packings of the set and returns one of them; the batch
    created with its choice is as correct as the default one and no slower than it was timed."""
    import torch
    ops = [oracle_ops(*c)[4] for c in CASES]
    arrays = [uh_arrays(op) for op in ops]
    built = [U.uh_desc_from_arrays(a) for a in arrays]
    descs = [d for d, _ in built]
    best, best_ms, default_ms = U.UHBatch.tune(descs, "c64", sample=0, reps=10)
    assert best.ctas_per_sm in (0, 1, 2)
    assert best.tile_bytes in (16384, 32768, 65536)
    assert best.item_cost in (1024, 4096, 16384)
    assert best.chunk_cost in (12288, 49152, 196608)
    assert best.pool_unit in (32768, 131072, 524288)
    assert 0 < best_ms <= default_ms
    batch = U.UHBatch(descs, "c64", best)
    off = batch.offsets
    xs = [I.complex_normal(op.tree.n, 30 + k) for k, op in enumerate(ops)]
    y = batch.matvec(torch.from_numpy(np.concatenate(xs)).to("cuda", torch.complex64))
    batch.check()
    yb = y.cpu().numpy().astype(np.complex128)
    for k, op in enumerate(ops):
        assert relerr(yb[off[k]:off[k + 1]], O.uh_matvec(op, xs[k])) <= TOL["c64"], k
    batch.close()


@pytest.mark.parametrize("name", ["sphere2048", "ellipsoid1000"])
def test_two_ctas_per_sm_op_parity(U, name):
    """A single operator packed for two CTAs per SM (uh_create_ex): the product, the extended-
    precision product and the factored form agree with the oracle; two calls are bitwise equal."""
    import torch
    from tests.test_gpu_matvec import WORKLOADS
    from tests.uh_testutil import stored_c64
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    for arrays, ref in ((uh_arrays(uh), uh), (uh_arrays(O.factor_coupling(uh, 3 * WORKLOADS[name][4])), None)):
        if ref is None:
            ref = O.factor_coupling(uh, 3 * WORKLOADS[name][4])
        op = U.UHOp.from_arrays(arrays, "c64", U.PackParams(0, 0, 0, 0, 2))
        st = op.stats()
        assert st["pack_ctas_per_sm"] == 2 and st["pack_tile_bytes"] == 24576
        x = I.complex_normal(tree.n, 40)
        xt = torch.from_numpy(x).to("cuda", torch.complex64)
        y1, y2 = op.matvec(xt), op.matvec(xt)
        op.check()
        assert torch.equal(y1, y2)
        assert relerr(y1.cpu().numpy().astype(np.complex128), O.uh_matvec(stored_c64(ref), x)) <= TOL["c64"]
        x2 = torch.from_numpy(x).to("cuda")
        ym = op.matvec_mixed(x2)
        op.check()
        assert relerr(ym.cpu().numpy(), O.uh_matvec(stored_c64(ref), x)) <= 1e-11
        op.close()


def test_two_ctas_per_sm_complex128_parity(U):
    """A complex128 program on two CTAs per SM: the product agrees with the oracle to 1e-12."""
    import torch
    from tests.test_gpu_matvec import WORKLOADS
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["ellipsoid1000"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128", U.PackParams(0, 0, 0, 0, 2))
    assert op.stats()["pack_ctas_per_sm"] == 2
    x = I.complex_normal(tree.n, 41)
    y = op.matvec(torch.from_numpy(x).to("cuda"))
    op.check()
    assert relerr(y.cpu().numpy(), O.uh_matvec(uh, x)) <= TOL["c128"]
    op.close()

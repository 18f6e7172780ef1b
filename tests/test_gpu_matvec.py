"""GPU parity of the single-RHS UH and H products against the FP64 oracle, through the C ABI.

The operator data are built by the oracle and handed to uh_create / h_create, so both sides
apply the same operator and only the summation order (c128) or the storage rounding (c64)
differs. Tolerances: relative 2-norm 1e-12 for complex128, 5e-6 for complex64 (FP32
accumulation), and element-wise |y_gpu - y_ref| <= tol * max|y_ref|.
"""
import math

import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import h_arrays, oracle_ops, relerr, uh_arrays

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 5e-6}


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


def _run(op, x, torch):
    xt = torch.from_numpy(x).to("cuda", torch.complex128 if op.c128 else torch.complex64)
    y = torch.full_like(xt, complex(float("nan"), float("nan")))  # poisoned output
    op.matvec(xt, y)
    op.check()  # raises if a bounded device-side wait ran out
    return y.cpu().numpy().astype(np.complex128)


def _check(y, yref, tol):
    assert np.isfinite(y).all()
    assert relerr(y, yref) <= tol
    assert np.max(np.abs(y - yref)) <= tol * np.max(np.abs(yref)) * 10


WORKLOADS = {
    # parity case: unit sphere N = 2048, k = 4, leaf 32, eta 1, eps 1e-6, ACA 1e-8
    "sphere2048": (2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0),
    # ragged: N not a power of two, noisy ellipsoid, leaf 24 (odd leaf sizes, uneven levels)
    "ellipsoid1000": (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01),
    # the same ellipsoid under strong admissibility (eq. (3.2)): a finer partition
    "ellipsoid1000_strong": (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01, 0, True),
}


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_calls_on_two_streams_run_in_call_order(U, prec):
    """Products of one op issued alternately on two streams, with no synchronisation between the
    streams and the first stream held back by a sleep kernel, equal bit for bit the same products
    issued on one stream: the library runs calls on one op in the order they are made (they share
    the op's scratch and per-call counters)."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), prec)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    xs = [torch.from_numpy(I.complex_normal(tree.n, 100 + k)).to("cuda", dt) for k in range(8)]
    ref = []
    for x in xs:
        y = torch.empty_like(x)
        op.matvec(x, y)
        ref.append(y)
    ys = [torch.full_like(x, complex(float("nan"), float("nan"))) for x in xs]
    torch.cuda.synchronize()
    op.check()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    if hasattr(torch.cuda, "_sleep"):
        with torch.cuda.stream(streams[0]):
            torch.cuda._sleep(40_000_000)  # about 20 ms: the first product starts late
    for k, x in enumerate(xs):
        op.matvec(x, ys[k], stream=streams[k & 1])
    torch.cuda.synchronize()
    op.check()
    for k in range(len(xs)):
        assert torch.equal(ys[k], ref[k]), k


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_uh_matvec_parity(U, name, prec):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    op = U.UHOp.from_arrays(uh_arrays(uh), prec)
    x = I.complex_normal(tree.n, 0)
    _check(_run(op, x, torch), O.uh_matvec(uh, x), TOL[prec])
    st = op.stats()
    c = uh.counts()
    assert (st["E_U"], st["E_V"], st["E_S"], st["E_D"]) == (c["E_U"], c["E_V"], c["E_S"], c["E_D"])
    assert st["csp"] == O.sparsity_constant(uh.adm)


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_h_matvec_parity(U, name, prec):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS[name])
    op = U.HOp.from_arrays(h_arrays(h), prec)
    x = I.complex_normal(tree.n, 1)
    _check(_run(op, x, torch), O.h_matvec(h, x), TOL[prec])


def test_uh_against_dense_product(U):
    """Parity case against the exact dense product: within Theorem 5.1 plus the ACA error."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128")
    x = I.complex_normal(tree.n, 0)
    y = _run(op, x, torch)
    A = O.dense_matrix(pts, 4.0)
    e_aca = np.linalg.norm(A - O.h_to_dense(hf), 2)
    assert np.linalg.norm(y - A @ x) <= (O.theorem51_bound(uh) + e_aca) * np.linalg.norm(x)
    assert relerr(y, A @ x) < 1e-5


def test_bitwise_deterministic(U):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c64")
    xt = torch.from_numpy(I.complex_normal(tree.n, 3)).to("cuda", torch.complex64)
    ys = [op.matvec(xt).clone() for _ in range(8)]
    torch.cuda.synchronize()
    for y in ys[1:]:
        assert torch.equal(y.view(torch.float32), ys[0].view(torch.float32))


def test_side_stream_and_reuse(U):
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128")
    s = torch.cuda.Stream()
    x1 = I.complex_normal(tree.n, 7)
    x2 = I.complex_normal(tree.n, 8)
    with torch.cuda.stream(s):
        a = torch.from_numpy(x1).cuda()
        b = torch.from_numpy(x2).cuda()
        ya = op.matvec(a)
        yb = op.matvec(b)
    s.synchronize()
    _check(ya.cpu().numpy(), O.uh_matvec(uh, x1), 1e-12)
    _check(yb.cpu().numpy(), O.uh_matvec(uh, x2), 1e-12)


def test_degenerate_rank_zero_bases(U):
    """eps = 1 truncates every basis to rank 0: only the near field remains."""
    import torch
    pts = I.fibonacci_sphere(512)
    tree = O.ClusterTree(pts, 16)
    adm, dense = O.block_tree(tree, 1.0)
    hf, _ = O.build_h(pts, tree, adm, dense, 2.0, 1e-8)
    uh = O.uniform_compression(hf, 1.0)
    assert all(u.shape[1] == 0 for u in uh.U.values())
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128")
    x = I.complex_normal(512, 0)
    _check(_run(op, x, torch), O.uh_matvec(uh, x), 1e-12)


@pytest.mark.parametrize("n,leaf", [(1, 8), (40, 64), (97, 16)])
def test_small_and_all_dense(U, n, leaf):
    import torch
    pts = I.fibonacci_sphere(n)
    tree, hf, h, uh = O.build_operators(pts, 3.0, leaf, 1.0, 1e-6, 1e-8)
    x = I.complex_normal(n, 2)
    for prec in ("c128", "c64"):
        op = U.UHOp.from_arrays(uh_arrays(uh), prec)
        _check(_run(op, x, torch), O.uh_matvec(uh, x), TOL[prec])
        hop = U.HOp.from_arrays(h_arrays(h), prec)
        _check(_run(hop, x, torch), O.h_matvec(h, x), TOL[prec])


def test_c64_storage_input(U):
    """Descriptor data given as complex64 (UH_DATA_C64) is accepted and used as stored."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    a = uh_arrays(uh, dtype=np.complex64)
    op = U.UHOp.from_arrays(a, "c64")
    x = I.complex_normal(tree.n, 0)
    _check(_run(op, x, torch), O.uh_matvec(uh, x), TOL["c64"])


def test_bounded_wait_runs_out_and_recovers(U):
    """A product whose dependency waits look for an epoch nobody publishes: every such wait runs
    out after ~1 ms of SM cycles, the kernel returns, uh_check reports UH_ETIMEOUT, and the next
    ordinary product is exact (the context stays usable)."""
    import torch
    pts, tree, hf, h, uh = oracle_ops(*WORKLOADS["sphere2048"])
    op = U.UHOp.from_arrays(uh_arrays(uh), "c128")
    x = I.complex_normal(tree.n, 0)
    xt = torch.from_numpy(x).cuda()
    y = torch.empty_like(xt)
    s = torch.cuda.current_stream().cuda_stream
    assert U.lib.uh_debug_stalled_matvec(op.handle, xt.data_ptr(), y.data_ptr(), 2_000_000, s) == U.UH_OK
    with pytest.raises(U.UHError) as e:
        op.check()
    assert e.value.code == U.UH_ETIMEOUT
    op.check()  # status cleared
    _check(_run(op, x, torch), O.uh_matvec(uh, x), 1e-12)

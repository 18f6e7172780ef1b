"""GPU tests of the serving runtime (uh_server_* / uh_solve_*): GMRES(30) solves of the collocation
operator with its Arnoldi products in complex64 (FP32 accumulation), the restart residual's
product in extended precision on the complex128 x, and orthogonalisation and update in FP64.
Checked against the FP64 oracle: the true residual ||b - A x|| / ||b|| with the oracle's own UH
operator and with the stored (complex64-rounded) operator, and the solution of the dense system
of that operator. A solve's result must be bitwise the same alone and among other solves."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr, stored_c64, uh_arrays

pytestmark = pytest.mark.gpu

SPHERE = (2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0)
ELLIPSOID = (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01)


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


@pytest.fixture(scope="module")
def ops(U):
    a = oracle_ops(*SPHERE)[4]
    b = oracle_ops(*ELLIPSOID)[4]
    return {"sphere": (a, U.UHOp.from_arrays(uh_arrays(a), "c64"), U.UHOp.from_arrays(uh_arrays(a), "c128")),
            "ellipsoid": (b, U.UHOp.from_arrays(uh_arrays(b), "c64"), None)}


def test_solve_converges_against_fp64_operator(U, ops):
    uh, op64, _ = ops["sphere"]
    srv = U.Server(max_active=4)
    b = I.complex_normal(uh.tree.n, 3)
    t = srv.submit(op64, b, tol=1e-6, restart=30, maxit=300)
    x, info = srv.wait(t)
    assert info["status"] == U.UH_OK and info["converged"] == 1
    assert info["rel_residual"] <= 1e-6
    # the reported residual is the true one of the stored operator, computed in FP64
    stored_res = np.linalg.norm(b - O.uh_matvec(stored_c64(uh), x)) / np.linalg.norm(b)
    assert abs(info["rel_residual"] - stored_res) <= 1e-4 * stored_res
    # against the FP64 operator the complex64 storage of the entries adds at most a few 1e-8
    true_res = np.linalg.norm(b - O.uh_matvec(uh, x)) / np.linalg.norm(b)
    assert true_res <= 1.05e-6, true_res
    xref = np.linalg.solve(O.uh_to_dense(uh), b)
    assert relerr(x, xref) <= 1e-5
    assert info["latency_s"] >= info["queue_s"] >= 0
    srv.close()


def test_solve_complex128_op_reaches_tight_tolerance(U, ops):
    uh, _, op128 = ops["sphere"]
    srv = U.Server()
    b = I.complex_normal(uh.tree.n, 4)
    x, info = srv.wait(srv.submit(op128, b, tol=1e-11, restart=20, maxit=400))
    assert info["converged"] == 1 and info["restarts"] >= 1
    assert np.linalg.norm(b - O.uh_matvec(uh, x)) / np.linalg.norm(b) <= 1e-10
    srv.close()


@pytest.mark.parametrize("tol", [1e-9, 1e-11])
def test_refinement_reaches_below_the_fp32_product(U, ops, tol):
    """Tolerances the FP32-accumulated product cannot resolve (its error is ~3e-7 of |A x|): the
    restarts with the extended-precision residual drive the stored operator's true residual
    below tol."""
    uh, op64, _ = ops["sphere"]
    srv = U.Server()
    b = I.complex_normal(uh.tree.n, 7)
    x, info = srv.wait(srv.submit(op64, b, tol=tol, restart=30, maxit=600))
    assert info["status"] == U.UH_OK and info["converged"] == 1, info
    assert info["restarts"] >= 2  # refinement: more than one cycle was needed
    stored_res = np.linalg.norm(b - O.uh_matvec(stored_c64(uh), x)) / np.linalg.norm(b)
    assert stored_res <= 1.05 * tol, stored_res
    assert abs(info["rel_residual"] - stored_res) <= 1e-3 * stored_res + 1e-13
    srv.close()


def test_same_result_alone_and_in_a_mix(U, ops):
    uh, op64, _ = ops["sphere"]
    uh2, op2, _ = ops["ellipsoid"]
    b = I.complex_normal(uh.tree.n, 5)
    srv = U.Server(max_active=8)
    x_alone, info_alone = srv.wait(srv.submit(op64, b))
    others = [srv.submit(op2, I.complex_normal(uh2.tree.n, 20 + k), tol=1e-7) for k in range(4)]
    others += [srv.submit(op64, I.complex_normal(uh.tree.n, 30 + k), restart=10) for k in range(2)]
    mine = srv.submit(op64, b)
    x_mix, info_mix = srv.wait(mine)
    for t in others:
        xo, io = srv.wait(t)
        assert io["converged"] == 1
    assert np.array_equal(x_alone, x_mix)
    assert info_alone["iterations"] == info_mix["iterations"]
    srv.close()


def test_paired_products_change_no_result(U, ops):
    """With multi-RHS scratch reserved on the op, solves of that op share their Arnoldi products
    (passes of two right-hand sides). A solve's x is still bitwise that of the same solve alone on
    an op without pairing, and of the same solve alone on the reserved op."""
    uh, op_plain, _ = ops["sphere"]
    op = U.UHOp.from_arrays(uh_arrays(uh), "c64")
    op.reserve(2)
    bs = [I.complex_normal(uh.tree.n, 60 + k) for k in range(6)]
    srv = U.Server(max_active=8)
    alone = [srv.wait(srv.submit(op_plain, b))[0] for b in bs]
    x_res, info_res = srv.wait(srv.submit(op, bs[0]))
    assert info_res["paired_steps"] == 0
    tickets = [srv.submit(op, b) for b in bs]
    res = [srv.wait(t) for t in tickets]
    srv.close()
    assert np.array_equal(x_res, alone[0])
    for (x, info), xa in zip(res, alone):
        assert info["converged"] == 1
        assert np.array_equal(x, xa)
    assert sum(info["paired_steps"] for _, info in res) > 0
    op.close()


def test_admission_busy_and_errors(U, ops):
    uh, op64, _ = ops["sphere"]
    b = I.complex_normal(uh.tree.n, 6)
    srv = U.Server(max_active=1, queue_capacity=1)
    tickets = [srv.submit(op64, b) for _ in range(3)]
    assert None in tickets[1:]  # one running or waiting, one waiting, the rest refused (UH_EBUSY)
    first = tickets[0]
    assert srv.poll(first) is None or True  # may already be done on a fast GPU
    for t in tickets:
        if t is not None:
            x, info = srv.wait(t)
            assert info["converged"] == 1
    with pytest.raises(U.UHError) as e:
        srv.poll(10 ** 9)
    assert e.value.code == U.UH_EINVAL
    small = U.Server(hbm_budget=1 << 20)
    with pytest.raises(U.UHError) as e:
        small.submit(op64, b)  # workspace above the budget
    assert e.value.code == U.UH_EINVAL
    small.close()
    srv.close()

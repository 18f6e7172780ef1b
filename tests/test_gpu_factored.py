"""GPU parity of the factored coefficient storage S_b = S_X,b S_Y,b^* (Section 4.2; uh_desc.S_rank)
against the FP64 oracle, through the C ABI.

The oracle factors its own operator (factor_coupling: the pair of Algorithm 2 recompressed at the
given eps, kept factored where k_b (l_tau + l_sigma) < l_tau l_sigma) and applies it with the
factored coupling (t_b = S_Y^* xhat_sigma, yhat_tau += S_X t_b); the same factors are handed to
uh_create, so only the summation order (complex128) or the storage rounding (complex64) differs.
The tolerances are those of the dense-S products: 1e-12 (complex128), 5e-6 (complex64 with FP32
accumulation), 1e-11 (extended precision), 1e-3 / 1e-4 (TF32 / BF16x3 multi-RHS), relative 2-norm
and element-wise against the largest output. The builders' factored option (host and device) is
checked against the oracle's dense-S operator within 10 eps.
"""
import functools

import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr, stored_c64, uh_arrays

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-12, "c64": 5e-6}
TOL_MIXED = 1e-11
TOL_MM = {"tf32": 1e-3, "bf16x3": 1e-4}

# (oracle workload, eps factor of the recompression): both forms occur in each, and at 30 eps
# every block of the sphere is factored
CASES = {
    "sphere2048": ((2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0), 1.0),
    "sphere2048_all": ((2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0), 30.0),
    "ellipsoid1000": ((1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01), 3.0),
    "ellipsoid1000_strong": ((1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01, 0, True), 3.0),
}


@pytest.fixture(scope="module")
def U():
    import torch  # noqa: F401
    from paper_2405_15573_gb300 import uh
    return uh


@functools.lru_cache(maxsize=None)
def _factored(name):
    wl, f = CASES[name]
    pts, tree, hf, h, uh = oracle_ops(*wl)
    return tree, uh, O.factor_coupling(uh, f * wl[4])


def _run(op, x, torch):
    xt = torch.from_numpy(x).to("cuda", torch.complex128 if op.c128 else torch.complex64)
    y = torch.full_like(xt, complex(float("nan"), float("nan")))  # poisoned output
    op.matvec(xt, y)
    op.check()
    return y.cpu().numpy().astype(np.complex128)


def _check(y, yref, tol):
    assert np.isfinite(y).all()
    assert relerr(y, yref) <= tol
    assert np.max(np.abs(y - yref)) <= tol * np.max(np.abs(yref)) * 10


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_factored_matvec_parity(U, name, prec):
    import torch
    tree, uh, fu = _factored(name)
    assert fu.F
    op = U.UHOp.from_arrays(uh_arrays(fu), prec)
    for seed in (0, 1):
        x = I.complex_normal(tree.n, seed)
        ref = fu if prec == "c128" else stored_c64(fu)
        _check(_run(op, x, torch), O.uh_matvec(ref, x), TOL[prec])
    st = op.stats()
    c = fu.counts()
    assert (st["E_U"], st["E_V"], st["E_S"], st["E_D"]) == (c["E_U"], c["E_V"], c["E_S"], c["E_D"])
    assert st["n_factored"] == len(fu.F) and st["sum_factored_rank"] == c["K"]
    # the factored operator streams fewer bytes than the dense-S one
    dense = U.UHOp.from_arrays(uh_arrays(uh), prec).stats()
    assert st["E_S"] < dense["E_S"]
    assert st["algo_bytes_matvec"] == dense["algo_bytes_matvec"] + st["elem_bytes"] * (
        st["E_S"] - dense["E_S"] + 2 * st["sum_factored_rank"])


@pytest.mark.parametrize("name", ["sphere2048", "ellipsoid1000"])
def test_factored_mixed_parity(U, name):
    """The extended-precision product (the refinement residual) with factored coefficients."""
    import torch
    tree, uh, fu = _factored(name)
    op = U.UHOp.from_arrays(uh_arrays(fu), "c64")
    x = I.complex_normal(tree.n, 4)
    xt = torch.from_numpy(x).to("cuda", torch.complex128)
    y = torch.full_like(xt, complex(float("nan"), float("nan")))
    op.matvec_mixed(xt, y)
    op.check()
    _check(y.cpu().numpy(), O.uh_matvec(stored_c64(fu), x), TOL_MIXED)


def test_factored_product_is_bitwise_repeatable(U):
    import torch
    tree, uh, fu = _factored("sphere2048")
    op = U.UHOp.from_arrays(uh_arrays(fu), "c64")
    x = I.complex_normal(tree.n, 5)
    y1 = _run(op, x, torch)
    y2 = _run(op, x, torch)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("mode", ["tf32", "bf16x3"])
@pytest.mark.parametrize("nrhs", [7, 64])
def test_factored_matmat_parity(U, mode, nrhs):
    """The tensor-core multi-RHS product assembles S_b from the stored factors when it packs."""
    import torch
    tree, uh, fu = _factored("ellipsoid1000")
    op = U.UHOp.from_arrays(uh_arrays(fu), "c64_" + mode)
    X = np.stack([I.complex_normal(tree.n, 10 + j) for j in range(nrhs)], axis=1)
    Xd = torch.from_numpy(X.T.copy()).to("cuda", torch.complex64).T
    Yd = torch.full((nrhs, tree.n), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda").T
    op.matmat(Xd, Yd, mode=mode)
    op.check()
    Y = Yd.cpu().numpy().astype(np.complex128)
    assert np.isfinite(Y).all()
    errs = [relerr(Y[:, j], O.uh_matvec(fu, X[:, j])) for j in range(nrhs)]
    assert max(errs) <= TOL_MM[mode], max(errs)


def test_factored_batch_parity(U):
    """One launch over operators with and without factored coefficients."""
    import torch
    ops = [_factored("sphere2048")[2], _factored("ellipsoid1000")[2], oracle_ops(512, 3.0, 16, 1.0, 1e-6, 1e-8)[4]]
    batch = U.UHBatch.from_arrays([uh_arrays(o) for o in ops], "c64")
    xs = [I.complex_normal(o.tree.n, 20 + i) for i, o in enumerate(ops)]
    x = torch.from_numpy(np.concatenate(xs)).to("cuda", torch.complex64)
    y = torch.full_like(x, complex(float("nan"), float("nan")))
    batch.matvec(x, y)
    batch.check()
    yc = y.cpu().numpy().astype(np.complex128)
    at = 0
    for o, xi in zip(ops, xs):
        _check(yc[at:at + o.tree.n], O.uh_matvec(stored_c64(o), xi), TOL["c64"])
        at += o.tree.n


def _points(n, axes, noise, seed=0):
    if axes == (1.0, 1.0, 1.0) and not noise:
        return I.fibonacci_sphere(n)
    return I.ellipsoid_points(n, axes, noise, seed)


@pytest.mark.parametrize("device", [False, True])
@pytest.mark.parametrize("name", ["sphere2048", "ellipsoid1000"])
def test_builder_factored_option(U, device, name):
    """uhb_params.factored on the host and the device builder: the factored blocks keep the rank
    rule of a plain SVD of the same builder's dense S_b at eps (within one, the last value decided
    within rounding), store fewer elements, and the product stays within 10 eps of the oracle's
    dense-S operator."""
    import torch
    wl, _ = CASES[name]
    n, k, leaf, eta, eps, tol, axes, noise = wl
    pts, tree, hf, h, uh = oracle_ops(*wl)
    p = _points(n, axes, noise)
    md = U.HelmholtzModel(p, k, leaf, eta, eps, tol, device=device)
    mf = U.HelmholtzModel(p, k, leaf, eta, eps, tol, device=device, factored=True)
    ad, af = md.uh_arrays(), mf.uh_arrays()
    assert af["S_rank"] is not None and (af["S_rank"] > 0).sum() > len(af["S_rank"]) // 10
    for key in ("row_rank", "col_rank", "adm_row", "adm_col"):
        assert np.array_equal(ad[key], af[key]), key
    for b in np.flatnonzero(af["S_rank"] >= 0)[::7]:
        lt, ls, kb = int(af["row_rank"][af["adm_row"][b]]), int(af["col_rank"][af["adm_col"][b]]), int(af["S_rank"][b])
        Sd = ad["S_data"][ad["S_off"][b]:ad["S_off"][b] + lt * ls].reshape(ls, lt).T
        o = af["S_off"][b]
        X = af["S_data"][o:o + lt * kb].reshape(kb, lt).T
        Y = af["S_data"][o + lt * kb:o + kb * (lt + ls)].reshape(kb, ls).T
        s = np.linalg.svd(Sd, compute_uv=False)
        assert abs(kb - int(np.sum(s > eps * s[0]))) <= 1
        assert kb * (lt + ls) < lt * ls
        assert np.linalg.norm(Sd - X @ Y.conj().T, 2) <= 2 * eps * s[0]
    x = I.complex_normal(n, 6)
    xt = torch.from_numpy(x).to("cuda", torch.complex128)
    opf = mf.uh_op("c128")
    y = opf.matvec(xt)
    opf.check()
    assert relerr(y.cpu().numpy(), O.uh_matvec(uh, x)) <= 10 * eps
    assert opf.stats()["E_S"] < md.uh_op("c128").stats()["E_S"]
    md.close()
    mf.close()

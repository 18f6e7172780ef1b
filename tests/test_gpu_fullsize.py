"""Parity at the headline size (unit sphere, N = 32768, k = 16, leaf 64, eta 1, eps 1e-6) in the
launch configuration the benchmark times. The operator comes from the library's builder; the
oracle applies the same operator (its Algorithm 5/6 products) in FP64, and the exact dense
rows (A x)_i = sum_j A_ij x_j of a sample of rows check the approximation itself."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.test_builder_cpu import _oracle_view
from tests.uh_testutil import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    from paper_2405_15573_gb300 import uh as U
    w = I.SPHERE_32768
    pts = w.points()
    m = U.HelmholtzModel(pts, w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    a = m.uh_arrays()
    Ub, Vb, Sb, near = _oracle_view(a)
    import types
    tree = types.SimpleNamespace(n=w.n, perm=a["perm"], begin=a["cl_begin"].tolist(), size=a["cl_size"].tolist())
    uh = O.UHMatrix(tree, sorted(Sb), sorted(near), Ub, Vb, Sb, near, {}, {})
    ha = m.h_arrays()
    low = {}
    for t, s, k, xo, yo in zip(ha["adm_row"], ha["adm_col"], ha["adm_rank"], ha["X_off"], ha["Y_off"]):
        mt, ms = int(a["cl_size"][t]), int(a["cl_size"][s])
        low[(int(t), int(s))] = (ha["X_data"][xo:xo + mt * k].reshape(k, mt).T,
                                 ha["Y_data"][yo:yo + ms * k].reshape(k, ms).T)
    h = O.HMatrix(tree, sorted(low), sorted(near), low, near)
    return w, pts, m, uh, h


def _gpu(op, x, dt):
    import torch
    xt = torch.from_numpy(x).to("cuda", dt)
    y = torch.full_like(xt, complex(float("nan"), float("nan")))
    op.matvec(xt, y)
    op.check()
    return y.cpu().numpy().astype(np.complex128)


def test_full_uh_c64_and_c128(full):
    import torch
    w, pts, m, uh, h = full
    x = w.x()
    yref = O.uh_matvec(uh, x)
    y64 = _gpu(m.uh_op("c64"), x, torch.complex64)
    assert np.isfinite(y64).all() and relerr(y64, yref) <= 5e-6
    assert np.max(np.abs(y64 - yref)) <= 5e-5 * np.max(np.abs(yref))
    y128 = _gpu(m.uh_op("c128"), x, torch.complex128)
    assert relerr(y128, yref) <= 1e-12
    # exact rows of A x: the approximation error of the compressed operator itself
    rows = np.random.default_rng(0).choice(w.n, 48, replace=False)
    exact = O.dense_rows_matvec(pts, w.wavenumber, rows, x)
    assert relerr(y64[rows], exact) < 1e-5


def test_full_h_c64(full):
    import torch
    w, pts, m, uh, h = full
    x = I.complex_normal(w.n, 1)
    yref = O.h_matvec(h, x)
    y = _gpu(m.h_op("c64"), x, torch.complex64)
    assert relerr(y, yref) <= 5e-6

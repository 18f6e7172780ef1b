"""Multi-RHS product at the large size: ellipsoid (1, 0.7, 0.4) with 1% radial noise, N = 131072,
k = 32, leaf 64, eta 1, eps 1e-4, 64 right-hand sides, in the launch configuration of the
library (passes of 64, three launches each). The operator comes from the library's builder; the
truth for 256 sampled rows is the exact dense product (A X)_i = sum_j A_ij X_j written out from
the matrix entries (oracle), so the error measured is that of the compressed operator (eps 1e-4)
plus the tensor-core rounding. Bound per column: 1e-3 relative 2-norm (both TF32 and BF16x3);
also at N = 32768 with 32 right-hand sides (sphere, eps 1e-6), where BF16x3 is held to 1e-4."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _colmajor(torch, X):
    return torch.from_numpy(np.ascontiguousarray(X.T).astype(np.complex64)).to("cuda").T


def _columns_error(Y, exact):
    return [float(np.linalg.norm(Y[:, j] - exact[:, j]) / np.linalg.norm(exact[:, j])) for j in range(Y.shape[1])]


@pytest.mark.parametrize("w, rows, tol_bf16", [(I.ELLIPSOID_131072_R64, 256, 1e-3), (I.SPHERE_32768_R32, 128, 1e-4)],
                         ids=["ellipsoid131072_R64", "sphere32768_R32"])
def test_matmat_sampled_rows(w, rows, tol_bf16):
    import torch
    from paper_2405_15573_gb300 import uh as U
    pts = w.points()
    m = U.HelmholtzModel(pts, w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    X = np.stack([I.complex_normal(w.n, w.x_seed + j) for j in range(w.nrhs)], axis=1)
    sample = np.random.default_rng(1).choice(w.n, rows, replace=False)
    exact = O.dense_rows_matvec(pts, w.wavenumber, sample, X)
    Xd = _colmajor(torch, X)
    for mode, tol in (("tf32", 1e-3), ("bf16x3", tol_bf16)):
        op = m.uh_op("c64_" + mode)
        Yd = torch.full((w.nrhs, w.n), complex(float("nan"), float("nan")), dtype=torch.complex64, device="cuda").T
        op.matmat(Xd, Yd, mode=mode)
        op.check()
        Y = Yd.cpu().numpy().astype(np.complex128)
        assert np.isfinite(Y).all()
        errs = _columns_error(Y[sample], exact)
        assert max(errs) <= tol, (mode, max(errs))
        del op
    m.close()

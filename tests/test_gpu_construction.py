"""Construction on the GPU (uhb_build_helmholtz_gpu: ACA with recompression, Section 2.3, and the
direct UH construction of Section 4.3, Algorithms 3 and 4, all on the device) against the FP64
oracle's construction from the same points: cluster ranks within one of the oracle's, and the
device-built operator's product (complex128) within 10 eps of the oracle operator's product.
The host builder's operator is the second reference: the same steps on the CPU."""
import numpy as np
import pytest

from oracle import uh_oracle as O
from paper_2405_15573_gb300 import inputs as I
from tests.uh_testutil import oracle_ops, relerr

pytestmark = pytest.mark.gpu

CASES = {
    # (n, k, leaf, eta, eps, tol_aca, axes, noise, seed, strong)
    "sphere2048": (2048, 4.0, 32, 1.0, 1e-6, 1e-8, (1.0, 1.0, 1.0), 0.0, 0, False),
    "ellipsoid1000": (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01, 0, False),
    "ellipsoid1000_strong": (1000, 6.0, 24, 1.0, 1e-5, 1e-8, (1.0, 0.7, 0.4), 0.01, 0, True),
}


def _points(case):
    n, k, leaf, eta, eps, tol, axes, noise, seed, strong = case
    if axes == (1.0, 1.0, 1.0) and not noise:
        return I.fibonacci_sphere(n)
    return I.ellipsoid_points(n, axes, noise, seed)


def _product(op, x, torch):
    xt = torch.from_numpy(x).to("cuda", torch.complex128)
    y = op.matvec(xt)
    op.check()
    return y.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_device_build_matches_oracle(name):
    import torch
    from paper_2405_15573_gb300 import uh as U
    case = CASES[name]
    n, k, leaf, eta, eps, tol, axes, noise, seed, strong = case
    pts, tree, hf, h, uh = oracle_ops(n, k, leaf, eta, eps, tol, axes, noise, seed, strong)
    m = U.HelmholtzModel(_points(case), k, leaf, eta, eps, tol, strong=strong, device=True)
    a = m.uh_arrays()
    # the same trees
    assert np.array_equal(a["perm"], tree.perm)
    assert np.array_equal(a["cl_size"], np.asarray(tree.size))
    # cluster ranks within one of the oracle's (Algorithm 2's SVD of the stacked matrix)
    lu, lv = uh.ranks()
    for c in range(tree.n_clusters):
        assert abs(int(a["row_rank"][c]) - lu.get(c, 0)) <= 1, ("row", c)
        assert abs(int(a["col_rank"][c]) - lv.get(c, 0)) <= 1, ("col", c)
    # the products: device-built UH and H operators against the oracle's, complex128
    for seed_x in (0, 1):
        x = I.complex_normal(n, seed_x)
        yu = _product(m.uh_op("c128"), x, torch)
        assert relerr(yu, O.uh_matvec(uh, x)) <= 10 * eps
        yh = _product(m.h_op("c128"), x, torch)
        assert relerr(yh, O.h_matvec(h, x)) <= 10 * eps
    info = m.info()
    assert info["seconds_aca"] >= 0 and info["lmax"] == max(a["row_rank"].max(), a["col_rank"].max())
    m.close()


def test_device_and_host_builders_agree():
    """The device and the host builder run the same steps: identical trees and blocks, ranks
    equal up to the last one decided within rounding, products within a few eps."""
    import torch
    from paper_2405_15573_gb300 import uh as U
    w = I.SPHERE_2048
    pts = w.points()
    md = U.HelmholtzModel(pts, w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca, device=True)
    mh = U.HelmholtzModel(pts, w.wavenumber, w.leaf, w.eta, w.eps, w.tol_aca)
    ad, ah = md.uh_arrays(), mh.uh_arrays()
    for key in ("perm", "cl_begin", "cl_size", "adm_row", "adm_col", "dense_row", "dense_col"):
        assert np.array_equal(ad[key], ah[key]), key
    assert np.abs(ad["row_rank"] - ah["row_rank"]).max() <= 1
    assert np.abs(ad["col_rank"] - ah["col_rank"]).max() <= 1
    assert np.mean(ad["row_rank"] == ah["row_rank"]) > 0.95
    # near field: identical entries (the same formula in FP64)
    assert np.allclose(ad["D_data"], ah["D_data"], rtol=1e-14, atol=1e-16)
    x = I.complex_normal(w.n, 3)
    yd = _product(md.uh_op("c128"), x, torch)
    yh = _product(mh.uh_op("c128"), x, torch)
    assert relerr(yd, yh) <= 3 * w.eps
    md.close()
    mh.close()


def test_device_build_rejects_bad_parameters():
    from paper_2405_15573_gb300 import uh as U
    with pytest.raises(U.UHError) as e:
        U.HelmholtzModel(I.fibonacci_sphere(64), 1.0, 0, 1.0, 1e-6, 1e-8, device=True)
    assert e.value.code == U.UH_EINVAL

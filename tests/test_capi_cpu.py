"""CPU-side checks of the C ABI: the library loads, exports every function include/uh.h declares,
and rejects invalid descriptors with UH_EINVAL before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import uh_oracle as O
from tests.uh_testutil import h_arrays, oracle_ops, uh_arrays

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def uh():
    from paper_2405_15573_gb300 import uh as U
    return U


def test_header_symbols_exported(uh):
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(h)
    assert "uh_matvec" in names and "h_matvec" in names and "uh_create" in names
    for name in names:
        assert hasattr(uh.lib, name), f"{name} declared but not exported"


def test_version_and_error_string(uh):
    assert "sm_103a" in uh.version()
    assert uh.lib.uh_last_error() is not None


def _small():
    _, _, hf, h, op = oracle_ops(512, 3.0, 16, 1.0, 1e-6, 1e-8)
    return uh_arrays(op), h_arrays(h)


def _expect_einval(uh, arrays, match, kind="uh"):
    desc, keep = (uh.uh_desc_from_arrays if kind == "uh" else uh.h_desc_from_arrays)(arrays)
    h = C.c_void_p()
    fn = uh.lib.uh_create if kind == "uh" else uh.lib.h_create
    rc = fn(C.byref(desc), uh.UH_PREC_C64, C.byref(h))
    assert rc == uh.UH_EINVAL
    assert h.value is None
    msg = uh.lib.uh_last_error().decode()
    assert re.search(match, msg), msg


def test_rejects_bad_permutation(uh):
    a, _ = _small()
    a = dict(a)
    p = a["perm"].copy()
    p[3] = p[4]
    a["perm"] = p
    _expect_einval(uh, a, "permutation")


def test_rejects_missing_and_double_coverage(uh):
    a, _ = _small()
    b = dict(a)
    b["dense_row"], b["dense_col"], b["D_off"] = a["dense_row"][1:], a["dense_col"][1:], a["D_off"][1:]
    _expect_einval(uh, b, "not covered")
    c = dict(a)
    c["dense_row"] = np.concatenate([a["dense_row"], a["dense_row"][:1]])
    c["dense_col"] = np.concatenate([a["dense_col"], a["dense_col"][:1]])
    c["D_off"] = np.concatenate([a["D_off"], a["D_off"][:1]])
    _expect_einval(uh, c, "covered twice")


def test_rejects_out_of_range_data_and_ranks(uh):
    a, h = _small()
    b = dict(a)
    b["S_off"] = a["S_off"].copy()
    b["S_off"][-1] = len(a["S_data"])
    _expect_einval(uh, b, "coupling matrix")
    c = dict(a)
    c["row_rank"] = a["row_rank"].copy()
    r = int(np.flatnonzero(a["row_rank"] > 0)[0])
    c["row_rank"][r] = 10 ** 6
    _expect_einval(uh, c, "row_rank")
    d = dict(a)
    d["cl_size"] = a["cl_size"].copy()
    d["cl_size"][1] = 10 ** 6
    _expect_einval(uh, d, "outside")
    e = dict(h)
    e["adm_rank"] = h["adm_rank"].copy()
    e["adm_rank"][0] = -1
    _expect_einval(uh, e, "adm_rank", kind="h")


def test_null_arguments(uh):
    h = C.c_void_p()
    assert uh.lib.uh_create(None, 0, C.byref(h)) == uh.UH_EINVAL
    assert uh.lib.uh_destroy(None) == uh.UH_OK
    assert uh.lib.uh_matvec(None, None, None, None) == uh.UH_EINVAL


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("ncta", [152, 148, 7, 1])
@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6), (1000, 6.0, 24, 1e-5), (97, 3.0, 16, 1e-6),
                                  (40, 3.0, 64, 1e-6)])
def test_packing_self_check_passes(uh, prec, ncta, case):
    """Validation, packing and the packer's check of every kernel address, for several CTA
    counts, without a GPU (uh_debug.h)."""
    n, k, leaf, eps = case
    axes, noise = ((1.0, 0.7, 0.4), 0.01) if n == 1000 else ((1.0, 1.0, 1.0), 0.0)
    _, _, hf, h, op = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
    for mk, fn, arr in ((uh.uh_desc_from_arrays, uh.lib.uh_pack_check, uh_arrays(op)),
                        (uh.h_desc_from_arrays, uh.lib.h_pack_check, h_arrays(h))):
        desc, keep = mk(arr)
        rc = fn(C.byref(desc), prec, ncta)
        assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("ncta", [152, 5, 1])
@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6), (1000, 6.0, 24, 1e-5), (40, 3.0, 64, 1e-6)])
def test_multi_rhs_packing_self_check_passes(uh, prec, ncta, case):
    """The tensor-core multi-RHS program (TF32 and BF16x3 tiles) is packed and every address the
    kernel derives from it checked, without a GPU; the H form rejects these precisions."""
    n, k, leaf, eps = case
    axes, noise = ((1.0, 0.7, 0.4), 0.01) if n == 1000 else ((1.0, 1.0, 1.0), 0.0)
    _, _, hf, h, op = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
    desc, keep = uh.uh_desc_from_arrays(uh_arrays(op))
    rc = uh.lib.uh_pack_check(C.byref(desc), prec, ncta)
    assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()
    hd, hkeep = uh.h_desc_from_arrays(h_arrays(h))
    assert uh.lib.h_pack_check(C.byref(hd), prec, ncta) == uh.UH_EINVAL


BATCH_CASES = [(512, 3.0, 16, 1e-6), (1000, 6.0, 24, 1e-5), (97, 3.0, 16, 1e-6), (40, 3.0, 64, 1e-6),
               (2048, 4.0, 32, 1e-6)]


def _batch_arrays():
    out = []
    for n, k, leaf, eps in BATCH_CASES:
        axes, noise = ((1.0, 0.7, 0.4), 0.01) if n == 1000 else ((1.0, 1.0, 1.0), 0.0)
        _, _, hf, h, op = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
        out.append(uh_arrays(op))
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("ncta", [152, 7, 1])
def test_batch_packing_self_check_passes(uh, prec, ncta):
    """Five operators of uneven size (one all dense, odd sizes) packed as one device program,
    every kernel address checked, without a GPU."""
    built = [uh.uh_desc_from_arrays(a) for a in _batch_arrays()]
    arr = uh._desc_array([d for d, _ in built])
    rc = uh.lib.uh_batch_pack_check(arr, len(built), prec, ncta)
    assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()


# every value the autotuner (uh_batch_tune) can choose, one knob at a time, and all at extremes
TUNER_PARAMS = [(16384, 0, 0, 0), (32768, 0, 0, 0), (0, 1024, 0, 0), (0, 16384, 0, 0), (0, 0, 12288, 0),
                (0, 0, 196608, 0), (0, 0, 0, 32768), (0, 0, 0, 524288), (16384, 1024, 12288, 32768),
                (16384, 16384, 196608, 524288)]


@pytest.mark.parametrize("params", TUNER_PARAMS)
@pytest.mark.parametrize("ncta", [152, 7])
def test_batch_packing_with_tuner_parameters(uh, params, ncta):
    built = [uh.uh_desc_from_arrays(a) for a in _batch_arrays()]
    arr = uh._desc_array([d for d, _ in built])
    pp = uh.PackParams(*params)
    rc = uh.lib.uh_batch_pack_check_ex(arr, len(built), 1, pp, ncta)
    assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()


def test_batch_rejects_bad_pack_parameters(uh):
    built = [uh.uh_desc_from_arrays(a) for a in _batch_arrays()]
    arr = uh._desc_array([d for d, _ in built])
    for bad in [(1024, 0, 0, 0), (131072, 0, 0, 0), (0, -1, 0, 0)]:
        rc = uh.lib.uh_batch_pack_check_ex(arr, len(built), 1, uh.PackParams(*bad), 7)
        assert rc == uh.UH_EINVAL and "pack parameters" in uh.lib.uh_last_error().decode()


def test_batch_rejects_bad_operator_and_precision(uh):
    arrays = _batch_arrays()
    bad = dict(arrays[2])
    p = bad["perm"].copy()
    p[0] = p[1]
    bad["perm"] = p
    arrays[2] = bad
    built = [uh.uh_desc_from_arrays(a) for a in arrays]
    arr = uh._desc_array([d for d, _ in built])
    assert uh.lib.uh_batch_pack_check(arr, len(built), 1, 7) == uh.UH_EINVAL
    assert "operator 2" in uh.lib.uh_last_error().decode()
    good = [uh.uh_desc_from_arrays(a) for a in _batch_arrays()[:2]]
    arr = uh._desc_array([d for d, _ in good])
    assert uh.lib.uh_batch_pack_check(arr, 2, uh.UH_PREC_C64_TF32, 7) == uh.UH_EINVAL
    assert uh.lib.uh_batch_pack_check(arr, 0, 1, 7) == uh.UH_EINVAL


def test_server_argument_checks(uh):
    h = C.c_void_p()
    assert uh.lib.uh_server_create(0, 1 << 30, 4, C.byref(h)) == uh.UH_EINVAL
    assert uh.lib.uh_server_create(4, 0, 4, C.byref(h)) == uh.UH_EINVAL
    assert uh.lib.uh_server_create(4, 1 << 30, 0, C.byref(h)) == uh.UH_EINVAL
    assert h.value is None
    assert uh.lib.uh_server_destroy(None) == uh.UH_OK
    t = C.c_uint64()
    assert uh.lib.uh_solve_submit(None, None, None, 1e-6, 30, 100, C.byref(t)) == uh.UH_EINVAL
    assert uh.lib.uh_solve_poll(None, 1, None, None) == uh.UH_EINVAL


def test_block_apply_noalloc_argument_checks(uh):
    """The binding rejects every inconsistent block product before the library is called, and
    the C entry point rejects sizes its grid cannot cover; neither needs a GPU to do so."""
    import torch
    cd = torch.complex128
    m, n, lt, ls = 40, 30, 5, 4

    def good():
        return dict(U=torch.zeros(lt, m, dtype=cd).T, S=torch.zeros(ls, lt, dtype=cd).T,
                    V=torch.zeros(ls, n, dtype=cd).T, x=torch.zeros(n, dtype=cd),
                    y=torch.zeros(m, dtype=cd))

    bad = [
        ("x", lambda a: torch.zeros(n, dtype=torch.float64), "complex64 or complex128"),
        ("y", lambda a: a["y"].to(torch.complex64), "y has dtype"),
        ("S", lambda a: a["S"].to(torch.complex64), "S has dtype"),
        ("U", lambda a: a["U"][:, 0].contiguous(), "U must be a matrix"),
        ("x", lambda a: torch.zeros(n + 1, dtype=cd), "x has 31 values"),
        ("y", lambda a: torch.zeros(m - 1, dtype=cd), "y has 39"),
        ("y", lambda a: torch.zeros(2 * m, dtype=cd)[::2], "contiguous vector"),
        ("S", lambda a: torch.zeros(ls, lt + 1, dtype=cd).T, r"S is \(6, 4\)"),
        ("U", lambda a: torch.zeros(m, lt, dtype=cd), "U must be column-major"),
        ("V", lambda a: a["V"], "must be a CUDA tensor"),  # all consistent, but on the host
    ]
    for name, make, match in bad:
        a = good()
        a[name] = make(a)
        with pytest.raises(ValueError, match=match):
            uh.block_apply_noalloc(a["U"], a["S"], a["V"], a["x"], a["y"])
    big = (0x7FFFFFFF * 256) + 1
    for mm, nn in ((big, 8), (8, big)):
        rc = uh.lib.uh_block_apply_noalloc(mm, nn, 1, 1, 16, mm, 16, 1, 16, nn, 16, 16,
                                           uh.UH_PREC_C128, None)
        assert rc == uh.UH_EINVAL and "above the limit" in uh.lib.uh_last_error().decode()


def _factored_arrays(n, k, leaf, eps, f=1.0):
    """An oracle operator with its coefficient matrices stored factored where smaller (Section
    4.2, recompressed at f * eps), flattened into the descriptor arrays (S_rank set)."""
    axes, noise = ((1.0, 0.7, 0.4), 0.01) if n == 1000 else ((1.0, 1.0, 1.0), 0.0)
    _, _, hf, h, op = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
    return uh_arrays(O.factor_coupling(op, f * eps))


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("ncta", [152, 7, 1])
@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6, 1.0), (1000, 6.0, 24, 1e-5, 3.0), (2048, 4.0, 32, 1e-6, 30.0)])
def test_factored_packing_self_check_passes(uh, prec, ncta, case):
    """Operators with factored and dense coefficient matrices (the t_b group, z4 and its scatter)
    are packed and every kernel address checked, for the streaming and the tensor-core programs."""
    a = _factored_arrays(*case)
    assert a["S_rank"] is not None and (a["S_rank"] >= 0).any()
    desc, keep = uh.uh_desc_from_arrays(a)
    rc = uh.lib.uh_pack_check(C.byref(desc), prec, ncta)
    assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()


@pytest.mark.parametrize("ncta", [152, 7])
def test_factored_batch_packing_self_check_passes(uh, ncta):
    """A batch mixing operators with and without factored coefficients."""
    arrays = _batch_arrays()[:3] + [_factored_arrays(2048, 4.0, 32, 1e-6), _factored_arrays(1000, 6.0, 24, 1e-5, 3.0)]
    built = [uh.uh_desc_from_arrays(a) for a in arrays]
    arr = uh._desc_array([d for d, _ in built])
    for prec in (0, 1):
        rc = uh.lib.uh_batch_pack_check(arr, len(built), prec, ncta)
        assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()


def test_rejects_bad_factored_ranks(uh):
    a = _factored_arrays(1000, 6.0, 24, 1e-5, 3.0)
    i = int(np.flatnonzero(a["S_rank"] > 0)[0])
    b = dict(a)
    b["S_rank"] = a["S_rank"].copy()
    b["S_rank"][i] = -2
    _expect_einval(uh, b, "S_rank")
    c = dict(a)
    c["S_rank"] = a["S_rank"].copy()
    r = int(a["row_rank"][a["adm_row"][i]])
    s = int(a["col_rank"][a["adm_col"][i]])
    c["S_rank"][i] = min(r, s) + 1
    _expect_einval(uh, c, "S_rank")
    d = dict(a)
    d["S_off"] = a["S_off"].copy()
    d["S_off"][i] = len(a["S_data"]) - 1  # the factors would run past the end of S_data
    _expect_einval(uh, d, "coupling matrix")


@pytest.mark.parametrize("ncta", [304, 14, 2])
@pytest.mark.parametrize("case", [(2048, 4.0, 32, 1e-6), (1000, 6.0, 24, 1e-5), (97, 3.0, 16, 1e-6),
                                  (40, 3.0, 64, 1e-6)])
def test_two_ctas_per_sm_packing_self_check_passes(uh, ncta, case):
    """Programs packed for two CTAs per SM (tiles up to 24 KB in 26 KB stages; the extended-
    precision stage checked as well), single operators, factored coefficients and a batch."""
    n, k, leaf, eps = case
    axes, noise = ((1.0, 0.7, 0.4), 0.01) if n == 1000 else ((1.0, 1.0, 1.0), 0.0)
    _, _, hf, h, op = oracle_ops(n, k, leaf, 1.0, eps, 1e-8, axes, noise)
    pp = uh.PackParams(0, 0, 0, 0, 2)
    desc, keep = uh.uh_desc_from_arrays(uh_arrays(op))
    for prec in (0, 1):
        rc = uh.lib.uh_pack_check_ex(C.byref(desc), prec, C.byref(pp), ncta)
        assert rc == uh.UH_OK, uh.lib.uh_last_error().decode()
    if n == 2048:
        fd, fkeep = uh.uh_desc_from_arrays(_factored_arrays(2048, 4.0, 32, 1e-6))
        assert uh.lib.uh_pack_check_ex(C.byref(fd), 1, C.byref(pp), ncta) == uh.UH_OK, uh.lib.uh_last_error().decode()
        built = [uh.uh_desc_from_arrays(a) for a in _batch_arrays()]
        arr = uh._desc_array([d for d, _ in built])
        assert uh.lib.uh_batch_pack_check_ex(arr, len(built), 1, pp, ncta) == uh.UH_OK, uh.lib.uh_last_error().decode()


def test_two_ctas_per_sm_complex128_and_bad_values(uh):
    """A complex128 program packs for two CTAs per SM too; out-of-range values are rejected."""
    a, _ = _small()
    desc, keep = uh.uh_desc_from_arrays(a)
    assert uh.lib.uh_pack_check_ex(C.byref(desc), 0, C.byref(uh.PackParams(0, 0, 0, 0, 2)), 304) == uh.UH_OK, \
        uh.lib.uh_last_error().decode()
    assert uh.lib.uh_pack_check_ex(C.byref(desc), 1, C.byref(uh.PackParams(0, 0, 0, 0, 3)), 304) == uh.UH_EINVAL
    assert "ctas_per_sm" in uh.lib.uh_last_error().decode()

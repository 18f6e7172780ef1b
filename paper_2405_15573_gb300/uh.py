"""ctypes binding of libuh.so (include/uh.h): argument marshalling only.

Every product runs in the library's CUDA kernels; this module only builds the C descriptors
from numpy arrays (or takes them from the host-side builder), passes device pointers of torch
tensors, and maps status codes to exceptions. There is no CPU fallback: if the library has not
been built, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libuh.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'`")
lib = C.CDLL(_LIB_PATH)

UH_OK, UH_EINVAL, UH_ENOMEM, UH_ECUDA, UH_ENOTREADY, UH_ETIMEOUT, UH_EBUSY = range(7)
UH_DATA_C128, UH_DATA_C64 = 0, 1
UH_PREC_C128, UH_PREC_C64, UH_PREC_C64_TF32, UH_PREC_C64_BF16X3 = 0, 1, 2, 3
_PREC = {"c128": UH_PREC_C128, "c64": UH_PREC_C64, "c64_tf32": UH_PREC_C64_TF32,
         "c64_bf16x3": UH_PREC_C64_BF16X3}
UH_MM_SIMT, UH_MM_TF32, UH_MM_BF16X3 = 0, 1, 2
_MM = {"simt": UH_MM_SIMT, "tf32": UH_MM_TF32, "bf16x3": UH_MM_BF16X3}

_p = C.c_void_p
_i32 = C.c_int32
_i64 = C.c_int64


class TreeDesc(C.Structure):
    _fields_ = [("n", _i64), ("perm", _p), ("n_clusters", _i32), ("cl_begin", _p), ("cl_size", _p)]


class DenseDesc(C.Structure):
    _fields_ = [("n_dense", _i64), ("row_cl", _p), ("col_cl", _p), ("off", _p), ("data", _p),
                ("len", _i64)]


class UHDesc(C.Structure):
    _fields_ = [("tree", TreeDesc), ("data_type", _i32),
                ("row_rank", _p), ("row_off", _p), ("U_data", _p), ("U_len", _i64),
                ("col_rank", _p), ("col_off", _p), ("V_data", _p), ("V_len", _i64),
                ("n_adm", _i64), ("adm_row", _p), ("adm_col", _p), ("S_off", _p), ("S_data", _p),
                ("S_len", _i64), ("dense", DenseDesc), ("S_rank", _p)]


class HDesc(C.Structure):
    _fields_ = [("tree", TreeDesc), ("data_type", _i32), ("n_adm", _i64),
                ("adm_row", _p), ("adm_col", _p), ("adm_rank", _p),
                ("X_off", _p), ("X_data", _p), ("X_len", _i64),
                ("Y_off", _p), ("Y_data", _p), ("Y_len", _i64), ("dense", DenseDesc)]


class Stats(C.Structure):
    _fields_ = [("n", _i64), ("precision", _i32), ("elem_bytes", _i32),
                ("n_row_bases", _i64), ("n_col_bases", _i64), ("n_adm", _i64), ("n_dense", _i64),
                ("E_U", _i64), ("E_V", _i64), ("E_S", _i64), ("E_D", _i64),
                ("sum_row_rank", _i64), ("sum_col_rank", _i64),
                ("rank_min", _i32), ("rank_max", _i32), ("rank_mean", C.c_double), ("csp", _i32),
                ("algo_bytes_matvec", _i64), ("device_bytes", _i64), ("packed_bytes", _i64),
                ("n_launches", _i32), ("n_items", _i64),
                ("matmat_mode", _i32), ("panel_bytes", _i64), ("panel_items", _i64),
                ("panel_mma_flops", _i64), ("pack_tile_bytes", _i64), ("pack_item_cost", _i64),
                ("pack_chunk_cost", _i64), ("pack_pool_unit", _i64), ("pack_ctas_per_sm", _i64), ("n_factored", _i64),
                ("sum_factored_rank", _i64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PackParams(C.Structure):
    """uh_pack_params: packing and scheduling of the streaming program (0 = default)."""
    _fields_ = [("tile_bytes", _i32), ("item_cost", _i32), ("chunk_cost", _i32), ("pool_unit", _i32),
                ("ctas_per_sm", _i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


lib.uh_last_error.restype = C.c_char_p
lib.uh_version.restype = C.c_char_p
for _name, _args in [
    ("uh_create", [C.POINTER(UHDesc), _i32, C.POINTER(_p)]),
    ("uh_create_ex", [C.POINTER(UHDesc), _i32, C.POINTER(PackParams), C.POINTER(_p)]),
    ("uh_pack_check_ex", [C.POINTER(UHDesc), _i32, C.POINTER(PackParams), _i32]),
    ("uh_destroy", [_p]),
    ("uh_matvec", [_p, _p, _p, _p]),
    ("uh_matmat", [_p, _i32, _p, _i64, _p, _i64, _i32, _p]),
    ("uh_reserve", [_p, _i32]),
    ("uh_stats", [_p, C.POINTER(Stats)]),
    ("h_create", [C.POINTER(HDesc), _i32, C.POINTER(_p)]),
    ("h_destroy", [_p]),
    ("h_matvec", [_p, _p, _p, _p]),
    ("h_matmat", [_p, _i32, _p, _i64, _p, _i64, _i32, _p]),
    ("h_reserve", [_p, _i32]),
    ("h_stats", [_p, C.POINTER(Stats)]),
    ("uh_check", [_p, _p]),
    ("uh_pack_check", [C.POINTER(UHDesc), _i32, _i32]),
    ("uh_debug_stalled_matvec", [_p, _p, _p, C.c_longlong, _p]),
    ("uh_debug_dfma_rate", [_i32, C.POINTER(C.c_double), _p]),
    ("h_pack_check", [C.POINTER(HDesc), _i32, _i32]),
    ("h_check", [_p, _p]),
    ("uh_matvec_mixed", [_p, _p, _p, _p]),
    ("uh_block_apply_noalloc", [_i64, _i64, _i32, _i32, _p, _i64, _p, _i64, _p, _i64, _p, _p, _i32, _p]),
    ("uh_batch_create", [C.POINTER(C.POINTER(UHDesc)), _i32, _i32, C.POINTER(_p)]),
    ("uh_batch_create_ex", [C.POINTER(C.POINTER(UHDesc)), _i32, _i32, C.POINTER(PackParams), C.POINTER(_p)]),
    ("uh_batch_tune", [C.POINTER(C.POINTER(UHDesc)), _i32, _i32, _i32, _i32, C.POINTER(PackParams),
                       C.POINTER(C.c_double), C.POINTER(C.c_double), _p]),
    ("uh_batch_destroy", [_p]),
    ("uh_batch_offsets", [_p, C.POINTER(_i64)]),
    ("uh_batch_matvec", [_p, _p, _p, _p]),
    ("uh_batch_check", [_p, _p]),
    ("uh_batch_stats", [_p, C.POINTER(Stats)]),
    ("uh_batch_pack_check", [C.POINTER(C.POINTER(UHDesc)), _i32, _i32, _i32]),
    ("uh_batch_pack_check_ex", [C.POINTER(C.POINTER(UHDesc)), _i32, _i32, C.POINTER(PackParams), _i32]),
    ("uh_server_create", [_i32, _i64, _i32, C.POINTER(_p)]),
    ("uh_server_destroy", [_p]),
    ("uh_solve_submit", [_p, _p, _p, C.c_double, _i32, _i32, C.POINTER(C.c_uint64)]),
    ("uh_solve_poll", [_p, C.c_uint64, _p, _p]),
]:
    getattr(lib, _name).argtypes = _args
    getattr(lib, _name).restype = C.c_int


class UHError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed ({code}): {lib.uh_last_error().decode()}")


def check(code: int, where: str) -> None:
    if code != UH_OK:
        raise UHError(code, where)


def version() -> str:
    return lib.uh_version().decode()


def _ptr(a) -> int | None:
    return None if a is None else a.ctypes.data


class _Keep:
    """Holds the numpy arrays a descriptor points into."""

    def __init__(self):
        self.arrays = []

    def __call__(self, a, dtype):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        self.arrays.append(a)
        return a


def _tree(keep, d, arrays):
    d.tree.n = int(arrays["n"])
    d.tree.perm = _ptr(keep(arrays.get("perm"), np.int64))
    cb = keep(arrays["cl_begin"], np.int64)
    d.tree.n_clusters = len(cb)
    d.tree.cl_begin = _ptr(cb)
    d.tree.cl_size = _ptr(keep(arrays["cl_size"], np.int64))


def _data(keep, a, c128):
    return keep(a, np.complex128 if c128 else np.complex64)


def _dense(keep, d, arrays, c128):
    row = keep(arrays["dense_row"], np.int32)
    d.dense.n_dense = len(row)
    d.dense.row_cl = _ptr(row)
    d.dense.col_cl = _ptr(keep(arrays["dense_col"], np.int32))
    d.dense.off = _ptr(keep(arrays["D_off"], np.int64))
    D = _data(keep, arrays["D_data"], c128)
    d.dense.data = _ptr(D)
    d.dense.len = len(D)


def uh_desc_from_arrays(arrays: dict):
    """Build a uh_desc from numpy arrays named like the descriptor fields (plus dense_row,
    dense_col, D_off, D_data). Returns (desc, keepalive)."""
    keep = _Keep()
    c128 = np.asarray(arrays["U_data"]).dtype != np.complex64
    d = UHDesc()
    _tree(keep, d, arrays)
    d.data_type = UH_DATA_C128 if c128 else UH_DATA_C64
    d.row_rank = _ptr(keep(arrays["row_rank"], np.int32))
    d.row_off = _ptr(keep(arrays["row_off"], np.int64))
    U = _data(keep, arrays["U_data"], c128)
    d.U_data, d.U_len = _ptr(U), len(U)
    d.col_rank = _ptr(keep(arrays["col_rank"], np.int32))
    d.col_off = _ptr(keep(arrays["col_off"], np.int64))
    V = _data(keep, arrays["V_data"], c128)
    d.V_data, d.V_len = _ptr(V), len(V)
    ar = keep(arrays["adm_row"], np.int32)
    d.n_adm = len(ar)
    d.adm_row = _ptr(ar)
    d.adm_col = _ptr(keep(arrays["adm_col"], np.int32))
    d.S_off = _ptr(keep(arrays["S_off"], np.int64))
    S = _data(keep, arrays["S_data"], c128)
    d.S_data, d.S_len = _ptr(S), len(S)
    if arrays.get("S_rank") is not None:
        d.S_rank = _ptr(keep(arrays["S_rank"], np.int32))
    _dense(keep, d, arrays, c128)
    return d, keep


def h_desc_from_arrays(arrays: dict):
    keep = _Keep()
    c128 = np.asarray(arrays["X_data"]).dtype != np.complex64
    d = HDesc()
    _tree(keep, d, arrays)
    d.data_type = UH_DATA_C128 if c128 else UH_DATA_C64
    ar = keep(arrays["adm_row"], np.int32)
    d.n_adm = len(ar)
    d.adm_row = _ptr(ar)
    d.adm_col = _ptr(keep(arrays["adm_col"], np.int32))
    d.adm_rank = _ptr(keep(arrays["adm_rank"], np.int32))
    d.X_off = _ptr(keep(arrays["X_off"], np.int64))
    X = _data(keep, arrays["X_data"], c128)
    d.X_data, d.X_len = _ptr(X), len(X)
    d.Y_off = _ptr(keep(arrays["Y_off"], np.int64))
    Y = _data(keep, arrays["Y_data"], c128)
    d.Y_data, d.Y_len = _ptr(Y), len(Y)
    _dense(keep, d, arrays, c128)
    return d, keep


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class _Op:
    _create = _destroy = _matvec = _matmat = _stats = _reserve = _check = None

    def __init__(self, desc, precision: str = "c64", params: "PackParams | None" = None):
        self.precision = precision
        self.c128 = precision == "c128"
        h = _p()
        if params is None:
            check(self._create(C.byref(desc), _PREC[precision], C.byref(h)), self._create.__name__)
        else:
            check(lib.uh_create_ex(C.byref(desc), _PREC[precision], C.byref(params), C.byref(h)), "uh_create_ex")
        self.handle = h
        s = Stats()
        check(self._stats(self.handle, C.byref(s)), "stats")
        self.n = s.n

    def stats(self) -> dict:
        s = Stats()
        check(self._stats(self.handle, C.byref(s)), "stats")
        return s.as_dict()

    def _check_vec(self, t, cols=None):
        import torch
        want = torch.complex128 if self.c128 else torch.complex64
        if not t.is_cuda or t.dtype != want:
            raise TypeError(f"expected a CUDA tensor of {want}, got {t.dtype} on {t.device}")
        if t.shape[0] != self.n:
            raise ValueError(f"length {t.shape[0]} != n = {self.n}")

    def matvec(self, x, y=None, stream=None):
        """y = A x for a CUDA tensor x (original ordering). Asynchronous on the stream."""
        import torch
        self._check_vec(x)
        if not x.is_contiguous():
            raise ValueError("x must be contiguous")
        if y is None:
            y = torch.empty_like(x)
        self._check_vec(y)
        check(self._matvec(self.handle, x.data_ptr(), y.data_ptr(), _stream_handle(stream)),
              "matvec")
        return y

    def matmat(self, X, Y=None, mode: str = "simt", stream=None):
        """Y = A X for an n x nrhs column-major CUDA tensor X (X.T contiguous, e.g.
        torch.empty(nrhs, n).T). mode: "simt", or "tf32" / "bf16x3" for an op created with
        precision "c64_tf32" / "c64_bf16x3". Asynchronous on the stream."""
        import torch
        self._check_vec(X)
        n, r = X.shape
        if X.stride(0) != 1:
            raise ValueError("X must be column-major (stride(0) == 1)")
        if Y is None:
            Y = torch.empty((r, n), dtype=X.dtype, device=X.device).T
        self._check_vec(Y)
        if Y.stride(0) != 1 or Y.shape != X.shape:
            raise ValueError("Y must be column-major with X's shape")
        check(self._matmat(self.handle, r, X.data_ptr(), max(X.stride(1), n), Y.data_ptr(),
                           max(Y.stride(1), n), _MM[mode], _stream_handle(stream)), "matmat")
        return Y

    def check(self, stream=None):
        """Synchronise the stream; raise UHError (UH_ETIMEOUT) if a device-side wait ran out."""
        check(self._check(self.handle, _stream_handle(stream)), "check")

    def reserve(self, max_nrhs: int):
        check(self._reserve(self.handle, max_nrhs), "reserve")

    def close(self):
        if getattr(self, "handle", None):
            self._destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_block_args(U, S, V, x, y):
    """Raises ValueError unless the five tensors describe one block product the library can run
    without touching memory outside them: one complex dtype, consistent sizes, column-major
    matrices, contiguous vectors, and every tensor on the current CUDA device."""
    import torch
    if x.dtype not in (torch.complex64, torch.complex128):
        raise ValueError(f"x must be complex64 or complex128, not {x.dtype}")
    for name, t in (("U", U), ("S", S), ("V", V), ("y", y)):
        if t.dtype != x.dtype:
            raise ValueError(f"{name} has dtype {t.dtype}, x has {x.dtype}")
    for name, t in (("U", U), ("S", S), ("V", V)):
        if t.dim() != 2:
            raise ValueError(f"{name} must be a matrix")
    for name, t in (("x", x), ("y", y)):
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous vector")
    m, lt = U.shape
    n, ls = V.shape
    if tuple(S.shape) != (lt, ls):
        raise ValueError(f"S is {tuple(S.shape)}, expected ({lt}, {ls}) from U and V")
    if x.numel() != n or y.numel() != m:
        raise ValueError(f"x has {x.numel()} values (needs {n}), y has {y.numel()} (needs {m})")
    for name, t, rows in (("U", U, m), ("S", S, lt), ("V", V, n)):
        if t.numel() and (t.stride(0) != 1 or t.stride(1) < rows):
            raise ValueError(f"{name} must be column-major (stride (1, >= {rows}))")
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    for name, t in (("U", U), ("S", S), ("V", V), ("x", x), ("y", y)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")


def block_apply_noalloc(U, S, V, x, y, stream=None):
    """y = U (S (V^* x)) for one UH block without any allocation by the library (uh.h,
    uh_block_apply_noalloc). U (m x lt), S (lt x ls), V (n x ls) are column-major CUDA tensors
    (tensor.T contiguous), x (n) and y (m) contiguous; all complex128 or all complex64."""
    _check_block_args(U, S, V, x, y)
    import torch
    c128 = x.dtype == torch.complex128
    m, lt = U.shape
    n, ls = V.shape
    check(lib.uh_block_apply_noalloc(m, n, lt, ls, U.data_ptr(), max(U.stride(1), m), S.data_ptr(),
                                     max(S.stride(1), lt), V.data_ptr(), max(V.stride(1), n),
                                     x.data_ptr(), y.data_ptr(),
                                     UH_PREC_C128 if c128 else UH_PREC_C64, _stream_handle(stream)),
          "uh_block_apply_noalloc")
    return y


class UHOp(_Op):
    """Device-resident uniform H-matrix (uh_create)."""
    _create = lib.uh_create
    _destroy = lib.uh_destroy
    _matvec = lib.uh_matvec
    _matmat = lib.uh_matmat
    _stats = lib.uh_stats
    _reserve = lib.uh_reserve
    _check = lib.uh_check

    @classmethod
    def from_arrays(cls, arrays: dict, precision: str = "c64", params: "PackParams | None" = None):
        desc, keep = uh_desc_from_arrays(arrays)
        return cls(desc, precision, params)

    def matvec_mixed(self, x, y=None, stream=None):
        """y = A x with the complex64-stored operator in extended-precision arithmetic
        (uh_matvec_mixed): x and y are contiguous complex128 CUDA tensors of length n."""
        import torch
        if self.c128:
            raise ValueError("matvec_mixed needs an op with complex64 storage")
        for name, t in (("x", x), ("y", y)):
            if t is None:
                continue
            if not t.is_cuda or t.dtype != torch.complex128 or t.dim() != 1 or t.shape[0] != self.n \
                    or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA tensor of {self.n} complex128")
        if y is None:
            y = torch.empty_like(x)
        check(lib.uh_matvec_mixed(self.handle, x.data_ptr(), y.data_ptr(), _stream_handle(stream)),
              "uh_matvec_mixed")
        return y


def _desc_array(descs):
    return (C.POINTER(UHDesc) * len(descs))(*[C.pointer(d) for d in descs])


class UHBatch:
    """Many independent UH operators applied in one launch (uh.h, uh_batch_*). x and y of
    matvec() hold the operators' vectors back to back: operator k at offsets[k]:offsets[k+1]."""

    def __init__(self, descs, precision: str = "c64", params: "PackParams | None" = None):
        self.precision = precision
        self.c128 = precision == "c128"
        self.count = len(descs)
        h = _p()
        check(lib.uh_batch_create_ex(_desc_array(descs), self.count, _PREC[precision],
                                     C.byref(params) if params is not None else None, C.byref(h)),
              "uh_batch_create_ex")
        self.handle = h
        off = (_i64 * (self.count + 1))()
        check(lib.uh_batch_offsets(self.handle, off), "uh_batch_offsets")
        self.offsets = np.array(off[:], dtype=np.int64)
        self.n = int(self.offsets[-1])

    @classmethod
    def from_arrays(cls, arrays_list, precision: str = "c64", params: "PackParams | None" = None):
        built = [uh_desc_from_arrays(a) for a in arrays_list]
        return cls([d for d, _ in built], precision, params)

    @staticmethod
    def tune(descs, precision: str = "c64", sample: int = 0, reps: int = 20, stream=None):
        """uh_batch_tune: (best PackParams, best ms, default ms) for this set of operators."""
        best = PackParams()
        bms, dms = C.c_double(0.0), C.c_double(0.0)
        check(lib.uh_batch_tune(_desc_array(descs), len(descs), _PREC[precision], sample, reps, C.byref(best),
                                C.byref(bms), C.byref(dms), _stream_handle(stream)), "uh_batch_tune")
        return best, bms.value, dms.value

    def stats(self) -> dict:
        s = Stats()
        check(lib.uh_batch_stats(self.handle, C.byref(s)), "uh_batch_stats")
        return s.as_dict()

    def matvec(self, x, y=None, stream=None):
        import torch
        want = torch.complex128 if self.c128 else torch.complex64
        if not x.is_cuda or x.dtype != want or x.shape[0] != self.n or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous CUDA tensor of {self.n} {want}")
        if y is None:
            y = torch.empty_like(x)
        if not y.is_cuda or y.dtype != want or y.shape[0] != self.n or not y.is_contiguous():
            raise ValueError(f"y must be a contiguous CUDA tensor of {self.n} {want}")
        check(lib.uh_batch_matvec(self.handle, x.data_ptr(), y.data_ptr(), _stream_handle(stream)),
              "uh_batch_matvec")
        return y

    def check(self, stream=None):
        check(lib.uh_batch_check(self.handle, _stream_handle(stream)), "uh_batch_check")

    def close(self):
        if getattr(self, "handle", None):
            lib.uh_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SolveInfo(C.Structure):
    _fields_ = [("status", _i32), ("converged", _i32), ("iterations", _i32), ("restarts", _i32),
                ("rel_residual", C.c_double), ("queue_s", C.c_double), ("latency_s", C.c_double),
                ("paired_steps", _i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Server:
    """GMRES serving runtime (uh.h, uh_server_* / uh_solve_*): submit(op, b) returns a ticket,
    poll(ticket) returns None until the solve has ended, then (x, info)."""

    def __init__(self, max_active: int = 8, hbm_budget: int = 8 << 30, queue_capacity: int = 64):
        h = _p()
        check(lib.uh_server_create(max_active, hbm_budget, queue_capacity, C.byref(h)), "uh_server_create")
        self.handle = h
        self._n = {}

    def submit(self, op, b, tol: float = 1e-6, restart: int = 30, maxit: int = 300):
        """Ticket of the solve op x = b (b: n complex values, copied), or None if the server is
        busy (UH_EBUSY)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        if b.shape != (op.n,):
            raise ValueError(f"b must have {op.n} entries")
        t = C.c_uint64()
        rc = lib.uh_solve_submit(self.handle, op.handle, b.ctypes.data, float(tol), restart, maxit, C.byref(t))
        if rc == UH_EBUSY:
            return None
        check(rc, "uh_solve_submit")
        self._n[t.value] = op.n
        return t.value

    def poll(self, ticket: int):
        n = self._n.get(ticket)
        x = np.empty(n, np.complex128) if n is not None else None
        info = SolveInfo()
        rc = lib.uh_solve_poll(self.handle, ticket, None if x is None else x.ctypes.data, C.byref(info))
        if rc == UH_ENOTREADY:
            return None
        self._n.pop(ticket, None)
        check(rc, "uh_solve_poll")
        return x, info.as_dict()

    def wait(self, ticket: int, timeout: float = 60.0, interval: float = 1e-4):
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.time() - t0 > timeout:
                raise TimeoutError(f"solve {ticket} not done after {timeout} s")
            time.sleep(interval)

    def close(self):
        if getattr(self, "handle", None):
            lib.uh_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HOp(_Op):
    """Device-resident H-matrix (h_create), the plain form."""
    _create = lib.h_create
    _destroy = lib.h_destroy
    _matvec = lib.h_matvec
    _matmat = lib.h_matmat
    _stats = lib.h_stats
    _reserve = lib.h_reserve
    _check = lib.h_check

    @classmethod
    def from_arrays(cls, arrays: dict, precision: str = "c64"):
        desc, keep = h_desc_from_arrays(arrays)
        return cls(desc, precision)


# ------------------------------------------------------------------ host-side builder (uh_build.h)

class BuildParams(C.Structure):
    _fields_ = [("wavenumber", C.c_double), ("leaf", _i32), ("eta", C.c_double),
                ("eps", C.c_double), ("tol_aca", C.c_double), ("nthreads", _i32), ("strong", _i32),
                ("factored", _i32)]


class BuildInfo(C.Structure):
    _fields_ = [("n", _i64), ("n_clusters", _i64), ("n_adm", _i64), ("n_dense", _i64),
                ("depth", _i32), ("csp", _i32), ("kmax_aca", _i32), ("kmax_h", _i32),
                ("lmax", _i32), ("seconds_tree", C.c_double), ("seconds_aca", C.c_double),
                ("seconds_bases", C.c_double), ("seconds_dense", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


lib.uhb_build_helmholtz.argtypes = [_i64, _p, C.POINTER(BuildParams), C.POINTER(_p)]
lib.uhb_build_helmholtz_gpu.argtypes = [_i64, _p, C.POINTER(BuildParams), C.POINTER(_p)]
lib.uhb_uh_desc.argtypes = [_p, C.POINTER(UHDesc)]
lib.uhb_h_desc.argtypes = [_p, C.POINTER(HDesc)]
lib.uhb_info.argtypes = [_p, C.POINTER(BuildInfo)]
lib.uhb_free.argtypes = [_p]
for _f in (lib.uhb_build_helmholtz, lib.uhb_build_helmholtz_gpu, lib.uhb_uh_desc, lib.uhb_h_desc, lib.uhb_info,
           lib.uhb_free):
    _f.restype = C.c_int


def _view(ptr, count, dtype):
    if count == 0 or not ptr:
        return np.zeros(0, dtype)
    nbytes = int(count) * np.dtype(dtype).itemsize
    buf = (C.c_char * nbytes).from_address(ptr)
    return np.frombuffer(buf, dtype=dtype, count=int(count))


class HelmholtzModel:
    """Synthetic Helmholtz collocation operator built on the host (uh_build.h) in both UH and
    H form. The arrays live in the library; uh_op()/h_op() upload them to the GPU."""

    def __init__(self, points, wavenumber, leaf, eta, eps, tol_aca, nthreads: int = 0, strong: bool = False,
                 device: bool = False, factored: bool = False):
        """device=True: the construction runs on the current CUDA device (uhb_build_helmholtz_gpu).
        factored=True: coefficient matrices stored factored where smaller (uhb_params.factored)."""
        pts = np.ascontiguousarray(points, dtype=np.float64)
        prm = BuildParams(float(wavenumber), int(leaf), float(eta), float(eps), float(tol_aca),
                          int(nthreads), 1 if strong else 0, 1 if factored else 0)
        h = _p()
        fn = lib.uhb_build_helmholtz_gpu if device else lib.uhb_build_helmholtz
        check(fn(len(pts), pts.ctypes.data, C.byref(prm), C.byref(h)), fn.__name__)
        self.handle = h
        self.n = len(pts)

    def info(self) -> dict:
        i = BuildInfo()
        check(lib.uhb_info(self.handle, C.byref(i)), "uhb_info")
        return i.as_dict()

    def uh_desc(self) -> UHDesc:
        d = UHDesc()
        check(lib.uhb_uh_desc(self.handle, C.byref(d)), "uhb_uh_desc")
        return d

    def h_desc(self) -> HDesc:
        d = HDesc()
        check(lib.uhb_h_desc(self.handle, C.byref(d)), "uhb_h_desc")
        return d

    def uh_op(self, precision: str = "c64", params: "PackParams | None" = None) -> "UHOp":
        return UHOp(self.uh_desc(), precision, params)

    def h_op(self, precision: str = "c64") -> "HOp":
        return HOp(self.h_desc(), precision)

    def _tree_arrays(self, t):
        ncl = t.n_clusters
        return dict(n=t.n, perm=_view(t.perm, t.n, np.int64),
                    cl_begin=_view(t.cl_begin, ncl, np.int64),
                    cl_size=_view(t.cl_size, ncl, np.int64))

    def _dense_arrays(self, d):
        k = d.n_dense
        return dict(dense_row=_view(d.row_cl, k, np.int32),
                    dense_col=_view(d.col_cl, k, np.int32),
                    D_off=_view(d.off, k, np.int64),
                    D_data=_view(d.data, d.len, np.complex128))

    def uh_arrays(self, copy: bool = True) -> dict:
        """The UH descriptor arrays (same names as uh_desc_from_arrays takes): copies, or with
        copy=False views into the model that are valid until close()."""
        d = self.uh_desc()
        ncl = d.tree.n_clusters
        a = self._tree_arrays(d.tree)
        a.update(row_rank=_view(d.row_rank, ncl, np.int32),
                 row_off=_view(d.row_off, ncl, np.int64),
                 U_data=_view(d.U_data, d.U_len, np.complex128),
                 col_rank=_view(d.col_rank, ncl, np.int32),
                 col_off=_view(d.col_off, ncl, np.int64),
                 V_data=_view(d.V_data, d.V_len, np.complex128),
                 adm_row=_view(d.adm_row, d.n_adm, np.int32),
                 adm_col=_view(d.adm_col, d.n_adm, np.int32),
                 S_off=_view(d.S_off, d.n_adm, np.int64),
                 S_data=_view(d.S_data, d.S_len, np.complex128),
                 S_rank=_view(d.S_rank, d.n_adm, np.int32) if d.S_rank else None)
        a.update(self._dense_arrays(d.dense))
        return {k: (v.copy() if copy and isinstance(v, np.ndarray) else v) for k, v in a.items()}

    def h_arrays(self) -> dict:
        d = self.h_desc()
        a = self._tree_arrays(d.tree)
        a.update(adm_row=_view(d.adm_row, d.n_adm, np.int32),
                 adm_col=_view(d.adm_col, d.n_adm, np.int32),
                 adm_rank=_view(d.adm_rank, d.n_adm, np.int32),
                 X_off=_view(d.X_off, d.n_adm, np.int64),
                 X_data=_view(d.X_data, d.X_len, np.complex128),
                 Y_off=_view(d.Y_off, d.n_adm, np.int64),
                 Y_data=_view(d.Y_data, d.Y_len, np.complex128))
        a.update(self._dense_arrays(d.dense))
        return {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in a.items()}

    def close(self):
        if getattr(self, "handle", None):
            lib.uhb_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

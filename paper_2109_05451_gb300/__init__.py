"""paper_2109_05451_gb300 -- H^2 matrix-vector product on one GB300 GPU.

A thin ctypes binding over ``libh2.so`` (``include/h2.h``): functions with the same
names as the C ABI, plus a small ``H2Operator`` convenience class. Arguments are
marshalled only; every step of the product runs in the library's CUDA kernels. Device
buffers are torch tensors (their ``data_ptr()``), streams are torch streams.

There is no CPU fallback: importing works without a GPU (the host build and the
structure queries are host code), but every device call raises if the library or the
GPU is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

H2_OK, H2_EINVAL, H2_ENOMEM, H2_ECUDA, H2_ETIMEOUT, H2_ESTATE, H2_ENOTCONV = 0, -1, -2, -3, -4, -5, 1
H2_ECANCELED = -6
H2_FP64, H2_FP32, H2_BF16X2, H2_FP32_MF = 0, 1, 2, 3
H2_K_EXP, H2_K_GAUSS, H2_K_IMQ, H2_K_POLY = 0, 1, 2, 3
H2_MAX_LEVELS = 32
KERNELS = {"exp": H2_K_EXP, "gauss": H2_K_GAUSS, "imq": H2_K_IMQ, "poly": H2_K_POLY}
PRECISIONS = {"fp64": H2_FP64, "fp32": H2_FP32, "bf16x2": H2_BF16X2, "fp32mf": H2_FP32_MF}


class H2Error(RuntimeError):
    def __init__(self, status: int, call: str):
        super().__init__(f"{call}: {h2_status_str(status)} ({status})")
        self.status = status


class h2_kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("b", C.c_double), ("deg", C.c_int)]


class h2_info(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("dim", C.c_int), ("depth", C.c_int), ("rank", C.c_int), ("leaf_size", C.c_int),
        ("cheb_order", C.c_int), ("eta", C.c_double), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
        ("n_coupling", C.c_int64), ("n_dense", C.c_int64), ("coupling_per_level", C.c_int64 * H2_MAX_LEVELS),
        ("max_coupling_per_row", C.c_int32), ("max_dense_per_row", C.c_int32), ("coupling_entries", C.c_int64),
        ("dense_entries", C.c_int64), ("basis_entries", C.c_int64), ("transfer_entries", C.c_int64),
        ("uploaded_prec", C.c_int), ("device_bytes", C.c_size_t),
    ]


class h2_request_result(C.Structure):
    _fields_ = [("request_id", C.c_int64), ("status", C.c_int), ("iters", C.c_int), ("true_relres", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class h2_compress_info(C.Structure):
    _fields_ = [("tau", C.c_double), ("norm_lowrank", C.c_double), ("dropped_energy", C.c_double), ("depth", C.c_int),
                ("rank_in", C.c_int), ("rank_out", C.c_int), ("level_rank", C.c_int * H2_MAX_LEVELS),
                ("ms", C.c_double * 4), ("flops", C.c_double * 4), ("jacobi_sweeps", C.c_int64),
                ("lowrank_bytes_in", C.c_size_t), ("lowrank_bytes_out", C.c_size_t)]


# name -> (restype, argtypes); every symbol declared in include/h2.h
_P, _I64, _I, _D, _SZ = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_size_t
SIGNATURES = {
    "h2_build": (_I, [_P, _I64, _I, h2_kernel, _I, _I, _D, C.POINTER(_P)]),
    "h2_upload": (_I, [_P, _I, _P]),
    "h2_workspace_bytes": (_SZ, [_P, _I]),
    "h2_matvec": (_I, [_P, _P, _P, _I, _D, _D, _P]),
    "h2_matvec_ws": (_I, [_P, _P, _P, _I, _D, _D, _P, _SZ, _P]),
    "h2_matvec_noalloc": (_I, [_P, _P, _P, _I, _D, _D, _P]),
    "h2_cg_solve": (_I, [_P, _D, _P, _P, _D, _I, C.POINTER(_I), C.POINTER(_D), _P]),
    "h2_get_info": (_I, [_P, C.POINTER(h2_info)]),
    "h2_get_perm": (_I, [_P, _P]),
    "h2_get_coupling_csr": (_I, [_P, _P, _P]),
    "h2_get_dense_csr": (_I, [_P, _P, _P]),
    "h2_get_bases": (_I, [_P, _P, _P]),
    "h2_set_timing": (_I, [_P, _I]),
    "h2_set_fp32_tensor": (_I, [_P, _I]),
    "h2_get_timing": (_I, [_P, _P, _P, _P]),
    "h2_destroy": (_I, [_P]),
    "h2_status_str": (C.c_char_p, [_I]),
    "h2_batch_create": (_I, [C.POINTER(_P), _I, C.POINTER(_P), C.POINTER(_P), C.POINTER(_I), _D, _D, _I,
                             C.POINTER(_P)]),
    "h2_batch_run": (_I, [_P, _P]),
    "h2_batch_check": (_I, [_P]),
    "h2_batch_describe": (_I, [_P, C.c_char_p, _SZ]),
    "h2_batch_destroy": (_I, [_P]),
    "h2_save": (_I, [_P, C.c_char_p]),
    "h2_compress": (_I, [_P, _D, _P, C.POINTER(_P), C.POINTER(h2_compress_info)]),
    "h2_get_level_ranks": (_I, [_P, C.POINTER(C.c_int)]),
    "h2_load": (_I, [C.c_char_p, C.POINTER(_P)]),
    "h2_server_create": (_I, [_SZ, _I, _I64, C.POINTER(_P)]),
    "h2_server_request_bytes": (_SZ, [_P]),
    "h2_server_submit": (_I, [_P, _P, _D, _P, _P, _D, _I, C.POINTER(_I64)]),
    "h2_server_submit_refined": (_I, [_P, _P, _P, _D, _P, _P, _D, _D, _I, C.POINTER(_I64)]),
    "h2_server_request_bytes_refined": (_SZ, [_P, _P]),
    "h2_server_poll": (_I, [_P, C.POINTER(h2_request_result), _I, C.POINTER(_I)]),
    "h2_server_wait": (_I, [_P, _D]),
    "h2_server_cancel": (_I, [_P, _I64]),
    "h2_server_destroy": (_I, [_P]),
    "h2_selftest_wait_timeout": (_I, [_I64]),
    "h2_measure_peak": (_I, [_I, _D, C.POINTER(_D), C.POINTER(_D)]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libh2.so (building it if missing or stale); raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libh2.so not built ({path}); run paper_2109_05451_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, call: str, allow=(H2_OK,)):
    if rc not in allow:
        raise H2Error(rc, call)
    return rc


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- C ABI, same names

def h2_status_str(status: int) -> str:
    return load().h2_status_str(int(status)).decode()


def h2_build(points, kernel, leaf_size: int, cheb_order: int, eta: float) -> int:
    """Build on the host; returns the opaque handle (an integer address)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    name, a, b, deg = kernel
    ker = h2_kernel(KERNELS[name], float(a), float(b), int(deg))
    h = C.c_void_p()
    _check(load().h2_build(_np_ptr(pts), n, dim, ker, int(leaf_size), int(cheb_order), float(eta), C.byref(h)),
           "h2_build")
    return h.value


def h2_upload(h: int, prec, stream=None) -> None:
    prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    _check(load().h2_upload(h, prec, _stream_ptr(stream)), "h2_upload")


def h2_workspace_bytes(h: int, nv: int) -> int:
    return int(load().h2_workspace_bytes(h, int(nv)))


def h2_matvec(h: int, X, Y, nv: int, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
    """X, Y: device tensors (n x nv column-major, i.e. shape (nv, n) contiguous or a
    Fortran-ordered (n, nv) view); pointers are passed through unchanged."""
    _check(load().h2_matvec(h, X.data_ptr(), Y.data_ptr(), int(nv), float(alpha), float(beta),
                            _stream_ptr(stream)), "h2_matvec")


def h2_matvec_ws(h: int, X, Y, nv: int, alpha: float, beta: float, workspace, ws_bytes: int, stream=None) -> None:
    _check(load().h2_matvec_ws(h, X.data_ptr(), Y.data_ptr(), int(nv), float(alpha), float(beta),
                               workspace.data_ptr(), int(ws_bytes), _stream_ptr(stream)), "h2_matvec_ws")


H2_NOALLOC_SCRATCH_BYTES = 64 << 20


def h2_matvec_noalloc(h: int, X, Y, nv: int, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
    """As h2_matvec, but the workspace is the library's fixed per-GPU scratch area: nothing
    is allocated, for callers that must not allocate device memory. Operators whose
    workspace exceeds H2_NOALLOC_SCRATCH_BYTES are rejected (H2_EINVAL). Calls that overlap
    on the GPU share the scratch area and race; order them on one stream."""
    _check(load().h2_matvec_noalloc(h, X.data_ptr(), Y.data_ptr(), int(nv), float(alpha), float(beta),
                                    _stream_ptr(stream)), "h2_matvec_noalloc")


def h2_cg_solve(h: int, sigma2: float, b, x, tol: float, maxit: int, stream=None):
    """Returns (status, iterations, true relative residual); status is H2_OK or H2_ENOTCONV."""
    it = C.c_int(0)
    rr = C.c_double(0.0)
    rc = load().h2_cg_solve(h, float(sigma2), b.data_ptr(), x.data_ptr(), float(tol), int(maxit), C.byref(it),
                            C.byref(rr), _stream_ptr(stream))
    _check(rc, "h2_cg_solve", allow=(H2_OK, H2_ENOTCONV))
    return rc, it.value, rr.value


def h2_save(h: int, path: str):
    _check(load().h2_save(h, os.fsencode(path)), "h2_save")


def h2_load(path: str) -> int:
    h = C.c_void_p()
    _check(load().h2_load(os.fsencode(path), C.byref(h)), "h2_load")
    return h.value


def h2_compress(h: int, tau: float, stream=None):
    """Sec. 5 recompression on the GPU: (new handle, h2_compress_info)."""
    out = C.c_void_p()
    info = h2_compress_info()
    _check(load().h2_compress(h, float(tau), _stream_ptr(stream), C.byref(out), C.byref(info)), "h2_compress")
    return out.value, info


def h2_get_level_ranks(h: int) -> list:
    depth = h2_get_info(h).depth
    r = (C.c_int * (depth + 1))()
    _check(load().h2_get_level_ranks(h, r), "h2_get_level_ranks")
    return list(r)


def h2_get_info(h: int) -> h2_info:
    info = h2_info()
    _check(load().h2_get_info(h, C.byref(info)), "h2_get_info")
    return info


def h2_get_perm(h: int) -> np.ndarray:
    info = h2_get_info(h)
    out = np.empty(info.n, dtype=np.int64)
    _check(load().h2_get_perm(h, _np_ptr(out)), "h2_get_perm")
    return out


def h2_get_coupling_csr(h: int):
    info = h2_get_info(h)
    rowptr = np.empty(info.n_nodes + 2, dtype=np.int64)
    col = np.empty(max(1, info.n_coupling), dtype=np.int32)
    _check(load().h2_get_coupling_csr(h, _np_ptr(rowptr), _np_ptr(col)), "h2_get_coupling_csr")
    return rowptr, col[:info.n_coupling]


def h2_get_dense_csr(h: int):
    info = h2_get_info(h)
    rowptr = np.empty(info.n_leaves + 1, dtype=np.int64)
    col = np.empty(max(1, info.n_dense), dtype=np.int32)
    _check(load().h2_get_dense_csr(h, _np_ptr(rowptr), _np_ptr(col)), "h2_get_dense_csr")
    return rowptr, col[:info.n_dense]


def h2_get_bases(h: int):
    info = h2_get_info(h)
    U = np.empty((info.n, info.rank))
    E = np.empty((info.n_nodes + 1, info.rank, info.rank))
    _check(load().h2_get_bases(h, _np_ptr(U), _np_ptr(E)), "h2_get_bases")
    return U, E


H2_NPHASES = 4
PHASES = ("upsweep", "stream", "top", "downsweep")


def h2_set_fp32_tensor(h: int, enable: bool) -> None:
    """FP32 passes of more than 8 vectors on the tensor cores (3xTF32; default) or on the CUDA cores."""
    _check(load().h2_set_fp32_tensor(h, int(bool(enable))), "h2_set_fp32_tensor")


def h2_set_timing(h: int, enable: bool) -> None:
    _check(load().h2_set_timing(h, int(bool(enable))), "h2_set_timing")


def h2_get_timing(h: int):
    """Waits for the recorded phase events; returns (ms per phase, launches per phase, products)."""
    ms = np.zeros(H2_NPHASES)
    launches = np.zeros(H2_NPHASES, dtype=np.int64)
    prods = np.zeros(1, dtype=np.int64)
    _check(load().h2_get_timing(h, _np_ptr(ms), _np_ptr(launches), _np_ptr(prods)), "h2_get_timing")
    return ms, launches, int(prods[0])


H2_PEAK_DFMA, H2_PEAK_FFMA, H2_PEAK_EX2 = 0, 1, 2
PEAK_UNITS = {"dfma": H2_PEAK_DFMA, "ffma": H2_PEAK_FFMA, "ex2": H2_PEAK_EX2}


def h2_measure_peak(unit, target_ms: float = 30.0):
    """Measured rate of one arithmetic unit of the current device: (rate, ms of the fastest
    launch); flop/s for "dfma" / "ffma", evaluations/s for "ex2"."""
    u = PEAK_UNITS[unit] if isinstance(unit, str) else int(unit)
    rate = C.c_double(0.0)
    ms = C.c_double(0.0)
    _check(load().h2_measure_peak(u, float(target_ms), C.byref(rate), C.byref(ms)), "h2_measure_peak")
    return rate.value, ms.value


def h2_destroy(h: int) -> None:
    if h:
        _check(load().h2_destroy(h), "h2_destroy")


# ---------------------------------------------------------------- convenience class

class H2Operator:
    """Owns one handle. ``matvec`` takes torch tensors of shape (n, nv) in column-major
    (Fortran) layout or (n,) vectors; the dtype must match the uploaded precision."""

    def __init__(self, points, kernel, leaf_size: int, cheb_order: int, eta: float, *, _handle=None):
        self.handle = _handle if _handle is not None else h2_build(points, kernel, leaf_size, cheb_order, eta)
        self.info = h2_get_info(self.handle)
        self.n = int(self.info.n)
        self.prec = None

    @classmethod
    def load(cls, path: str) -> "H2Operator":
        """An operator read from a file written by ``save`` (not uploaded)."""
        return cls(None, None, 0, 0, 0.0, _handle=h2_load(path))

    def save(self, path: str) -> None:
        h2_save(self.handle, path)

    def compress(self, tau: float, stream=None) -> "H2Operator":
        """A new operator compressed to relative tolerance tau (Sec. 5, on the GPU, FP64);
        not uploaded. Its h2_compress_info is kept as ``compress_info``."""
        hc, info = h2_compress(self.handle, tau, stream)
        op = H2Operator(None, None, 0, 0, 0.0, _handle=hc)
        op.compress_info = info
        return op

    @property
    def level_ranks(self) -> list:
        return h2_get_level_ranks(self.handle)

    def upload(self, prec="fp32", stream=None):
        h2_upload(self.handle, prec, stream)
        self.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        self.info = h2_get_info(self.handle)
        return self

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.prec == H2_FP64 else torch.float32

    def new_vectors(self, nv: int, fill=None):
        """A device (n, nv) column-major tensor of the operator's dtype."""
        import torch
        t = torch.empty((nv, self.n), dtype=self.dtype, device="cuda")
        if fill is not None:
            t.fill_(fill)
        return t.t()

    def matvec(self, X, Y=None, alpha: float = 1.0, beta: float = 0.0, stream=None):
        nv = 1 if X.dim() == 1 else X.shape[1]
        _check_colmajor(X, self.n, nv, self.dtype)
        if Y is None:
            Y = self.new_vectors(nv).squeeze(1) if X.dim() == 1 else self.new_vectors(nv)
            beta = 0.0
        _check_colmajor(Y, self.n, nv, self.dtype)
        h2_matvec(self.handle, X, Y, nv, alpha, beta, stream)
        return Y

    def close(self):
        if getattr(self, "handle", None):
            h2_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_colmajor(t, n: int, nv: int, dtype):
    if not t.is_cuda or t.dtype != dtype:
        raise ValueError(f"expected a CUDA tensor of dtype {dtype}")
    if t.dim() == 1:
        ok = t.shape[0] == n and nv == 1 and t.stride(0) == 1
    else:
        ok = tuple(t.shape) == (n, nv) and t.stride(0) == 1 and (nv == 1 or t.stride(1) == n)
    if not ok:
        raise ValueError("expected an (n, nv) column-major tensor with leading dimension n")


class H2Server:
    """CG serving loop (h2_server_*): solves of (A + sigma2 I) x = b on resident operators,
    admitted in FIFO order as slots and slot memory free up, running concurrently on the GPU.
    Holds each request's host arrays until its result is polled."""

    def __init__(self, slot_memory_bytes: int, max_slots: int, max_points: int):
        h = C.c_void_p()
        _check(load().h2_server_create(int(slot_memory_bytes), int(max_slots), int(max_points), C.byref(h)),
               "h2_server_create")
        self.handle = h.value
        self._live = {}  # request id -> (b, x)

    @staticmethod
    def request_bytes(op: "H2Operator") -> int:
        return int(load().h2_server_request_bytes(op.handle))

    @staticmethod
    def request_bytes_refined(op: "H2Operator", op64: "H2Operator") -> int:
        return int(load().h2_server_request_bytes_refined(op.handle, op64.handle))

    def submit(self, op: "H2Operator", b: np.ndarray, tol: float, maxit: int, sigma2: float = 0.0,
               op64: "H2Operator" = None, inner_tol: float = 1e-3) -> int:
        """Queue a CG solve; with op64 (an FP64 upload of the same operator) a mixed-precision
        refinement: inner CG on op to inner_tol, outer FP64 residuals on op64 until tol."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if b.shape != (op.n,):
            raise ValueError("b must have n entries")
        x = np.empty_like(b)
        rid = C.c_int64(0)
        if op64 is None:
            _check(load().h2_server_submit(self.handle, op.handle, float(sigma2), _np_ptr(b), _np_ptr(x), float(tol),
                                           int(maxit), C.byref(rid)), "h2_server_submit")
        else:
            _check(load().h2_server_submit_refined(self.handle, op.handle, op64.handle, float(sigma2), _np_ptr(b),
                                                   _np_ptr(x), float(tol), float(inner_tol), int(maxit),
                                                   C.byref(rid)), "h2_server_submit_refined")
        self._live[rid.value] = (b, x)
        return rid.value

    def poll(self, max_results: int = 256) -> list:
        """Completed requests: dicts with id, status, iters, true_relres, times and x."""
        buf = (h2_request_result * max_results)()
        n = C.c_int(0)
        _check(load().h2_server_poll(self.handle, buf, max_results, C.byref(n)), "h2_server_poll")
        out = []
        for r in buf[: n.value]:
            b, x = self._live.pop(r.request_id)
            out.append({"id": r.request_id, "status": r.status, "iters": r.iters, "true_relres": r.true_relres,
                        "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done, "x": x})
        return out

    def cancel(self, request_id: int) -> int:
        """Cancel a queued or running request; its result (status H2_ECANCELED) is still polled."""
        return int(load().h2_server_cancel(self.handle, int(request_id)))

    def wait(self, timeout_s: float = 600.0) -> int:
        rc = load().h2_server_wait(self.handle, float(timeout_s))
        _check(rc, "h2_server_wait", allow=(H2_OK, H2_ETIMEOUT))
        return rc

    def close(self):
        if getattr(self, "handle", None):
            load().h2_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


H2_BATCH_AUTOTUNE = 1
H2_BATCH_MEMBER_SWEEPS = 2


class H2Batch:
    """Batched products of uneven operators (h2_batch_*): Y_i = alpha A_i X_i + beta Y_i for
    every member, captured once as a CUDA graph and replayed by run(). Xs, Ys: CUDA tensors
    (n_i, nv_i), column-major, of the members' element type; kept alive by the batch."""

    def __init__(self, ops, Xs, Ys, alpha: float = 1.0, beta: float = 0.0, autotune: bool = False,
                 member_sweeps: bool = False):
        if not (len(ops) == len(Xs) == len(Ys)) or not ops:
            raise ValueError("ops, Xs and Ys must have the same nonzero length")
        nvs = []
        for op, X, Y in zip(ops, Xs, Ys):
            nv = 1 if X.dim() == 1 else X.shape[1]
            _check_colmajor(X, op.n, nv, op.dtype)
            _check_colmajor(Y, op.n, nv, op.dtype)
            nvs.append(nv)
        n = len(ops)
        hs = (C.c_void_p * n)(*[op.handle for op in ops])
        xs = (C.c_void_p * n)(*[X.data_ptr() for X in Xs])
        ys = (C.c_void_p * n)(*[Y.data_ptr() for Y in Ys])
        nv_arr = (C.c_int * n)(*nvs)
        h = C.c_void_p()
        _check(load().h2_batch_create(hs, n, xs, ys, nv_arr, float(alpha), float(beta),
                                      (H2_BATCH_AUTOTUNE if autotune else 0)
                                      | (H2_BATCH_MEMBER_SWEEPS if member_sweeps else 0), C.byref(h)),
               "h2_batch_create")
        self.handle = h.value
        self._keep = (list(ops), list(Xs), list(Ys))

    def run(self, stream=None):
        _check(load().h2_batch_run(self.handle, _stream_ptr(stream)), "h2_batch_run")

    def check(self):
        _check(load().h2_batch_check(self.handle), "h2_batch_check")

    def describe(self) -> str:
        buf = C.create_string_buffer(4096)
        _check(load().h2_batch_describe(self.handle, buf, 4096), "h2_batch_describe")
        return buf.value.decode()

    def close(self):
        if getattr(self, "handle", None):
            load().h2_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

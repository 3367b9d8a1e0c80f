"""Thin Python binding of libspx's C ABI (include/spx.h).

Every function has the name of the C entry point it calls and only marshals
arguments: torch tensors become device (or host) pointers, status codes
become ``SpxError``.  All computation happens in the CUDA library; there is
no CPU fallback -- if ``libspx.so`` is missing or cannot be loaded, importing
the library raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

# ------------------------------------------------------------------ constants (spx.h)
SPX_OK, SPX_ERR_INVALID, SPX_ERR_TOO_LARGE, SPX_ERR_OOM, SPX_ERR_CUDA = 0, 1, 2, 3, 4
SPX_ERR_UNSUPPORTED, SPX_ERR_TIMEOUT, SPX_ERR_NOT_FOUND = 5, 6, 7
SPX_CSR, SPX_ELL, SPX_COO, SPX_HYB = 0, 1, 2, 3
SPX_F64, SPX_F32 = 0, 1
SPX_CG, SPX_BICGSTAB, SPX_GMRES, SPX_CGS = 0, 1, 2, 3
SPX_PRECOND_JACOBI = 0x100
SPX_PRECOND_BLOCK_JACOBI = 0x200
SPX_PRECOND_BLOCK_SHIFT = 16
SPX_PRECOND_BLOCK_ADAPTIVE = 0x400
SPX_SOLVE_ONE_CLUSTER = 0x800


def SPX_PRECOND_BLOCK(bs: int) -> int:
    """Block-Jacobi flag with block size bs (1, 2, 4, 8, 16 or 32), OR-ed into a solver code."""
    return SPX_PRECOND_BLOCK_JACOBI | (int(bs) << SPX_PRECOND_BLOCK_SHIFT)
SPX_PREC_F64, SPX_PREC_F32, SPX_PREC_MIXED = 0, 1, 2
SPX_CONVERGED, SPX_MAX_ITER, SPX_BREAKDOWN, SPX_STAGNATED, SPX_SOLVE_TIMEOUT = 0, 1, 2, 3, 4
SPX_KERNEL_AUTO, SPX_KERNEL_CSR_VECTOR, SPX_KERNEL_CSR_MERGE, SPX_KERNEL_ELL, SPX_KERNEL_COO = 0, 1, 2, 3, 4
SPX_KERNEL_CSR_SPLIT = 5
SPX_KERNEL_CSR_ROWS = 6
SPX_KERNEL_CSR_TILED = 7
SPX_HOST_INPUT, SPX_MIXED_SHADOW = 1, 2
(SPX_PART_ROW_PTR, SPX_PART_COL, SPX_PART_VAL, SPX_PART_ELL_COL, SPX_PART_ELL_VAL, SPX_PART_COO_ROW,
 SPX_PART_COO_COL, SPX_PART_COO_VAL, SPX_PART_VAL_F32) = range(9)

FORMATS = {"csr": SPX_CSR, "ell": SPX_ELL, "coo": SPX_COO, "hyb": SPX_HYB}
SOLVERS = {"cg": SPX_CG, "bicgstab": SPX_BICGSTAB, "gmres": SPX_GMRES, "cgs": SPX_CGS}
PRECISIONS = {"f64": SPX_PREC_F64, "f32": SPX_PREC_F32, "mixed": SPX_PREC_MIXED}
STATUS_NAMES = {SPX_CONVERGED: "converged", SPX_MAX_ITER: "max_iter", SPX_BREAKDOWN: "breakdown",
                SPX_STAGNATED: "stagnated", SPX_SOLVE_TIMEOUT: "timeout"}


class SpxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


def _status_name(s):
    return {0: "SPX_OK", 1: "SPX_ERR_INVALID", 2: "SPX_ERR_TOO_LARGE", 3: "SPX_ERR_OOM", 4: "SPX_ERR_CUDA",
            5: "SPX_ERR_UNSUPPORTED", 6: "SPX_ERR_TIMEOUT", 7: "SPX_ERR_NOT_FOUND"}.get(s, str(s))


class spx_matrix_info(C.Structure):
    _fields_ = [("format", C.c_int32), ("dtype", C.c_int32), ("nrows", C.c_int64), ("ncols", C.c_int64),
                ("nnz", C.c_int64), ("ell_width", C.c_int64), ("ell_ld", C.c_int64), ("coo_nnz", C.c_int64),
                ("max_row_len", C.c_int64), ("mean_row_len", C.c_double), ("device_bytes", C.c_int64),
                ("kernel", C.c_int32), ("kernel_param", C.c_int32), ("has_f32_shadow", C.c_int32)]


class spx_solve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iterations", C.c_int64),
                ("relres_recurrence", C.c_double), ("relres_true", C.c_double), ("time_ms", C.c_double),
                ("inner_iterations", C.c_int64)]


class spx_server_result(C.Structure):
    _fields_ = [("id", C.c_int64), ("error", C.c_int32), ("pad", C.c_int32), ("info", spx_solve_info),
                ("submit_ms", C.c_double), ("admit_ms", C.c_double), ("done_ms", C.c_double),
                ("upload_ms", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("download_ms", C.c_double), ("batched", C.c_int32), ("pad2", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# C signatures: name -> (restype, argtypes)
_P, _I, _I64, _D, _U, _SZ = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint, C.c_size_t
_PP = C.POINTER(C.c_void_p)
SIGNATURES = {
    "spx_ctx_create": (_I, [_PP, _I, _P, ALLOC_FN, FREE_FN, _P]),
    "spx_ctx_destroy": (_I, [_P]),
    "spx_ctx_set_stream": (_I, [_P, _P]),
    "spx_matrix_create": (_I, [_P, _PP, _I, _I, _I64, _I64, _I64, _P, _P, _P, _I, _I64, _U]),
    "spx_matrix_destroy": (_I, [_P]),
    "spx_matrix_get_info": (_I, [_P, C.POINTER(spx_matrix_info)]),
    "spx_matrix_export": (_I, [_P, _P, _I, _P, _SZ, C.POINTER(C.c_size_t)]),
    "spx_matrix_set_kernel": (_I, [_P, _I, _I]),
    "spx_matrix_tune": (_I, [_P, _P, _I, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "spx_spmv": (_I, [_P, _P, _P, _P]),
    "spx_spmv_axpby": (_I, [_P, _P, _D, _P, _D, _P]),
    "spx_spmv_host": (_I, [_P, _P, _P, _P]),
    "spx_spmv_csr_noalloc": (_I, [_P, _I, _I64, _I64, _I64, _P, _P, _P, _P, _P]),
    "spx_dot": (_I, [_P, _I, _I64, _P, _P, _P]),
    "spx_axpby": (_I, [_P, _I, _I64, _D, _P, _D, _P]),
    "spx_solve": (_I, [_P, _P, _P, _P, _I, _D, _I64, _I, _I, C.POINTER(spx_solve_info)]),
    "spx_solve_fixed": (_I, [_P, _P, _P, _P, _I, _I64, _I, _I, C.POINTER(spx_solve_info)]),
    "spx_batch_create": (_I, [_P, _PP, _I, _I64, _P, _P, _P, _P, _P, _U]),
    "spx_batch_destroy": (_I, [_P]),
    "spx_batch_solve": (_I, [_P, _P, _P, _P, _I, _D, _I64, _I, _P]),
    "spx_batch_tune": (_I, [_P, _P, _I, _I, C.POINTER(C.c_int)]),
    "spx_server_create": (_I, [_P, _PP, _I64, _I]),
    "spx_server_submit": (_I, [_P, _I64, _I64, _P, _P, _P, _P, _P, _I, _D, _I64, _I, _I, C.POINTER(C.c_int64)]),
    "spx_server_submit_matrix": (_I, [_P, _P, _P, _P, _I, _D, _I64, _I, _I, C.POINTER(C.c_int64)]),
    "spx_server_poll": (_I, [_P, C.POINTER(spx_server_result), _I, _I, C.POINTER(C.c_int)]),
    "spx_server_set_batching": (_I, [_P, _I64, C.POINTER(C.c_int64)]),
    "spx_ctx_set_grid_sms": (_I, [_P, _I, C.POINTER(C.c_int)]),
    "spx_server_set_slot_sms": (_I, [_P, _I, C.POINTER(C.c_int)]),
    "spx_server_set_cluster_rows": (_I, [_P, _I64, C.POINTER(C.c_int64)]),
    "spx_probe_gather": (_I, [_P, _I64, _P, _P, _I, _P]),
    "spx_ctx_check": (_I, [_P]),
    "spx_selftest_wait_timeout": (_I, [_P, _I]),
    "spx_server_pending": (_I, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "spx_server_destroy": (_I, [_P]),
    "spx_last_error": (C.c_char_p, []),
    "spx_status_str": (C.c_char_p, [_I]),
    "spx_version": (_I, []),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libspx.so (building it first if it is missing or stale and nvcc exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libspx.so not found at {_build.LIB}; run paper_2103_10116_gb300.build.build()")
            lib = C.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
        return _lib


def _check(status: int):
    if status != SPX_OK:
        raise SpxError(status, load().spx_last_error().decode())


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensors passed to libspx must be contiguous")
        return t.data_ptr()
    return int(t)


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return SPX_F64
    if t.dtype == torch.float32:
        return SPX_F32
    raise TypeError(f"unsupported value dtype {t.dtype}")


# ------------------------------------------------------------------ allocator
_alloc_refs = []


def _torch_allocator(device: int):
    def _alloc(size, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), device, int(stream or 0))
        except Exception:  # out of memory -> NULL, reported by the library
            return None

    def _free(ptr, size, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _alloc_refs.append((a, f))  # callbacks must outlive every context that uses them
    return a, f


# ------------------------------------------------------------------ context
def spx_ctx_create(device: int = 0, stream=None, allocator: str = "torch") -> int:
    """Create a context on `device` bound to `stream` (torch Stream, raw handle or None =
    torch's current stream).  allocator: "torch" (caching allocator) or "cuda" (cudaMallocAsync)."""
    if stream is None:
        stream = torch.cuda.current_stream(device)
    handle = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)
    if allocator == "torch":
        a, f = _torch_allocator(device)
    else:
        a, f = ALLOC_FN(), FREE_FN()
    out = C.c_void_p()
    _check(load().spx_ctx_create(C.byref(out), device, handle, a, f, None))
    return out.value


def spx_ctx_destroy(ctx: int):
    _check(load().spx_ctx_destroy(ctx))


def spx_ctx_set_grid_sms(ctx: int, sms: int) -> int:
    """Size the context's launch grids for `sms` SMs (<= 0: the whole device); returns the value in force."""
    eff = C.c_int()
    _check(load().spx_ctx_set_grid_sms(ctx, int(sms), C.byref(eff)))
    return eff.value


def spx_ctx_set_stream(ctx: int, stream):
    handle = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)
    _check(load().spx_ctx_set_stream(ctx, handle))


# ------------------------------------------------------------------ matrices
def spx_matrix_create(ctx: int, fmt, row_ptr: torch.Tensor, col_idx: torch.Tensor, values: torch.Tensor,
                      ncols: int | None = None, dtype=None, hyb_width: int = -1, flags: int = 0) -> int:
    """Create a matrix in format `fmt` ("csr"/"ell"/"coo"/"hyb" or an SPX_* code) from CSR
    tensors (all on the device, or all on the host: SPX_HOST_INPUT is then added)."""
    fmt = FORMATS.get(fmt, fmt)
    nrows = row_ptr.numel() - 1
    ncols = nrows if ncols is None else ncols
    if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
        raise TypeError("row_ptr and col_idx must be int32")
    vdt = _dt(values)
    mdt = vdt if dtype is None else ({torch.float64: SPX_F64, torch.float32: SPX_F32}.get(dtype, dtype))
    if not row_ptr.is_cuda:
        flags |= SPX_HOST_INPUT
    out = C.c_void_p()
    _check(load().spx_matrix_create(ctx, C.byref(out), fmt, mdt, nrows, ncols, col_idx.numel(), _ptr(row_ptr),
                                    _ptr(col_idx), _ptr(values), vdt, hyb_width, flags))
    return out.value


def spx_matrix_destroy(A: int):
    _check(load().spx_matrix_destroy(A))


def spx_matrix_get_info(A: int) -> dict:
    info = spx_matrix_info()
    _check(load().spx_matrix_get_info(A, C.byref(info)))
    return {k: getattr(info, k) for k, _ in spx_matrix_info._fields_}


def spx_matrix_export(ctx: int, A: int, part: int, device: int = 0) -> torch.Tensor:
    """Copy an internal array of A into a new device tensor (int32 or the value dtype)."""
    info = spx_matrix_get_info(A)
    fdt = torch.float64 if info["dtype"] == SPX_F64 else torch.float32
    n, nnz, w, ld, cn = info["nrows"], info["nnz"], info["ell_width"], info["ell_ld"], info["coo_nnz"]
    shapes = {SPX_PART_ROW_PTR: (n + 1, torch.int32), SPX_PART_COL: (nnz, torch.int32),
              SPX_PART_VAL: (nnz, fdt), SPX_PART_ELL_COL: (w * ld, torch.int32), SPX_PART_ELL_VAL: (w * ld, fdt),
              SPX_PART_COO_ROW: (cn, torch.int32), SPX_PART_COO_COL: (cn, torch.int32),
              SPX_PART_COO_VAL: (cn, fdt)}
    if part == SPX_PART_VAL_F32:
        m = nnz if info["format"] == SPX_CSR else (w * ld if info["format"] in (SPX_ELL, SPX_HYB) else cn)
        shapes[part] = (m, torch.float32)
    if part not in shapes:
        raise SpxError(SPX_ERR_NOT_FOUND, "unknown part")
    num, dt = shapes[part]
    dst = torch.empty(max(num, 1), dtype=dt, device=f"cuda:{device}")
    written = C.c_size_t()
    _check(load().spx_matrix_export(ctx, A, part, _ptr(dst), dst.numel() * dst.element_size(), C.byref(written)))
    return dst[: written.value // dst.element_size()]


def spx_matrix_set_kernel(A: int, kernel: int, param: int = 0):
    _check(load().spx_matrix_set_kernel(A, kernel, param))


def spx_matrix_tune(ctx: int, A: int, reps: int = 10) -> tuple:
    """Time every SpMV kernel variant for A and keep the fastest; returns (kernel, param, us per product)."""
    k, p, us = C.c_int(), C.c_int(), C.c_float()
    _check(load().spx_matrix_tune(ctx, A, int(reps), C.byref(k), C.byref(p), C.byref(us)))
    return k.value, p.value, us.value


def tune_key(A: int, device_name: str) -> str:
    """Cache key of an autotuned choice: the GPU and the matrix's format, dtype and shape statistics
    (sizes to two significant digits, row lengths to the nearest power of two)."""
    import math
    i = spx_matrix_get_info(A)

    def sig(v):
        v = int(v)
        return 0 if v <= 0 else int(float(f"{v:.2g}"))

    def p2(v):
        return 0 if v <= 0 else 1 << int(math.ceil(math.log2(max(1.0, float(v)))))
    return (f"{device_name}|fmt{i['format']}|dt{i['dtype']}|n{sig(i['nrows'])}|nnz{sig(i['nnz'])}"
            f"|max{p2(i['max_row_len'])}|mean{p2(i['mean_row_len'])}|ell{i['ell_width']}")


def tune_cached(ctx: int, A: int, cache_path: str | None = None, reps: int = 10, device: int = 0,
                device_name: str | None = None, tuner=None) -> tuple:
    """Autotune with a JSON cache (default: $SPX_TUNE_CACHE or ~/.cache/spx/tune.json): a matrix whose key
    (tune_key) is in the cache gets the stored kernel without timing; otherwise spx_matrix_tune runs and
    the choice is stored.  Returns (kernel, param, us or None when it came from the cache).  `tuner`
    replaces spx_matrix_tune (same signature), e.g. to test the cache without a GPU."""
    import json
    import os
    path = cache_path or os.environ.get("SPX_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "spx",
                                                                        "tune.json")
    key = tune_key(A, device_name if device_name is not None else torch.cuda.get_device_name(device))
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        k, p = cache[key]["kernel"], cache[key]["param"]
        spx_matrix_set_kernel(A, k, p)
        return k, p, None
    k, p, us = (tuner or spx_matrix_tune)(ctx, A, reps)
    cache[key] = {"kernel": k, "param": p, "us": us}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return k, p, us


# ------------------------------------------------------------------ SpMV / BLAS-1
def spx_spmv(ctx: int, A: int, x: torch.Tensor, y: torch.Tensor):
    _check(load().spx_spmv(ctx, A, _ptr(x), _ptr(y)))


def spx_spmv_axpby(ctx: int, A: int, alpha: float, x: torch.Tensor, beta: float, y: torch.Tensor):
    _check(load().spx_spmv_axpby(ctx, A, float(alpha), _ptr(x), float(beta), _ptr(y)))


def spx_spmv_host(ctx: int, A: int, x_host: torch.Tensor, y_host: torch.Tensor):
    """End-to-end SpMV on host tensors (pin them for full copy bandwidth)."""
    if x_host.is_cuda or y_host.is_cuda:
        raise ValueError("spx_spmv_host takes host tensors")
    _check(load().spx_spmv_host(ctx, A, _ptr(x_host), _ptr(y_host)))


def spx_spmv_csr_noalloc(row_ptr: torch.Tensor, col_idx: torch.Tensor, values: torch.Tensor, x: torch.Tensor,
                         y: torch.Tensor, ncols: int | None = None, stream=None):
    """y = A x straight from device CSR tensors; allocates nothing (fixed scratch inside the
    library).  stream: torch Stream / raw handle / None (torch's current stream)."""
    if stream is None:
        stream = torch.cuda.current_stream(values.device)
    handle = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)
    n = row_ptr.numel() - 1
    _check(load().spx_spmv_csr_noalloc(handle, _dt(values), n, n if ncols is None else ncols, col_idx.numel(),
                                       _ptr(row_ptr), _ptr(col_idx), _ptr(values), _ptr(x), _ptr(y)))


def spx_dot(ctx: int, x: torch.Tensor, y: torch.Tensor, result: torch.Tensor):
    _check(load().spx_dot(ctx, _dt(x), x.numel(), _ptr(x), _ptr(y), _ptr(result)))


def spx_axpby(ctx: int, alpha: float, x: torch.Tensor, beta: float, y: torch.Tensor):
    _check(load().spx_axpby(ctx, _dt(x), x.numel(), float(alpha), _ptr(x), float(beta), _ptr(y)))


# ------------------------------------------------------------------ solvers
@dataclass
class SolveInfo:
    status: int
    restarts: int
    iterations: int
    relres_recurrence: float
    relres_true: float
    time_ms: float
    inner_iterations: int

    @property
    def status_name(self):
        return STATUS_NAMES.get(self.status, str(self.status))


def _info(i: spx_solve_info) -> SolveInfo:
    return SolveInfo(i.status, i.restarts, i.iterations, i.relres_recurrence, i.relres_true, i.time_ms,
                     i.inner_iterations)


def _solver_code(solver, precond, block_size=8):
    """precond: None, "jacobi", "block_jacobi" (blocks of block_size rows) or
    "adaptive_block_jacobi" (the same with FP32 storage of well-conditioned blocks)."""
    code = SOLVERS.get(solver, solver)
    if precond == "jacobi":
        code |= SPX_PRECOND_JACOBI
    elif precond == "block_jacobi":
        code |= SPX_PRECOND_BLOCK(block_size)
    elif precond == "adaptive_block_jacobi":
        code |= SPX_PRECOND_BLOCK(block_size) | SPX_PRECOND_BLOCK_ADAPTIVE
    elif precond is not None:
        raise ValueError(f"unknown preconditioner {precond!r}")
    return code


def spx_solve(ctx: int, A: int, b: torch.Tensor, x: torch.Tensor, solver="cg", tol: float = 1e-10,
              max_iter: int = 10000, restart: int = 30, precision="f64", precond=None,
              block_size: int = 8, one_cluster: bool = False) -> SolveInfo:
    """one_cluster: the whole solve in one launch on one thread-block cluster (SPX_SOLVE_ONE_CLUSTER)."""
    info = spx_solve_info()
    code = _solver_code(solver, precond, block_size) | (SPX_SOLVE_ONE_CLUSTER if one_cluster else 0)
    _check(load().spx_solve(ctx, A, _ptr(b), _ptr(x), code, float(tol), int(max_iter), int(restart),
                            PRECISIONS.get(precision, precision), C.byref(info)))
    return _info(info)


def spx_solve_fixed(ctx: int, A: int, b: torch.Tensor, x: torch.Tensor, solver="cg", iterations: int = 1000,
                    restart: int = 30, precision="f64", precond=None, block_size: int = 8) -> SolveInfo:
    info = spx_solve_info()
    _check(load().spx_solve_fixed(ctx, A, _ptr(b), _ptr(x), _solver_code(solver, precond, block_size),
                                  int(iterations), int(restart), PRECISIONS.get(precision, precision),
                                  C.byref(info)))
    return _info(info)


# ------------------------------------------------------------------ batched
def spx_batch_create(ctx: int, row_off, nnz_off, row_ptr: torch.Tensor, col_idx: torch.Tensor,
                     values: torch.Tensor, flags: int = 0) -> int:
    import numpy as np
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    no = np.ascontiguousarray(nnz_off, dtype=np.int64)
    out = C.c_void_p()
    _check(load().spx_batch_create(ctx, C.byref(out), _dt(values), ro.shape[0] - 1, ro.ctypes.data,
                                   no.ctypes.data, _ptr(row_ptr), _ptr(col_idx), _ptr(values), flags))
    return out.value


def spx_batch_destroy(B: int):
    _check(load().spx_batch_destroy(B))


def spx_batch_solve(ctx: int, B: int, b: torch.Tensor, x: torch.Tensor, nsys: int, solver="cg",
                    tol: float = 1e-10, max_iter: int = 10000, precision="f64") -> list[SolveInfo]:
    infos = (spx_solve_info * max(nsys, 1))()
    _check(load().spx_batch_solve(ctx, B, _ptr(b), _ptr(x), SOLVERS.get(solver, solver), float(tol),
                                  int(max_iter), PRECISIONS.get(precision, precision), C.cast(infos, C.c_void_p)))
    return [_info(infos[i]) for i in range(nsys)]


def spx_batch_tune(ctx: int, B: int, solver="cg", precision="f64") -> int:
    chosen = C.c_int()
    _check(load().spx_batch_tune(ctx, B, SOLVERS.get(solver, solver), PRECISIONS.get(precision, precision),
                                 C.byref(chosen)))
    return chosen.value


# ------------------------------------------------------------------ serving
def spx_server_create(ctx: int, budget_bytes: int = 0, max_slots: int = 8) -> int:
    out = C.c_void_p()
    _check(load().spx_server_create(ctx, C.byref(out), int(budget_bytes), int(max_slots)))
    return out.value


def spx_server_submit(S: int, row_ptr, col_idx, values, b, x, solver="cg", tol: float = 1e-8,
                      max_iter: int = 100000, restart: int = 30, precision="mixed") -> int:
    """Queue a solve on HOST numpy arrays (int32 row_ptr / col_idx, float64 values / b / x).
    The caller keeps every array alive and x untouched until the request completes."""
    import numpy as np
    for a, dt in ((row_ptr, np.int32), (col_idx, np.int32), (values, np.float64), (b, np.float64),
                  (x, np.float64)):
        if not (isinstance(a, np.ndarray) and a.dtype == dt and a.flags.c_contiguous):
            raise TypeError("spx_server_submit takes contiguous numpy arrays (int32 indices, float64 values)")
    rid = C.c_int64()
    _check(load().spx_server_submit(S, row_ptr.shape[0] - 1, col_idx.shape[0], row_ptr.ctypes.data,
                                    col_idx.ctypes.data, values.ctypes.data, b.ctypes.data, x.ctypes.data,
                                    SOLVERS.get(solver, solver), float(tol), int(max_iter), int(restart),
                                    PRECISIONS.get(precision, precision), C.byref(rid)))
    return rid.value


def spx_server_submit_matrix(S: int, A: int, b, x, solver="cg", tol: float = 1e-8, max_iter: int = 100000,
                             restart: int = 30, precision="mixed") -> int:
    """Queue a solve on a resident matrix handle A (FP64, square) with HOST numpy b and x
    (float64); A, b and x stay alive and untouched until the request completes."""
    import numpy as np
    for a in (b, x):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError("spx_server_submit_matrix takes contiguous float64 numpy b and x")
    rid = C.c_int64()
    _check(load().spx_server_submit_matrix(S, A, b.ctypes.data, x.ctypes.data, SOLVERS.get(solver, solver),
                                           float(tol), int(max_iter), int(restart),
                                           PRECISIONS.get(precision, precision), C.byref(rid)))
    return rid.value


def spx_server_poll(S: int, max_results: int = 256, wait_ms: int = 0) -> list[dict]:
    buf = (spx_server_result * max(1, max_results))()
    cnt = C.c_int()
    _check(load().spx_server_poll(S, buf, max_results, int(wait_ms), C.byref(cnt)))
    out = []
    for i in range(cnt.value):
        r = buf[i]
        out.append({"id": r.id, "error": r.error, "info": _info(r.info), "submit_ms": r.submit_ms,
                    "admit_ms": r.admit_ms, "done_ms": r.done_ms, "upload_ms": r.upload_ms,
                    "setup_ms": r.setup_ms, "solve_ms": r.solve_ms, "download_ms": r.download_ms,
                    "batched": r.batched == 1, "route": ("slot", "batch", "cluster")[r.batched]})
    return out


def spx_ctx_check(ctx: int):
    """Raise SpxError(SPX_ERR_TIMEOUT) if a bounded device-side wait gave up since the last check."""
    _check(load().spx_ctx_check(ctx))


def spx_selftest_wait_timeout(ctx: int, which: int = 0):
    _check(load().spx_selftest_wait_timeout(ctx, int(which)))


def spx_probe_gather(ctx: int, col_idx: torch.Tensor, x: torch.Tensor, out: torch.Tensor):
    """Gather-only floor of an SpMV on col_idx's pattern (measurement aid)."""
    _check(load().spx_probe_gather(ctx, col_idx.numel(), _ptr(col_idx), _ptr(x), _dt(x), _ptr(out)))


def spx_server_set_batching(S: int, max_rows: int) -> int:
    eff = C.c_int64(0)
    _check(load().spx_server_set_batching(S, int(max_rows), C.byref(eff)))
    return eff.value


def spx_server_set_slot_sms(S: int, sms: int) -> int:
    """Grid share of the server's slots (0: whole device, the default; -1: by row length; below -1: report
    only); returns the setting in force."""
    eff = C.c_int()
    _check(load().spx_server_set_slot_sms(S, int(sms), C.byref(eff)))
    return eff.value


def spx_server_set_cluster_rows(S: int, max_rows: int) -> int:
    """Route slot requests of at most max_rows rows to the one-cluster solve (0: none;
    negative: report only); returns the limit in force."""
    eff = C.c_int64()
    _check(load().spx_server_set_cluster_rows(S, int(max_rows), C.byref(eff)))
    return eff.value


def spx_server_pending(S: int) -> tuple[int, int, int]:
    q, r, b = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().spx_server_pending(S, C.byref(q), C.byref(r), C.byref(b)))
    return q.value, r.value, b.value


def spx_server_destroy(S: int):
    _check(load().spx_server_destroy(S))


# ------------------------------------------------------------------ errors
def spx_last_error() -> str:
    return load().spx_last_error().decode()


def spx_status_str(status: int) -> str:
    return load().spx_status_str(status).decode()


def spx_version() -> int:
    return load().spx_version()

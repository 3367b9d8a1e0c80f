"""Plain CPU oracle for the sparse hot path (SpMV, format conversions, CG,
BiCGSTAB, GMRES(m), mixed-precision iterative refinement).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library product
(``paper_2103_10116_gb300``) never imports, loads or calls it, and the two share
no code: the arithmetic lives in ``spx_oracle.c`` (plain sequential C, IEEE
double, compiled with ``-O2 -ffp-contract=off``), this module only marshals numpy
arrays into it.

Each function cites the passage of the paper (arXiv 2103.10116) it follows;
the C source states the algorithm in the paper's order and notation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spx_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, C.CDLL] = {}

CONVERGED, MAX_ITER, BREAKDOWN, STAGNATED = 0, 1, 2, 3
STATUS_NAMES = {CONVERGED: "converged", MAX_ITER: "max_iter", BREAKDOWN: "breakdown",
                STAGNATED: "stagnated"}


class _Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("restarts", C.c_int32), ("iterations", C.c_int64),
                ("relres_recurrence", C.c_double), ("relres_true", C.c_double)]


@dataclass
class SolveInfo:
    status: int
    iterations: int
    restarts: int
    relres_recurrence: float
    relres_true: float


def build(mutant: int = 0, openmp: bool = False) -> str:
    """Compile the oracle with gcc; ``mutant`` > 0 plants a known mistake (used
    only by the mutation tests that show the pins catch it).  ``openmp`` builds
    the all-cores variant of the plain SpMV used by the CPU baseline (same
    arithmetic, rows shared among threads)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "liboracle_omp.so" if openmp else f"liboracle_m{mutant}.so")
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           f"-DORC_MUTANT={mutant}"]
    if openmp:
        cmd += ["-O3", "-fopenmp", "-DORC_OPENMP"]
    cmd += [_SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_OMP = None


def spmv_csr_plain_omp(rp, col, val, x) -> np.ndarray:
    """spmv_csr_plain on all host cores (OpenMP over rows; the same bits)."""
    global _OMP
    with _LOCK:
        if _OMP is None:
            _OMP = C.CDLL(build(openmp=True))
            _OMP.orc_spmv_csr_plain.restype = None
            _OMP.orc_spmv_csr_plain.argtypes = [C.c_int64] + [C.c_void_p] * 5
    rp, col, val = _csr(rp, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    _OMP.orc_spmv_csr_plain(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else the host's cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def _lib(mutant: int = 0) -> C.CDLL:
    with _LOCK:
        if mutant not in _LIBS:
            lib = C.CDLL(build(mutant))
            i64, dbl, p = C.c_int64, C.c_double, C.c_void_p
            lib.orc_csr_check.restype = C.c_int
            lib.orc_csr_check.argtypes = [i64, i64, i64, p, p]
            for name in ("orc_spmv_csr", "orc_spmv_csr_absbound", "orc_spmv_csr_plain"):
                getattr(lib, name).restype = None
                getattr(lib, name).argtypes = [i64, p, p, p, p, p]
            lib.orc_csr_to_coo_rows.argtypes = [i64, p, p]
            lib.orc_max_row_len.restype = i64
            lib.orc_max_row_len.argtypes = [i64, p]
            lib.orc_csr_to_ell.argtypes = [i64, i64, i64, p, p, p, C.c_int, p, p]
            lib.orc_hyb_coo_count.restype = i64
            lib.orc_hyb_coo_count.argtypes = [i64, p, i64]
            lib.orc_csr_to_hyb.argtypes = [i64, i64, i64, p, p, p, C.c_int, p, p, p, p, p]
            lib.orc_hyb_auto_width.restype = i64
            lib.orc_hyb_auto_width.argtypes = [i64, p, C.c_int]
            for name in ("orc_cg", "orc_bicgstab", "orc_cgs", "orc_cg_jacobi", "orc_bicgstab_jacobi",
                         "orc_cgs_jacobi"):
                getattr(lib, name).restype = C.c_int
                getattr(lib, name).argtypes = [i64, p, p, p, p, p, dbl, i64, C.POINTER(_Info), p]
            for name in ("orc_gmres", "orc_gmres_jacobi"):
                getattr(lib, name).restype = C.c_int
                getattr(lib, name).argtypes = [i64, p, p, p, p, p, C.c_int, dbl, i64, C.POINTER(_Info), p]
            for name in ("orc_cg_bjacobi", "orc_bicgstab_bjacobi", "orc_cgs_bjacobi"):
                getattr(lib, name).restype = C.c_int
                getattr(lib, name).argtypes = [i64, p, p, p, p, p, dbl, i64, C.POINTER(_Info), p, C.c_int,
                                               C.c_int]
            lib.orc_gmres_bjacobi.restype = C.c_int
            lib.orc_gmres_bjacobi.argtypes = [i64, p, p, p, p, p, C.c_int, dbl, i64, C.POINTER(_Info), p,
                                              C.c_int, C.c_int]
            lib.orc_block_jacobi_inv.restype = C.c_int
            lib.orc_block_jacobi_inv.argtypes = [i64, p, p, p, C.c_int, p]
            lib.orc_block_jacobi_inv_adaptive.restype = C.c_int
            lib.orc_block_jacobi_inv_adaptive.argtypes = [i64, p, p, p, C.c_int, p, p]
            lib.orc_ir.restype = C.c_int
            lib.orc_ir.argtypes = [i64, p, p, p, C.c_int, p, p, dbl, dbl, C.c_int, i64,
                                   C.POINTER(_Info)]
            lib.orc_cg_reliable.restype = C.c_int
            lib.orc_cg_reliable.argtypes = [i64, p, p, p, p, p, dbl, dbl, i64, C.POINTER(_Info)]
            lib.orc_spmv_repeat.argtypes = [i64, p, p, p, p, p, C.c_int]
            _LIBS[mutant] = lib
        return _LIBS[mutant]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _csr(rp, col, val):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return rp, col, val


def csr_check(n, ncols, rp, col, mutant=0) -> bool:
    """CSR well-formedness (Section 5: row pointers index a row-sorted COO)."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if rp.shape[0] != n + 1:
        return False
    return _lib(mutant).orc_csr_check(n, ncols, int(col.shape[0]), _ptr(rp), _ptr(col)) == 0


def spmv_csr(rp, col, val, x, mutant=0) -> np.ndarray:
    """y = A x for CSR A (Section 5), compensated summation in index order."""
    rp, col, val = _csr(rp, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    _lib(mutant).orc_spmv_csr(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def spmv_csr_plain(rp, col, val, x) -> np.ndarray:
    """The literal index-order definition of Section 5 without compensation."""
    rp, col, val = _csr(rp, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    _lib().orc_spmv_csr_plain(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def spmv_absbound(rp, col, val, x, mutant=0) -> np.ndarray:
    """(|A| |x|)_i: the scale against which a row's rounding error is judged."""
    rp, col, val = _csr(rp, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    _lib(mutant).orc_spmv_csr_absbound(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y))
    return y


def spmv_repeat(rp, col, val, x, reps: int) -> np.ndarray:
    rp, col, val = _csr(rp, col, val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    _lib().orc_spmv_repeat(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(x), _ptr(y), reps)
    return y


def csr_to_coo_rows(rp) -> np.ndarray:
    """COO row indices of a CSR matrix (Section 5: CSR replaces these by pointers)."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    n = rp.shape[0] - 1
    row = np.empty(int(rp[-1]), dtype=np.int32)
    _lib().orc_csr_to_coo_rows(n, _ptr(rp), _ptr(row))
    return row


def max_row_len(rp) -> int:
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    return int(_lib().orc_max_row_len(rp.shape[0] - 1, _ptr(rp)))


def csr_to_ell(rp, col, val, width: int, ld: int):
    """Column-major padded ELL: slot (i, j) at j*ld + i, padding col=-1, value +0.0."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val)
    n = rp.shape[0] - 1
    ecol = np.empty(width * ld, dtype=np.int32)
    evals = np.empty(width * ld, dtype=val.dtype)
    _lib().orc_csr_to_ell(n, ld, width, _ptr(rp), _ptr(col), _ptr(val), val.itemsize,
                          _ptr(ecol), _ptr(evals))
    return ecol, evals


def hyb_coo_count(rp, width: int) -> int:
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    return int(_lib().orc_hyb_coo_count(rp.shape[0] - 1, _ptr(rp), width))


def csr_to_hyb(rp, col, val, width: int, ld: int):
    """HYB = ELL of the given width + COO (CSR order) of what does not fit."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val)
    n = rp.shape[0] - 1
    nc = hyb_coo_count(rp, width)
    ecol = np.empty(width * ld, dtype=np.int32)
    evals = np.empty(width * ld, dtype=val.dtype)
    crow = np.empty(nc, dtype=np.int32)
    ccol = np.empty(nc, dtype=np.int32)
    cval = np.empty(nc, dtype=val.dtype)
    _lib().orc_csr_to_hyb(n, ld, width, _ptr(rp), _ptr(col), _ptr(val), val.itemsize,
                          _ptr(ecol), _ptr(evals), _ptr(crow), _ptr(ccol), _ptr(cval))
    return ecol, evals, crow, ccol, cval


def hyb_auto_width(rp, vbytes: int) -> int:
    """Footprint-optimal ELL width of a HYB matrix."""
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    return int(_lib().orc_hyb_auto_width(rp.shape[0] - 1, _ptr(rp), vbytes))


def block_jacobi_inv(rp, col, val, bs: int, mutant=0, adaptive=False):
    """Inverses of the bs x bs diagonal blocks of A (block-Jacobi, listed among
    the library's preconditioners in Section 2), shape (ceil(n / bs), bs, bs).
    adaptive=True: also the per-block storage flags (1 = FP64, 0 = FP32, the
    block's inverse then rounded to FP32); returns (inverses, flags)."""
    rp, col, val = _csr(rp, col, val)
    n = rp.shape[0] - 1
    nb = (n + bs - 1) // bs
    out = np.empty((max(nb, 1), bs, bs), dtype=np.float64)
    if adaptive:
        flags = np.zeros(max(nb, 1), dtype=np.uint8)
        st = _lib(mutant).orc_block_jacobi_inv_adaptive(n, _ptr(rp), _ptr(col), _ptr(val), int(bs), _ptr(out),
                                                        _ptr(flags))
    else:
        st = _lib(mutant).orc_block_jacobi_inv(n, _ptr(rp), _ptr(col), _ptr(val), int(bs), _ptr(out))
    if st != 0:
        raise ValueError("block size must be at least 1")
    return (out[:nb], flags[:nb]) if adaptive else out[:nb]


def _solve(fn, args, rp, col, val, b, x0, with_hist, maxit, mutant, tail=()):
    rp, col, val = _csr(rp, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rp.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = _Info()
    hist = np.full(maxit + 2, np.nan) if with_hist else None
    getattr(_lib(mutant), fn)(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(b), _ptr(x), *args,
                              C.byref(info), _ptr(hist) if hist is not None else None, *tail)
    si = SolveInfo(info.status, info.iterations, info.restarts, info.relres_recurrence,
                   info.relres_true)
    if with_hist:
        return x, si, hist[: info.iterations + 1]
    return x, si


def _fn(base, precond, block_size):
    """Entry point and trailing arguments for a preconditioner choice."""
    if precond is None:
        return base, ()
    if precond == "jacobi":
        return base + "_jacobi", ()
    if precond in ("block_jacobi", "adaptive_block_jacobi"):
        if int(block_size) < 1:
            raise ValueError("block_size must be at least 1")
        return base + "_bjacobi", (int(block_size), int(precond == "adaptive_block_jacobi"))
    raise ValueError(f"unknown preconditioner {precond!r}")


def cg(rp, col, val, b, tol=1e-10, maxit=10000, x0=None, hist=False, mutant=0, precond=None, block_size=8):
    """Conjugate Gradient for SPD A (Section 5 names CG; textbook form);
    precond="jacobi": preconditioned CG with M = diag(A); "block_jacobi": M =
    the block diagonal of A with blocks of block_size rows."""
    fn, tail = _fn("orc_cg", precond, block_size)
    return _solve(fn, [float(tol), int(maxit)], rp, col, val, b, x0, hist, maxit, mutant, tail)


def bicgstab(rp, col, val, b, tol=1e-10, maxit=10000, x0=None, hist=False, mutant=0, precond=None,
             block_size=8):
    """BiCGSTAB for general A (Section 5 names BiCGSTAB; van der Vorst form);
    precond="jacobi" / "block_jacobi": right preconditioning with M = diag(A) /
    the block diagonal of A."""
    fn, tail = _fn("orc_bicgstab", precond, block_size)
    return _solve(fn, [float(tol), int(maxit)], rp, col, val, b, x0, hist, maxit, mutant, tail)


def cgs(rp, col, val, b, tol=1e-10, maxit=10000, x0=None, hist=False, mutant=0, precond=None, block_size=8):
    """Conjugate Gradient Squared (Sonneveld) for general A (Section 5 names CGS);
    precond="jacobi" / "block_jacobi": right preconditioning with M = diag(A) /
    the block diagonal of A."""
    fn, tail = _fn("orc_cgs", precond, block_size)
    return _solve(fn, [float(tol), int(maxit)], rp, col, val, b, x0, hist, maxit, mutant, tail)


def gmres(rp, col, val, b, m=30, tol=1e-10, maxit=10000, x0=None, hist=False, mutant=0, precond=None,
          block_size=8):
    """Restarted GMRES(m), MGS Arnoldi + Givens rotations (Section 5 names GMRES);
    precond="jacobi" / "block_jacobi": right preconditioning with M = diag(A) /
    the block diagonal of A."""
    fn, tail = _fn("orc_gmres", precond, block_size)
    return _solve(fn, [int(m), float(tol), int(maxit)], rp, col, val, b, x0, hist, maxit, mutant, tail)


def ir(rp, col, val, b, solver="cg", tol=1e-10, inner_tol=1e-4, max_outer=20,
       maxit_inner=500, x0=None, mutant=0):
    """FP64 iterative refinement around an FP32 CG / BiCGSTAB / CGS inner solve
    (at most maxit_inner inner iterations per refinement cycle)."""
    rp, col, val = _csr(rp, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rp.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    info = _Info()
    _lib(mutant).orc_ir(n, _ptr(rp), _ptr(col), _ptr(val), {"cg": 0, "bicgstab": 1, "cgs": 3}[solver], _ptr(b),
                  _ptr(x), float(tol), float(inner_tol), int(max_outer), int(maxit_inner),
                  C.byref(info))
    return x, SolveInfo(info.status, info.iterations, info.restarts, info.relres_recurrence,
                        info.relres_true)


def cg_reliable(rp, col, val, b, tol=1e-10, delta=0.1, maxit=100000, x0=None, mutant=0):
    """Mixed-precision CG with reliable updates: FP32 iterations, FP64 residual
    replacement whenever the FP32 residual fell by delta (see the C source)."""
    rp, col, val = _csr(rp, col, val)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = rp.shape[0] - 1
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    inf = _Info()
    _lib(mutant).orc_cg_reliable(n, _ptr(rp), _ptr(col), _ptr(val), _ptr(b), _ptr(x), float(tol), float(delta),
                                 int(maxit), C.byref(inf))
    return x, SolveInfo(inf.status, inf.iterations, inf.restarts, inf.relres_recurrence, inf.relres_true)

"""Seeded synthetic inputs: sparse matrices in CSR form and vectors.

This module holds none of the method's arithmetic (no products, no solves):
it only lays out matrix structure and draws values from numpy's PCG64
generator, so that the CUDA path and the CPU oracle can be fed identical
inputs.  Every generator returns ``(row_ptr int32[n+1], col int32[nnz],
val float64[nnz])`` with columns sorted inside each row.

Workloads (the paper measures on SuiteSparse matrices, Table 1, which are not
available here; these synthetic families stand in for them and span the same
4-60 nonzeros-per-row range):
  * 2D 5-point and 3D 7-point Laplacians (diagonal 4 / 6, neighbours -1);
  * 3D 27-point stencil (diagonal 26, the 26 neighbours -1);
  * 3D upwind convection-diffusion, Peclet 10, nonsymmetric;
  * power-law rows: Pareto(tail 1.5) row lengths fitted to a mean, capped;
    distinct uniform columns; N(0,1) values;
  * ragged 2D Laplacian plus a diagonal shift (batched systems);
  * diagonally dominant random rows (served systems).
"""
from __future__ import annotations

import math

import numpy as np


def _finish(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """Rows must already be sorted (and columns sorted within a row)."""
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    if rp[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz does not fit int32 indices")
    return rp.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64)


def _stencil(shape: tuple[int, ...], offsets: list[tuple[int, ...]], weights: list[float]):
    """Generic constant-coefficient stencil on a grid with Dirichlet boundary.
    offsets are (dz, dy, dx) style tuples, last axis fastest in the numbering."""
    dims = len(shape)
    n = int(np.prod(shape))
    # sort offsets by the column they produce so that columns come out sorted
    strides = [int(np.prod(shape[d + 1:])) for d in range(dims)]
    order = sorted(range(len(offsets)), key=lambda k: sum(o * s for o, s in zip(offsets[k], strides)))
    offsets = [offsets[k] for k in order]
    weights = [weights[k] for k in order]
    coords = np.indices(shape).reshape(dims, n)
    cols = np.empty((n, len(offsets)), dtype=np.int64)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    valid = np.ones((n, len(offsets)), dtype=bool)
    for k, (off, w) in enumerate(zip(offsets, weights)):
        c = np.zeros(n, dtype=np.int64)
        ok = np.ones(n, dtype=bool)
        for d in range(dims):
            q = coords[d] + off[d]
            ok &= (q >= 0) & (q < shape[d])
            c += q * strides[d]
        cols[:, k] = c
        vals[:, k] = w
        valid[:, k] = ok
    rows = np.repeat(np.arange(n, dtype=np.int64), len(offsets)).reshape(n, len(offsets))
    return _finish(n, rows[valid], cols[valid], vals[valid])


def laplace2d_5pt(nx: int, ny: int | None = None):
    """5-point 2D Laplacian on an nx-by-ny grid: diagonal 4, neighbours -1."""
    ny = nx if ny is None else ny
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    w = [4.0, -1.0, -1.0, -1.0, -1.0]
    return _stencil((ny, nx), offs, w)


def laplace3d_7pt(m: int):
    """7-point 3D Laplacian on an m^3 grid: diagonal 6, neighbours -1."""
    offs = [(0, 0, 0)] + [tuple(s if a == d else 0 for a in range(3)) for d in range(3) for s in (-1, 1)]
    w = [6.0] + [-1.0] * 6
    return _stencil((m, m, m), offs, w)


def stencil3d_27pt(m: int):
    """27-point 3D stencil on an m^3 grid: diagonal 26, all 26 neighbours -1.
    It equals 27 I - T (x) T (x) T with T = tridiag(1, 1, 1), hence SPD."""
    offs, w = [], []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                offs.append((dz, dy, dx))
                w.append(26.0 if (dz, dy, dx) == (0, 0, 0) else -1.0)
    return _stencil((m, m, m), offs, w)


def convdiff3d_upwind(m: int, peclet: float = 10.0):
    """-Laplace(u) + w . grad(u) on the unit cube, m^3 interior points,
    h = 1/(m+1), w = peclet * (1,1,1)/sqrt(3), first-order upwind, scaled by h^2.
    Row: diagonal 6 + h*sum(w), backward neighbour -1 - h*w_d, forward -1."""
    h = 1.0 / (m + 1)
    wd = peclet / math.sqrt(3.0)
    offs = [(0, 0, 0)]
    w = [6.0 + 3.0 * h * wd]
    for d in range(3):
        for s in (-1, 1):
            offs.append(tuple(s if a == d else 0 for a in range(3)))
            w.append(-1.0 - h * wd if s == -1 else -1.0)
    return _stencil((m, m, m), offs, w)


def powerlaw_lengths(n: int, mean: float = 16.0, max_len: int = 20000, tail: float = 1.5,
                     seed: int = 2) -> np.ndarray:
    """Row lengths L = min(max_len, floor(x_m * U^(-1/tail))) with U ~ U(0,1]
    and x_m fitted by bisection so that the sample mean equals ``mean``."""
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)  # (0, 1]
    g = u ** (-1.0 / tail)

    def lens(xm):
        return np.minimum(max_len, np.floor(xm * g)).astype(np.int64)

    lo, hi = 1.0, float(mean)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if lens(mid).mean() < mean:
            lo = mid
        else:
            hi = mid
    return lens(hi)


def powerlaw(n: int, mean: float = 16.0, max_len: int = 20000, tail: float = 1.5, seed: int = 2,
             ncols: int | None = None):
    """Random sparse matrix with power-law (Pareto tail 1.5) row lengths, distinct
    uniform random columns per row and N(0,1) values."""
    ncols = n if ncols is None else ncols
    L = np.minimum(powerlaw_lengths(n, mean, max_len, tail, seed), ncols)
    rng = np.random.default_rng(seed + 1000)
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    cols = rng.integers(0, ncols, size=rows.shape[0], dtype=np.int64)
    # make columns distinct inside each row: redraw duplicates until none are left
    while True:
        key = rows * ncols + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        rows, cols = rows[order], cols[order]
        dup = np.zeros(key.shape[0], dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        cols[dup] = rng.integers(0, ncols, size=nd, dtype=np.int64)
    vals = np.random.default_rng(seed + 2000).standard_normal(rows.shape[0])
    return _finish(n, rows, cols, vals)


def ragged_laplace2d(n: int, shift: float):
    """n-row principal block of a 2D grid Laplacian of width nx = round(sqrt(n)):
    node i sits at (i mod nx, i // nx); neighbours i+-1 on the same grid row
    and i+-nx inside [0, n); diagonal 4 + shift, neighbours -1.  SPD for shift > 0."""
    nx = max(1, int(round(math.sqrt(n))))
    i = np.arange(n, dtype=np.int64)
    cand = np.stack([i - nx, i - 1, i, i + 1, i + nx], axis=1)
    ok = np.stack([i - nx >= 0, (i % nx) != 0, np.ones(n, bool), ((i + 1) % nx != 0) & (i + 1 < n),
                   i + nx < n], axis=1)
    vals = np.where(cand == i[:, None], 4.0 + shift, -1.0)
    rows = np.repeat(i, 5).reshape(n, 5)
    return _finish(n, rows[ok], cand[ok], vals[ok])


def batch_sizes(nsys: int, nmin: int, nmax: int, seed: int = 4):
    """Row counts ~ U{nmin..nmax} and diagonal shifts ~ U[0.01, 1]."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(nmin, nmax + 1, size=nsys)
    shifts = rng.uniform(0.01, 1.0, size=nsys)
    return sizes, shifts


def batch_ragged_laplace(nsys: int, nmin: int = 100, nmax: int = 10000, seed: int = 4):
    """Concatenated batch of independent ragged 2D Laplacian systems.
    Returns (row_off int64[nsys+1], nnz_off int64[nsys+1], rp, col, val) where
    rp / col are LOCAL to each system (rp restarts at 0 for every system and
    occupies rp[row_off[s] + s : row_off[s+1] + s + 1])."""
    sizes, shifts = batch_sizes(nsys, nmin, nmax, seed)
    rps, cols, vals = [], [], []
    row_off = np.zeros(nsys + 1, dtype=np.int64)
    nnz_off = np.zeros(nsys + 1, dtype=np.int64)
    for s in range(nsys):
        rp, c, v = ragged_laplace2d(int(sizes[s]), float(shifts[s]))
        rps.append(rp)
        cols.append(c)
        vals.append(v)
        row_off[s + 1] = row_off[s] + sizes[s]
        nnz_off[s + 1] = nnz_off[s] + c.shape[0]
    return row_off, nnz_off, np.concatenate(rps), np.concatenate(cols), np.concatenate(vals)


def diagdom_random(n: int, seed: int, nnz_min: int = 8, nnz_max: int = 32):
    """Nonsymmetric, strictly diagonally dominant random rows: row length
    ~ U{nnz_min..nnz_max} including the diagonal, distinct uniform off-diagonal
    columns, off-diagonal values N(0,1), diagonal = 2 * sum |off-diagonal|."""
    rng = np.random.default_rng(seed)
    L = np.minimum(rng.integers(nnz_min, nnz_max + 1, size=n), n)
    noff = L - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), noff)
    cols = rng.integers(0, max(n - 1, 1), size=rows.shape[0], dtype=np.int64)
    cols = cols + (cols >= rows)  # skip the diagonal
    if n == 1:
        rows = rows[:0]
        cols = cols[:0]
    while True:
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        rows, cols, key = rows[order], cols[order], key[order]
        dup = np.zeros(key.shape[0], dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        c = rng.integers(0, n - 1, size=nd, dtype=np.int64)
        cols[dup] = c + (c >= rows[dup])
    off = rng.standard_normal(rows.shape[0])
    dsum = np.bincount(rows, weights=np.abs(off), minlength=n)
    diag = 2.0 * dsum
    diag[diag == 0.0] = 1.0
    allr = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    allc = np.concatenate([cols, np.arange(n, dtype=np.int64)])
    allv = np.concatenate([off, diag])
    order = np.lexsort((allc, allr))
    return _finish(n, allr[order], allc[order], allv[order])


class DiagDomFamily:
    """Diagonally dominant random rows for any size n <= n_max, from one master
    draw, so that a stream of requests of continuously distributed sizes needs
    no per-request generation beyond one pass over the column indices.

    Row i has L_i ~ U{nnz_min..nnz_max} entries (at most n): the diagonal first,
    then m = L_i - 1 off-diagonal columns, values N(0, 1) off the diagonal and
    2 * sum |off-diagonal| on it (strictly diagonally dominant, nonsymmetric).
    The off-diagonal columns of the size-n matrix are a stratified uniform
    sample of [0, n) without i: with the n - 1 candidates cut into m integer
    strata [floor(j (n-1) / m), floor((j+1) (n-1) / m)), the j-th column is
    uniform in stratum j, moved past the diagonal; they are distinct for
    n - 1 >= m.  Row pointers and values of the size-n matrix are prefixes of
    the master arrays (views); only the columns depend on n."""

    def __init__(self, n_max: int, seed: int, nnz_min: int = 8, nnz_max: int = 32):
        rng = np.random.default_rng(seed)
        L = rng.integers(nnz_min, nnz_max + 1, size=n_max).astype(np.int64)
        self.n_max = n_max
        self.nnz_max = nnz_max
        self.rp = np.zeros(n_max + 1, np.int32)
        self.rp[1:] = np.cumsum(L)
        nnz = int(self.rp[-1])
        self.row = np.repeat(np.arange(n_max, dtype=np.int64), L)
        j = np.arange(nnz, dtype=np.int64) - np.repeat(self.rp[:-1].astype(np.int64), L)  # 0 = diagonal
        self.diag = j == 0
        self.j = np.maximum(j - 1, 0)           # stratum of an off-diagonal entry
        self.m = np.maximum(L - 1, 1)[self.row]  # strata in its row
        self.v = rng.random(nnz)                 # position inside the stratum
        off = ~self.diag
        vals = rng.standard_normal(nnz)
        dsum = np.bincount(self.row[off], weights=np.abs(vals[off]), minlength=n_max)
        vals[self.diag] = 2.0 * dsum
        self.val = vals

    def matrix(self, n: int):
        """(row_ptr, col, val) of the size-n member (n - 1 >= nnz_max - 1)."""
        if not (self.nnz_max <= n <= self.n_max):
            raise ValueError("size outside the family")
        nnz = int(self.rp[n])
        row, j, m = self.row[:nnz], self.j[:nnz], self.m[:nnz]
        lo = j * (n - 1) // m
        w = (j + 1) * (n - 1) // m - lo
        c = lo + np.minimum((self.v[:nnz] * w).astype(np.int64), w - 1)
        c += c >= row
        col = np.where(self.diag[:nnz], row, c).astype(np.int32)
        return self.rp[: n + 1], col, self.val[:nnz]


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """x ~ U[lo, hi] in double."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)

"""Bounds of the row-block SpMV kernels' bulk copies, checked on the CPU.

The row-block CSR and COO kernels copy each tile of 128 rows into a shared-memory
stage with 1-D bulk copies (`cp.async.bulk`), whose source and size must be
multiples of 16 bytes.  This file restates the tile arithmetic of the kernels
(copy start rounded down to 16 bytes, size rounded up, stage slots sized from the
largest tile) and checks, for the test and benchmark matrices, that

* every copy starts on a 16-byte boundary and moves a multiple of 16 bytes;
* every copy stays inside the library's device array, which is allocated with
  its size rounded up to 16 bytes plus 64 bytes of padding;
* every copy fits its stage slot, and every shared-memory read of the reduction
  (row pointers, columns, values, for 1, 2 or 4 threads per row) lands in data
  the copy brought in;
* with several threads per row, the lanes of a row take each entry exactly once.

No GPU is needed; a mistake here is a fault there, so this runs before any
GPU test of a new matrix shape."""
import numpy as np
import pytest

from paper_2103_10116_gb300 import synth

ROWS = 128
PAD = 64
SMEM_OPTIN = 232448  # bytes of shared memory a block may opt into on sm_103a


def _r16(v):
    return (np.asarray(v, dtype=np.int64) + 15) // 16 * 16


def _alloc(nbytes):
    return int(_r16(nbytes)) + PAD


MATS = {
    "lap2d_64": lambda: synth.laplace2d_5pt(64),
    "st27_23": lambda: synth.stencil3d_27pt(23),
    "convdiff_20": lambda: synth.convdiff3d_upwind(20),
    "powerlaw_60k": lambda: synth.powerlaw(60000, mean=16, max_len=6000, seed=5),
    "ragged_tail": lambda: synth.laplace2d_5pt(37),  # n = 1369: a last tile of 89 rows
    "stencil27_100": lambda: synth.stencil3d_27pt(100),
    "poisson128": lambda: synth.laplace3d_7pt(128),
}
_cache = {}


def _rp(name):
    if name not in _cache:
        _cache[name] = np.asarray(MATS[name]()[0], dtype=np.int64)
    return _cache[name]


def _lane_count(L, sub, tpr):
    """Entries lane `sub` of a row of length L takes (sub + tpr*u for u below this count)."""
    return L if tpr == 1 else (L - sub + tpr - 1) // tpr


def _lane_partition_ok(lengths, tpr, count=_lane_count):
    for L in np.unique(lengths):
        L = int(L)
        taken = [sub + tpr * u for sub in range(tpr) for u in range(count(L, sub, tpr))]
        if sorted(taken) != list(range(L)):
            return False
    return True


@pytest.mark.parametrize("V", [8, 4], ids=["f64", "f32"])
@pytest.mark.parametrize("name", list(MATS))
def test_csr_row_block_copies_stay_in_bounds(name, V):
    rp = _rp(name)
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    ntiles = -(-n // ROWS)
    t = np.arange(ntiles, dtype=np.int64)
    r0 = t * ROWS
    r1 = np.minimum(n, r0 + ROWS)
    j0, j1 = rp[r0], rp[r1]
    cap = int((j1 - j0).max())
    VA = 16 // V
    rp_bytes = (ROWS + 8) * 4
    col_bytes = ((cap + 8) * 4 + 15) & ~15
    val_bytes = ((cap + 8) * V + 15) & ~15
    smem = 2 * (rp_bytes + col_bytes + val_bytes) + 32 + 16
    if smem > SMEM_OPTIN:  # the launcher returns SPX_ERR_TOO_LARGE; nothing is copied
        assert name == "powerlaw_60k"
        return
    ra = r0 & ~3
    rbytes = ((r1 + 1 - ra + 3) & ~3) * 4
    ca = j0 & ~3
    va = j0 & ~(VA - 1)
    has = j1 > j0
    cbytes = np.where(has, ((j1 - ca + 3) & ~3) * 4, 0)
    vbytes = np.where(has, ((j1 - va + VA - 1) & ~(VA - 1)) * V, 0)
    for start, size in ((ra * 4, rbytes), (ca * 4, cbytes), (va * V, vbytes)):
        assert np.all(start % 16 == 0) and np.all(size % 16 == 0)
    assert np.all(ra * 4 + rbytes <= _alloc((n + 1) * 4))
    assert np.all(np.where(has, ca * 4 + cbytes, 0) <= _alloc(nnz * 4))
    assert np.all(np.where(has, va * V + vbytes, 0) <= _alloc(nnz * V))
    assert np.all(rbytes <= rp_bytes) and np.all(cbytes <= col_bytes) and np.all(vbytes <= val_bytes)
    # reads of the reduction: s_rp[(r0 - ra) + q + 1] for the tile's last row; the last entry of the tile
    assert np.all((r1 - ra + 1) * 4 <= rbytes)
    assert np.all(np.where(has, (j1 - ca) * 4 <= cbytes, True))
    assert np.all(np.where(has, (j1 - va) * V <= vbytes, True))
    lengths = np.diff(rp)
    for tpr in (1, 2, 4):
        assert _lane_partition_ok(lengths, tpr)


@pytest.mark.parametrize("V", [8, 4], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["lap2d_64", "st27_23", "convdiff_20", "ragged_tail", "poisson128"])
def test_coo_row_block_copies_stay_in_bounds(name, V):
    rp = _rp(name)
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    crow = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    ntiles = -(-n // ROWS)
    bounds = np.searchsorted(crow, np.minimum(n, np.arange(ntiles + 1, dtype=np.int64) * ROWS), side="left")
    e0, e1 = bounds[:-1], bounds[1:]
    cap = int((e1 - e0).max())
    VA = 16 // V
    idx_bytes = ((cap + 8) * 4 + 15) & ~15
    val_bytes = ((cap + 8) * V + 15) & ~15
    assert 2 * (2 * idx_bytes + val_bytes) + 32 + 16 <= SMEM_OPTIN
    ia = e0 & ~3
    va = e0 & ~(VA - 1)
    has = e1 > e0
    ibytes = np.where(has, ((e1 - ia + 3) & ~3) * 4, 0)
    vbytes = np.where(has, ((e1 - va + VA - 1) & ~(VA - 1)) * V, 0)
    for start, size in ((ia * 4, ibytes), (va * V, vbytes)):
        assert np.all(start % 16 == 0) and np.all(size % 16 == 0)
    assert np.all(np.where(has, ia * 4 + ibytes, 0) <= _alloc(nnz * 4))
    assert np.all(np.where(has, va * V + vbytes, 0) <= _alloc(nnz * V))
    assert np.all(ibytes <= idx_bytes) and np.all(vbytes <= val_bytes)
    assert np.all(np.where(has, (e1 - ia) * 4 <= ibytes, True))
    assert np.all(np.where(has, (e1 - va) * V <= vbytes, True))
    # every staged row index belongs to the tile, so the row marks s_first/s_end[row - r0] stay in [0, ROWS)
    t_of_entry = np.repeat(np.arange(ntiles), e1 - e0)
    assert np.all((crow - t_of_entry * ROWS >= 0) & (crow - t_of_entry * ROWS < ROWS))


def test_lane_partition_detects_a_wrong_split():
    """The partition check itself: a count that drops the last entry of odd rows fails it."""
    lengths = np.array([0, 1, 5, 27])
    assert _lane_partition_ok(lengths, 2) and _lane_partition_ok(lengths, 4)
    assert not _lane_partition_ok(lengths, 2, count=lambda L, sub, tpr: L // tpr)

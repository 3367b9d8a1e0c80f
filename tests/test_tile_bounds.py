"""Bounds of the tiled SpMV kernels' bulk copies, checked on the CPU.

The row-block CSR and COO kernels copy each tile of 128 rows, and the merge-path
CSR kernel each tile of merge items (row ends and nonzeros), into a shared-memory
stage with 1-D bulk copies (`cp.async.bulk`), whose source and size must be
multiples of 16 bytes.  This file restates the tile arithmetic of the kernels
(the merge-path tile map, copy start rounded down to 16 bytes, size rounded up,
stage slots sized from the largest tile) and checks, for the test and benchmark
matrices, that

* every copy starts on a 16-byte boundary and moves a multiple of 16 bytes;
* every copy stays inside the library's device array, which is allocated with
  its size rounded up to 16 bytes plus 64 bytes of padding;
* every copy fits its stage slot (for the merge-path kernel, together with the
  row sums stored after it), and every shared-memory read of the reduction
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


def _long_row():
    """Rows of 3 entries and one of 50,000: longer than any merge tile's slack."""
    lens = np.full(3000, 3, np.int64)
    lens[7] = 50000
    rp = np.zeros(lens.size + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    return rp, None, None


MATS = {
    "lap2d_64": lambda: synth.laplace2d_5pt(64),
    "st27_23": lambda: synth.stencil3d_27pt(23),
    "convdiff_20": lambda: synth.convdiff3d_upwind(20),
    "powerlaw_60k": lambda: synth.powerlaw(60000, mean=16, max_len=6000, seed=5),
    "ragged_tail": lambda: synth.laplace2d_5pt(37),  # n = 1369: a last tile of 89 rows
    "stencil27_100": lambda: synth.stencil3d_27pt(100),
    "poisson128": lambda: synth.laplace3d_7pt(128),
    "long_row": _long_row,
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
        assert name in ("powerlaw_60k", "long_row")
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


def _merge_tiles(rp, tile, slack):
    """Tile boundaries (row, nonzero) of the merge-path CSR kernel: the merge of the row ends
    with the nonzeros cut every `tile` items, each cut moved forward to the next row end when
    that is at most `slack` items away."""
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    ntiles = -(-(n + nnz) // tile)
    d = np.minimum(np.arange(ntiles + 1, dtype=np.int64) * tile, n + nnz)
    # the first row i with i + rp[i + 1] >= d (row ends before the cut), within the feasible range
    i = np.searchsorted(np.arange(n, dtype=np.int64) + rp[1:], d, side="left")
    i = np.clip(i, np.maximum(0, d - nnz), np.minimum(d, n))
    j = d - i
    inner = (i < n) & (j > rp[np.minimum(i, n)])
    dn = i + 1 + rp[np.minimum(i + 1, n)]
    snap = inner & (dn - d <= slack)
    i = np.where(snap, i + 1, i)
    j = np.where(snap, rp[np.minimum(i, n)], j)
    return i, j


@pytest.mark.parametrize("ipt", [4, 8, 16])
@pytest.mark.parametrize("V", [8, 4], ids=["f64", "f32"])
@pytest.mark.parametrize("name", ["lap2d_64", "st27_23", "convdiff_20", "powerlaw_60k", "ragged_tail", "long_row"])
def test_merge_path_copies_stay_in_bounds(name, V, ipt):
    rp = _rp(name)
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    block = 256
    tile = block * ipt
    slack = tile // 4
    stage = (4 + V) * (tile + slack) + 256
    smem = 2 * stage + block * 4 + block * V + (block + 1) * 4 + 12 + 32 + 16
    assert smem <= SMEM_OPTIN
    ti, tj = _merge_tiles(rp, tile, slack)
    assert ti[0] == 0 and tj[0] == 0 and ti[-1] == n and tj[-1] == nnz
    assert np.all(np.diff(ti) >= 0) and np.all(np.diff(tj) >= 0)
    i0, j0, i1, j1 = ti[:-1], tj[:-1], ti[1:], tj[1:]
    assert np.all((i1 - i0) + (j1 - j0) <= tile + slack)
    VA = 16 // V
    ra = i0 & ~3
    rend = np.minimum(i1 + 2, n + 1)
    rbytes = ((rend - ra + 3) & ~3) * 4
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
    # the copies, then one row sum per row end of the tile, fit the stage
    assert np.all(rbytes + cbytes + vbytes + V * (i1 - i0) <= stage)
    # rp[i0 .. min(i1 + 1, n)] and the tile's nonzeros were copied
    assert np.all((np.minimum(i1 + 1, n) - ra + 1) * 4 <= rbytes)
    assert np.all(np.where(has, (j1 - ca) * 4 <= cbytes, True))
    assert np.all(np.where(has, (j1 - va) * V <= vbytes, True))
    if name == "long_row":  # the 50,000-entry row straddles tiles: the cut inside it was not snapped
        assert np.any((j0 > rp[np.minimum(i0, n)]) & (i0 < n))


def test_lane_partition_detects_a_wrong_split():
    """The partition check itself: a count that drops the last entry of odd rows fails it."""
    lengths = np.array([0, 1, 5, 27])
    assert _lane_partition_ok(lengths, 2) and _lane_partition_ok(lengths, 4)
    assert not _lane_partition_ok(lengths, 2, count=lambda L, sub, tpr: L // tpr)


@pytest.mark.parametrize("R,V", [(1, 8), (2, 8), (1, 4), (2, 4), (4, 4)])
def test_ell_vector_loads_stay_in_bounds(R, V):
    """The ELL kernel gives each thread R consecutive rows and reads each slab's R
    columns and values with one vector load: slab j, rows [i, i + R), i = g*R.  The
    column-major arrays have ld = n rounded up to 32 rows per slab (HYB's ELL part
    too), so every load is aligned to its own size and stays inside its slab.  The
    rows-per-thread choices the library accepts (1 or 2 in FP64, up to 4 in FP32)
    keep each vector load within 16 bytes."""
    n = np.arange(1, 4200, dtype=np.int64)
    ld = (n + 31) // 32 * 32
    last = ((n + R - 1) // R - 1) * R  # first row of the last group
    assert np.all(last + R <= ld)
    assert np.all(ld % R == 0)  # slab starts j*ld and group starts i are multiples of R
    assert R * V <= 16 and R * 4 <= 16


# ---------------------------------------------------------------- tiled nnz-split CSR
def _tiled_layout(nnz, ipt, vec):
    """Destination of source entry k in the tile-transposed layout (the index
    arithmetic of the transposition kernel), over the padded range."""
    chunk = 32 * ipt
    nchunks = -(-nnz // chunk)
    total = nchunks * chunk
    k = np.arange(total, dtype=np.int64)
    c = k // chunk
    wi = k - c * chunk
    lane, u = wi // ipt, wi % ipt
    return c * chunk + (u // vec) * 32 * vec + lane * vec + u % vec, total


def _tiled_descriptors(rp, ipt):
    """trow / tmask / slow flags as the descriptor kernels define them."""
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    ngran = -(-nnz // (32 * ipt)) * 32
    trow = np.zeros(ngran, np.int64)
    a = np.arange(ngran, dtype=np.int64) * ipt
    act = a < nnz
    trow[act] = np.searchsorted(rp[1:], a[act], side="right")  # first r with rp[r+1] > a
    tmask = np.zeros(ngran + 1, np.int64)
    slow = np.zeros(ngran, bool)
    for r in range(n):
        p = int(rp[r])
        g, u = divmod(p, ipt)
        if rp[r + 1] > p:
            tmask[g] |= 1 << u
        elif u != 0 and p < nnz:
            slow[g] = True
    return trow, tmask, slow, ngran


def _tiled_walk(rp, col, val, x, ipt):
    """The lanes' walk over their granules using only the descriptors (and the
    row pointers where a granule is flagged), summing each row's pieces: must
    give the SpMV."""
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    trow, tmask, slow, ngran = _tiled_descriptors(rp, ipt)
    y = np.zeros(n)
    for g in range(ngran):
        a = g * ipt
        cnt = max(0, min(ipt, nnz - a))
        if cnt == 0:
            continue
        r = int(trow[g])
        assert rp[r] <= a < rp[r + 1]  # the row holding the granule's first entry, never empty
        for s in range(cnt):
            if s > 0 and (tmask[g] >> s) & 1:
                r += 1
                if slow[g]:
                    while rp[r + 1] == rp[r]:
                        r += 1
                assert rp[r] == a + s  # the row that starts here
            assert rp[r] <= a + s < rp[r + 1]
            y[r] += val[a + s] * x[col[a + s]]
        ends_b = a + ipt >= nnz or (tmask[g + 1] & 1)
        assert bool(ends_b) == (rp[r + 1] == min(a + ipt, nnz) or a + ipt >= nnz)
    return y


def _empty_rows_matrix():
    rng = np.random.default_rng(3)
    lens = rng.integers(0, 40, size=700)
    lens[rng.random(700) < 0.3] = 0
    lens[:5] = 0
    lens[-7:] = 0
    lens[300] = 2500
    rp = np.zeros(lens.size + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    col = rng.integers(0, lens.size, size=int(rp[-1]))
    val = rng.integers(-8, 9, size=int(rp[-1])).astype(np.float64)
    return rp, col, val


@pytest.mark.parametrize("ipt", [16, 32])
@pytest.mark.parametrize("mname", ["lap2d_64", "powerlaw_60k", "ragged_tail", "empty_rows"])
def test_tiled_csr_layout_and_descriptors(mname, ipt):
    if mname == "empty_rows":
        rp, col, val = _empty_rows_matrix()
    else:
        rp, col, val = MATS[mname]()
        rp = np.asarray(rp, np.int64)
    nnz = int(rp[-1])
    for vec, esize in ((4, 4), (2, 8), (4, 4)):  # columns, FP64 values, FP32 values
        dst, total = _tiled_layout(nnz, ipt, vec)
        # a permutation of the padded range: every slot written once, all inside the allocation
        assert dst.min() == 0 and dst.max() == total - 1 and np.unique(dst).size == total
        assert (total * esize + 16) <= _alloc(total * esize + 16)
        # the kernel's 16-byte loads: lane l, slot group q of chunk c reads
        # [c*CHUNK + q*32*vec + l*vec, +vec): aligned and inside the chunk
        chunk = 32 * ipt
        q = np.arange(ipt // vec)[:, None]
        lane = np.arange(32)[None, :]
        off = q * 32 * vec + lane * vec
        assert (off * esize % 16 == 0).all() and off.min() == 0 and (off + vec).max() == chunk
        # lane l's slot u is the source entry l*ipt + u of the chunk
        src = np.empty(total, np.int64)
        src[dst] = np.arange(total)
        u = np.arange(ipt)
        for l in (0, 5, 31):
            got = src[(u // vec) * 32 * vec + l * vec + u % vec]
            assert np.array_equal(got, l * ipt + u)
    trow, tmask, slow, ngran = _tiled_descriptors(rp, ipt)
    assert tmask.shape[0] == ngran + 1  # the kernel reads tmask[g + 1] for every granule
    assert (trow < rp.shape[0] - 1).all() and (trow >= 0).all()
    if mname != "empty_rows":
        assert not slow.any()
    else:
        assert slow.any()
    # the descriptor walk reproduces the product exactly on integer data
    x = np.random.default_rng(1).integers(-8, 9, size=rp.shape[0] - 1).astype(np.float64)
    if mname != "empty_rows":
        val = np.round(np.asarray(val) * 4)  # small integers: exact sums in any order
    y = _tiled_walk(rp, np.asarray(col), np.asarray(val, np.float64), x, ipt)
    yref = np.zeros(rp.shape[0] - 1)
    rows = np.repeat(np.arange(rp.shape[0] - 1), np.diff(rp))
    np.add.at(yref, rows, np.asarray(val, np.float64) * x[np.asarray(col)])
    assert np.array_equal(y, yref)


# ------------------------------------------------------------------ cluster solves
# The two cluster kernels split a system's rows over the blocks of one cluster:
# the small-system CG gives block k the slice [k R, (k+1) R) of R = 2^lg rows,
# lg the least with CL << lg >= n, and keeps it in shared memory (4 vectors of R
# values, R at most 4096); the one-cluster solve of any size gives block k
# [min(n, k R), min(n, k R + R)) with R = ceil(n / CL) rounded up to 32.  Every
# row must belong to exactly one block, a block's slice must start on a multiple
# of 32 rows (its threads' rows then fall in whole warps' sectors), and the small
# CG's slices must fit the shared memory it asks for.


def _cluster_small_slices(n, cl):
    lg = 0
    while (cl << lg) < n:
        lg += 1
    r = 1 << lg
    return r, [(min(n, k * r), min(n, (k + 1) * r)) for k in range(cl)]


def _cluster_solve_slices(n, cl):
    r = ((n + cl - 1) // cl + 31) & ~31
    return r, [(min(n, k * r), min(n, k * r + r)) for k in range(cl)]


@pytest.mark.parametrize("cl", [8, 16])
def test_cluster_row_slices_partition_the_rows(cl):
    sizes = [1, 2, 5, 31, 32, 33, 4095, 4096, 4097, 8000, 32761, 65535, 65536, 68921, 10**6, 2**30]
    for n in sizes:
        for slices_of, small in ((_cluster_solve_slices, False), (_cluster_small_slices, True)):
            if small and n > cl * 4096:
                continue  # the small CG takes at most 4096 rows per block
            r, sl = slices_of(n, cl)
            covered = 0
            for k, (lo, hi) in enumerate(sl):
                assert 0 <= lo <= hi <= n
                assert hi - lo <= r
                if hi > lo:
                    assert lo == covered, (n, cl, k)  # contiguous, in rank order, no overlap
                    covered = hi
                if not small:
                    assert lo % 32 == 0 or lo == n
            assert covered == n, (n, cl)
            if small:
                assert r <= 4096 and 4 * r * 8 <= SMEM_OPTIN  # four FP64 slices in shared memory
            else:
                assert r % 32 == 0 and r * cl >= n

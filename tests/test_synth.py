"""The seeded input generators: the exact-size random family of the serving
workload (CPU only)."""
import numpy as np
import pytest
import torch

from paper_2103_10116_gb300 import synth


@pytest.fixture(scope="module")
def fam():
    return synth.DiagDomFamily(60_000, seed=7)


@pytest.mark.parametrize("n", [1000, 1001, 4567, 60_000])
def test_family_member_is_diagonally_dominant_with_distinct_columns(fam, n):
    rp, col, val = fam.matrix(n)
    assert rp.shape[0] == n + 1 and rp[0] == 0 and col.shape[0] == rp[-1] == val.shape[0]
    L = np.diff(rp)
    assert L.min() >= 8 and L.max() <= 32
    assert col.min() >= 0 and col.max() < n
    rows = np.repeat(np.arange(n), L)
    key = rows.astype(np.int64) * n + col
    assert np.unique(key).size == key.size          # distinct columns in every row
    isd = col == rows
    assert isd.sum() == n and np.all(col[rp[:-1]] == np.arange(n))  # the diagonal first
    off = np.zeros(n)
    np.add.at(off, rows[~isd], np.abs(val[~isd]))
    assert np.allclose(val[isd], 2 * off) and np.all(val[isd] > 0)


def test_family_columns_are_uniform(fam):
    # each stratum is uniform, so the columns are: a chi-square-free check on deciles
    _, col, _ = fam.matrix(50_000)
    hist = np.bincount(col * 10 // 50_000, minlength=10) / col.size
    assert np.all(np.abs(hist - 0.1) < 0.01)


def test_bench_family_columns_match_the_generator(fam):
    import bench
    t = lambda a: torch.from_numpy(a)
    for n in (1000, 31337, 60_000):
        nnz = int(fam.rp[n])
        got = bench.family_columns(t(fam.j), t(fam.m), t(fam.v), t(fam.row), t(fam.diag), n, nnz).numpy()
        assert np.array_equal(got, fam.matrix(n)[1])

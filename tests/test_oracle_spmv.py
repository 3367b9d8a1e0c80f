"""Pins for the oracle's SpMV, CSR check and storage conversions (CPU only).

Each pin comes from outside the oracle: exact dense products on integer data,
closed-form Laplacian eigenpairs, hand-worked layouts (tests/golden), and
brute force over every ELL width.  Mutation tests rebuild the oracle with a
planted mistake and show that a pin fails.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import laplace1d, random_int_csr, to_dense

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- SpMV pins
def test_spmv_hand_worked_example():
    g = _golden("spmv_4x4.json")
    y = oracle.spmv_csr(g["row_ptr"], g["col"], g["val"], g["x"])
    assert np.array_equal(y, np.array(g["y"]))
    assert np.array_equal(to_dense(g["row_ptr"], g["col"], g["val"]), np.array(g["dense"], float))


@pytest.mark.parametrize("seed", range(12))
def test_spmv_exact_against_dense_on_integers(seed):
    # Integer A and x with |entries| <= 8 and short rows: every partial sum is an
    # exactly representable integer, so any summation order gives the same bits.
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    ncols = int(rng.integers(1, 40))
    rp, col, val = random_int_csr(rng, n, ncols)
    x = rng.integers(-8, 9, size=ncols).astype(np.float64)
    y = oracle.spmv_csr(rp, col, val, x)
    assert np.array_equal(y, to_dense(rp, col, val, ncols) @ x)
    assert np.array_equal(oracle.spmv_csr_plain(rp, col, val, x), y)


def test_openmp_build_gives_the_same_bits():
    # the all-cores CPU baseline runs the plain definition with rows shared among
    # threads: each row is still summed alone in index order, so the bits match
    rng = np.random.default_rng(9)
    rp, col, val = random_int_csr(rng, 5000, 5000, max_len=30)
    val = val * 0.3127
    x = rng.standard_normal(5000)
    assert np.array_equal(oracle.spmv_csr_plain_omp(rp, col, val, x), oracle.spmv_csr_plain(rp, col, val, x))


def test_spmv_empty_matrix_and_rows():
    rp = np.zeros(6, np.int32)
    y = oracle.spmv_csr(rp, np.zeros(0, np.int32), np.zeros(0), np.ones(3))
    assert np.array_equal(y, np.zeros(5))


@pytest.mark.parametrize("m", [5, 17])
def test_laplace1d_eigenpairs(m):
    # tridiag(-1,2,-1): lambda_j = 2 - 2 cos(j pi/(m+1)), v_j(i) = sin(i j pi/(m+1)).
    rp, col, val = laplace1d(m)
    i = np.arange(1, m + 1)
    for j in (1, 2, m // 2, m):
        v = np.sin(i * j * np.pi / (m + 1))
        lam = 2.0 - 2.0 * np.cos(j * np.pi / (m + 1))
        r = oracle.spmv_csr(rp, col, val, v) - lam * v
        assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(v)


@pytest.mark.parametrize("m", [6, 11])
def test_laplace2d_eigenpairs(m):
    # 5-point: lambda_jk = 4 - 2cos(j pi/(m+1)) - 2cos(k pi/(m+1)), product-sine vector.
    rp, col, val = synth.laplace2d_5pt(m)
    iy, ix = np.meshgrid(np.arange(1, m + 1), np.arange(1, m + 1), indexing="ij")
    for j, k in [(1, 1), (2, 3), (m, 1), (m, m)]:
        v = (np.sin(ix * j * np.pi / (m + 1)) * np.sin(iy * k * np.pi / (m + 1))).ravel()
        lam = 4 - 2 * np.cos(j * np.pi / (m + 1)) - 2 * np.cos(k * np.pi / (m + 1))
        r = oracle.spmv_csr(rp, col, val, v) - lam * v
        assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(v)


def _sines3(m, jx, jy, jz):
    iz, iy, ix = np.meshgrid(*(np.arange(1, m + 1),) * 3, indexing="ij")
    th = np.pi / (m + 1)
    return (np.sin(ix * jx * th) * np.sin(iy * jy * th) * np.sin(iz * jz * th)).ravel()


@pytest.mark.parametrize("m", [4, 9])
def test_laplace3d_7pt_eigenpairs(m):
    rp, col, val = synth.laplace3d_7pt(m)
    assert col.shape[0] == 7 * m**3 - 6 * m**2
    th = np.pi / (m + 1)
    for js in [(1, 1, 1), (2, 1, m), (m, m, m)]:
        v = _sines3(m, *js)
        lam = 6 - 2 * sum(np.cos(j * th) for j in js)
        r = oracle.spmv_csr(rp, col, val, v) - lam * v
        assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(v)


@pytest.mark.parametrize("m", [3, 8])
def test_stencil27_eigenpairs(m):
    # 27 I - T(x)T(x)T with T = tridiag(1,1,1): lambda = 27 - prod_d (1 + 2cos(j_d pi/(m+1))).
    rp, col, val = synth.stencil3d_27pt(m)
    assert col.shape[0] == (3 * m - 2) ** 3
    th = np.pi / (m + 1)
    for js in [(1, 1, 1), (1, 2, 3), (m, 1, m)]:
        v = _sines3(m, *js)
        lam = 27 - np.prod([1 + 2 * np.cos(j * th) for j in js])
        r = oracle.spmv_csr(rp, col, val, v) - lam * v
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(v)


def test_convdiff_row_sums():
    # Upwind rows sum to zero at interior points (consistency of the scheme) and
    # are positive where a Dirichlet neighbour was dropped.
    m = 6
    rp, col, val = synth.convdiff3d_upwind(m)
    s = oracle.spmv_csr(rp, col, val, np.ones(m**3)).reshape(m, m, m)
    assert np.all(np.abs(s[1:-1, 1:-1, 1:-1]) <= 1e-14)
    assert np.all(s[0] > 0) and np.all(s[:, 0] > 0) and np.all(s[:, :, 0] > 0)
    d = to_dense(rp, col, val)
    assert not np.allclose(d, d.T)


def test_compensated_sum_is_correctly_rounded_scale():
    # Exact rational arithmetic (fractions) gives the true row sums; the
    # compensated oracle must sit within a couple of ulps of the exact value
    # measured against (|A||x|)_i, far inside any kernel tolerance.
    from fractions import Fraction
    rng = np.random.default_rng(3)
    rp, col, val = random_int_csr(rng, 30, 30)
    val = val * 0.37
    x = rng.standard_normal(30)
    y = oracle.spmv_csr(rp, col, val, x)
    bound = oracle.spmv_absbound(rp, col, val, x)
    for i in range(30):
        exact = sum((Fraction(float(val[k])) * Fraction(float(x[col[k]]))
                     for k in range(rp[i], rp[i + 1])), Fraction(0))
        assert abs(Fraction(float(y[i])) - exact) <= Fraction(2.3e-16) * Fraction(float(bound[i]))
        assert bound[i] >= abs(y[i])


@pytest.mark.parametrize("seed", range(12))
def test_absbound_exact_against_dense_on_integers(seed):
    # (|A||x|)_i scales every GPU parity tolerance, so it is pinned exactly:
    # on integer A and x (|entries| <= 8, short rows) every partial sum is an
    # exact integer, and the bound must equal the dense product |A|.|x| bit for
    # bit.  Duplicates count once each (|a|+|b|, not |a+b|), as the dense
    # matrix of absolute entries below does.
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 40))
    ncols = int(rng.integers(1, 40))
    rp, col, val = random_int_csr(rng, n, ncols)
    x = rng.integers(-8, 9, size=ncols).astype(np.float64)
    absdense = np.zeros((n, ncols))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            absdense[i, col[k]] += abs(val[k])
    got = oracle.spmv_absbound(rp, col, val, x)
    assert np.array_equal(got, absdense @ np.abs(x))
    # and it bounds the product itself, with equality on non-negative data
    assert np.all(got >= np.abs(oracle.spmv_csr(rp, col, val, x)))
    assert np.array_equal(oracle.spmv_absbound(rp, col, np.abs(val), np.abs(x)),
                          oracle.spmv_csr(rp, col, np.abs(val), np.abs(x)))


@pytest.mark.parametrize("mutant", [12, 13])
def test_planted_absbound_mistakes_are_caught(mutant):
    # 12 doubles the bound (a loosened tolerance), 13 reads x at the row index
    # instead of the column index: the exact dense pin above fails for both.
    caught = False
    for seed in range(6):
        rng = np.random.default_rng(seed)
        rp, col, val = random_int_csr(rng, 20, 20, empty_frac=0.0)
        x = rng.integers(-8, 9, size=20).astype(np.float64)
        absdense = np.abs(to_dense(rp, col, np.abs(val)))
        got = oracle.spmv_absbound(rp, col, val, x, mutant=mutant)
        caught |= not np.array_equal(got, absdense @ np.abs(x))
    assert caught


# ---------------------------------------------------------------- CSR check
def test_csr_check():
    g = _golden("spmv_4x4.json")
    assert oracle.csr_check(4, 4, g["row_ptr"], g["col"])
    assert not oracle.csr_check(4, 4, [0, 2, 1, 5, 7], g["col"])         # decreasing
    assert not oracle.csr_check(4, 4, [1, 2, 2, 5, 7], g["col"])         # rp[0] != 0
    assert not oracle.csr_check(4, 3, g["row_ptr"], g["col"])            # col >= ncols
    bad = list(g["col"])
    bad[3] = -1
    assert not oracle.csr_check(4, 4, g["row_ptr"], bad)                 # negative col
    assert not oracle.csr_check(4, 4, [0, 2, 2, 5, 6], g["col"])         # rp[n] != nnz


# ---------------------------------------------------------------- conversions
def test_conversions_hand_worked():
    g = _golden("spmv_4x4.json")
    rp, col, val = (np.array(g["row_ptr"], np.int32), np.array(g["col"], np.int32),
                    np.array(g["val"]))
    assert np.array_equal(oracle.csr_to_coo_rows(rp), g["coo_row"])
    assert oracle.max_row_len(rp) == g["ell_width"]
    ec, ev = oracle.csr_to_ell(rp, col, val, g["ell_width"], g["ell_ld"])
    assert np.array_equal(ec, g["ell_col"]) and np.array_equal(ev, g["ell_val"])
    ec, ev, cr, cc, cv = oracle.csr_to_hyb(rp, col, val, g["hyb_width"], g["ell_ld"])
    assert np.array_equal(ec, g["hyb_ell_col"]) and np.array_equal(ev, g["hyb_ell_val"])
    assert np.array_equal(cr, g["hyb_coo_row"]) and np.array_equal(cc, g["hyb_coo_col"])
    assert np.array_equal(cv, g["hyb_coo_val"])


def _dense_from_ell(ec, ev, n, ld, k, ncols):
    d = np.zeros((n, ncols))
    for j in range(k):
        for i in range(ld):
            c = ec[j * ld + i]
            if c >= 0:
                assert i < n
                d[i, c] += ev[j * ld + i]
            else:
                assert ev[j * ld + i].tobytes() == bytes(ev.itemsize)
    return d


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_conversions_reconstruct_dense(seed, dtype):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 30))
    rp, col, val = random_int_csr(rng, n, n, max_len=9)
    val = val.astype(dtype)
    dense = to_dense(rp, col, val.astype(np.float64))
    # COO keeps CSR order
    rows = oracle.csr_to_coo_rows(rp)
    assert np.array_equal(rows, np.repeat(np.arange(n), np.diff(rp)))
    # ELL
    k = oracle.max_row_len(rp)
    ld = ((n + 31) // 32) * 32
    ec, ev = oracle.csr_to_ell(rp, col, val, k, ld)
    assert np.array_equal(_dense_from_ell(ec, ev, n, ld, k, n), dense)
    # within-row order kept: slot j of row i holds entry rp[i]+j
    for i in range(n):
        for j in range(rp[i + 1] - rp[i]):
            assert ec[j * ld + i] == col[rp[i] + j]
            assert ev[j * ld + i].tobytes() == val[rp[i] + j].tobytes()
    # HYB at every width
    for w in range(0, k + 2):
        ec, ev, cr, cc, cv = oracle.csr_to_hyb(rp, col, val, w, ld)
        assert cr.shape[0] == oracle.hyb_coo_count(rp, w) == sum(max(0, int(L) - w) for L in np.diff(rp))
        d = _dense_from_ell(ec, ev, n, ld, w, n)
        for a, b_, c in zip(cr, cc, cv):
            d[a, b_] += c
        assert np.array_equal(d, dense)
        assert np.all(np.diff(cr) >= 0)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("vbytes", [8, 4])
def test_hyb_auto_width_minimises_footprint(seed, vbytes):
    # Brute force: the footprint (V+4) k n + (V+8) * overflow over every width;
    # the rule must return the smallest minimiser.
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 200))
    lens = np.minimum(synth.powerlaw_lengths(n, mean=6, max_len=60, seed=seed), 60)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(lens)
    foot = [(vbytes + 4) * k * n + (vbytes + 8) * int(np.maximum(lens - k, 0).sum())
            for k in range(int(lens.max()) + 1)]
    assert oracle.hyb_auto_width(rp, vbytes) == int(np.argmin(foot))


def test_hyb_auto_width_27pt_is_pure_ell():
    rp, _, _ = synth.stencil3d_27pt(40)  # 86% interior rows of length 27
    assert oracle.hyb_auto_width(rp, 8) == 27


# ---------------------------------------------------------------- mutants
@pytest.mark.parametrize("mutant", [1, 2])
def test_planted_spmv_mistakes_are_caught(mutant):
    caught = False
    for seed in range(6):
        rng = np.random.default_rng(seed)
        rp, col, val = random_int_csr(rng, 20, 20, empty_frac=0.0)
        x = rng.integers(-8, 9, size=20).astype(np.float64)
        y = oracle.spmv_csr(rp, col, val, x, mutant=mutant)
        caught |= not np.array_equal(y, to_dense(rp, col, val) @ x)
    assert caught

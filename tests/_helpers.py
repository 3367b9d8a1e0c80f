"""Small test helpers: dense copies and random tiny CSR matrices.  Nothing here
is used by the library or by the oracle."""
import numpy as np


def to_dense(rp, col, val, ncols=None):
    n = len(rp) - 1
    ncols = n if ncols is None else ncols
    d = np.zeros((n, ncols))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            d[i, col[k]] += val[k]
    return d


def random_int_csr(rng, n, ncols=None, max_len=6, allow_dup=True, lo=-8, hi=8,
                   empty_frac=0.2):
    """Tiny CSR with integer values: empty rows, unsorted and duplicate columns
    and explicit zeros all occur."""
    ncols = n if ncols is None else ncols
    rp = [0]
    cols, vals = [], []
    for _ in range(n):
        L = 0 if rng.random() < empty_frac else int(rng.integers(1, max_len + 1))
        if not allow_dup:
            L = min(L, ncols)
            c = rng.choice(ncols, size=L, replace=False)
        else:
            c = rng.integers(0, ncols, size=L)
        cols.extend(int(v) for v in c)
        vals.extend(float(v) for v in rng.integers(lo, hi + 1, size=L))
        rp.append(len(cols))
    return (np.array(rp, dtype=np.int32), np.array(cols, dtype=np.int32),
            np.array(vals, dtype=np.float64))


def csr_from_dense(d):
    rp, cols, vals = [0], [], []
    for i in range(d.shape[0]):
        for j in range(d.shape[1]):
            if d[i, j] != 0.0:
                cols.append(j)
                vals.append(d[i, j])
        rp.append(len(cols))
    return (np.array(rp, dtype=np.int32), np.array(cols, dtype=np.int32),
            np.array(vals, dtype=np.float64))


def laplace1d(m):
    """tridiag(-1, 2, -1) of size m, assembled here independently of synth."""
    d = np.zeros((m, m))
    for i in range(m):
        d[i, i] = 2.0
        if i > 0:
            d[i, i - 1] = -1.0
        if i + 1 < m:
            d[i, i + 1] = -1.0
    return csr_from_dense(d)


# ---------------------------------------------------------------- parity tolerances
# FP64 SpMV: ||y - y_ref|| <= 1e-12 ||y_ref|| and, per row,
# |y_i - y_ref,i| <= 1e-12 (|A||x|)_i.  FP32: the same form at 1e-5 against the
# FP64 oracle applied to the FP32-rounded A and x.  y_ref is the compensated
# oracle, whose own error is negligible at these scales.
TOL = {"f64": 1e-12, "f32": 1e-5}


def assert_spmv_close(y, yref, bound, rel):
    y = np.asarray(y, dtype=np.float64)
    err = np.abs(y - yref)
    bad = err > rel * bound + 1e-300
    assert not bad.any(), (f"{bad.sum()} rows off; worst row {int(np.argmax(err - rel * bound))}: "
                           f"err {err.max():.3e} bound {bound[np.argmax(err - rel * bound)]:.3e}")
    ny = np.linalg.norm(yref)
    if ny > 0:
        assert np.linalg.norm(y - yref) <= rel * ny


# ---------------------------------------------------------------- residual slack
def residual_limit(rp, col, val, b, x, tol):
    """Largest oracle-formed relative residual ||b - A x|| / ||b|| that is
    consistent with a solver that reported its own FP64 true residual <= tol.

    The two evaluations of r = b - A x (the library's and the oracle's) sum the
    same terms in different orders.  Each lies within gamma_{L+1} (|b| + |A||x|)
    of the exact residual, componentwise, where L is the longest row and
    gamma_k = k u / (1 - k u), u = 2^-53 (Higham, Accuracy and Stability of
    Numerical Algorithms, 2nd ed., section 3.5).  Their difference is then at
    most 2 gamma_{L+1} || |b| + |A||x| ||_2, which is added to tol after dividing
    by ||b||."""
    import oracle
    rp = np.asarray(rp)
    L = int(np.diff(rp).max()) if rp.shape[0] > 1 else 0
    u = 2.0 ** -53
    g = (L + 1) * u / (1 - (L + 1) * u)
    s = np.abs(np.asarray(b, dtype=np.float64)) + oracle.spmv_absbound(rp, col, val, x)
    return tol + 2 * g * np.linalg.norm(s) / np.linalg.norm(b)

"""Pins for the oracle's mixed-precision CG with reliable updates (FP32
iterations, FP64 residual replacement, the Krylov direction kept) - CPU only.

* On c I with c a power of two each FP32 iteration is exact, so the first
  update leaves the FP32 rounding of b as the residual (|r_i| <= 2^-24 |b_i|)
  and the second one leaves at most 2^-48 |b_i|: two iterations, two updates.
* Keeping the Krylov space means the iteration count of FP64 CG (within 5%)
  on Laplacian problems, and the true FP64 residual, formed here from the
  dense matrix, meets tol.
* Planted mistakes: trusting the FP32 recurrence instead of recomputing the
  residual in FP64, and restarting the Krylov space at each update."""
import numpy as np
import pytest

import oracle
from paper_2103_10116_gb300 import synth
from tests._helpers import residual_limit, to_dense


def test_scaled_identity_two_exact_steps():
    n = 300
    c = 4.0
    rp = np.arange(n + 1, dtype=np.int32)
    col = np.arange(n, dtype=np.int32)
    val = np.full(n, c)
    b = np.random.default_rng(2).standard_normal(n) * 3.7
    x, info = oracle.cg_reliable(rp, col, val, b, tol=1e-10)
    assert info.status == oracle.CONVERGED
    assert info.iterations == 2 and info.restarts == 2
    assert np.all(np.abs(b - c * x) <= 2.0 ** -48 * np.abs(b))
    # after one step and one update: the FP32 rounding of b, and no better
    x1, i1 = oracle.cg_reliable(rp, col, val, b, tol=1e-10, maxit=1)
    assert i1.iterations == 1 and i1.restarts == 1
    r1 = b - c * x1
    assert np.all(np.abs(r1) <= 2.0 ** -24 * np.abs(b))
    assert np.array_equal(x1, b.astype(np.float32).astype(np.float64) / c)


def _problem(name):
    rp, col, val = {"lap2d_48": lambda: synth.laplace2d_5pt(48), "lap3d_16": lambda: synth.laplace3d_7pt(16),
                    "shifted": lambda: synth.ragged_laplace2d(3000, 0.05)}[name]()
    n = rp.shape[0] - 1
    xs = np.random.default_rng(3).uniform(-1, 1, n)
    return rp, col, val, xs, to_dense(rp, col, val) @ xs


@pytest.mark.parametrize("name", ["lap2d_48", "lap3d_16", "shifted"])
def test_keeps_cg_iteration_count_and_reaches_tol(name):
    rp, col, val, xs, b = _problem(name)
    d = to_dense(rp, col, val)
    _, ci = oracle.cg(rp, col, val, b, tol=1e-10)
    x, ri = oracle.cg_reliable(rp, col, val, b, tol=1e-10)
    assert ri.status == oracle.CONVERGED
    assert np.linalg.norm(b - d @ x) / np.linalg.norm(b) <= residual_limit(rp, col, val, b, x, 1e-10)
    assert abs(ri.iterations - ci.iterations) <= max(3, ci.iterations // 20), (ri, ci)
    assert ri.restarts >= 3  # the residual was replaced along the way (delta = 0.1 per update)


@pytest.mark.parametrize("mutant", [15, 16])
def test_planted_reliable_update_mistakes_are_caught(mutant):
    caught = False
    for name in ("lap2d_48", "lap3d_16"):
        rp, col, val, xs, b = _problem(name)
        d = to_dense(rp, col, val)
        _, ci = oracle.cg(rp, col, val, b, tol=1e-10)
        x, ri = oracle.cg_reliable(rp, col, val, b, tol=1e-10, maxit=5000, mutant=mutant)
        rel = np.linalg.norm(b - d @ x) / np.linalg.norm(b)
        caught |= rel > residual_limit(rp, col, val, b, x, 1e-10) or abs(ri.iterations - ci.iterations) > max(3, ci.iterations // 20)
    assert caught

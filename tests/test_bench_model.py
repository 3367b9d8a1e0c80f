"""The benchmark's byte model against the numbers the paper prints
(Section 5 footprints, Section 6.3 intensities and bounds), CPU only."""
import json
import os

import pytest

import bench

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_intensity.json")


def test_bytes_per_nonzero_match_section5():
    g = json.load(open(GOLD))
    n = 1_000_000
    for key, per in g["bytes_per_nnz"].items():
        fmt, dt = key.split("_")
        V = 8 if dt == "f64" else 4
        # drop x, y and row pointers as the paper's simplification does
        b = bench.algorithmic_bytes(fmt, V, 0, 0, n)
        if fmt == "csr":
            b -= 4  # the (n+1)-th row pointer of an empty row set
        assert b == per * n


def test_intensity_and_bounds_match_section63():
    g = json.load(open(GOLD))
    for key, val in g["intensity"].items():
        fmt, dt = key.split("_")
        assert bench.paper_intensity(fmt, 8 if dt == "f64" else 4) == pytest.approx(val)
    for e in g["bound_gflops"]:
        bound = bench.paper_intensity(e["format"], 8 if e["dtype"] == "f64" else 4) * e["gbs"]
        assert abs(bound - e["gflops"]) <= e["rounding"]


def test_full_byte_model_counts_vectors_and_pointers():
    n, nnz = 1000, 27000
    assert bench.algorithmic_bytes("csr", 8, n, n, nnz) == 12 * nnz + 4 * (n + 1) + 16 * n
    assert bench.algorithmic_bytes("ell", 8, n, n, nnz, ell_w=27) == 12 * 27 * n + 16 * n
    assert bench.algorithmic_bytes("coo", 4, n, n, nnz) == 12 * nnz + 8 * n
    assert bench.algorithmic_bytes("hyb", 8, n, n, nnz, ell_w=6, coo_nnz=500) == 12 * 6 * n + 16 * 500 + 16 * n

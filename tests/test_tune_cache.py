"""The autotuner's JSON cache (host logic; the tuner and the matrix handle are
faked, so no GPU is needed)."""
import json

import pytest

from paper_2103_10116_gb300 import spx


def _fake(monkeypatch, infos, calls):
    monkeypatch.setattr(spx, "spx_matrix_get_info", lambda A: infos[A])
    monkeypatch.setattr(spx, "spx_matrix_set_kernel", lambda A, k, p=0: calls.append(("set", A, k, p)))


def _info(n, nnz, mx, mean, fmt=0, dt=0, ellw=0):
    return {"format": fmt, "dtype": dt, "nrows": n, "nnz": nnz, "max_row_len": mx, "mean_row_len": mean,
            "ell_width": ellw}


def test_tune_then_hit(tmp_path, monkeypatch):
    calls = []
    infos = {1: _info(1_000_000, 26_463_592, 27, 26.46), 2: _info(1_000_000, 26_463_592, 27, 26.46)}
    _fake(monkeypatch, infos, calls)
    tuned = []

    def tuner(ctx, A, reps):
        tuned.append(A)
        return (6, 2, 83.5)
    path = tmp_path / "tune.json"
    assert spx.tune_cached(0, 1, str(path), device_name="GPU-A", tuner=tuner) == (6, 2, 83.5)
    data = json.loads(path.read_text())
    assert len(data) == 1 and list(data.values())[0] == {"kernel": 6, "param": 2, "us": 83.5}
    # same shape statistics, same GPU: from the cache, no timing, the kernel is set
    assert spx.tune_cached(0, 2, str(path), device_name="GPU-A", tuner=tuner) == (6, 2, None)
    assert tuned == [1] and calls == [("set", 2, 6, 2)]


def test_key_separates_gpus_formats_and_shapes(tmp_path, monkeypatch):
    calls = []
    base = _info(2_000_000, 32_000_000, 20000, 16.0)
    infos = {1: base, 2: dict(base, format=2), 3: dict(base, nnz=64_000_000), 4: dict(base, max_row_len=100),
             5: dict(base, nnz=32_400_000)}
    _fake(monkeypatch, infos, calls)
    keys = {spx.tune_key(a, "GPU-A") for a in infos} | {spx.tune_key(1, "GPU-B")}
    # 5 differs from 1 only below two significant digits of nnz: same key
    assert spx.tune_key(5, "GPU-A") == spx.tune_key(1, "GPU-A")
    assert len(keys) == 5


def test_unreadable_cache_is_retuned(tmp_path, monkeypatch):
    calls = []
    _fake(monkeypatch, {1: _info(4096, 20224, 5, 4.9)}, calls)
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    out = spx.tune_cached(0, 1, str(path), device_name="GPU-A", tuner=lambda c, A, r: (2, 8, 3.1))
    assert out == (2, 8, 3.1) and json.loads(path.read_text())

"""The SVD work-split autotuner: table handling on the host, tuning and tuned SVDs on the GPU."""
import numpy as np
import pytest

from paper_2211_07983_gb300 import autotune


def test_cap_shapes_and_probe_matrix():
    # n = 12, D = 64: caps 1 2 4 8 16 32 64 32 ...; shapes (2 cap[b], 2 cap[b+2]) with sides <= 128
    shapes = autotune.cap_shapes(12, 64)
    assert (64, 64) in shapes and (128, 32) in shapes and (32, 128) in shapes and (2, 8) in shapes
    assert all(max(s) <= 128 for s in shapes)
    assert autotune.cap_shapes(40, 256) and all(max(s) <= 128 for s in autotune.cap_shapes(40, 256))
    A = autotune.probe_matrix(64, 32, seed=3)
    s = np.linalg.svd(A, compute_uv=False)
    assert A.shape == (64, 32) and np.allclose(s[:16], np.geomspace(1.0, 1e-6, 16), rtol=1e-9)
    assert s[16] < 1e-14
    assert np.array_equal(A, autotune.probe_matrix(64, 32, seed=3))


def test_table_save_load_and_validation(tmp_path):
    from paper_2211_07983_gb300 import _lib
    rows = [{"m_cap": 64, "n_cap": 64, "jg32": 16, "jg64": 8, "rule_ms": 1.0, "best_ms": 0.9}]
    path = str(tmp_path / "t.json")
    autotune.save(rows, path)
    assert autotune.load(path) == rows
    assert autotune.load(str(tmp_path / "none.json")) is None
    lib = _lib.load()
    bad = np.array([[64, 64, 12, 8]], dtype=np.int32)      # 12 lanes is not a choice
    assert lib.mps_set_svd_tiles(1, bad.ctypes.data) == 1   # MPS_EINVAL
    bad = np.array([[1, 64, 8, 8]], dtype=np.int32)
    assert lib.mps_set_svd_tiles(1, bad.ctypes.data) == 1
    assert lib.mps_set_svd_tiles(-1, None) == 1
    assert lib.mps_set_svd_tiles(0, None) == 0              # clears the table


def test_tune_and_ensure_logic(tmp_path, monkeypatch):
    """tune keeps a split only when it beats the rule by the margin; ensure tunes only the shapes
    the saved table lacks, saves the union and installs it (timings and installation faked)."""
    calls, installed = [], []

    def fake_time(A, g32, g64, reps):
        calls.append((A.shape, g32, g64))
        if A.shape == (64, 64):
            return {(0, 0): 1.0, (16, 8): 0.90}.get((g32, g64), 1.2)   # 10% better: kept
        return {(0, 0): 1.0, (32, 32): 0.99}.get((g32, g64), 1.1)      # 1% better: rule kept
    monkeypatch.setattr(autotune, "time_svd", fake_time)
    monkeypatch.setattr(autotune, "apply", lambda rows: installed.append(list(rows)))
    rows = autotune.tune([(64, 64), (8, 32)], reps=1)
    assert [(r["jg32"], r["jg64"]) for r in rows] == [(16, 8), (0, 0)]
    assert len(calls) == 2 * 10
    path = str(tmp_path / "tiles.json")
    calls.clear()
    out = autotune.ensure([(64, 64)], path=path)
    assert len(calls) == 10 and autotune.load(path) == out and installed[-1] == out
    calls.clear()
    out2 = autotune.ensure([(64, 64), (8, 32)], path=path)   # only the new shape is timed
    assert {c[0] for c in calls} == {(8, 32)} and len(out2) == 2
    calls.clear()
    autotune.ensure([(8, 32)], path=path)                    # everything cached: nothing timed
    assert calls == [] and installed[-1] == out2


@pytest.mark.gpu
def test_tuned_svd_variants_match_lapack():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import build
    build.build()
    import paper_2211_07983_gb300 as M
    try:
        for (m, n) in ((64, 64), (128, 32), (16, 64), (8, 8)):
            A = autotune.probe_matrix(m, n, seed=1)
            s_ref = np.linalg.svd(A, compute_uv=False)
            assert autotune.time_svd(A, 0, 0, 2) > 0.0
            for g32 in autotune.CHOICES:
                for g64 in autotune.CHOICES:
                    autotune.apply([{"m_cap": m, "n_cap": n, "jg32": g32, "jg64": g64}])
                    s, V, W, k = M.svd(A, D=min(m, n), eps=0.0)
                    r = len(s_ref) // 2
                    assert np.allclose(s[:r], s_ref[:r], rtol=1e-11, atol=0), (m, n, g32, g64)
        rows = autotune.tune([(64, 64), (16, 64)], reps=2)
        assert [(r["m_cap"], r["n_cap"]) for r in rows] == [(64, 64), (16, 64)]
        assert all(r["best_ms"] <= r["rule_ms"] for r in rows)
        assert all(r["jg32"] in (0, 8, 16, 32) and r["jg64"] in (0, 8, 16, 32) for r in rows)
    finally:
        autotune.apply([])

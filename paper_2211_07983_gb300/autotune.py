"""Autotuner of the gate SVD's work split, with a table persisted as JSON.

The one-CTA Jacobi SVD (one CTA per matrix, step S3) hands each column pair of a round to 8, 16 or
32 lanes, chosen separately for its FP32 preconditioning sweeps and its FP64 sweeps. The library
has a rule for the choice (from the number of pairs). `tune` times every combination on seeded
probe matrices of each bond-cap shape a workload meets, through mps_svd_tune. It keeps a
combination only when it beats the rule by more than `margin`. `apply` installs the result
(mps_set_svd_tiles), and `ensure` loads a saved table or tunes and saves one.

The probe matrix of an m x n shape has rank min(m, n)/2 and singular values falling geometrically
from 1 to 1e-6, like the two-site matrices of a UCC circuit (half of their columns numerically
zero, a wide spread of kept values).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import _lib
from ._lib import check

CHOICES = (8, 16, 32)
MAX_SIDE = 128   # larger matrices take the cooperative SVD, which has no such choice


def probe_matrix(m: int, n: int, seed: int = 0) -> np.ndarray:
    """Seeded m x n complex probe matrix (row-major), rank min(m, n)/2."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919 * m + n))
    r = max(1, min(m, n) // 2)
    U = np.linalg.qr(rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r)))[0]
    V = np.linalg.qr(rng.standard_normal((n, r)) + 1j * rng.standard_normal((n, r)))[0]
    s = np.geomspace(1.0, 1e-6, r)
    return np.ascontiguousarray((U * s) @ V.conj().T)


def cap_shapes(n: int, D: int) -> list[tuple[int, int]]:
    """The (m_cap, n_cap) two-site matrix shapes of an n-qubit state with bond cap D that run on
    the one-CTA SVD (both sides at most 128)."""
    cap = [min(2 ** min(b, n - b), D) for b in range(n + 1)]
    shapes = {(2 * cap[b], 2 * cap[b + 2]) for b in range(n - 1)}
    return sorted(sh for sh in shapes if max(sh) <= MAX_SIDE)


def time_svd(A: np.ndarray, jg32: int, jg64: int, reps: int) -> float:
    """mps_svd_tune: mean ms of one SVD of A with the given lanes per pair (0 = the rule)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    ms = np.zeros(1)
    check(_lib.load().mps_svd_tune(A.shape[0], A.shape[1], A.ctypes.data, jg32, jg64, reps, ms.ctypes.data))
    return float(ms[0])


def tune(shapes, reps: int = 10, margin: float = 0.03, seed: int = 0) -> list[dict]:
    """Time the rule and the 9 combinations per shape; return one row per shape."""
    rows = []
    for m, n in shapes:
        A = probe_matrix(m, n, seed)
        rule = time_svd(A, 0, 0, reps)
        best, best_ms = (0, 0), rule
        for g32 in CHOICES:
            for g64 in CHOICES:
                t = time_svd(A, g32, g64, reps)
                if t < best_ms:
                    best, best_ms = (g32, g64), t
        if best_ms > (1.0 - margin) * rule:   # not clearly better: keep the rule
            best, best_ms = (0, 0), rule
        rows.append({"m_cap": m, "n_cap": n, "jg32": best[0], "jg64": best[1], "rule_ms": rule, "best_ms": best_ms})
    return rows


def apply(rows) -> None:
    """Install a tuned table (rows of tune()) for every later gate SVD; [] clears it."""
    ent = np.array([[r["m_cap"], r["n_cap"], r["jg32"], r["jg64"]] for r in rows], dtype=np.int32).reshape(-1, 4)
    ent = np.ascontiguousarray(ent)
    check(_lib.load().mps_set_svd_tiles(len(ent), ent.ctypes.data if len(ent) else None))


def default_path() -> str:
    """$XDG_CACHE_HOME (or ~/.cache)/paper_2211_07983_gb300/svd_tiles_<GPU name>.json."""
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_").replace("/", "_")
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_2211_07983_gb300", f"svd_tiles_{name}.json")


def save(rows, path: str) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump({"version": 1, "rows": rows}, f, indent=1)


def load(path: str) -> list[dict] | None:
    if not os.path.exists(path):
        return None
    with open(path) as f:
        data = json.load(f)
    if data.get("version") != 1:
        return None
    return data["rows"]


def ensure(shapes, path: str | None = None, reps: int = 10) -> list[dict]:
    """Load the saved table if it covers `shapes`, else tune them (plus what it had) and save;
    then install it."""
    path = path or default_path()
    rows = load(path) or []
    have = {(r["m_cap"], r["n_cap"]) for r in rows}
    missing = [sh for sh in shapes if tuple(sh) not in have]
    if missing:
        rows = rows + tune(missing, reps=reps)
        save(rows, path)
    apply(rows)
    return rows

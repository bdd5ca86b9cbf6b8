"""Helpers shared by the GPU parity tests (error norms, device setup)."""

import numpy as np
import pytest

# Tolerances of the float32 force path against the float64 oracle.
RMS_TOL = 1e-5    # ||a - a_ref||_2 / ||a_ref||_2
MAX_TOL = 1e-4    # max_i |a_i - a_ref,i| / max(|a_ref,i|, 1e-3 rms|a_ref|)


def need_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def err_norms(a, ref):
    """(rms relative error, max relative error with a floor) over particles."""
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.linalg.norm(a - ref)
    den = np.linalg.norm(ref)
    rms = num / den if den > 0 else num
    mag = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(mag * mag)) if mag.size else 0.0
    per = np.linalg.norm(a - ref, axis=1) / np.maximum(mag, max(floor, 1e-30))
    return float(rms), float(per.max() if per.size else 0.0)


def sample_targets(cell_start, perm, N, S, crowded_cells=64, per_cell=8, seed=0):
    """S seeded random targets plus a few particles of the most crowded cells.

    cell_start and perm come from the oracle's binning (never the GPU's)."""
    rng = np.random.default_rng(seed)
    t = rng.choice(N, size=min(S, N), replace=False)
    cs = np.asarray(cell_start, np.int64)
    cnt = np.diff(cs)
    top = np.argsort(-cnt, kind="stable")[:crowded_cells]
    extra = []
    for c in top:
        k = int(cnt[c])
        if k == 0:
            continue
        extra.append(np.asarray(perm)[cs[c] + rng.choice(k, size=min(per_cell, k), replace=False)])
    if extra:
        t = np.concatenate([t, np.concatenate(extra)])
    return np.unique(t)

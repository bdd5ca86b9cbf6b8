"""The autotuner's search, run end to end on a small workload.

tune_workload times the split threshold with the symmetric force kernel, then
the launch shapes of both force kernels and both adjoints, and writes its
choice to a JSON cache.  Here it writes into a temporary cache; the test reads
the entry back through the same functions the benchmark uses and runs both
force kernels and the gather adjoint with the chosen shapes against the
float64 oracle.
"""

import json

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, make_config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_cuda()


@pytest.fixture(scope="module")
def hs():
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


def test_tune_workload_writes_cache_and_chosen_shapes_are_correct(torch, hs, tmp_path):
    from paper_1211_4864_gb300 import autotune

    path = str(tmp_path / "cache.json")
    res = autotune.tune_workload("uniform4096", splits=(32, 64, 128), quick=True, path=path)
    cache = json.load(open(path))
    key = autotune._key("uniform4096")
    assert list(cache) == [key]
    ent = cache[key]
    assert set(ent) == {"force", "symmetric", "adjoint", "adjoint_symmetric"}
    assert res["best"] == ent
    # the split threshold is the fastest of the ones timed, each with its full table
    T = ent["force"]["split_T"]
    assert T in (32, 64, 128)
    assert set(res["table"]) == {32, 64, 128}
    best_ms = {t: min(ms for _, ms in rows if ms is not None) for t, rows in res["table"].items()}
    assert best_ms[T] == min(best_ms.values())
    # every chosen shape is one of the candidates the tuner offers
    offered = [c.__dict__ for c in autotune.candidates(quick=True)]
    for mode in ("force", "symmetric", "adjoint", "adjoint_symmetric"):
        assert ent[mode]["launch"] in offered, mode
    assert autotune.cached_split("uniform4096", default=-1, path=path) == T

    w = make_config("uniform4096")
    c = default_coeffs(w.rcut, w.eps)
    prm = hs.SRParams(w.eps, w.rcut, c)
    sr = hs.ShortRange(w.L, w.vol_off, w.rcut, cell_min=w.cell_min, split_T=T)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    a = sr.force(prm, launch=autotune.cached("uniform4096", "force", path=path))
    a_sym = sr.force_symmetric(prm, launch=autotune.cached("uniform4096", "symmetric", path=path))
    lam = np.random.default_rng(5).normal(size=(3, w.N)).astype(np.float32)
    g, _ = sr.adjoint(prm, torch.tensor(lam, device="cuda"), want_gm=False,
                      launch=autotune.cached("uniform4096", "adjoint", path=path))
    torch.cuda.synchronize()
    sr.check_status()
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), w.eps, w.rcut, c.astype(np.float64))
    for name, out in (("gather", a), ("symmetric", a_sym)):
        rms, mx = err_norms(out.cpu().numpy().T, ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (name, rms, mx)
    ref_g, _ = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), w.eps, w.rcut, c.astype(np.float64),
                                       lam.T.astype(np.float64))
    rms, _ = err_norms(g.cpu().numpy().T, ref_g)
    assert rms < RMS_TOL, rms

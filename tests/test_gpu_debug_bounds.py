"""The debug build's bounds checks (libhacc_sr_debug.so, HACC_DEBUG_BOUNDS).

The debug build checks every index a task of the pair kernels leads to -- the
task count, its order entry and record, its volume and cell, its slot range
and each entry of its cell's neighbour list -- before using it, and skips a
task that fails with HACC_STATUS_BOUNDS in the device status word.  On clean
input it must give the product build's results (the gather kernels bit for
bit); on lists or tasks corrupted on purpose it must report the corruption
instead of reading out of range, and the next call on rebuilt lists must be
clean again.  The corruptions stay inside the arrays: only the values that
the kernels would use as indices are wrong, and the checks run before any such
value is used.
"""

import numpy as np
import pytest

import oracle
from gpu_util import RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, uniform_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0
BOUNDS = 16  # HACC_STATUS_BOUNDS


@pytest.fixture(scope="module")
def torch():
    return need_cuda()


@pytest.fixture(scope="module")
def hs():
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


@pytest.fixture
def debug_lib(hs):
    from paper_1211_4864_gb300 import _lib
    prev = _lib.use_library(debug=True)
    try:
        yield _lib
    finally:
        _lib._lib = prev


def _case(torch, hs, seed=21):
    w = uniform_box(4096, 16.0, seed=seed)
    c = default_coeffs(RC, EPS)
    prm = hs.SRParams(EPS, RC, c)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=48)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    lam = torch.tensor(np.random.default_rng(seed).normal(size=(3, w.N)).astype(np.float32), device="cuda")
    return w, c, prm, sr, pos, m, lam


def _all_calls(sr, prm, lam):
    a = sr.force(prm)
    s = sr.force_symmetric(prm)
    g, _ = sr.adjoint(prm, lam, want_gm=False)
    gs, _ = sr.adjoint_symmetric(prm, lam, want_gm=False)
    return a, s, g, gs


def test_debug_build_matches_product_build_on_clean_input(torch, hs):
    from paper_1211_4864_gb300 import _lib
    w, c, prm, sr, pos, m, lam = _case(torch, hs)
    sr.prepare(pos, m)
    ref = [t.clone() for t in _all_calls(sr, prm, lam)]
    pairs = sr.pair_count()
    within = sr.pairs_within_cutoff(prm)
    torch.cuda.synchronize()
    sr.check_status()
    prev = _lib.use_library(debug=True)
    try:
        assert _lib.load().hacc_version().decode().endswith("debug-bounds")
        sr.prepare(pos, m)
        got = _all_calls(sr, prm, lam)
        within_dbg = sr.pairs_within_cutoff(prm)
        torch.cuda.synchronize()
        assert hs.hacc_get_status(sr.status) == 0
        assert sr.pair_count() == pairs and within_dbg == within
        assert torch.equal(got[0], ref[0]) and torch.equal(got[2], ref[2])  # gather kernels: bit for bit
        for g, r in zip(got, ref):
            rms, _ = err_norms(g.cpu().numpy().T, r.cpu().numpy().T)
            assert rms < 1e-6
    finally:
        _lib._lib = prev
    A = oracle.sr_force(w.x, w.y, w.z, w.m, 16.0, EPS, RC, c.astype(np.float64))
    rms, _ = err_norms(ref[0].cpu().numpy().T, A)
    assert rms < RMS_TOL


def test_debug_build_binning_is_the_product_binning(torch, hs):
    """The debug build also checks every slot the binning's counting passes
    store to; on clean input it reports nothing and bins bit for bit as the
    product build (clustered particles over several tiles, two passes)."""
    from paper_1211_4864_gb300 import _lib
    from synth.workloads import clustered_box
    w = clustered_box(32, 20, seed=9)
    sr = hs.ShortRange(w.L, w.vol_off, RC)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    outs = []
    for debug in (False, True):
        prev = _lib.use_library(debug=debug)
        try:
            sr.status.zero_()
            sr.bin(pos[0], pos[1], pos[2], m)
            torch.cuda.synchronize()
            assert hs.hacc_get_status(sr.status) == 0
            outs.append([t.cpu().numpy().copy() for t in (sr.cell_of, sr.cell_start, sr.perm, sr.sorted4)])
        finally:
            _lib._lib = prev
    for g, r in zip(outs[1], outs[0]):
        assert np.array_equal(g.view(np.int32), r.view(np.int32))


@pytest.mark.parametrize("what", ["list entry", "list image code", "task slots", "task count"])
def test_corrupted_lists_and_tasks_are_reported_not_read(torch, hs, debug_lib, what):
    w, c, prm, sr, pos, m, lam = _case(torch, hs, seed=22)
    sr.prepare(pos, m)
    torch.cuda.synchronize()
    sr.check_status()
    if what == "list entry":
        sr.nbr_cell[5] = sr.n_cells + 1000
    elif what == "list image code":
        sr.nbr_shift[40] = 77
    elif what == "task slots":
        k = int(sr.task_order[3].item())
        sr.tasks[k, 2] = w.N + 50
    else:
        sr.n_tasks[0] = sr.task_cap + 5
    for name, call in (("force", lambda: sr.force(prm)), ("force_symmetric", lambda: sr.force_symmetric(prm)),
                       ("adjoint", lambda: sr.adjoint(prm, lam, want_gm=True)),
                       ("adjoint_symmetric", lambda: sr.adjoint_symmetric(prm, lam, want_gm=False)),
                       ("potential", lambda: sr.potential(prm))):
        sr.status.zero_()
        call()
        torch.cuda.synchronize()
        st = hs.hacc_get_status(sr.status)
        assert st & BOUNDS, (what, name, st)
    # rebuilt lists: clean again and correct
    sr.prepare(pos, m)
    sr.status.zero_()
    a = sr.force(prm)
    torch.cuda.synchronize()
    assert hs.hacc_get_status(sr.status) == 0
    A = oracle.sr_force(w.x, w.y, w.z, w.m, 16.0, EPS, RC, c.astype(np.float64))
    rms, _ = err_norms(a.cpu().numpy().T, A)
    assert rms < RMS_TOL

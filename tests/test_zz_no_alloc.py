"""hacc_bin_noalloc: binning for callers that cannot allocate device memory.

Such a caller (a plugin inside an application that owns all device memory, or
code running where cudaMalloc is not allowed) cannot hand hacc_bin a
workspace; hacc_bin_noalloc uses the library's fixed device scratch array
instead.  Its output must be identical, bit for bit, to hacc_bin's on the same
input, call after call, whatever the previous call left in that array.  This
file is collected last so that a run stopping at the first failure has run
every other test first.
"""

import ctypes

import numpy as np
import pytest

from synth import uniform_box
from synth.workloads import clustered_box


def _run(hs, torch, w, noalloc):
    sr = hs.ShortRange(w.L, w.vol_off, w.rcut)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    if noalloc:
        hs.hacc_bin_noalloc(sr.mesh, pos[0], pos[1], pos[2], m, sr.binned, sr.status)
    else:
        hs.hacc_bin(sr.mesh, pos[0], pos[1], pos[2], m, sr.binned, sr.ws, sr.status)
    torch.cuda.synchronize()
    assert int(sr.status.item()) == 0
    return [t.cpu().numpy().copy() for t in (sr.cell_of, sr.cell_start, sr.perm, sr.sorted4, sr.mass_varies)]


@pytest.mark.gpu
def test_noalloc_binning_matches_workspace_binning_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4864_gb300 as hs
    hs.load()
    # different problems back to back through the shared scratch array (the last one with
    # varied masses: the equal-mass flag set, as by hacc_bin)
    varied = uniform_box(3000, 14.0, seed=4)
    varied.m[:] = np.random.default_rng(4).uniform(0.5, 2.0, varied.N).astype(np.float32)
    for w in (clustered_box(24, 6, seed=12), uniform_box(4096, 16.0, seed=1), varied):
        got = _run(hs, torch, w, noalloc=True)
        ref = _run(hs, torch, w, noalloc=False)
        for g, r in zip(got, ref):
            assert g.shape == r.shape
            assert np.array_equal(g.view(np.int32), r.view(np.int32))


@pytest.mark.gpu
def test_noalloc_binning_at_its_documented_limit():
    """262,144 clustered particles (the documented capacity of the fixed
    scratch array; two counting passes over 64 tiles): bit for bit what
    hacc_bin gives with a workspace."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4864_gb300 as hs
    hs.load()
    w = clustered_box(64, 100, seed=4)
    assert w.N == 262144
    got = _run(hs, torch, w, noalloc=True)
    ref = _run(hs, torch, w, noalloc=False)
    for g, r in zip(got, ref):
        assert np.array_equal(g.view(np.int32), r.view(np.int32))


def test_noalloc_rejects_problems_beyond_its_scratch():
    """Too large for the fixed array: a clear capacity error, checked on the
    host before any device work."""
    from paper_1211_4864_gb300 import _lib
    from paper_1211_4864_gb300._lib import hacc_binned, hacc_mesh
    lib = _lib.load()
    mesh = hacc_mesh()
    mesh.V = 1
    mesh.N = 1 << 22
    mesh.n_cells = 1 << 18
    out = hacc_binned()
    rc = lib.hacc_bin_noalloc(ctypes.byref(mesh), None, None, None, None, ctypes.byref(out), None, None)
    assert rc == _lib.HACC_ERR_CAPACITY


def test_noalloc_capacity_matches_the_documented_limit():
    """The scratch array holds hacc_bin's workspace for 262,144 particles in
    any number of cells (the workspace does not grow with the cells) but not
    for 400,000; a problem that needs more is refused with a capacity error on
    the host, before any device work."""
    from paper_1211_4864_gb300 import _lib
    from paper_1211_4864_gb300._lib import hacc_binned, hacc_mesh
    lib = _lib.load()
    limit = 9 << 20
    mesh = hacc_mesh()
    mesh.V = 1
    mesh.N = 262144
    for nc in (1, 500000, (1 << 31) - 1):
        mesh.n_cells = nc
        assert lib.hacc_bin_workspace_size(ctypes.byref(mesh)) <= limit
    mesh.N = 400000
    assert lib.hacc_bin_workspace_size(ctypes.byref(mesh)) > limit
    out = hacc_binned()
    rc = lib.hacc_bin_noalloc(ctypes.byref(mesh), None, None, None, None, ctypes.byref(out), None, None)
    assert rc == _lib.HACC_ERR_CAPACITY

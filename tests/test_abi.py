"""The C-ABI library builds, loads and exports every symbol the header
declares; host-only calls (planning, workspace queries) agree with the
oracle's mesh definitions.  No GPU needed."""

import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1211_4864_gb300 import _build, _lib
from paper_1211_4864_gb300._lib import hacc_mesh, hacc_volume

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "hacc_sr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hacc_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"
    assert set(_lib.SIGNATURES) == set(names)


def test_debug_build_exports_the_same_symbols():
    """libhacc_sr_debug.so (bounds-checked pair kernels) is built beside the
    product library by __graft_entry__.build() and exports the same ABI."""
    if not os.path.exists(_build.LIB_DEBUG):
        pytest.skip("debug library not built")
    dbg = ctypes.CDLL(_build.LIB_DEBUG)
    for n in _header_functions():
        assert hasattr(dbg, n), n
    dbg.hacc_version.restype = ctypes.c_char_p
    assert dbg.hacc_version().decode().endswith("debug-bounds")
    assert os.path.dirname(_build.LIB_DEBUG) == os.path.dirname(_build.LIB)


def test_library_is_in_tree_and_for_sm103a(lib):
    assert os.path.dirname(_build.LIB) == os.path.join(ROOT, "paper_1211_4864_gb300")
    assert "sm_103a" in lib.hacc_version().decode()
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def _plan(L, vol_off, cell_min, rcut):
    V = len(L)
    Ls = np.asarray(L, np.float32)
    vo = np.asarray(vol_off, np.int64)
    table = (hacc_volume * V)()
    mesh = hacc_mesh()
    rc = _lib.load().hacc_mesh_plan(V, Ls.ctypes.data, vo.ctypes.data, float(cell_min), float(rcut), table,
                                    ctypes.byref(mesh))
    return rc, table, mesh


@pytest.mark.parametrize("L,cell_min,rcut", [(16.0, 3.0, 3.0), (128.0, 3.0, 3.0), (256.0, 3.0, 3.0),
                                             (13.0, 1.4, 3.0), (9.0, 3.0, 3.0), (17.3, 2.5, 2.0)])
def test_plan_matches_oracle_mesh(L, cell_min, rcut):
    rc, table, mesh = _plan([L], [0, 1000], cell_min, rcut)
    assert rc == 0
    n, w, iw = oracle.mesh(L, cell_min)
    t = table[0]
    assert t.n == n
    assert np.float32(t.w).view(np.int32) == np.float32(w).view(np.int32)
    assert np.float32(t.inv_w).view(np.int32) == np.float32(iw).view(np.int32)
    assert t.R == oracle.reach(w, rcut)
    off, _, _ = oracle.lists_volume(n, w, rcut)
    assert t.S * n ** 3 == off[-1]
    assert mesh.n_cells == n ** 3 and mesh.n_entries == off[-1] and mesh.N == 1000


def test_plan_batched_bases():
    L = [16.0, 20.5, 9.0]
    vo = [0, 100, 100, 350]
    rc, table, mesh = _plan(L, vo, 3.0, 3.0)
    assert rc == 0
    cb = eb = 0
    for v in range(3):
        t = table[v]
        assert (t.p_begin, t.p_end) == (vo[v], vo[v + 1])
        assert t.cell_base == cb and t.entry_base == eb
        cb += t.n ** 3
        eb += t.n ** 3 * t.S
    assert mesh.n_cells == cb and mesh.n_entries == eb and mesh.V == 3


@pytest.mark.parametrize("L,vo,cell_min,rcut", [
    ([8.0], [0, 10], 3.0, 3.0),      # n = 2 < 3
    ([5.0], [0, 10], 1.0, 3.0),      # L < 2 r_c
    ([16.0], [1, 10], 3.0, 3.0),     # vol_off[0] != 0
    ([16.0], [0, -1], 3.0, 3.0),     # decreasing
    ([16.0], [0, 10], 0.0, 3.0),     # cell_min = 0
    ([16.0], [0, 10], 3.0, -1.0),    # rcut < 0
    ([float("nan")], [0, 10], 3.0, 3.0),
    ([13.0], [0, 10], 1.0, 3.0),     # R = 3 needs n >= 7: n = 13 fine -> but L/2 = 6.5 ok; see next
])
def test_plan_rejects_invalid(L, vo, cell_min, rcut):
    rc, _, _ = _plan(L, vo, cell_min, rcut)
    if L == [13.0]:
        assert rc == 0
    else:
        assert rc == _lib.HACC_ERR_INVALID


def test_workspace_queries_positive(lib):
    rc, table, mesh = _plan([64.0], [0, 262144], 3.0, 3.0)
    assert rc == 0
    for fn in ("hacc_bin_workspace_size", "hacc_lists_workspace_size", "hacc_force_workspace_size"):
        assert getattr(lib, fn)(ctypes.byref(mesh)) > 0
    assert lib.hacc_task_capacity(ctypes.byref(mesh), 32) >= 262144 // 32
    assert lib.hacc_moments_workspace_size(10) > 0


def test_device_calls_reject_bad_arguments_on_host(lib):
    """Argument checks run before any CUDA call (safe without a GPU)."""
    rc, table, mesh = _plan([16.0], [0, 10], 3.0, 3.0)
    assert lib.hacc_bin(None, None, None, None, None, None, None, None, None, None, 0, None,
                        None) == _lib.HACC_ERR_INVALID
    assert lib.hacc_kick(None, -1, None, None, None, None, None, None, 0.0, None, None, None, 0.0,
                         None) == _lib.HACC_ERR_INVALID
    assert lib.hacc_moments(5, None, None, None, None, None, None, None, None, None, None, 0,
                            None) == _lib.HACC_ERR_INVALID
    # 32-bit slots and keys: N and n_cells below 2^31 (checked before any device work; the
    # pointers are never dereferenced)
    for n, nc in (((1 << 31), 27), (1000, (1 << 31))):
        big = _lib.hacc_mesh()
        big.vols = 16
        big.V = 1
        big.N = n
        big.n_cells = nc
        out = _lib.hacc_binned()
        assert lib.hacc_bin(ctypes.byref(big), None, None, None, None, None, None, None, ctypes.byref(out), None,
                            0, ctypes.c_void_p(16), None) == _lib.HACC_ERR_INVALID

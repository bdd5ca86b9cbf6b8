"""CPU float64 oracle of the short-range force path.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never imports it; the product path never imports this.

The arithmetic lives in ``hacc_oracle.c`` (plain C, float64, OpenMP over
target particles); this module compiles it with gcc on first use and wraps it
with numpy.  See the C file for the definitions and the passages they follow.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hacc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libhacc_oracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -ffp-contract=off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _SO)
    return _SO


def configure(L):
    """Declare the argument and result types of a loaded oracle library."""
    L.ora_num_threads.restype = ctypes.c_int
    L.ora_mesh.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    L.ora_bin.argtypes = [_f32p, _f32p, _f32p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          _f32p, ctypes.c_int64, ctypes.c_float, ctypes.c_int32, ctypes.c_float,
                          ctypes.c_float, _i32p, _i32p, _i32p, _f32p]
    L.ora_bin.restype = ctypes.c_int
    L.ora_reach.argtypes = [ctypes.c_float, ctypes.c_float]
    L.ora_reach.restype = ctypes.c_int32
    L.ora_lists.argtypes = [ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.ora_lists.restype = ctypes.c_int64
    L.ora_rcb_build.argtypes = [_f32p, _f32p, _f32p, _f32p, ctypes.c_int64, ctypes.c_float, ctypes.c_int32,
                                ctypes.c_int32, _i32p, _i32p, _i32p, _f32p]
    L.ora_rcb_build.restype = ctypes.c_int64
    L.ora_rcb_lists.argtypes = [ctypes.c_int64, _i32p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.ora_rcb_lists.restype = ctypes.c_int64
    L.ora_tasks.argtypes = [_i32p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]
    L.ora_tasks.restype = ctypes.c_int64
    L.ora_fsr.argtypes = [ctypes.c_double, ctypes.c_double, _f64p]
    L.ora_fsr.restype = ctypes.c_double
    L.ora_dfsr.argtypes = [ctypes.c_double, ctypes.c_double, _f64p]
    L.ora_dfsr.restype = ctypes.c_double
    L.ora_sr_force.argtypes = [_f64p, _f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, _f64p, _i64p,
                               ctypes.c_int64, _f64p, _f64p, _f64p]
    L.ora_pair_potential.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _f64p]
    L.ora_pair_potential.restype = ctypes.c_double
    L.ora_sr_potential.argtypes = [_f64p, _f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, _f64p, _i64p, ctypes.c_int64, _f64p]
    L.ora_pair_count.argtypes = [_f64p, _f64p, _f64p, ctypes.c_int64, ctypes.c_double,
                                 ctypes.c_double, _i64p, ctypes.c_int64]
    L.ora_pair_count.restype = ctypes.c_int64
    L.ora_sr_force_adjoint.argtypes = [_f64p, _f64p, _f64p, _f64p, ctypes.c_int64,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       _f64p, _f64p, _f64p, _f64p, _i64p, ctypes.c_int64,
                                       _f64p, _f64p, _f64p, ctypes.c_void_p]
    L.ora_kick_drift.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                 ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_double]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(ctypes.CDLL(build()))
    return _lib


def num_threads() -> int:
    return int(lib().ora_num_threads())


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------------------
# mesh, binning, lists
# ---------------------------------------------------------------------------

def mesh(L: float, cell_min: float) -> tuple[int, np.float32, np.float32]:
    n = ctypes.c_int32()
    w = ctypes.c_float()
    iw = ctypes.c_float()
    lib().ora_mesh(float(L), float(cell_min), ctypes.byref(n), ctypes.byref(w), ctypes.byref(iw))
    return int(n.value), np.float32(w.value), np.float32(iw.value)


def bin_volume(x, y, z, m, L: float, cell_min: float, disp=None) -> dict:
    """Reference binning of one periodic volume (see ora_bin); disp: optional
    float32 displacements [3, N] (the position is then x + d)."""
    n, w, iw = mesh(L, cell_min)
    N = int(np.asarray(x).shape[0])
    cell_of = np.zeros(N, np.int32)
    cell_start = np.zeros(n ** 3 + 1, np.int32)
    perm = np.zeros(N, np.int32)
    sorted4 = np.zeros((N, 4), np.float32)
    if disp is None:
        dptr = (None, None, None)
    else:
        d = [_c32(disp[k]) for k in range(3)]
        dptr = tuple(a.ctypes.data for a in d)
    rc = lib().ora_bin(_c32(x), _c32(y), _c32(z), dptr[0], dptr[1], dptr[2], _c32(m), N, float(L), n,
                       float(w), float(iw), cell_of, cell_start, perm, sorted4.reshape(-1))
    assert rc == 0
    return dict(n=n, w=w, inv_w=iw, cell_of=cell_of, cell_start=cell_start, perm=perm,
                sorted4=sorted4)


def lists_volume(n: int, w: float, rcut: float):
    """Reference cell-pair lists of one volume: (nbr_off int64[n^3+1], nbr_cell, nbr_shift)."""
    L_ = lib()
    cnt = L_.ora_lists(int(n), float(w), float(rcut), None, None, None)
    if cnt < 0:
        raise ValueError("mesh too coarse for a unique periodic image")
    off = np.zeros(n ** 3 + 1, np.int64)
    cell = np.zeros(cnt, np.int32)
    shift = np.zeros(cnt, np.int8)
    L_.ora_lists(int(n), float(w), float(rcut), off.ctypes.data, cell.ctypes.data, shift.ctypes.data)
    return off, cell, shift


def rcb_volume(x, y, z, m, L: float, leaf_max: int, max_depth: int = 48) -> dict:
    """Reference RCB fat-leaf tree of one volume (see ora_rcb_build):
    perm, leaf_start[n_leaves + 1], leaf_qbox[n_leaves, 6] (integer lo xyz,
    hi xyz on the 2^21 grid), sorted4 (leaf-relative offsets and mass)."""
    N = int(np.asarray(x).shape[0])
    perm = np.zeros(max(N, 1), np.int32)
    leaf_start = np.zeros(N + 2, np.int32)
    qbox = np.zeros((N + 1) * 6, np.int32)
    sorted4 = np.zeros((max(N, 1), 4), np.float32)
    nl = lib().ora_rcb_build(_c32(x), _c32(y), _c32(z), _c32(m), N, float(L), int(leaf_max), int(max_depth), perm,
                             leaf_start, qbox, sorted4.reshape(-1))
    assert nl >= 0
    return dict(n_leaves=int(nl), perm=perm[:N], leaf_start=leaf_start[:nl + 1],
                leaf_qbox=qbox[:6 * nl].reshape(nl, 6), sorted4=sorted4[:N])


def rcb_lists(leaf_qbox: np.ndarray, L: float, rcut: float, targets=None):
    """Reference leaf interaction lists (see ora_rcb_lists) of every leaf, or of
    the leaves `targets`: (nbr_off int64[count + 1], nbr_leaf int32, nbr_shift int8)."""
    q = np.ascontiguousarray(leaf_qbox, dtype=np.int32).reshape(-1)
    nl = q.shape[0] // 6
    L_ = lib()
    if targets is None:
        tp, nt = None, nl
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        tp, nt = tg.ctypes.data, tg.shape[0]
    cnt = L_.ora_rcb_lists(nl, q, float(L), float(rcut), tp, nt, None, None, None)
    off = np.zeros(nt + 1, np.int64)
    leaf = np.zeros(max(cnt, 1), np.int32)
    shift = np.zeros(max(cnt, 1), np.int8)
    L_.ora_rcb_lists(nl, q, float(L), float(rcut), tp, nt, off.ctypes.data, leaf.ctypes.data, shift.ctypes.data)
    return off, leaf[:cnt], shift[:cnt]


def reach(w: float, rcut: float) -> int:
    return int(lib().ora_reach(float(w), float(rcut)))


def tasks(cell_start: np.ndarray, T: int) -> np.ndarray:
    """Reference task list [(cell, begin, end)] (int32 [n_tasks, 3])."""
    cs = np.ascontiguousarray(cell_start, dtype=np.int32)
    nc = cs.shape[0] - 1
    cnt = lib().ora_tasks(cs, nc, int(T), None)
    out = np.zeros((cnt, 3), np.int32)
    lib().ora_tasks(cs, nc, int(T), out.ctypes.data)
    return out


# ---------------------------------------------------------------------------
# force, adjoint, kick
# ---------------------------------------------------------------------------

def fsr(s: float, eps: float, c) -> float:
    return float(lib().ora_fsr(float(s), float(eps), _c64(c)))


def dfsr(s: float, eps: float, c) -> float:
    return float(lib().ora_dfsr(float(s), float(eps), _c64(c)))


def _targets(N, targets):
    if targets is None:
        return np.arange(N, dtype=np.int64)
    return np.ascontiguousarray(targets, dtype=np.int64)


def sr_force(x, y, z, m, L, eps, rcut, c, targets=None) -> np.ndarray:
    """float64 accelerations [S, 3] of the targets (all particles if None)."""
    x, y, z, m = _c64(x), _c64(y), _c64(z), _c64(m)
    N = x.shape[0]
    t = _targets(N, targets)
    S = t.shape[0]
    ax, ay, az = np.zeros(S), np.zeros(S), np.zeros(S)
    lib().ora_sr_force(x, y, z, m, N, float(L), float(eps), float(rcut), _c64(c), t, S, ax, ay, az)
    return np.stack([ax, ay, az], axis=1)


def pair_potential(s: float, eps: float, rcut: float, c) -> float:
    return float(lib().ora_pair_potential(float(s), float(eps), float(rcut), _c64(c)))


def sr_potential(x, y, z, m, L, eps, rcut, c, targets=None) -> np.ndarray:
    """float64 short-range potential phi [S] of the targets (all if None)."""
    x, y, z, m = _c64(x), _c64(y), _c64(z), _c64(m)
    N = x.shape[0]
    t = _targets(N, targets)
    phi = np.zeros(t.shape[0])
    lib().ora_sr_potential(x, y, z, m, N, float(L), float(eps), float(rcut), _c64(c), t, t.shape[0], phi)
    return phi


def pair_count(x, y, z, L, rcut, targets=None) -> int:
    """Ordered pairs (i in targets, j != i) closer than the cutoff."""
    x, y, z = _c64(x), _c64(y), _c64(z)
    t = _targets(x.shape[0], targets)
    return int(lib().ora_pair_count(x, y, z, x.shape[0], float(L), float(rcut), t, t.shape[0]))


def sr_force_adjoint(x, y, z, m, L, eps, rcut, c, lam, targets=None, want_gm=True):
    """float64 (dL/dx [S, 3], dL/dm [S]) for the cotangent lam [N, 3] = dL/da."""
    x, y, z, m = _c64(x), _c64(y), _c64(z), _c64(m)
    lam = np.asarray(lam, dtype=np.float64)
    N = x.shape[0]
    t = _targets(N, targets)
    S = t.shape[0]
    gx, gy, gz = np.zeros(S), np.zeros(S), np.zeros(S)
    gm = np.zeros(S) if want_gm else None
    lib().ora_sr_force_adjoint(x, y, z, m, N, float(L), float(eps), float(rcut), _c64(c),
                               _c64(lam[:, 0]), _c64(lam[:, 1]), _c64(lam[:, 2]), t, S,
                               gx, gy, gz, gm.ctypes.data if want_gm else None)
    return np.stack([gx, gy, gz], axis=1), gm


def kick_drift(v, a, dt_k, x=None, dt_d=0.0):
    """float64 kick v += dt_k a, then optional drift x += dt_d v (new arrays)."""
    v = np.array(v, dtype=np.float64, order="C")
    vx, vy, vz = [np.ascontiguousarray(v[:, k]) for k in range(3)]
    a = np.asarray(a, dtype=np.float64)
    N = v.shape[0]
    if x is not None:
        x = np.array(x, dtype=np.float64, order="C")
        px, py, pz = [np.ascontiguousarray(x[:, k]) for k in range(3)]
        lib().ora_kick_drift(N, vx, vy, vz, _c64(a[:, 0]), _c64(a[:, 1]), _c64(a[:, 2]),
                             float(dt_k), px.ctypes.data, py.ctypes.data, pz.ctypes.data,
                             float(dt_d))
        return np.stack([vx, vy, vz], 1), np.stack([px, py, pz], 1)
    lib().ora_kick_drift(N, vx, vy, vz, _c64(a[:, 0]), _c64(a[:, 1]), _c64(a[:, 2]),
                         float(dt_k), None, None, None, 0.0)
    return np.stack([vx, vy, vz], 1), None

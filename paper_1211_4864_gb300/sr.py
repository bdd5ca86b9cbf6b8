"""PyTorch-facing binding of the short-range force library.

The functions named ``hacc_*`` mirror the C ABI one to one and only marshal
arguments (torch tensors -> device pointers, the current CUDA stream).  The
``ShortRange`` class owns the device buffers of one mesh (PyTorch allocates
them) and sequences the calls; ``sr_force_autograd`` and ``kick_drift_autograd``
wrap the calls as ``torch.autograd.Function``s whose backward passes call the
hand-written adjoint and kick kernels.  No arithmetic of the method runs in
Python or in PyTorch ops.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import (HaccError, check, hacc_binned, hacc_launch, hacc_lists, hacc_mesh, hacc_sr_params,
                   hacc_tree, hacc_volume)


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if t.numel() == 0:
        return None
    if not t.is_cuda:
        raise HaccError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise HaccError("expected a contiguous tensor")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


@dataclass
class SRParams:
    """Force-law parameters: softening eps, cutoff rcut, poly[5] coefficients."""

    eps: float
    rcut: float
    c: np.ndarray

    def c_struct(self) -> hacc_sr_params:
        p = hacc_sr_params()
        p.eps = float(self.eps)
        p.rcut = float(self.rcut)
        cc = np.asarray(self.c, dtype=np.float32)
        if cc.shape != (6,):
            raise HaccError("need exactly six polynomial coefficients")
        for k in range(6):
            p.c[k] = float(cc[k])
        return p


@dataclass
class Launch:
    warps_per_cta: int = 8
    ctas_per_sm: int = 2
    jtile: int = 64
    stages: int = 4
    wait_cycles: int = 0  # bound of each tile wait in SM cycles; 0 = the library default (~1 s)

    def c_struct(self) -> hacc_launch:
        return hacc_launch(self.warps_per_cta, self.ctas_per_sm, self.jtile, self.stages, self.wait_cycles)


# ---------------------------------------------------------------------------
# one-to-one wrappers of the C ABI
# ---------------------------------------------------------------------------

def hacc_version() -> str:
    return _lib.load().hacc_version().decode()


def hacc_get_status(status) -> int:
    """The device status word `status` (a CUDA int32 tensor of one element),
    once the current stream has finished its enqueued work."""
    v = ctypes.c_uint32()
    check(_lib.load().hacc_get_status(_ptr(status), ctypes.byref(v), _stream()), "hacc_get_status")
    return int(v.value)


def hacc_kernel_launches() -> int:
    return int(_lib.load().hacc_kernel_launches())


def hacc_mesh_plan(L, vol_off, cell_min: float, rcut: float):
    """Host planning; returns (ctypes volume table, hacc_mesh)."""
    L = np.ascontiguousarray(np.atleast_1d(L), dtype=np.float32)
    vol_off = np.ascontiguousarray(vol_off, dtype=np.int64)
    V = L.shape[0]
    if vol_off.shape != (V + 1,):
        raise HaccError("vol_off must have V + 1 entries")
    table = (hacc_volume * V)()
    mesh = hacc_mesh()
    check(_lib.load().hacc_mesh_plan(V, L.ctypes.data, vol_off.ctypes.data, float(cell_min), float(rcut),
                                     table, ctypes.byref(mesh)), "hacc_mesh_plan")
    return table, mesh


def hacc_bin(mesh, x, y, z, m, binned, ws, status, dx=None, dy=None, dz=None):
    check(_lib.load().hacc_bin(ctypes.byref(mesh), _ptr(x), _ptr(y), _ptr(z), _ptr(dx), _ptr(dy), _ptr(dz), _ptr(m),
                               ctypes.byref(binned), _ptr(ws), ws.numel(), _ptr(status), _stream()), "hacc_bin")


def hacc_bin_noalloc(mesh, x, y, z, m, binned, status):
    """hacc_bin without a workspace: the library's fixed device scratch array
    stands in for it (for callers that cannot allocate device memory)."""
    check(_lib.load().hacc_bin_noalloc(ctypes.byref(mesh), _ptr(x), _ptr(y), _ptr(z), _ptr(m),
                                       ctypes.byref(binned), _ptr(status), _stream()), "hacc_bin_noalloc")


def hacc_build_lists(mesh, binned, lists, ws, status):
    check(_lib.load().hacc_build_lists(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists), _ptr(ws),
                                       ws.numel(), _ptr(status), _stream()), "hacc_build_lists")


def hacc_rcb_build(mesh, x, y, z, m, tree, binned, ws, status):
    """RCB fat-leaf tree (synchronises the current stream once per tree level)."""
    check(_lib.load().hacc_rcb_build(ctypes.byref(mesh), _ptr(x), _ptr(y), _ptr(z), _ptr(m), ctypes.byref(tree),
                                     ctypes.byref(binned), _ptr(ws), ws.numel(), _ptr(status), _stream()),
          "hacc_rcb_build")


def hacc_rcb_lists(mesh, tree, lists, entry_cap: int, n_entries, ws, status):
    check(_lib.load().hacc_rcb_lists(ctypes.byref(mesh), ctypes.byref(tree), ctypes.byref(lists), int(entry_cap),
                                     _ptr(n_entries), _ptr(ws), ws.numel(), _ptr(status), _stream()),
          "hacc_rcb_lists")


def hacc_drift_offsets(mesh, binned, vx, vy, vz, dt: float, skin: float, status):
    check(_lib.load().hacc_drift_offsets(ctypes.byref(mesh), ctypes.byref(binned), _ptr(vx), _ptr(vy), _ptr(vz),
                                         float(dt), float(skin), _ptr(status), _stream()), "hacc_drift_offsets")


def hacc_sr_force(mesh, binned, lists, params: SRParams, ax, ay, az, ws, status, launch: Launch | None = None):
    p = params.c_struct()
    lc = launch.c_struct() if launch is not None else None
    check(_lib.load().hacc_sr_force(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists), ctypes.byref(p),
                                    _ptr(ax), _ptr(ay), _ptr(az), ctypes.byref(lc) if lc else None, _ptr(ws),
                                    ws.numel(), _ptr(status), _stream()), "hacc_sr_force")


def hacc_sr_force_symmetric(mesh, binned, lists, params: SRParams, ax, ay, az, ws, status,
                            launch: Launch | None = None):
    p = params.c_struct()
    lc = launch.c_struct() if launch is not None else None
    check(_lib.load().hacc_sr_force_symmetric(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists),
                                              ctypes.byref(p), _ptr(ax), _ptr(ay), _ptr(az),
                                              ctypes.byref(lc) if lc else None, _ptr(ws), ws.numel(), _ptr(status),
                                              _stream()), "hacc_sr_force_symmetric")


def hacc_sr_force_adjoint(mesh, binned, lists, params: SRParams, gax, gay, gaz, gx, gy, gz, gm, ws, status,
                          launch: Launch | None = None):
    p = params.c_struct()
    lc = launch.c_struct() if launch is not None else None
    check(_lib.load().hacc_sr_force_adjoint(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists),
                                            ctypes.byref(p), _ptr(gax), _ptr(gay), _ptr(gaz), _ptr(gx), _ptr(gy),
                                            _ptr(gz), _ptr(gm), ctypes.byref(lc) if lc else None, _ptr(ws),
                                            ws.numel(), _ptr(status), _stream()), "hacc_sr_force_adjoint")


def hacc_sr_force_adjoint_symmetric(mesh, binned, lists, params: SRParams, gax, gay, gaz, gx, gy, gz, gm, ws,
                                    status, launch: Launch | None = None):
    p = params.c_struct()
    lc = launch.c_struct() if launch is not None else None
    check(_lib.load().hacc_sr_force_adjoint_symmetric(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists),
                                                      ctypes.byref(p), _ptr(gax), _ptr(gay), _ptr(gaz), _ptr(gx),
                                                      _ptr(gy), _ptr(gz), _ptr(gm),
                                                      ctypes.byref(lc) if lc else None, _ptr(ws), ws.numel(),
                                                      _ptr(status), _stream()), "hacc_sr_force_adjoint_symmetric")


def hacc_count_pairs(mesh, binned, lists, params: SRParams, out):
    p = params.c_struct()
    check(_lib.load().hacc_count_pairs(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists),
                                       ctypes.byref(p), _ptr(out), _stream()), "hacc_count_pairs")


def hacc_kick(mesh, N, vx, vy, vz, ax, ay, az, dt_kick, x=None, y=None, z=None, dt_drift=0.0):
    check(_lib.load().hacc_kick(ctypes.byref(mesh) if mesh is not None else None, int(N), _ptr(vx), _ptr(vy),
                                _ptr(vz), _ptr(ax), _ptr(ay), _ptr(az), float(dt_kick), _ptr(x), _ptr(y), _ptr(z),
                                float(dt_drift), _stream()), "hacc_kick")


def hacc_moments(N, m, vx, vy, vz, ax, ay, az, out, ws, phi=None):
    check(_lib.load().hacc_moments(int(N), _ptr(m), _ptr(vx), _ptr(vy), _ptr(vz), _ptr(ax), _ptr(ay), _ptr(az),
                                   _ptr(phi), _ptr(out), _ptr(ws), ws.numel(), _stream()), "hacc_moments")


def hacc_sr_potential(mesh, binned, lists, params: SRParams, phi, ws, status, launch: Launch | None = None):
    p = params.c_struct()
    lc = launch.c_struct() if launch is not None else None
    check(_lib.load().hacc_sr_potential(ctypes.byref(mesh), ctypes.byref(binned), ctypes.byref(lists),
                                        ctypes.byref(p), _ptr(phi), ctypes.byref(lc) if lc else None, _ptr(ws),
                                        ws.numel(), _ptr(status), _stream()), "hacc_sr_potential")


# ---------------------------------------------------------------------------
# buffers of one mesh
# ---------------------------------------------------------------------------

class ShortRange:
    """Device buffers and the call sequence for one chaining mesh of V volumes.

    ``L`` (per volume box sides) and ``vol_off`` (particle ranges) are host
    arrays; positions, masses, velocities and accelerations are float32 CUDA
    tensors of length N in input order.
    """

    def __init__(self, L, vol_off, rcut: float, cell_min: float | None = None, split_T: int = 32,
                 device: str | torch.device = "cuda", builder: str = "mesh", leaf_max: int = 64,
                 max_depth: int = 48, skin: float = 0.0, equal_mass_path: bool = True):
        """builder: "mesh" (chaining mesh, hacc_bin + hacc_build_lists) or "rcb"
        (the paper's RCB fat-leaf tree, hacc_rcb_build + hacc_rcb_lists, leaves
        of at most leaf_max particles; its build synchronises the stream).
        skin (mesh only): lists built for rcut + skin, so that binned particles
        may drift up to skin/2 (drift_offsets) before the next binning.
        equal_mass_path: let the binning flag equal masses (hacc_binned
        mass_varies) so that the force calls take their equal-mass path;
        False passes no flag and always runs the general path."""
        if builder not in ("mesh", "rcb"):
            raise HaccError(f"unknown list builder {builder!r}")
        if skin < 0 or (skin > 0 and builder != "mesh"):
            raise HaccError("a skin needs the chaining mesh and must be non-negative")
        self.builder = builder
        self.skin = float(skin)
        self.device = torch.device(device)
        self.rcut = float(rcut)
        self.cell_min = float(cell_min if cell_min is not None else rcut + skin)
        self.table, self.mesh = hacc_mesh_plan(L, vol_off, self.cell_min, self.rcut + self.skin)
        self.V = int(self.mesh.V)
        self.N = int(self.mesh.N)
        self.n_cells = int(self.mesh.n_cells)
        self.n_entries = int(self.mesh.n_entries)
        raw = bytes(self.table)
        self.vols = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(self.device)
        self.mesh.vols = self.vols.data_ptr()
        lib = _lib.load()
        dev = self.device
        i32, i64 = torch.int32, torch.int64
        N = self.N
        self.cell_of = torch.empty(N, dtype=i32, device=dev)
        self.perm = torch.empty(N, dtype=i32, device=dev)
        self.sorted4 = torch.empty((N, 4), dtype=torch.float32, device=dev)
        self.split_T = int(split_T)
        self.n_tasks = torch.zeros(1, dtype=i32, device=dev)
        self.n_pairs = torch.zeros(1, dtype=i64, device=dev)
        self.mass_varies = torch.ones(1, dtype=i32, device=dev) if equal_mass_path else None
        if builder == "mesh":
            self.cell_start = torch.empty(self.n_cells + 1, dtype=i32, device=dev)
            self.binned = hacc_binned(_ptr(self.cell_of), _ptr(self.cell_start), _ptr(self.perm),
                                      _ptr(self.sorted4), None, _ptr(self.mass_varies))
            self.task_cap = int(lib.hacc_task_capacity(ctypes.byref(self.mesh), self.split_T))
            self.nbr_off = torch.empty(self.n_cells + 1, dtype=i64, device=dev)
            self.entry_cap = self.n_entries
            build_ws = max(lib.hacc_bin_workspace_size(ctypes.byref(self.mesh)),
                           lib.hacc_lists_workspace_size(ctypes.byref(self.mesh)))
        else:
            # a leaf holds at least one particle: N leaves (and fewer internal nodes) always fit
            self.leaf_cap = lc = max(N, 1)
            self.n_leaves = torch.zeros(1, dtype=i32, device=dev)
            self.n_nodes = torch.zeros(1, dtype=i32, device=dev)
            self.cell_start = self.leaf_start = torch.empty(lc + 1, dtype=i32, device=dev)
            self.leaf_qbox = torch.empty((lc, 6), dtype=i32, device=dev)
            self.leaf_origin = torch.empty((lc, 4), dtype=torch.float32, device=dev)
            self.node_qbox = torch.empty((lc, 6), dtype=i32, device=dev)
            self.node_child = torch.empty((lc, 2), dtype=i32, device=dev)
            self.root = torch.empty(self.V, dtype=i32, device=dev)
            self.tree = hacc_tree(int(leaf_max), int(max_depth), lc, _ptr(self.n_leaves), _ptr(self.n_nodes),
                                  _ptr(self.leaf_start), _ptr(self.leaf_qbox), _ptr(self.leaf_origin),
                                  _ptr(self.node_qbox), _ptr(self.node_child), _ptr(self.root))
            self.binned = hacc_binned(_ptr(self.cell_of), _ptr(self.leaf_start), _ptr(self.perm),
                                      _ptr(self.sorted4), _ptr(self.leaf_origin), _ptr(self.mass_varies))
            # each leaf gives ceil(size / T) tasks
            self.task_cap = lc + N // self.split_T + 1
            self.nbr_off = torch.empty(lc + 1, dtype=i64, device=dev)
            self.n_entries_dev = torch.zeros(1, dtype=i64, device=dev)
            self.entry_cap = 0
            self._lstatus = torch.zeros(1, dtype=i32, device=dev)
            build_ws = max(lib.hacc_rcb_build_workspace_size(ctypes.byref(self.mesh), int(leaf_max)),
                           lib.hacc_rcb_lists_workspace_size(ctypes.byref(self.mesh), lc, self.task_cap))
        self.tasks = torch.empty((max(self.task_cap, 1), 4), dtype=i32, device=dev)
        self.task_order = torch.empty(max(self.task_cap, 1), dtype=i32, device=dev)
        self._alloc_entries(self.entry_cap)
        ws_bytes = max(build_ws, lib.hacc_force_workspace_size(ctypes.byref(self.mesh)))
        self.ws = torch.empty(int(ws_bytes), dtype=torch.uint8, device=dev)
        # the moments keep their own (small) scratch, so that they may run on another stream
        # while the next binning, lists or force call uses ws
        self.mom_ws = torch.empty(int(lib.hacc_moments_workspace_size(N)), dtype=torch.uint8, device=dev)
        self.status = torch.zeros(1, dtype=i32, device=dev)

    def _alloc_entries(self, cap: int):
        self.entry_cap = int(cap)
        self.nbr_cell = torch.empty(max(self.entry_cap, 1), dtype=torch.int32, device=self.device)
        self.nbr_shift = torch.empty(max(self.entry_cap, 1), dtype=torch.int8, device=self.device)
        self.lists = hacc_lists(_ptr(self.nbr_off), _ptr(self.nbr_cell), _ptr(self.nbr_shift), _ptr(self.tasks),
                                _ptr(self.n_tasks), _ptr(self.n_pairs), _ptr(self.task_order), self.task_cap,
                                self.split_T, 0)

    # -- calls ------------------------------------------------------------
    def bin(self, x, y, z, m, disp=None):
        if self.builder != "mesh":
            raise HaccError("bin() belongs to the chaining mesh; the tree is built by prepare()")
        if disp is None:
            hacc_bin(self.mesh, x, y, z, m, self.binned, self.ws, self.status)
        else:
            hacc_bin(self.mesh, x, y, z, m, self.binned, self.ws, self.status, disp[0], disp[1], disp[2])

    def build_lists(self):
        if self.builder != "mesh":
            raise HaccError("build_lists() belongs to the chaining mesh; the tree is built by prepare()")
        hacc_build_lists(self.mesh, self.binned, self.lists, self.ws, self.status)

    def build_tree(self, x, y, z, m):
        """RCB tree and its leaf lists (builder "rcb").  Synchronises: the build
        reads the number of groups left per level, and the lists grow to fit."""
        hacc_rcb_build(self.mesh, x, y, z, m, self.tree, self.binned, self.ws, self.status)
        self.check_status()  # a tree that ran out of capacity must not be walked
        while True:
            self._lstatus.zero_()
            hacc_rcb_lists(self.mesh, self.tree, self.lists, self.entry_cap, self.n_entries_dev, self.ws,
                           self._lstatus)
            need = int(self.n_entries_dev.item())
            if need <= self.entry_cap:
                break
            self._alloc_entries(need + need // 4 + 1024)
        s = int(self._lstatus.item())
        if s:
            raise HaccError(f"device status {s:#x} from the tree lists")
        self.n_entries = need
        self.n_cells = int(self.n_leaves.item())

    def force(self, params: SRParams, out=None, launch: Launch | None = None):
        if out is None:
            out = torch.empty((3, self.N), dtype=torch.float32, device=self.device)
        hacc_sr_force(self.mesh, self.binned, self.lists, params, out[0], out[1], out[2], self.ws, self.status,
                      launch)
        return out

    def force_symmetric(self, params: SRParams, out=None, launch: Launch | None = None):
        """Same forces from half the pair evaluations (Newton's third law;
        not bitwise reproducible)."""
        if out is None:
            out = torch.empty((3, self.N), dtype=torch.float32, device=self.device)
        hacc_sr_force_symmetric(self.mesh, self.binned, self.lists, params, out[0], out[1], out[2], self.ws,
                                self.status, launch)
        return out

    def adjoint(self, params: SRParams, lam, out=None, want_gm: bool = True, launch: Launch | None = None):
        """lam: [3, N] cotangent of the accelerations; returns (gx [3, N], gm [N] or None)."""
        if out is None:
            out = torch.empty((3, self.N), dtype=torch.float32, device=self.device)
        gm = torch.empty(self.N, dtype=torch.float32, device=self.device) if want_gm else None
        lam = lam.contiguous()
        hacc_sr_force_adjoint(self.mesh, self.binned, self.lists, params, lam[0], lam[1], lam[2], out[0], out[1],
                              out[2], gm, self.ws, self.status, launch)
        return out, gm

    def adjoint_symmetric(self, params: SRParams, lam, out=None, want_gm: bool = True,
                          launch: Launch | None = None):
        """adjoint() with each pair evaluated once (not bitwise reproducible)."""
        if out is None:
            out = torch.empty((3, self.N), dtype=torch.float32, device=self.device)
        gm = torch.empty(self.N, dtype=torch.float32, device=self.device) if want_gm else None
        lam = lam.contiguous()
        hacc_sr_force_adjoint_symmetric(self.mesh, self.binned, self.lists, params, lam[0], lam[1], lam[2], out[0],
                                        out[1], out[2], gm, self.ws, self.status, launch)
        return out, gm

    def kick(self, v, a, dt_kick, pos=None, dt_drift=0.0, wrap=True):
        """v += dt_kick a; then pos += dt_drift v (wrapped into the boxes if wrap)."""
        if pos is None:
            hacc_kick(None, self.N, v[0], v[1], v[2], a[0], a[1], a[2], dt_kick)
        else:
            hacc_kick(self.mesh if wrap else None, self.N, v[0], v[1], v[2], a[0], a[1], a[2], dt_kick, pos[0],
                      pos[1], pos[2], dt_drift)

    def drift_offsets(self, v, dt):
        """The stream map on the binned records (offsets += dt v) so that the
        pair calls can run again without re-binning; a particle that leaves its
        cell by more than skin/2 sets HACC_STATUS_SKIN."""
        hacc_drift_offsets(self.mesh, self.binned, v[0], v[1], v[2], dt, self.skin, self.status)

    def stream(self, v, pos, dt, wrap=True):
        """The stream map alone: pos += dt v (float64, wrapped if wrap); v unchanged."""
        hacc_kick(self.mesh if wrap else None, self.N, v[0], v[1], v[2], None, None, None, 0.0, pos[0], pos[1],
                  pos[2], dt)

    def moments(self, m, v=None, a=None, phi=None):
        """FP64 [sum m v (3), sum m a (3), kinetic energy, sum m |a|, potential energy]."""
        out = torch.empty(9, dtype=torch.float64, device=self.device)
        vx = vy = vz = ax = ay = az = None
        if v is not None:
            vx, vy, vz = v[0], v[1], v[2]
        if a is not None:
            ax, ay, az = a[0], a[1], a[2]
        hacc_moments(self.N, m, vx, vy, vz, ax, ay, az, out, self.mom_ws, phi)
        return out

    def potential(self, params: SRParams, out=None, launch: Launch | None = None):
        """Short-range potential phi [N] of every particle (same binning and lists as force)."""
        if out is None:
            out = torch.empty(self.N, dtype=torch.float32, device=self.device)
        hacc_sr_potential(self.mesh, self.binned, self.lists, params, out, self.ws, self.status, launch)
        return out

    def sks_subcycles(self, pos, v, m, params: SRParams, h: float, n_c: int, a=None,
                      launch: Launch | None = None, rebin_every: int = 1):
        """n_c short-range sub-cycles S(h/2) K(h) S(h/2) of the split-operator
        step (Eq. 6), in place on pos [3, N] (wrapped into the boxes) and
        v [3, N]: stream h/2, re-bin, force, kick h, stream h/2.  With
        rebin_every = k > 1 (and a skin) only every k-th sub-cycle re-bins; in
        between, the binned offsets are streamed with the positions
        (drift_offsets) and the lists are reused.  Every call is a library
        kernel, so the sequence can be captured in a CUDA graph."""
        if a is None:
            a = torch.empty_like(v)
        k = max(1, int(rebin_every))
        for c in range(n_c):
            self.stream(v, pos, 0.5 * h)
            if c % k == 0:
                self.prepare(pos, m)
            else:
                self.drift_offsets(v, 0.5 * h)
            self.force(params, a, launch=launch)
            self.kick(v, a, h, pos, 0.5 * h)
            if (c + 1) % k != 0 and c + 1 < n_c:  # the next force reuses these records
                self.drift_offsets(v, 0.5 * h)
        return a

    def set_equal_mass_path(self, enabled: bool):
        """Pass (enabled) or withhold the equal-mass flag of the binned
        particles; from the next prepare on, the force calls take the
        equal-mass path when every mass is equal, or the general path always."""
        if enabled and self.mass_varies is None:
            self.mass_varies = torch.ones(1, dtype=torch.int32, device=self.device)
        elif enabled:
            self.mass_varies.fill_(1)
        self.binned.mass_varies = _ptr(self.mass_varies) if enabled else None

    @property
    def equal_mass(self) -> bool:
        """True when the last binning found every mass equal (the force calls
        then take the equal-mass path); reads the device flag."""
        return self.binned.mass_varies is not None and int(self.mass_varies.item()) == 0

    def prepare(self, pos, m, disp=None):
        """Binning and lists for positions pos [3, N] (plus displacements disp
        [3, N], if given: the position is then pos + disp) and masses m [N]."""
        if self.builder == "rcb":
            if disp is not None:
                raise HaccError("the tree builder takes absolute positions only")
            self.build_tree(pos[0], pos[1], pos[2], m)
            return
        self.bin(pos[0], pos[1], pos[2], m, disp)
        self.build_lists()

    def check_status(self):
        s = hacc_get_status(self.status)
        if s:
            self.status.zero_()
            raise HaccError(f"device status {s:#x}")

    def pair_count(self) -> int:
        """Candidate ordered pairs (j != i) the pair kernels evaluate."""
        return int(self.n_pairs.item())

    def pairs_within_cutoff(self, params: SRParams) -> int:
        """Ordered pairs (j != i) inside the cutoff, decided as the pair kernels decide."""
        out = torch.zeros(1, dtype=torch.int64, device=self.device)
        hacc_count_pairs(self.mesh, self.binned, self.lists, params, out)
        return int(out.item())


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class _SRForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos, disp, m, solver: ShortRange, params: SRParams, symmetric: bool):
        solver.prepare(pos, m, disp)
        a = solver.force_symmetric(params) if symmetric else solver.force(params)
        ctx.save_for_backward(pos, disp, m)
        ctx.solver = solver
        ctx.params = params
        ctx.symmetric = symmetric
        return a

    @staticmethod
    def backward(ctx, ga):
        pos, disp, m = ctx.saved_tensors
        solver = ctx.solver
        # the pair terms are recomputed: re-bin the saved positions, then the adjoint
        solver.prepare(pos, m, disp)
        adj = solver.adjoint_symmetric if ctx.symmetric else solver.adjoint
        gpos, gm = adj(ctx.params, ga.contiguous(), want_gm=ctx.needs_input_grad[2])
        # the position is pos + disp: both receive the same cotangent
        return gpos, gpos if ctx.needs_input_grad[1] else None, gm, None, None, None


class _KickDrift(torch.autograd.Function):
    """v' = v + dt_k a ; x' = x + dt_d v' (no wrap), forward and VJP by hacc_kick."""

    @staticmethod
    def forward(ctx, v, pos, a, dt_k: float, dt_d: float):
        v2 = v.clone()
        p2 = pos.clone()
        N = v.shape[1]
        hacc_kick(None, N, v2[0], v2[1], v2[2], a[0], a[1], a[2], dt_k, p2[0], p2[1], p2[2], dt_d)
        ctx.dt = (dt_k, dt_d)
        return v2, p2

    @staticmethod
    def backward(ctx, gv2, gp2):
        dt_k, dt_d = ctx.dt
        if gv2 is None:
            gv2 = torch.zeros_like(gp2)
        if gp2 is None:
            gp2 = torch.zeros_like(gv2)
        gp2 = gp2.contiguous()
        gv = gv2.contiguous().clone()
        N = gv.shape[1]
        # gv = gv' + dt_d gx'   (v' feeds x')
        hacc_kick(None, N, gv[0], gv[1], gv[2], gp2[0], gp2[1], gp2[2], dt_d)
        # ga = dt_k gv
        ga = torch.zeros_like(gv)
        hacc_kick(None, N, ga[0], ga[1], ga[2], gv[0], gv[1], gv[2], dt_k)
        return gv, gp2, ga, None, None


def sr_force_autograd(pos, m, solver: ShortRange, params: SRParams, disp=None, symmetric: bool = False):
    """Accelerations [3, N] at positions pos [3, N] (+ disp [3, N] if given);
    differentiable in pos, disp and m.  symmetric: the Newton-III kernels
    (each pair evaluated once) for the forward and the adjoint; otherwise the
    gather kernels (bitwise reproducible)."""
    return _SRForce.apply(pos.contiguous(), None if disp is None else disp.contiguous(), m.contiguous(), solver,
                          params, bool(symmetric))


def kick_drift_autograd(v, pos, a, dt_k: float, dt_d: float):
    """(v + dt_k a, pos + dt_d (v + dt_k a)); differentiable."""
    return _KickDrift.apply(v.contiguous(), pos.contiguous(), a.contiguous(), dt_k, dt_d)


def trajectory_autograd(x0, v0, m, solver: ShortRange, params: SRParams, dt: float, steps: int,
                        symmetric: bool = False):
    """`steps` short-range kick-drift steps (the kick and stream maps of the
    paper's split-operator step, Eq. 6) from positions x0 [3, N] and velocities
    v0 [3, N].  Positions stay x0 + disp with a float32 displacement that the
    drift updates, so they keep float32 precision of the displacement rather
    than of the box.  Returns (disp, v) after the last step; differentiable in
    x0, v0 and m (symmetric: see sr_force_autograd)."""
    disp = torch.zeros_like(x0)
    v = v0
    for _ in range(steps):
        a = sr_force_autograd(x0, m, solver, params, disp, symmetric)
        v, disp = kick_drift_autograd(v, disp, a, dt, dt)
    return disp, v

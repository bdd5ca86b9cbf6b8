"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Binning, lists and tasks must be bit-exact; forces within 1e-5 rms and 1e-4
max relative error of the float64 oracle; the adjoint within the gradient
tolerances.  Every input is seeded and synthetic.
"""

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda, sample_targets
from synth import default_coeffs, make_config, uniform_box
from synth.workloads import Workload, batched_volumes, clustered_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0


@pytest.fixture(scope="module")
def torch():
    return need_cuda()


@pytest.fixture(scope="module")
def hs():
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


def params(hs, eps=EPS, rc=RC, c=None):
    if c is None:
        c = default_coeffs(rc, eps)
    return hs.SRParams(eps, rc, np.asarray(c, np.float32))


def to_dev(torch, w: Workload):
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    return pos, m


def run_force(torch, hs, w: Workload, prm, cell_min=None, split_T=32, launch=None):
    sr = hs.ShortRange(w.L, w.vol_off, prm.rcut, cell_min=cell_min, split_T=split_T)
    pos, m = to_dev(torch, w)
    sr.prepare(pos, m)
    a = sr.force(prm, launch=launch)
    torch.cuda.synchronize()
    sr.check_status()
    return sr, pos, m, a.cpu().numpy().T.astype(np.float64)


def oracle_force(w: Workload, prm, targets=None, v=0):
    b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
    return oracle.sr_force(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), prm.eps, prm.rcut,
                           prm.c.astype(np.float64), targets)


# --------------------------------------------------------------------------
# binning / lists / tasks: bit-exact
# --------------------------------------------------------------------------

def check_bin_lists(torch, hs, w: Workload, cell_min, rcut, split_T=32):
    sr = hs.ShortRange(w.L, w.vol_off, rcut, cell_min=cell_min, split_T=split_T)
    pos, m = to_dev(torch, w)
    sr.prepare(pos, m)
    torch.cuda.synchronize()
    sr.check_status()
    cell_of = sr.cell_of.cpu().numpy()
    cs = sr.cell_start.cpu().numpy()
    perm = sr.perm.cpu().numpy()
    s4 = sr.sorted4.cpu().numpy()
    off = sr.nbr_off.cpu().numpy()
    ncell = sr.nbr_cell.cpu().numpy()
    nsh = sr.nbr_shift.cpu().numpy()
    nt = int(sr.n_tasks.item())
    tasks = sr.tasks.cpu().numpy()[:nt]
    exp_tasks, exp_pairs = [], 0
    cbase = ebase = 0
    for v in range(w.V):
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        ob = oracle.bin_volume(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), cell_min)
        n = ob["n"]
        nc = n ** 3
        assert np.array_equal(cell_of[b:e], ob["cell_of"] + cbase)
        assert np.array_equal(cs[cbase:cbase + nc + 1], ob["cell_start"] + b)
        assert np.array_equal(perm[b:e], ob["perm"] + b)
        assert np.array_equal(s4[b:e].view(np.int32), ob["sorted4"].view(np.int32))
        o_off, o_cell, o_sh = oracle.lists_volume(n, ob["w"], rcut)
        assert np.array_equal(off[cbase:cbase + nc + 1], o_off + ebase)
        ne = int(o_off[-1])
        assert np.array_equal(ncell[ebase:ebase + ne], o_cell + cbase)
        assert np.array_equal(nsh[ebase:ebase + ne], o_sh)
        t = oracle.tasks(ob["cell_start"], split_T)
        if t.size:
            t = t.astype(np.int64)
            t[:, 0] += cbase
            t[:, 1:] += b
            exp_tasks.append(np.concatenate([t, np.full((t.shape[0], 1), v)], 1))
        # candidate pairs the force visits: per cell, count * sum of listed counts, minus self
        cnt = np.diff(ob["cell_start"]).astype(np.int64)
        nb = np.add.reduceat(cnt[o_cell], o_off[:-1]) if ne else np.zeros(nc, np.int64)
        exp_pairs += int((cnt * nb).sum()) - (e - b)
        cbase += nc
        ebase += ne
    exp = np.concatenate(exp_tasks) if exp_tasks else np.zeros((0, 4), np.int64)
    assert np.array_equal(tasks.astype(np.int64), exp)
    assert sr.pair_count() == exp_pairs
    # the work order is one valid schedule: a permutation, heaviest cost class
    # first, ties in task order
    order = sr.task_order.cpu().numpy()[:nt].astype(np.int64)
    assert np.array_equal(np.sort(order), np.arange(nt))
    if nt:
        cnt_all = np.diff(cs.astype(np.int64))
        nj = np.array([cnt_all[ncell[off[c]:off[c + 1]]].sum() for c in exp[:, 0]], np.int64)
        cost = (exp[:, 2] - exp[:, 1]) * np.maximum(nj, 1)
        cls = 63 - np.floor(np.log2(cost.astype(np.float64))).astype(np.int64)
        assert np.array_equal(order, np.argsort(cls, kind="stable"))
    return sr


def test_bin_lists_tasks_bit_exact_uniform(torch, hs):
    check_bin_lists(torch, hs, make_config("uniform4096"), 3.0, 3.0)


@pytest.mark.parametrize("N", [200, 3000, 40000, 70000])
def test_bin_bit_exact_when_one_cell_holds_most_particles(torch, hs, N):
    """Degenerate clustering: most particles in one cell, the rest uniform,
    over one to 18 tiles of the binning's counting passes: nearly every item
    of a tile shares one digit, so the ranks among equal digits span whole
    warps and tiles."""
    rng = np.random.default_rng(N)
    L = np.float32(27.0)
    k = N * 9 // 10
    p = np.concatenate([rng.random((k, 3)) * 3.0 + 12.0, rng.random((N - k, 3)) * float(L)])
    p = p[rng.permutation(N)].astype(np.float32)
    w = Workload("crowded", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), np.ones(N, np.float32),
                 np.zeros(N, np.float32), np.zeros(N, np.float32), np.zeros(N, np.float32),
                 np.array([L], np.float32), np.array([0, N], np.int64))
    sr = check_bin_lists(torch, hs, w, 3.0, 3.0, split_T=128)
    assert int(np.diff(sr.cell_start.cpu().numpy()).max()) >= k


def test_bin_bit_exact_for_cells_of_every_size_class(torch, hs):
    """Empty cells and cells of 1 to 1025 particles (sizes on both sides of
    the powers of two up to a warp's 32 lanes and beyond, so that runs of one
    digit start and end anywhere in a warp's items), in a shuffled input
    order; bit-exact against the oracle."""
    sizes = [0, 1, 2, 15, 16, 17, 31, 32, 33, 0, 63, 64, 65, 127, 128, 129, 255, 256, 257, 0, 511, 512, 513, 1,
             1023, 1024, 1025]
    rng = np.random.default_rng(77)
    L = np.float32(9.0)  # 3 cells per side of width 3: 27 cells, one size each
    parts = []
    for c, k in enumerate(sizes):
        cx, cy, cz = c % 3, (c // 3) % 3, c // 9
        parts.append((rng.random((k, 3)) * 2.9 + 0.05 + 3.0 * np.array([cx, cy, cz])))
    p = np.concatenate(parts)[rng.permutation(sum(sizes))].astype(np.float32)
    N = p.shape[0]
    w = Workload("boundaries", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), np.ones(N, np.float32),
                 np.zeros(N, np.float32), np.zeros(N, np.float32), np.zeros(N, np.float32),
                 np.array([L], np.float32), np.array([0, N], np.int64))
    sr = check_bin_lists(torch, hs, w, 3.0, 3.0, split_T=128)
    assert sorted(np.diff(sr.cell_start.cpu().numpy()).tolist()) == sorted(sizes)


def check_bin(torch, hs, w: Workload, cell_min, rcut, disp=None):
    """Binning alone (no lists), bit-exact against the oracle per volume."""
    sr = hs.ShortRange(w.L, w.vol_off, rcut, cell_min=cell_min)
    pos, m = to_dev(torch, w)
    d = None if disp is None else torch.tensor(disp, device="cuda")
    sr.bin(pos[0], pos[1], pos[2], m, None if d is None else (d[0], d[1], d[2]))
    torch.cuda.synchronize()
    sr.check_status()
    cell_of, cs = sr.cell_of.cpu().numpy(), sr.cell_start.cpu().numpy()
    perm, s4 = sr.perm.cpu().numpy(), sr.sorted4.cpu().numpy()
    cbase = 0
    for v in range(w.V):
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        ob = oracle.bin_volume(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), cell_min,
                               disp=None if disp is None else disp[:, b:e])
        nc = ob["n"] ** 3
        assert np.array_equal(cell_of[b:e], ob["cell_of"] + cbase)
        assert np.array_equal(cs[cbase:cbase + nc + 1], ob["cell_start"] + b)
        assert np.array_equal(perm[b:e], ob["perm"] + b)
        assert np.array_equal(s4[b:e].view(np.int32), ob["sorted4"].view(np.int32))
        cbase += nc
    assert cbase == sr.n_cells
    return sr


def _half_clustered(N, L, seed):
    """N particles in a box of side L: half uniform, half in eight tight
    clumps (runs of equal cells in the input order), positions slightly
    outside the box included."""
    rng = np.random.default_rng(seed)
    k = N // 2
    centres = rng.random((8, 3)) * L
    clump = centres[rng.integers(0, 8, N - k)] + rng.normal(size=(N - k, 3)) * 0.7
    p = np.concatenate([rng.random((k, 3)) * L, clump]).astype(np.float32)
    return Workload("half_clustered", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(),
                    rng.uniform(0.5, 2.0, N).astype(np.float32), np.zeros(N, np.float32),
                    np.zeros(N, np.float32), np.zeros(N, np.float32), np.array([L], np.float32),
                    np.array([0, N], np.int64))


# (N, L, cell_min, rcut): one counting pass (at most 1024 cells: keys of ten bits), two
# (2197 and 9261 cells) and three (102^3 = 1,061,208 cells: keys of 21 bits); N on both
# sides of the 4096-particle tile of the passes, and several tiles with a ragged tail
BIN_PASS_CASES = [(1, 27.0, 3.0, 3.0), (4095, 27.0, 3.0, 3.0), (4097, 27.0, 3.0, 3.0),
                  (4096, 40.0, 3.0, 3.0), (3 * 4096 + 17, 40.0, 3.0, 3.0), (20000, 64.0, 3.0, 3.0),
                  (3 * 4096 + 5, 102.0, 1.0, 1.0)]


@pytest.mark.parametrize("N,L,cell_min,rcut", BIN_PASS_CASES)
def test_bin_bit_exact_across_tiles_and_pass_counts(torch, hs, N, L, cell_min, rcut):
    check_bin(torch, hs, _half_clustered(N, np.float32(L), seed=N), cell_min, rcut)


def test_bin_with_displacements_bit_exact(torch, hs):
    """Positions given as a reference plus a float32 displacement: the
    position formed, wrapped and offset in float64 (two counting passes,
    several tiles), bit-exact against the oracle."""
    N, L = 3 * 4096 + 300, np.float32(40.0)
    w = _half_clustered(N, L, seed=91)
    rng = np.random.default_rng(91)
    disp = (rng.normal(size=(3, N)) * 2.0).astype(np.float32)
    disp[0, :4] = [0.5 * L, -0.5 * L, 1e-7, -1e-7]
    check_bin(torch, hs, w, 3.0, 3.0, disp=disp)


def test_bin_lists_bit_exact_fine_mesh_and_edge_positions(torch, hs):
    """Cells narrower than r_c (reach 2: 125-cell stencils), coordinates on
    and outside the box edges, a ragged split size."""
    rng = np.random.default_rng(5)
    L = np.float32(19.7)
    N = 5000
    x = (rng.random(N) * 3 * L - L).astype(np.float32)
    y = (rng.random(N) * L).astype(np.float32)
    z = (rng.normal(size=N) * 6).astype(np.float32)
    x[:5] = [0.0, -0.0, L, np.nextafter(L, np.float32(0)), np.float32(-1e-9)]
    w = Workload("edges", x, y, z, np.ones(N, np.float32), x * 0, x * 0, x * 0, np.array([L], np.float32),
                 np.array([0, N], np.int64))
    check_bin_lists(torch, hs, w, 1.6, 3.0, split_T=7)


def test_bin_lists_bit_exact_reach8(torch, hs):
    """Cells of 0.4 grid units against r_c = 3 (reach 8: a 17^3 stencil, more
    offsets than the list kernel's per-block predicate table holds, so every
    offset is decided directly; the other list tests run on the table), in two
    volumes of 17 and 18 cells per side."""
    wa = uniform_box(400, 7.0, seed=43)
    wb = uniform_box(500, 7.5, seed=44)
    cat = lambda f: np.concatenate([getattr(wa, f), getattr(wb, f)])
    w = Workload("reach8", cat("x"), cat("y"), cat("z"), cat("m"), cat("vx"), cat("vy"), cat("vz"),
                 np.array([7.0, 7.5], np.float32), np.array([0, 400, 900], np.int64))
    check_bin_lists(torch, hs, w, 0.4, 3.0, split_T=16)


def test_bin_lists_bit_exact_batched_volumes(torch, hs):
    w = batched_volumes(12, n_lo=800, n_hi=6000, seed=8)
    check_bin_lists(torch, hs, w, 3.0, 3.0, split_T=32)


def test_bin_lists_bit_exact_clustered_large_cells(torch, hs):
    """Halo cells with hundreds of particles: many tasks per cell."""
    w = clustered_box(24, 6, seed=12)
    check_bin_lists(torch, hs, w, 3.0, 3.0, split_T=13)


# --------------------------------------------------------------------------
# force
# --------------------------------------------------------------------------

def test_force_uniform4096_full_oracle(torch, hs):
    w = make_config("uniform4096")
    prm = params(hs)
    sr, _, _, a = run_force(torch, hs, w, prm)
    ref = oracle_force(w, prm)
    rms, mx = err_norms(a, ref)
    assert rms < RMS_TOL, rms
    assert mx < MAX_TOL, mx


@pytest.mark.parametrize("launch", [None, (4, 1, 32, 2), (8, 1, 128, 4), (8, 2, 64, 3), (2, 4, 256, 2)])
def test_force_launch_shapes_agree(torch, hs, launch):
    w = uniform_box(3000, 14.0, seed=17)
    prm = params(hs)
    L = hs.Launch(*launch) if launch else None
    _, _, _, a = run_force(torch, hs, w, prm, launch=L)
    ref = oracle_force(w, prm)
    rms, mx = err_norms(a, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_force_clustered_and_fine_mesh(torch, hs):
    """Clustered particles (cells of hundreds), split into many tasks, plus a
    mesh finer than the cutoff (lists longer than a warp)."""
    w = clustered_box(24, 6, seed=12)
    prm = params(hs)
    ref = oracle_force(w, prm)
    for cell_min, T in [(3.0, 32), (3.0, 5), (3.0, 64), (3.0, 47), (1.5, 64)]:
        _, _, _, a = run_force(torch, hs, w, prm, cell_min=cell_min, split_T=T)
        rms, mx = err_norms(a, ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (cell_min, T, rms, mx)


def test_force_edge_cases(torch, hs):
    prm = params(hs)
    L = np.float32(12.0)

    def one(pts, m=None):
        pts = np.asarray(pts, np.float32)
        N = pts.shape[0]
        mm = np.ones(N, np.float32) if m is None else np.asarray(m, np.float32)
        w = Workload("edge", pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(), mm, mm * 0, mm * 0, mm * 0,
                     np.array([L], np.float32), np.array([0, N], np.int64))
        _, _, _, a = run_force(torch, hs, w, prm)
        return a, oracle_force(w, prm)

    # a single particle feels nothing
    a, ref = one([[1.0, 2.0, 3.0]])
    assert np.all(a == 0.0) and np.all(ref == 0.0)
    # a pair across the periodic boundary
    a, ref = one([[0.5, 6.0, 6.0], [11.5, 6.0, 6.0]], m=[1.0, 2.0])
    assert np.allclose(a, ref, rtol=2e-6, atol=0)
    # beyond the cutoff: exactly zero
    a, ref = one([[1.0, 1.0, 1.0], [4.5, 1.0, 1.0]])
    assert np.all(a == 0.0)
    # everything in one cell, coincident pair included (softening keeps it finite)
    rng = np.random.default_rng(3)
    pts = 5.0 + rng.random((70, 3)) * 0.9
    pts[1] = pts[0]
    a, ref = one(pts)
    rms, mx = err_norms(a, ref)
    assert np.all(np.isfinite(a)) and rms < RMS_TOL and mx < MAX_TOL
    # perfect lattice: zero force by symmetry
    g = np.arange(12) + 0.5
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    a, _ = one(np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1))
    assert np.max(np.abs(a)) < 1e-5


def test_empty_input_and_empty_volume(torch, hs):
    """N = 0 runs every call and returns nothing; a batch whose middle volume
    holds no particles bins, lists and forces the others correctly."""
    prm = params(hs)
    e = np.zeros(0, np.float32)
    w0 = Workload("empty", e, e, e, e, e, e, e, np.array([12.0], np.float32), np.array([0, 0], np.int64))
    sr = hs.ShortRange(w0.L, w0.vol_off, RC)
    pos = torch.zeros((3, 0), device="cuda")
    m = torch.zeros(0, device="cuda")
    sr.prepare(pos, m)
    a = sr.force(prm)
    torch.cuda.synchronize()
    sr.check_status()
    assert a.shape == (3, 0) and int(sr.n_tasks.item()) == 0 and sr.pair_count() == 0
    assert np.all(sr.cell_start.cpu().numpy() == 0)
    # three volumes, the middle one empty
    wa, wb = uniform_box(700, 10.0, seed=31), uniform_box(900, 11.0, seed=32)
    cat = lambda f: np.concatenate([getattr(wa, f), getattr(wb, f)])
    w = Workload("gap", cat("x"), cat("y"), cat("z"), cat("m"), cat("vx"), cat("vy"), cat("vz"),
                 np.array([10.0, 9.5, 11.0], np.float32), np.array([0, 700, 700, 1600], np.int64))
    _, _, _, a = run_force(torch, hs, w, prm)
    for v, ww, (b, e_) in ((0, wa, (0, 700)), (2, wb, (700, 1600))):
        rms, mx = err_norms(a[b:e_], oracle_force(ww, prm))
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)
    check_bin_lists(torch, hs, w, 3.0, 3.0)


def test_force_zero_coefficients_is_truncated_newton(torch, hs):
    w = uniform_box(2000, 12.0, seed=4)
    prm = params(hs, c=np.zeros(6, np.float32), eps=0.05)
    _, _, _, a = run_force(torch, hs, w, prm)
    ref = oracle_force(w, prm)
    rms, mx = err_norms(a, ref)
    assert rms < RMS_TOL and mx < MAX_TOL


def test_force_batched_volumes(torch, hs):
    w = batched_volumes(10, n_lo=800, n_hi=5000, seed=6)
    prm = params(hs)
    _, _, _, a = run_force(torch, hs, w, prm)
    for v in range(w.V):
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        rms, mx = err_norms(a[b:e], oracle_force(w, prm, v=v))
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)


def test_force_newton3_and_moments(torch, hs):
    w = uniform_box(20000, 28.0, seed=9)
    prm = params(hs)
    sr, pos, m, a = run_force(torch, hs, w, prm)
    at = torch.tensor(a.T.astype(np.float32), device="cuda").contiguous()
    v = torch.zeros_like(at)
    mom = sr.moments(m, v, at).cpu().numpy()
    # sum m a vanishes up to float32 rounding of the individual forces
    assert np.all(np.abs(mom[3:6]) < 1e-5 * mom[7])
    ref = (w.m[:, None].astype(np.float64) * a).sum(0)
    assert np.allclose(mom[3:6], ref, rtol=0, atol=1e-9 * mom[7])
    assert mom[7] == pytest.approx(np.sum(np.linalg.norm(a, axis=1)), rel=1e-12)


@pytest.mark.parametrize("maker", ["uniform", "clustered", "fine"])
def test_pairs_within_cutoff_count(torch, hs, maker):
    """The kernels' within-cutoff pair count equals the oracle's brute-force
    count, up to pairs whose s sits within float32 rounding of r_c^2."""
    prm = params(hs)
    if maker == "uniform":
        w, cm = uniform_box(3000, 14.0, seed=17), 3.0
    elif maker == "clustered":
        w, cm = clustered_box(24, 6, seed=12), 3.0
    else:
        w, cm = uniform_box(3000, 14.0, seed=18), 1.5
    sr, _, _, _ = run_force(torch, hs, w, prm, cell_min=cm)
    got = sr.pairs_within_cutoff(prm)
    ref = oracle.pair_count(w.x, w.y, w.z, float(w.L[0]), RC)
    assert abs(got - ref) <= max(2, ref // 1_000_000), (got, ref)
    assert got <= sr.pair_count()


def test_capacity_overflow_sets_status_not_fault(torch, hs):
    w = uniform_box(4096, 16.0, seed=1)
    sr = hs.ShortRange(w.L, w.vol_off, RC)
    sr.lists.task_cap = 5   # far too small: the call must flag it, not write past it
    pos, m = to_dev(torch, w)
    sr.prepare(pos, m)
    torch.cuda.synchronize()
    assert int(sr.status.item()) & 1
    assert int(sr.n_tasks.item()) == 5


def test_nonfinite_position_flagged(torch, hs):
    w = uniform_box(500, 12.0, seed=2)
    w.x[7] = np.nan
    sr = hs.ShortRange(w.L, w.vol_off, RC)
    pos, m = to_dev(torch, w)
    sr.prepare(pos, m)
    # the library's own status read (waits for the stream) agrees with a plain tensor read
    assert hs.hacc_get_status(sr.status) & 4
    torch.cuda.synchronize()
    assert int(sr.status.item()) & 4
    with pytest.raises(hs.HaccError):
        sr.check_status()


# --------------------------------------------------------------------------
# adjoint and kick
# --------------------------------------------------------------------------

def test_adjoint_against_oracle(torch, hs):
    w = clustered_box(20, 4, seed=21)
    rng = np.random.default_rng(22)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    prm = params(hs)
    sr, pos, m, _ = run_force(torch, hs, w, prm)
    g, gm = sr.adjoint(prm, torch.tensor(lam.T.copy(), device="cuda"))
    torch.cuda.synchronize()
    sr.check_status()
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC, prm.c.astype(np.float64), lam)
    rms, mx = err_norms(g.cpu().numpy().T, rg)
    assert rms < RMS_TOL, rms
    grms = np.linalg.norm(gm.cpu().numpy() - rgm) / np.linalg.norm(rgm)
    assert grms < RMS_TOL, grms


def test_kick_drift_against_oracle(torch, hs):
    rng = np.random.default_rng(30)
    N = 10000
    L = 32.0
    x = (rng.random((N, 3)) * L).astype(np.float32)
    v = rng.normal(size=(N, 3)).astype(np.float32)
    a = rng.normal(size=(N, 3)).astype(np.float32)
    sr = hs.ShortRange(np.array([L], np.float32), np.array([0, N]), RC)
    vt = torch.tensor(v.T.copy(), device="cuda")
    xt = torch.tensor(x.T.copy(), device="cuda")
    at = torch.tensor(a.T.copy(), device="cuda")
    sr.kick(vt, at, 0.01, xt, 0.02, wrap=False)
    v_ref, x_ref = oracle.kick_drift(v, a, 0.01, x, 0.02)
    assert np.allclose(vt.cpu().numpy().T, v_ref, rtol=1e-6, atol=1e-7)
    assert np.allclose(xt.cpu().numpy().T, x_ref, rtol=0, atol=4e-6)
    # wrapped drift stays in [0, L)
    xt2 = torch.tensor(x.T.copy(), device="cuda")
    sr.kick(vt, at, 0.0, xt2, 50.0, wrap=True)
    xs = xt2.cpu().numpy()
    assert xs.min() >= 0.0 and xs.max() < L
    # the stream map alone (no accelerations): velocities untouched, x += dt v
    v2 = torch.tensor(v.T.copy(), device="cuda")
    xt3 = torch.tensor(x.T.copy(), device="cuda")
    sr.stream(v2, xt3, 0.02, wrap=False)
    _, x_ref3 = oracle.kick_drift(v, np.zeros_like(a), 0.0, x, 0.02)
    assert torch.equal(v2, torch.tensor(v.T.copy(), device="cuda"))
    assert np.allclose(xt3.cpu().numpy().T, x_ref3, rtol=0, atol=4e-6)
    with pytest.raises(hs.HaccError):  # neither a kick nor a drift
        hs.hacc_kick(None, N, v2[0], v2[1], v2[2], None, None, None, 0.0)


def test_moments_double_float_against_float64(torch, hs):
    """hacc_moments forms its terms and per-thread sums in double-float on the
    float32 pipe: on inputs spanning six decades, of both signs, with sums that
    cancel, every moment matches the float64 sum of the same float32 inputs to
    1e-12 of the sum of the terms' magnitudes."""
    N = 1_000_003
    rng = np.random.default_rng(41)
    scale = lambda: 10.0 ** rng.uniform(-3, 3, N)
    m = rng.uniform(0.5, 2.0, N).astype(np.float32)
    v = (rng.normal(size=(3, N)) * scale()).astype(np.float32)
    a = (rng.normal(size=(3, N)) * scale()).astype(np.float32)
    a[:, N // 2:] = -a[:, :N - N // 2]  # the second half cancels the first (up to one column)
    phi = (rng.normal(size=N) * scale()).astype(np.float32)
    L = np.array([64.0], np.float32)
    sr = hs.ShortRange(L, np.array([0, N], np.int64), RC)
    dev = lambda x: torch.tensor(x, device="cuda")
    got = sr.moments(dev(m), dev(v), dev(a), dev(phi)).cpu().numpy()
    m64, v64, a64, p64 = (x.astype(np.float64) for x in (m, v, a, phi))
    terms = [m64 * v64[0], m64 * v64[1], m64 * v64[2], m64 * a64[0], m64 * a64[1], m64 * a64[2],
             0.5 * m64 * (v64 ** 2).sum(0), m64 * np.sqrt((a64 ** 2).sum(0)), 0.5 * m64 * p64]
    for k, t in enumerate(terms):
        assert abs(got[k] - t.sum()) <= 1e-12 * np.abs(t).sum(), (k, got[k], t.sum())
    # the same sums with v or a left out, and the order-fixed result repeats bit for bit
    got2 = sr.moments(dev(m), None, dev(a), None).cpu().numpy()
    assert np.all(got2[[0, 1, 2, 6, 8]] == 0.0) and np.array_equal(got2[[3, 4, 5, 7]], got[[3, 4, 5, 7]])

"""GPU parity of the RCB fat-leaf tree builder (Sec. III) against the oracle.

The tree (slot order, leaf starts, integer leaf boxes, float32 origins and
offsets) and the leaf lists must be bit-exact; forces, potentials and
adjoints computed on the tree's leaves must meet the float32 tolerances
against the float64 brute-force oracle.  Every input is seeded and synthetic.
"""

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, uniform_box
from synth.workloads import Workload, clustered_box

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


def params(hs):
    return hs.SRParams(EPS, RC, default_coeffs(RC, EPS))


def build(torch, hs, w: Workload, leaf_max=64, max_depth=48, split_T=64):
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=split_T, builder="rcb", leaf_max=leaf_max, max_depth=max_depth)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    torch.cuda.synchronize()
    sr.check_status()
    return sr, pos, m


def concat(parts, L, name):
    """Volumes given as (x, y, z) float32 arrays, one box side each."""
    x = np.concatenate([p[0] for p in parts]).astype(np.float32)
    y = np.concatenate([p[1] for p in parts]).astype(np.float32)
    z = np.concatenate([p[2] for p in parts]).astype(np.float32)
    n = np.array([len(p[0]) for p in parts])
    vo = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    zeros = np.zeros(len(x), np.float32)
    rng = np.random.default_rng(12)
    m = rng.uniform(0.5, 1.5, len(x)).astype(np.float32)
    return Workload(name=name, x=x, y=y, z=z, m=m, vx=zeros, vy=zeros, vz=zeros,
                    L=np.asarray(L, np.float32), vol_off=vo)


def check_tree_bit_exact(sr, w: Workload, leaf_max, max_depth=48, list_targets=None):
    """Per volume: the GPU tree and lists equal the oracle's (leaf ids offset by
    the leaves of the earlier volumes).  list_targets: leaves per volume whose
    lists are compared (None: all)."""
    nl = int(sr.n_leaves.item())
    ls = sr.leaf_start.cpu().numpy()[:nl + 1]
    perm = sr.perm.cpu().numpy()
    s4 = sr.sorted4.cpu().numpy()
    qb = sr.leaf_qbox.cpu().numpy()[:nl]
    org = sr.leaf_origin.cpu().numpy()[:nl]
    cell_of = sr.cell_of.cpu().numpy()
    off = sr.nbr_off.cpu().numpy()[:nl + 1]
    nbr = sr.nbr_cell.cpu().numpy()[:sr.n_entries]
    shf = sr.nbr_shift.cpu().numpy()[:sr.n_entries]
    assert ls[0] == 0 and ls[-1] == w.N
    nt = int(sr.n_tasks.item())
    tasks = sr.tasks.cpu().numpy()[:nt]
    base = 0
    tbase = 0
    pairs = -w.N
    for v in range(w.V):
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        L = float(w.L[v])
        r = oracle.rcb_volume(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], L, leaf_max, max_depth)
        k = r["n_leaves"]
        assert np.array_equal(ls[base:base + k + 1], r["leaf_start"] + b)
        assert np.array_equal(perm[b:e], r["perm"] + b)
        assert np.array_equal(s4[b:e].view(np.int32), r["sorted4"].view(np.int32))
        assert np.array_equal(qb[base:base + k], r["leaf_qbox"])
        scale = L / 2.0 ** 21
        o_ref = (r["leaf_qbox"][:, :3].astype(np.float64) * scale).astype(np.float32)
        assert np.array_equal(org[base:base + k, :3].view(np.int32), o_ref.view(np.int32))
        for l in range(k):
            assert np.all(cell_of[perm[ls[base + l]:ls[base + l + 1]]] == base + l)
        t_ref = oracle.tasks(r["leaf_start"].astype(np.int32), sr.split_T)
        t_got = tasks[tbase:tbase + t_ref.shape[0]]
        assert np.array_equal(t_got[:, 0], t_ref[:, 0] + base)
        assert np.array_equal(t_got[:, 1:3], t_ref[:, 1:3] + b) and np.all(t_got[:, 3] == v)
        tbase += t_ref.shape[0]
        tg = None if list_targets is None else np.unique(
            np.random.default_rng(v).choice(k, min(k, list_targets), replace=False))
        roff, rleaf, rsh = oracle.rcb_lists(r["leaf_qbox"], L, RC, tg)
        if tg is None:
            size = np.diff(r["leaf_start"].astype(np.int64))
            pairs += int(sum(size[l] * size[rleaf[roff[l]:roff[l + 1]]].sum() for l in range(k)))
        leaves = range(k) if tg is None else tg
        for t, l in enumerate(leaves):
            g0, g1 = off[base + l], off[base + l + 1]
            assert g1 - g0 == roff[t + 1] - roff[t], (v, l)
            assert np.array_equal(nbr[g0:g1], rleaf[roff[t]:roff[t + 1]] + base)
            assert np.array_equal(shf[g0:g1], rsh[roff[t]:roff[t + 1]])
        base += k
    assert base == nl and tbase == nt
    if list_targets is None:
        assert sr.pair_count() == pairs


@pytest.mark.parametrize("case,leaf_max", [("uniform", 64), ("uniform", 1), ("clustered", 32), ("clustered", 7)])
def test_tree_and_lists_bit_exact(torch, hs, case, leaf_max):
    if case == "uniform":
        w = uniform_box(4096 if leaf_max > 1 else 600, 16.0, seed=1)
    else:
        w = clustered_box(20, 4, seed=21)
    sr, _, _ = build(torch, hs, w, leaf_max=leaf_max)
    check_tree_bit_exact(sr, w, leaf_max)


def test_batched_volumes_with_empty_tiny_and_coincident(torch, hs):
    """Empty volumes, a volume that is one leaf, a volume of coincident points
    (groups whose box is a point are halved by position), and ordinary ones."""
    rng = np.random.default_rng(3)
    u = lambda n, L: [(rng.random(n) * L).astype(np.float32) for _ in range(3)]
    same = [np.full(150, 4.25, np.float32)] * 3
    parts = [u(0, 10.0), u(5, 10.0), u(700, 11.0), same, u(0, 9.0), u(1500, 14.5)]
    w = concat(parts, [10.0, 10.0, 11.0, 9.0, 9.0, 14.5], "batched_edge")
    sr, _, _ = build(torch, hs, w, leaf_max=16)
    check_tree_bit_exact(sr, w, 16)
    root = sr.root.cpu().numpy()
    assert root[0] == np.iinfo(np.int32).min and root[4] == np.iinfo(np.int32).min
    assert root[1] == -1 - 0  # one leaf: the second volume's five particles form leaf 0


def test_depth_cap_gives_large_leaves_split_into_tasks(torch, hs):
    """max_depth 2: at most 4 leaves per volume, each cut into tasks of split_T."""
    w = uniform_box(3000, 16.0, seed=4)
    prm = params(hs)
    sr, pos, m = build(torch, hs, w, leaf_max=8, max_depth=2, split_T=32)
    check_tree_bit_exact(sr, w, 8, max_depth=2)
    assert int(sr.n_leaves.item()) == 4
    a = sr.force(prm)
    torch.cuda.synchronize()
    sr.check_status()
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, 16.0, EPS, RC, prm.c.astype(np.float64))
    rms, mx = err_norms(a.cpu().numpy().T, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


@pytest.mark.parametrize("case", ["uniform", "clustered"])
def test_force_potential_adjoint_on_tree_leaves(torch, hs, case):
    w = uniform_box(4096, 16.0, seed=1) if case == "uniform" else clustered_box(20, 4, seed=21)
    rng = np.random.default_rng(8)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    prm = params(hs)
    sr, pos, m = build(torch, hs, w, leaf_max=48, split_T=64)
    a = sr.force(prm)
    phi = sr.potential(prm)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    g, gm = sr.adjoint(prm, torch.tensor(lam.T.copy(), device="cuda"))
    torch.cuda.synchronize()
    sr.check_status()
    L = float(w.L[0])
    c64 = prm.c.astype(np.float64)
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, L, EPS, RC, c64)
    rms, mx = err_norms(a.cpu().numpy().T, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    pref = oracle.sr_potential(w.x, w.y, w.z, w.m, L, EPS, RC, c64)
    got = phi.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - pref) / np.linalg.norm(pref) < RMS_TOL
    tg = rng.choice(w.N, 256, replace=False)
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, L, EPS, RC, c64, lam, tg)
    rms, _ = err_norms(g.cpu().numpy().T[tg], rg)
    assert rms < RMS_TOL, rms
    assert np.linalg.norm(gm.cpu().numpy()[tg] - rgm) / np.linalg.norm(rgm) < RMS_TOL
    # the pair kernels found the oracle's pairs inside the cutoff (up to pairs whose s
    # sits within float32 rounding of r_c^2)
    got, want = sr.pairs_within_cutoff(prm), oracle.pair_count(w.x, w.y, w.z, L, RC)
    assert abs(got - want) <= max(2, want // 1_000_000), (got, want)


def test_same_forces_as_chaining_mesh(torch, hs):
    """The two list builders visit different candidates but the same pairs
    inside the cutoff: forces agree to float32 rounding."""
    w = clustered_box(24, 6, seed=5)
    prm = params(hs)
    sr, pos, m = build(torch, hs, w, leaf_max=64)
    a_t = sr.force(prm)
    mesh = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    mesh.prepare(pos, m)
    a_m = mesh.force(prm)
    torch.cuda.synchronize()
    sr.check_status()
    mesh.check_status()
    rms, mx = err_norms(a_t.cpu().numpy().T, a_m.cpu().numpy().T.astype(np.float64))
    # two float32 sums of the same pairs in different orders: each within the oracle tolerances
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    t, mm = sr.pairs_within_cutoff(prm), mesh.pairs_within_cutoff(prm)
    assert abs(t - mm) <= max(2, mm // 1_000_000), (t, mm)


def test_rebuild_on_moved_particles_is_reproducible(torch, hs):
    """Two builds of the same input give identical arrays (no leftovers of a
    previous, different tree leak into the next)."""
    w1 = clustered_box(16, 3, seed=6)
    w2 = clustered_box(16, 3, seed=7)
    sr, _, _ = build(torch, hs, w1, leaf_max=32)
    first = (sr.perm.clone(), sr.sorted4.clone(), sr.nbr_cell[:sr.n_entries].clone())
    pos2 = torch.tensor(np.stack([w2.x, w2.y, w2.z]), device="cuda")
    sr.prepare(pos2, torch.tensor(w2.m, device="cuda"))
    pos1 = torch.tensor(np.stack([w1.x, w1.y, w1.z]), device="cuda")
    sr.prepare(pos1, torch.tensor(w1.m, device="cuda"))
    torch.cuda.synchronize()
    sr.check_status()
    assert torch.equal(first[0], sr.perm) and torch.equal(first[1], sr.sorted4)
    assert torch.equal(first[2], sr.nbr_cell[:sr.n_entries])


def test_tree_capacity_overflow_is_flagged_not_written_past(torch, hs):
    """A leaf capacity far below the leaf count: the build flags
    HACC_STATUS_CAPACITY, writes nothing past the arrays, and prepare()
    raises before any walk of the incomplete tree."""
    w = uniform_box(3000, 14.0, seed=13)
    sr = hs.ShortRange(w.L, w.vol_off, RC, builder="rcb", leaf_max=8)
    sentinel = torch.full((64,), -7, dtype=torch.int32, device="cuda")
    sr.leaf_start = torch.cat([sr.leaf_start[:11], sentinel])  # room for 10 leaves, then a guard band
    sr.tree.leaf_start = sr.leaf_start.data_ptr()
    sr.tree.leaf_cap = 10
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    with pytest.raises(hs.HaccError):
        sr.prepare(pos, torch.tensor(w.m, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(sr.leaf_start[11:], sentinel)
    assert int(sr.n_leaves.item()) == 10

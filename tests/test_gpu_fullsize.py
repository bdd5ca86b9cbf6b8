"""Full-size parity in the launch configuration the benchmark times.

At the benchmark sizes the O(N^2) oracle is too slow for every particle, so
forces and adjoints are compared on seeded samples (random particles plus
particles of the most crowded cells, chosen from the oracle's own binning);
binning, lists and tasks are compared bit for bit in full (their oracles are
linear in N); and properties that hold at any size are checked on every
particle: Newton's third law for forces, and zero net position gradient
(translation invariance) for the adjoint.
"""

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda, sample_targets
from synth import default_coeffs, make_config

pytestmark = pytest.mark.gpu


def _tuned(config):
    from paper_1211_4864_gb300 import autotune
    return (autotune.cached(config), autotune.cached_split(config, 64), autotune.cached(config, "adjoint"),
            autotune.cached(config, "symmetric"), autotune.cached(config, "adjoint_symmetric"))


def _setup(config):
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    w = make_config(config)
    launch, T, launch_adj, launch_sym, launch_adj_sym = _tuned(config)
    prm = hs.SRParams(w.eps, w.rcut, default_coeffs(w.rcut, w.eps))
    sr = hs.ShortRange(w.L, w.vol_off, w.rcut, cell_min=w.cell_min, split_T=T)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    a = sr.force(prm, launch=launch)
    torch.cuda.synchronize()
    sr.check_status()
    return dict(torch=torch, hs=hs, w=w, prm=prm, sr=sr, pos=pos, m=m, a=a, launch=launch, launch_adj=launch_adj,
                launch_sym=launch_sym, launch_adj_sym=launch_adj_sym)


@pytest.fixture(scope="module")
def clustered():
    return _setup("clustered256")


def _bin_bit_exact(ctx, v=0):
    w, sr = ctx["w"], ctx["sr"]
    b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
    ob = oracle.bin_volume(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), w.cell_min)
    base = int(ctx["table_base"][v]) if "table_base" in ctx else 0
    n3 = ob["n"] ** 3
    assert np.array_equal(sr.cell_start.cpu().numpy()[base:base + n3 + 1], ob["cell_start"] + b)
    assert np.array_equal(sr.perm.cpu().numpy()[b:e], ob["perm"] + b)
    assert np.array_equal(sr.sorted4.cpu().numpy()[b:e].view(np.int32), ob["sorted4"].view(np.int32))
    return ob


def test_clustered256_binning_lists_tasks_bit_exact(clustered):
    ob = _bin_bit_exact(clustered)
    sr = clustered["sr"]
    off, cell, sh = oracle.lists_volume(ob["n"], ob["w"], 3.0)
    assert np.array_equal(sr.nbr_off.cpu().numpy(), off)
    assert np.array_equal(sr.nbr_cell.cpu().numpy(), cell)
    assert np.array_equal(sr.nbr_shift.cpu().numpy(), sh)
    t = oracle.tasks(ob["cell_start"], sr.split_T)
    nt = int(sr.n_tasks.item())
    assert nt == t.shape[0]
    assert np.array_equal(sr.tasks.cpu().numpy()[:nt, :3], t)


def test_clustered256_forces_sampled(clustered):
    w, prm = clustered["w"], clustered["prm"]
    ob = oracle.bin_volume(w.x, w.y, w.z, w.m, float(w.L[0]), w.cell_min)
    tg = sample_targets(ob["cell_start"], ob["perm"], w.N, 384, crowded_cells=32, per_cell=4, seed=3)
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut, prm.c.astype(np.float64), tg)
    got = clustered["a"].cpu().numpy().T[tg].astype(np.float64)
    rms, mx = err_norms(got, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_clustered256_symmetric_kernel_sampled_and_against_gather(clustered):
    """The Newton-III symmetric kernel in the benchmark's launch shape: every
    particle against the gather kernel, samples against the oracle, zero net
    force."""
    torch, w, prm, sr = clustered["torch"], clustered["w"], clustered["prm"], clustered["sr"]
    s = sr.force_symmetric(prm, launch=clustered["launch_sym"])
    mom = sr.moments(clustered["m"], None, s).cpu().numpy()
    torch.cuda.synchronize()
    sr.check_status()
    S = s.cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(S, clustered["a"].cpu().numpy().T.astype(np.float64))
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    ob = oracle.bin_volume(w.x, w.y, w.z, w.m, float(w.L[0]), w.cell_min)
    tg = sample_targets(ob["cell_start"], ob["perm"], w.N, 256, crowded_cells=16, per_cell=4, seed=8)
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut, prm.c.astype(np.float64), tg)
    rms, mx = err_norms(S[tg], ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    assert np.all(np.abs(mom[3:6]) < 1e-6 * mom[7]), mom


def test_clustered256_newton_third_law(clustered):
    sr, m, a = clustered["sr"], clustered["m"], clustered["a"]
    mom = sr.moments(m, None, a).cpu().numpy()
    assert np.all(np.abs(mom[3:6]) < 1e-6 * mom[7]), mom


def test_clustered256_adjoint_sampled_and_translation_invariant(clustered):
    torch, w, prm, sr = clustered["torch"], clustered["w"], clustered["prm"], clustered["sr"]
    rng = np.random.default_rng(21)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    g, gm = sr.adjoint(prm, torch.tensor(lam.T.copy(), device="cuda"), launch=clustered["launch_adj"])
    torch.cuda.synchronize()
    sr.check_status()
    G = g.cpu().numpy().T.astype(np.float64)
    # every particle: the position gradient of a translation-invariant loss sums to zero
    assert np.linalg.norm(G.sum(0)) < 1e-6 * np.abs(G).sum()
    tg = rng.choice(w.N, 128, replace=False)
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut,
                                      prm.c.astype(np.float64), lam, tg)
    rms, _ = err_norms(G[tg], rg)
    assert rms < RMS_TOL, rms
    assert np.linalg.norm(gm.cpu().numpy()[tg] - rgm) / np.linalg.norm(rgm) < RMS_TOL


def test_clustered256_symmetric_adjoint_sampled_and_against_gather(clustered):
    """The symmetric adjoint in the benchmark's launch shape: every particle
    against the gather adjoint, samples against the oracle, zero net
    position gradient."""
    torch, w, prm, sr = clustered["torch"], clustered["w"], clustered["prm"], clustered["sr"]
    rng = np.random.default_rng(23)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    lt = torch.tensor(lam.T.copy(), device="cuda")
    gs, gms = sr.adjoint_symmetric(prm, lt, launch=clustered["launch_adj_sym"])
    gg, gmg = sr.adjoint(prm, lt, launch=clustered["launch_adj"])
    torch.cuda.synchronize()
    sr.check_status()
    S, G = gs.cpu().numpy().T.astype(np.float64), gg.cpu().numpy().T.astype(np.float64)
    assert np.linalg.norm(S.sum(0)) < 1e-6 * np.abs(S).sum()
    rms, _ = err_norms(S, G)
    assert rms < RMS_TOL, rms
    tg = rng.choice(w.N, 128, replace=False)
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut,
                                      prm.c.astype(np.float64), lam, tg)
    rms, _ = err_norms(S[tg], rg)
    assert rms < RMS_TOL, rms
    assert np.linalg.norm(gms.cpu().numpy()[tg] - rgm) / np.linalg.norm(rgm) < RMS_TOL


def test_lattice128_forces_sampled_and_kick():
    ctx = _setup("lattice128")
    w, prm, sr, torch = ctx["w"], ctx["prm"], ctx["sr"], ctx["torch"]
    _bin_bit_exact(ctx)
    rng = np.random.default_rng(5)
    tg = rng.choice(w.N, 1024, replace=False)
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut, prm.c.astype(np.float64), tg)
    A = ctx["a"].cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(A[tg], ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    v = torch.zeros_like(ctx["a"])
    sr.kick(v, ctx["a"], w.dt)
    torch.cuda.synchronize()
    assert np.allclose(v.cpu().numpy().T[tg], w.dt * A[tg], rtol=1e-6, atol=0)


def test_batched256_sampled_volumes():
    ctx = _setup("batched256")
    w, prm, sr = ctx["w"], ctx["prm"], ctx["sr"]
    ctx["table_base"] = [ctx["sr"].table[v].cell_base for v in range(w.V)]
    A = ctx["a"].cpu().numpy().T.astype(np.float64)
    S = sr.force_symmetric(prm, launch=ctx["launch_sym"])
    ctx["torch"].cuda.synchronize()
    sr.check_status()
    S = S.cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(S, A)  # the symmetric kernel over all 256 volumes against the gather kernel
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    rng = np.random.default_rng(6)
    for v in sorted(set([0, 127, 128, 255]) | set(rng.choice(w.V, 4, replace=False).tolist())):
        _bin_bit_exact(ctx, v)
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        tg = rng.choice(e - b, min(256, e - b), replace=False)
        ref = oracle.sr_force(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), prm.eps, prm.rcut,
                              prm.c.astype(np.float64), tg)
        rms, mx = err_norms(A[b:e][tg], ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)
        rms, mx = err_norms(S[b:e][tg], ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)


def test_clustered256_rcb_tree_bit_exact_and_forces(clustered):
    """The RCB fat-leaf tree of the full clustered workload: tree bit-exact, the
    lists of sampled leaves bit-exact, forces equal to the chaining mesh's to
    float32 rounding on every particle and to the oracle on samples."""
    from test_gpu_rcb import check_tree_bit_exact
    torch, hs, w, prm = clustered["torch"], clustered["hs"], clustered["w"], clustered["prm"]
    tr = hs.ShortRange(w.L, w.vol_off, w.rcut, split_T=64, builder="rcb", leaf_max=64)
    tr.prepare(clustered["pos"], clustered["m"])
    a = tr.force(prm, launch=clustered["launch"])
    torch.cuda.synchronize()
    tr.check_status()
    check_tree_bit_exact(tr, w, 64, list_targets=12)
    A, M = a.cpu().numpy().T.astype(np.float64), clustered["a"].cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(A, M)
    # two float32 sums of the same pairs in different orders: each within the oracle tolerances
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    rng = np.random.default_rng(11)
    tg = rng.choice(w.N, 128, replace=False)
    ref = oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), prm.eps, prm.rcut, prm.c.astype(np.float64), tg)
    rms, mx = err_norms(A[tg], ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


def test_binning_bit_exact_beyond_2_26_particles():
    """More than 2^26 particles (16,385 tiles per counting pass, indices of 27
    bits, 16 million digit counts in each scan): bit-exact against the oracle
    (uniform particles, about one per grid cell cubed)."""
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    N = (1 << 26) + 4099
    L = np.float32(np.ceil(N ** (1.0 / 3.0)))
    rng = np.random.default_rng(26)
    x = (rng.random(N, dtype=np.float32) * L).astype(np.float32)
    y = (rng.random(N, dtype=np.float32) * L).astype(np.float32)
    z = (rng.random(N, dtype=np.float32) * L).astype(np.float32)
    m = np.ones(N, np.float32)
    sr = hs.ShortRange(np.array([L], np.float32), np.array([0, N], np.int64), 3.0)
    sr.bin(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"), torch.tensor(z, device="cuda"),
           torch.tensor(m, device="cuda"))
    torch.cuda.synchronize()
    sr.check_status()
    ob = oracle.bin_volume(x, y, z, m, float(L), 3.0)
    assert np.array_equal(sr.cell_of.cpu().numpy(), ob["cell_of"])
    assert np.array_equal(sr.cell_start.cpu().numpy(), ob["cell_start"])
    assert np.array_equal(sr.perm.cpu().numpy(), ob["perm"])
    assert np.array_equal(sr.sorted4.cpu().numpy().view(np.int32), ob["sorted4"].view(np.int32))

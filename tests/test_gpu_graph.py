"""Batched sub-volumes in one CUDA-graph replay: binning + lists + force +
kick of many independent periodic volumes captured once and replayed.  With
the gather kernel the replay must reproduce the eager calls bit for bit
(every kernel is deterministic: each particle's sum is owned by one warp in a
fixed order), also after new positions are copied into the captured input
buffers; with the symmetric kernel, to float32 rounding."""

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs
from synth.workloads import batched_volumes

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager_and_oracle():
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    w = batched_volumes(16, n_lo=800, n_hi=20000, seed=6)
    prm = hs.SRParams(0.01, 3.0, default_coeffs())
    sr = hs.ShortRange(w.L, w.vol_off, 3.0, split_T=64)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    a = torch.empty_like(pos)
    v = torch.zeros_like(pos)

    def step():
        sr.prepare(pos, m)
        sr.force(prm, a)
        sr.kick(v, a, 0.01)

    # eager reference
    step()
    torch.cuda.synchronize()
    sr.check_status()
    a_eager, v_eager = a.clone(), v.clone()

    # capture (after the eager warm-up on the same buffers)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        v.zero_()
        with torch.cuda.graph(g, stream=s):
            step()
    torch.cuda.current_stream().wait_stream(s)
    v.zero_()
    a.zero_()
    g.replay()
    torch.cuda.synchronize()
    sr.check_status()
    assert torch.equal(a, a_eager)
    assert torch.equal(v, v_eager)

    # new positions through the same graph
    rng = np.random.default_rng(9)
    shift = torch.tensor(rng.uniform(0, 1, (3, 1)).astype(np.float32), device="cuda")
    pos.add_(shift)
    v.zero_()
    g.replay()
    torch.cuda.synchronize()
    sr.check_status()
    a_graph2 = a.clone()
    v.zero_()
    step()
    torch.cuda.synchronize()
    assert torch.equal(a_graph2, a)
    # and the replayed forces still match the oracle, volume by volume (sampled)
    P = pos.cpu().numpy()
    A = a_graph2.cpu().numpy().T.astype(np.float64)
    for vol in (0, 7, 15):
        b, e = int(w.vol_off[vol]), int(w.vol_off[vol + 1])
        Lv = float(w.L[vol])
        ref = oracle.sr_force(P[0, b:e], P[1, b:e], P[2, b:e], w.m[b:e], Lv, 0.01, 3.0,
                              prm.c.astype(np.float64))
        rms, mx = err_norms(A[b:e], ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (vol, rms, mx)


def test_graph_replay_of_the_symmetric_step():
    """The benchmark's batched step (symmetric force, 128-particle tasks) in one
    CUDA-graph replay: the float64 atomics make it reproducible only to
    rounding, so the replay is compared with the eager step at float32
    rounding and with the oracle at the parity tolerances."""
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    w = batched_volumes(16, n_lo=800, n_hi=20000, seed=8)
    prm = hs.SRParams(0.01, 3.0, default_coeffs())
    sr = hs.ShortRange(w.L, w.vol_off, 3.0, split_T=128)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    a = torch.empty_like(pos)
    v = torch.zeros_like(pos)

    def step():
        sr.prepare(pos, m)
        sr.force_symmetric(prm, a)
        sr.kick(v, a, 0.01)

    step()
    torch.cuda.synchronize()
    sr.check_status()
    a_eager = a.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step()
    torch.cuda.current_stream().wait_stream(s)
    a.zero_()
    g.replay()
    torch.cuda.synchronize()
    sr.check_status()
    A = a.cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(A, a_eager.cpu().numpy().T.astype(np.float64))
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    for vol in (0, 9, 15):
        b, e = int(w.vol_off[vol]), int(w.vol_off[vol + 1])
        ref = oracle.sr_force(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[vol]), 0.01, 3.0,
                              prm.c.astype(np.float64))
        rms, mx = err_norms(A[b:e], ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (vol, rms, mx)

"""Gradient parity of the differentiation workload at its own size.

64^3 = 262,144 clustered particles (60 % uniform, 40 % in 100 NFW halos, seed
4) in a box of 64 grid units, four kick-drift steps of dt = 0.01 from rest,
loss sum_i w_i . (x_4,i - x_0,i)^2 with w seeded N(0, 1) (seed 40).  The GPU
gradient through the hand-written adjoints (both kernel pairs, via
torch.autograd) is compared with the float64 reference gradient of the
oracle, a brute-force O(N^2) computation of every force and adjoint of the
trajectory (about 8e11 float64 pair evaluations: minutes on the host cores).
"""

import numpy as np
import pytest

from gpu_util import need_cuda
from oracle import diff
from synth import default_coeffs, make_config

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GRAD_RMS_TOL = 1e-5  # GPU float32 gradient vs float64 reference gradient


@pytest.fixture(scope="module")
def workload():
    w = make_config("diff64")
    c = default_coeffs(w.rcut, w.eps)
    x0 = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    v0 = np.zeros_like(x0)
    wt = w.extra["loss_w"].astype(np.float64)
    return w, c, x0, v0, wt


@pytest.fixture(scope="module")
def gpu_grads(workload):
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    w, c, x0, v0, wt = workload
    prm = hs.SRParams(w.eps, w.rcut, c)
    sr = hs.ShortRange(w.L, w.vol_off, w.rcut, split_T=64)
    out = {}
    for sym in (False, True):
        xt = torch.tensor(x0.T.astype(np.float32), device="cuda", requires_grad=True)
        vt = torch.tensor(v0.T.astype(np.float32), device="cuda", requires_grad=True)
        mt = torch.tensor(w.m, device="cuda", requires_grad=True)
        disp, _ = hs.trajectory_autograd(xt, vt, mt, sr, prm, w.dt, int(w.extra["steps"]), symmetric=sym)
        wt_t = torch.tensor(wt.T.astype(np.float32), device="cuda")
        loss = (wt_t * disp * disp).sum()
        loss.backward()
        torch.cuda.synchronize()
        sr.check_status()
        out["symmetric" if sym else "gather"] = (
            float(loss.item()), xt.grad.cpu().numpy().T.astype(np.float64),
            vt.grad.cpu().numpy().T.astype(np.float64), mt.grad.cpu().numpy().astype(np.float64))
    return out


@pytest.fixture(scope="module")
def reference(workload):
    w, c, x0, v0, wt = workload
    m = w.m.astype(np.float64)
    L = float(w.L[0])
    steps = int(w.extra["steps"])
    g = diff.gradient(x0, v0, m, L, w.eps, w.rcut, c.astype(np.float64), w.dt, steps, wt)
    xs, _ = diff.trajectory(x0, v0, m, L, w.eps, w.rcut, c.astype(np.float64), w.dt, steps)
    dx = xs[-1] - xs[0]
    return float(np.sum(wt * dx * dx)), g


@pytest.mark.parametrize("pair", ["gather", "symmetric"])
def test_diff64_loss_and_gradient_against_float64_reference(gpu_grads, reference, pair):
    ref_loss, (rx, rv, rm) = reference
    loss, gx, gv, gm = gpu_grads[pair]
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for name, g, r in (("dL/dx0", gx, rx), ("dL/dv0", gv, rv), ("dL/dm", gm, rm)):
        rms = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert rms < GRAD_RMS_TOL, (pair, name, rms)

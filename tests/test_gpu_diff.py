"""Differentiation: gradients of a four-step short-range trajectory through the
hand-written adjoint (torch.autograd.Function over the C ABI) against the
float64 oracle's reference gradient and float64 finite differences, with the
gather kernels and with the Newton-III symmetric kernels.

Loss: sum_i w_i . (x_S,i - x_0,i)^2 over S kick-drift steps of dt (the kick
and stream maps of the paper's split-operator step, Eq. 6), w seeded N(0, 1).
"""

import numpy as np
import pytest

import oracle
from gpu_util import need_cuda
from oracle import diff
from synth import default_coeffs
from synth.workloads import clustered_box

pytestmark = pytest.mark.gpu

EPS, RC, DT, STEPS = 0.01, 3.0, 0.01, 4
GRAD_RMS_TOL = 1e-5    # GPU float32 gradient vs float64 reference gradient
FD_REL_TOL = 1e-3      # GPU float32 gradient vs float64 finite differences


@pytest.fixture(scope="module", params=[False, True], ids=["gather", "symmetric"])
def case(request):
    torch = need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    w = clustered_box(16, 3, seed=4)
    rng = np.random.default_rng(40)
    wt = rng.normal(size=(w.N, 3))
    v0 = (rng.normal(size=(w.N, 3)) * 0.1).astype(np.float32)
    c = default_coeffs(RC, EPS)
    prm = hs.SRParams(EPS, RC, c)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    x0 = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda", requires_grad=True)
    vt = torch.tensor(v0.T.copy(), device="cuda", requires_grad=True)
    mt = torch.tensor(w.m, device="cuda", requires_grad=True)
    disp, v = hs.trajectory_autograd(x0, vt, mt, sr, prm, DT, STEPS, symmetric=request.param)
    wt_t = torch.tensor(wt.T.astype(np.float32), device="cuda")
    loss = (wt_t * disp * disp).sum()
    loss.backward()
    torch.cuda.synchronize()
    sr.check_status()
    x0_np = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    ref = diff.gradient(x0_np, v0.astype(np.float64), w.m.astype(np.float64), float(w.L[0]), EPS, RC,
                        c.astype(np.float64), DT, STEPS, wt)
    got = (x0.grad.cpu().numpy().T.astype(np.float64), vt.grad.cpu().numpy().T.astype(np.float64),
           mt.grad.cpu().numpy().astype(np.float64))
    ref_loss = diff.loss(x0_np, v0.astype(np.float64), w.m.astype(np.float64), float(w.L[0]), EPS, RC,
                         c.astype(np.float64), DT, STEPS, wt)
    return dict(w=w, wt=wt, v0=v0, c=c, got=got, ref=ref, loss=float(loss.item()), ref_loss=ref_loss,
                x0=x0_np)


def test_loss_matches_float64_trajectory(case):
    assert case["loss"] == pytest.approx(case["ref_loss"], rel=1e-5)


@pytest.mark.parametrize("k,name", [(0, "dL/dx0"), (1, "dL/dv0"), (2, "dL/dm")])
def test_gradient_against_float64_reference(case, k, name):
    g, r = case["got"][k], case["ref"][k]
    rms = np.linalg.norm(g - r) / np.linalg.norm(r)
    assert rms < GRAD_RMS_TOL, (name, rms)


def test_gradient_against_finite_differences(case):
    """Central differences of the float64 loss on a few coordinates (h chosen
    where the loss is smooth: no pair of the sampled particle within h of r_c)."""
    w, wt, v0, c, x0 = case["w"], case["wt"], case["v0"], case["c"], case["x0"]
    gx, gv, gm = case["got"]
    L = float(w.L[0])
    m = w.m.astype(np.float64)
    rng = np.random.default_rng(7)
    checked = 0
    for i in rng.choice(w.N, 12, replace=False):
        d = x0 - x0[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        if np.any(np.abs(r - RC) < 5e-3):
            continue
        for axis in range(3):
            fd = diff.finite_difference(x0, v0.astype(np.float64), m, L, EPS, RC, c.astype(np.float64), DT,
                                        STEPS, wt, "x", (i, axis), 1e-4)
            assert gx[i, axis] == pytest.approx(fd, rel=FD_REL_TOL, abs=1e-6 * np.abs(gx).max())
            fdv = diff.finite_difference(x0, v0.astype(np.float64), m, L, EPS, RC, c.astype(np.float64), DT,
                                         STEPS, wt, "v", (i, axis), 1e-4)
            assert gv[i, axis] == pytest.approx(fdv, rel=FD_REL_TOL, abs=1e-6 * np.abs(gv).max())
        checked += 1
        if checked == 4:
            break
    assert checked >= 2

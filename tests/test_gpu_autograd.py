"""dJ/dgamma through torch.autograd (LKSObjective over the C ABI) against the oracle, torch's
gradcheck, and central finite differences of the GPU FP64 path (eps = 1e-4, as the paper's
Sec. 2.6 verification does) at seeded design cells."""
import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2506_23895_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2506_23895_gb300 import autograd, lks
    return torch, lks, autograd


def _clamped(w, lo=0.05, hi=0.95):
    return np.clip(w.gamma, lo, hi)


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_backward_matches_oracle_gradient(T, name):
    torch, lks, ag = T
    w = W.small_channel2d() if name == "2d" else W.small_duct3d()
    gam = _clamped(w)
    Jo, go = oracle.gradient(w.problem, gam, w.motion)
    s = lks.Solver(w.problem, lks.FP64)
    s.set_motion(w.motion)
    g = torch.tensor(gam, device="cuda", requires_grad=True)
    J = ag.objective(g, s)
    J.backward()
    assert abs(J.item() - Jo) <= 1e-11 * abs(Jo)
    gg = g.grad.cpu().numpy()
    assert np.max(np.abs(gg - go)) <= 1e-11 * np.max(np.abs(go))
    # a second differentiation of the same solver (new forward, new adjoint)
    g2 = torch.tensor(gam * 0.9, device="cuda", requires_grad=True)
    (2.0 * ag.objective(g2, s)).backward()
    Jo2, go2 = oracle.gradient(w.problem, gam * 0.9, w.motion)
    assert np.max(np.abs(g2.grad.cpu().numpy() - 2.0 * go2)) <= 2e-11 * np.max(np.abs(go2))
    s.close()


def test_gradcheck_fp64(T):
    torch, lks, ag = T
    w = W.small_channel2d(nx=20, ny=16, LD=5, n_steps=24)
    s = lks.Solver(w.problem, lks.FP64)
    s.set_motion(w.motion)
    g = torch.tensor(_clamped(w, 0.1, 0.9), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: ag.objective(x, s), (g,), eps=1e-6, atol=1e-9,
                                    rtol=1e-5)
    s.close()


def test_central_differences_at_seeded_cells(T):
    """GPU FP64 adjoint vs central FD (eps = 1e-4) at 16 seeded cells with gamma in [0.2, 0.8]
    among the largest sensitivities, on a 128^2 channel with a 48^2 rotating design (the
    workload-0 geometry, 400 steps)."""
    torch, lks, ag = T
    w = W.config(0, n_steps=400)
    s = lks.Solver(w.problem, lks.FP64)
    s.set_motion(w.motion)
    s.set_design(w.gamma)
    s.forward()
    g = s.adjoint()
    flat = g.reshape(-1)
    gam = w.gamma.reshape(-1)
    thr = np.quantile(np.abs(flat), 0.99)
    cand = np.where((gam > 0.2) & (gam < 0.8) & (np.abs(flat) >= thr))[0]
    cells = np.random.default_rng(16).choice(cand, size=min(16, cand.size), replace=False)
    assert cells.size >= 8
    eps = 1e-4
    for c in cells:
        gp = gam.copy()
        gm = gam.copy()
        gp[c] += eps
        gm[c] -= eps
        s.set_design(gp.reshape(g.shape))
        Jp = s.forward()
        s.set_design(gm.reshape(g.shape))
        Jm = s.forward()
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - flat[c]) <= 1e-4 * abs(flat[c]) + 1e-12 * np.abs(flat).max()
    s.close()
    # the FP32 path's gradient against the FP64 one on the same problem
    s32 = lks.Solver(w.problem, lks.FP32)
    s32.set_motion(w.motion)
    s32.set_design(w.gamma)
    J32 = s32.forward()
    g32 = s32.adjoint()
    s32.close()
    assert np.linalg.norm(g32 - g) <= 1e-4 * np.linalg.norm(g)


def test_central_differences_on_the_512_channel_geometry(T):
    """Workload 1's geometry: a 512^2 channel with a 192^2 design that rotates and translates
    sinusoidally (amplitude 20 cells, period 2000 steps), here over one full translation period
    (2000 steps, J1 over the last 200).  dJ/dgamma through torch.autograd with a snapshot budget
    that forces binomial checkpointing with recomputation, against central differences
    (eps = 1e-4, Sec. 2.6) of the GPU FP64 path at 16 seeded cells with gamma in [0.2, 0.8]
    among the largest sensitivities; then the FP32 path against FP64 within the stated
    tolerances (1e-5 on J, 1e-4 relative L2 on dJ/dgamma)."""
    torch, lks, ag = T
    w = W.config(1, n_steps=2000)
    p = w.problem
    state_bytes = p.nodes * 32
    s = lks.Solver(p, lks.FP64, ckpt_bytes=60 * state_bytes)
    s.set_motion(w.motion)
    gam = torch.tensor(w.gamma, device="cuda", requires_grad=True)
    J = ag.objective(gam, s)
    J.backward()
    st = s.stats()
    assert st["recomputed_steps"] > 0
    g = gam.grad.cpu().numpy()
    flat = g.reshape(-1)
    gflat = w.gamma.reshape(-1)
    thr = np.quantile(np.abs(flat), 0.99)
    cand = np.where((gflat > 0.2) & (gflat < 0.8) & (np.abs(flat) >= thr))[0]
    cells = np.random.default_rng(1).choice(cand, size=min(16, cand.size), replace=False)
    assert cells.size == 16
    eps = 1e-4
    for c in cells:
        gp = gflat.copy()
        gm = gflat.copy()
        gp[c] += eps
        gm[c] -= eps
        s.set_design(gp.reshape(w.gamma.shape))
        Jp = s.forward()
        s.set_design(gm.reshape(w.gamma.shape))
        Jm = s.forward()
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - flat[c]) <= 1e-4 * abs(flat[c]) + 1e-12 * np.abs(flat).max()
    s.close()
    s32 = lks.Solver(p, lks.FP32, ckpt_bytes=60 * p.nodes * 16)
    s32.set_motion(w.motion)
    s32.set_design(w.gamma)
    J32 = s32.forward()
    g32 = s32.adjoint()
    s32.close()
    assert abs(J32 - J.item()) <= 1e-5 * abs(J.item())
    assert np.linalg.norm(g32 - g) <= 1e-4 * np.linalg.norm(g)


def test_fp32_against_fp64_over_long_horizons(T):
    """The FP32 path against the plain FP64 GPU path (which matches the oracle to 1e-11) on the
    benchmark's 256^3 duct over 2000 steps (J over the last 200) and on the 512^2 channel over
    its full 20000 steps: J within 1e-5 relative and dJ/dgamma within 1e-4 relative L2.  With
    single-precision weights that break the lattice identities (a per-step velocity gain of
    3e-8) the duct's J error is 6e-5 at 2000 steps and the channel's gradient error 3e-4."""
    torch, lks, ag = T
    for w in (W.config(4, n_steps=2000), W.config(1)):
        res = {}
        for prec in (lks.FP64, lks.FP32):
            s = lks.Solver(w.problem, prec)
            s.set_motion(w.motion)
            s.set_design(w.gamma)
            res[prec] = (s.forward(), s.adjoint())
            s.close()
        (J64, g64), (J32, g32) = res[lks.FP64], res[lks.FP32]
        assert abs(J32 - J64) <= 1e-5 * abs(J64), w.problem.name
        assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64), w.problem.name

"""The adjoint of Sec. 2.4 as printed (LKS_FLAG_PAPER_ALKS) against the oracle's restatement of
the same variant, and its gap to the exact discrete adjoint and to central differences on the
128^2 channel geometry (the paper reports that its adjoint and finite differences "agree
fairly", Sec. 2.6)."""
import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2506_23895_gb300 import build as B
    B.build()
    import torch
    assert torch.cuda.is_available()
    from paper_2506_23895_gb300 import lks
    return lks


def _grad(L, w, flags):
    s = L.Solver(w.problem, L.FP64, flags=flags)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    J = s.forward()
    g = s.adjoint()
    s.close()
    return J, g


@pytest.mark.parametrize("name", ["2d_J1", "3d_J2"])
def test_printed_variant_matches_oracle(L, name):
    w = W.small_channel2d() if name == "2d_J1" else W.small_duct3d()
    Jo, go = oracle.gradient_printed(w.problem, w.gamma, w.motion)
    J, g = _grad(L, w, L.FLAG_PAPER_ALKS)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert np.max(np.abs(g - go)) <= 1e-11 * np.max(np.abs(go))


def test_printed_variant_gap_to_exact_and_finite_differences(L):
    w = W.config(0, n_steps=400)
    _, ge = _grad(L, w, 0)
    _, gp = _grad(L, w, L.FLAG_PAPER_ALKS)
    gap = np.linalg.norm(gp - ge) / np.linalg.norm(ge)
    cos = float((gp * ge).sum() / np.linalg.norm(gp) / np.linalg.norm(ge))
    assert 0.05 < gap < 0.8 and cos > 0.8      # "agree fairly", not exactly
    # central differences side with the exact adjoint
    s = L.Solver(w.problem, L.FP64)
    s.set_motion(w.motion)
    flat_e, flat_p, gam = ge.reshape(-1), gp.reshape(-1), w.gamma.reshape(-1)
    cand = np.where((gam > 0.2) & (gam < 0.8) &
                    (np.abs(flat_e) >= np.quantile(np.abs(flat_e), 0.99)))[0]
    cells = np.random.default_rng(7).choice(cand, size=min(6, cand.size), replace=False)
    err_e, err_p = [], []
    for c in cells:
        Js = []
        for sgn in (1, -1):
            gg = gam.copy()
            gg[c] += sgn * 1e-4
            s.set_design(gg.reshape(ge.shape))
            Js.append(s.forward())
        fd = (Js[0] - Js[1]) / 2e-4
        err_e.append(abs(fd - flat_e[c]) / abs(fd))
        err_p.append(abs(fd - flat_p[c]) / abs(fd))
    s.close()
    assert max(err_e) < 1e-4
    assert np.median(err_p) > 10 * max(err_e)

"""The design chain on the GPU (lks_set_filter, lks_volume) against the oracle: the solver sees
H(F gamma) and lks_adjoint returns dJ/dgamma through the projection and the transposed
filter; the volume constraint G and its gradient."""
import numpy as np
import pytest

import oracle
from oracle import design_chain as D
from paper_2506_23895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2506_23895_gb300 import build as B
    B.build()
    from paper_2506_23895_gb300 import lks
    import torch
    assert torch.cuda.is_available()
    return lks


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def run(L, w, prec, R, beta):
    s = L.Solver(w.problem, prec)
    s.set_design(w.gamma)
    s.set_filter(R, beta)
    s.set_motion(w.motion)
    J = s.forward()
    g = s.adjoint()
    vol = s.volume(0.4)
    s.close()
    return J, g, vol


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_filtered_gradient_fp64_matches_oracle(L, name):
    w = W.small_channel2d() if name == "2d" else W.small_duct3d()
    R, beta = 2.4, 4.0
    gb = D.physical(w.gamma, R, beta)
    Jo, go_b = oracle.gradient(w.problem, gb, w.motion)
    go = D.chain_T(w.gamma, go_b, R, beta)
    J, g, (G, dG) = run(L, w, L.FP64, R, beta)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert rel_max(g, go) < 1e-11
    Go, dGo = D.volume(w.gamma, 0.4, R, beta)
    assert abs(G - Go) < 1e-12
    assert rel_max(dG, dGo) < 1e-12


@pytest.mark.parametrize("name", ["2d", "3d"])
def test_filtered_gradient_fp32_within_tolerance(L, name):
    w = W.small_channel2d() if name == "2d" else W.small_duct3d()
    R, beta = 2.4, 2.0
    gb = D.physical(w.gamma, R, beta)
    Jo, go_b = oracle.gradient(w.problem, gb, w.motion)
    go = D.chain_T(w.gamma, go_b, R, beta)
    J, g, _ = run(L, w, L.FP32, R, beta)
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4


def test_filter_off_restores_plain_gradient_and_volume(L):
    w = W.small_channel2d()
    s = L.Solver(w.problem, L.FP64)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    s.set_filter(2.4, 8.0)
    s.forward()
    s.set_filter(0.0)
    J = s.forward()
    g = s.adjoint()
    G, dG = s.volume(0.5)
    s.close()
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert rel_max(g, go) < 1e-11
    assert abs(G - (w.gamma.mean() / 0.5 - 1.0)) < 1e-13
    assert np.allclose(dG, 1.0 / (0.5 * w.gamma.size))


def test_filter_argument_checks(L):
    w = W.small_channel2d()
    s = L.Solver(w.problem, L.FP32)
    for args in ((-1.0, 1.0, 0.5), (2.4, 0.0, 0.5), (2.4, 1.0, 1.0)):
        with pytest.raises(L.LksError) as e:
            s.set_filter(*args)
        assert e.value.status == 1
    with pytest.raises(L.LksError) as e:
        s.volume(0.5)
    assert e.value.status == 2
    s.close()

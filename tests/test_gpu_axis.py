"""Rotation about a general 3D axis on the GPU (cell-list transfer) against the oracle."""
import numpy as np
import pytest

import oracle
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


CASES = {
    "tilted_J2": lambda: W.small_duct3d(n_steps=16, rot_axis=W.unit((1.0, 1.0, 3.0)),
                                        omega=0.02, trans_amp=0.5),
    "tilted_J1": lambda: W.small_duct3d(n_steps=14, rot_axis=W.unit((0.0, 1.0, 0.3)),
                                        omega=0.02, trans_amp=0.4, obj_kind=W.OBJ_PRESSURE,
                                        seed=23),
    "ragged": lambda: W.small_duct3d(nx=33, ny=29, nz=31, LD=9, n_steps=12,
                                     rot_axis=W.unit((2.0, -1.0, 2.0)), omega=0.01,
                                     trans_amp=0.8, seed=24),
}


def test_transfer_fp64_matches_oracle(L):
    w = CASES["ragged"]()
    s = L.Solver(w.problem, L.FP64)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    for n in (1, 6, 12):
        k, us = s.transfer(n)
        ko, uso = oracle.transfer(w.problem, w.gamma, w.motion[n])
        assert rel_max(k, ko) < 1e-13
        assert np.max(np.abs(us - uso)) < 1e-13 * max(np.max(np.abs(uso)), 1e-3)
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_forward_adjoint_fp64_match_oracle(L, name):
    w = CASES[name]()
    Jo, fo = oracle.forward(w.problem, w.gamma, w.motion)
    _, go = oracle.gradient(w.problem, w.gamma, w.motion)
    s = L.Solver(w.problem, L.FP64)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    J = s.forward()
    st = s.get_state()
    g = s.adjoint()
    s.close()
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert rel_max(st, fo) < 1e-11
    assert rel_max(g, go) < 1e-11


@pytest.mark.parametrize("name", ["tilted_J2", "ragged"])
def test_fp32_fused_within_tolerance(L, name):
    w = CASES[name]()
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    s = L.Solver(w.problem, L.FP32)
    assert s.kernels == "fused3d"
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    J = s.forward()
    g = s.adjoint()
    s.close()
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4


def test_explicit_z_axis_is_the_default_path_and_bad_axes_are_rejected(L):
    w = W.small_duct3d(n_steps=10)
    res = []
    for axis in ((0.0, 0.0, 1.0), (0.0, 0.0, 0.0)):
        w.problem.rot_axis = axis
        s = L.Solver(w.problem, L.FP32)
        s.set_design(w.gamma)
        s.set_motion(w.motion)
        res.append((s.forward(), s.adjoint()))
        s.close()
    assert res[0][0] == res[1][0] and np.array_equal(res[0][1], res[1][1])
    w.problem.rot_axis = (0.0, 0.6, 0.6)   # not a unit vector
    with pytest.raises(L.LksError):
        L.Solver(w.problem, L.FP32)

"""Pins of the oracle's static solids and warm-started adjoint.

Static solids (the inner wall of the 2D pump, Sec. 3.2, and the fixed outer cylinder of the
appendix's rotating-cylinder check) enter the implicit Brinkman update with solid velocity 0:
u = (u* + kappa u_S) / (1 + kappa + kappa_s).  A warm-started adjoint (state and adjoint
fields reused from the previous optimisation step, Secs. 3.2 and 3.3) is the exact adjoint of
J + <lambda_term, s^N>, which the complex step of that augmented objective pins.
"""
import numpy as np

import oracle
from paper_2506_23895_gb300 import workloads as W


def test_uniform_static_field_damps_uniform_flow_geometrically():
    n = (7, 6, 1)
    p = W.periodic_box(2, n, A=0.3, n_steps=5)
    u = (0.03, -0.02, 0.0)
    s0 = W.initial_state(p, u=[np.full((1, 6, 7), v) for v in u])
    ks = np.full((1, 6, 7), 0.25)
    for N in (1, 4):
        _, fin = oracle.forward(p, None, np.zeros((6, 8)), n_steps=N, init_state=s0, kstatic=ks)
        assert np.allclose(fin[0], 1.0, atol=1e-15)
        assert np.allclose(fin[1], u[0] / 1.25 ** N, rtol=1e-14, atol=0)
        assert np.allclose(fin[2], u[1] / 1.25 ** N, rtol=1e-14, atol=0)


def test_zero_static_field_changes_nothing():
    w = W.small_channel2d()
    J0, f0 = oracle.forward(w.problem, w.gamma, w.motion)
    J1, f1 = oracle.forward(w.problem, w.gamma, w.motion, kstatic=np.zeros((1,) + w.problem.n[1::-1]))
    assert J0 == J1 and np.array_equal(f0, f1)


def _with_block(w):
    nx, ny, _ = w.problem.n
    box = (2, 4, 2, ny - 3, 0, 0) if w.problem.dim == 2 else (2, 3, 2, 5, 2, 5)
    return W.static_box(w.problem, box, 30.0)


def test_adjoint_with_static_solid_matches_complex_step():
    for w in (W.small_channel2d(n_steps=30), W.small_duct3d(n_steps=14)):
        ks = _with_block(w)
        J, g = oracle.gradient(w.problem, w.gamma, w.motion, kstatic=ks)
        Jn, _ = oracle.gradient(w.problem, w.gamma, w.motion)
        assert abs(J - Jn) > 1e-6 * abs(Jn)          # the block changes the flow
        d = np.random.default_rng(11).standard_normal(g.shape)
        dJ, _ = oracle.complex_step(w.problem, w.gamma, w.motion, d, kstatic=ks)
        assert abs(dJ - (g * d).sum()) <= 1e-11 * np.abs(g * d).sum()


def test_terminal_adjoint_term_matches_complex_step_of_augmented_objective():
    w = W.small_channel2d(n_steps=24)
    rng = np.random.default_rng(12)
    lam = 1e-3 * rng.standard_normal((4, 1, w.problem.n[1], w.problem.n[0]))
    J, g, lam0 = oracle.gradient(w.problem, w.gamma, w.motion, lam_term=lam, want_lam0=True)
    J0, g0 = oracle.gradient(w.problem, w.gamma, w.motion)
    assert np.linalg.norm(g - g0) > 1e-3 * np.linalg.norm(g0)
    d = rng.standard_normal(g.shape)
    dJ, Jr = oracle.complex_step(w.problem, w.gamma, w.motion, d, lam_term=lam)
    assert abs(Jr - J) < 1e-14 * abs(J)
    assert abs(dJ - (g * d).sum()) <= 1e-11 * np.abs(g * d).sum()
    assert np.abs(lam0).max() > 0


def test_lambda0_is_the_gradient_with_respect_to_the_initial_state():
    w = W.small_channel2d(n_steps=20)
    p = w.problem
    rng = np.random.default_rng(13)
    s0 = W.initial_state(p) + 1e-3 * rng.standard_normal((4, 1, p.n[1], p.n[0]))
    s0[3] = 0.0
    _, _, lam0 = oracle.gradient(p, w.gamma, w.motion, init_state=s0, want_lam0=True)
    d = rng.standard_normal(s0.shape)
    d[3] = 0.0
    eps = 1e-6
    Jp, _ = oracle.forward(p, w.gamma, w.motion, init_state=s0 + eps * d)
    Jm, _ = oracle.forward(p, w.gamma, w.motion, init_state=s0 - eps * d)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(fd - (lam0 * d).sum()) <= 1e-7 * abs(fd)

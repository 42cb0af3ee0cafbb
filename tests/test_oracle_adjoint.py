"""Pins of the oracle's exact discrete adjoint (Secs. 2.4, 2.6).

The adjoint gradient is checked against differentiation of the forward code by two routes
that share nothing with the reverse sweep: the complex step (J(gamma + i h e)/h, exact to
rounding for this analytic map) and central finite differences as in the paper's Sec. 2.6
verification (eps = 1e-4), plus the second-order decay of the Taylor remainder.  The
problems carry every boundary type (inlet, outlet, moving wall), both objective kinds and a
design grid that rotates and translates, so a wrong transpose anywhere shows up.
"""
import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W

CASES = {
    "2d_J1": lambda: W.small_channel2d(obj_kind=W.OBJ_PRESSURE),
    "2d_J2": lambda: W.small_channel2d(obj_kind=W.OBJ_VELOCITY, n_steps=36, seed=21),
    "3d_J2": lambda: W.small_duct3d(obj_kind=W.OBJ_VELOCITY),
    "3d_J1": lambda: W.small_duct3d(obj_kind=W.OBJ_PRESSURE, n_steps=18, seed=22),
}


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_complex_step_per_cell(name):
    w = CASES[name]()
    J, g = oracle.gradient(w.problem, w.gamma, w.motion)
    assert np.abs(g).max() > 0
    rng = np.random.default_rng(3)
    flat = g.reshape(-1)
    cells = rng.choice(flat.size, size=min(12, flat.size), replace=False)
    for c in cells:
        d = np.zeros(flat.size)
        d[c] = 1.0
        dJ, Jr = oracle.complex_step(w.problem, w.gamma, w.motion, d.reshape(g.shape))
        assert abs(Jr - J) < 1e-14 * abs(J) + 1e-17
        assert abs(dJ - flat[c]) <= 1e-11 * np.abs(flat).max()
    # one dense random direction
    d = rng.standard_normal(g.shape)
    dJ, _ = oracle.complex_step(w.problem, w.gamma, w.motion, d)
    assert abs(dJ - (g * d).sum()) <= 1e-11 * np.abs(g * d).sum()


@pytest.mark.parametrize("name", ["2d_J1", "3d_J2"])
def test_adjoint_matches_central_differences(name):
    w = CASES[name]()
    J, g = oracle.gradient(w.problem, w.gamma, w.motion)
    flat = g.reshape(-1)
    order = np.argsort(-np.abs(flat))
    eps = 1e-4
    for c in order[:4]:
        gp = w.gamma.copy().reshape(-1)
        gm = gp.copy()
        gp[c] += eps
        gm[c] -= eps
        Jp, _ = oracle.forward(w.problem, gp.reshape(g.shape), w.motion)
        Jm, _ = oracle.forward(w.problem, gm.reshape(g.shape), w.motion)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - flat[c]) <= 1e-5 * abs(flat[c])


def test_taylor_remainder_is_second_order():
    w = CASES["2d_J2"]()
    J, g = oracle.gradient(w.problem, w.gamma, w.motion)
    d = np.random.default_rng(5).standard_normal(g.shape) * 0.05
    rem = []
    for h in (0.08, 0.04, 0.02):
        Jh, _ = oracle.forward(w.problem, w.gamma + h * d, w.motion)
        rem.append(abs(Jh - J - h * (g * d).sum()))
    assert 3.2 < rem[0] / rem[1] < 4.8 and 3.2 < rem[1] / rem[2] < 4.8


def test_printed_alks_variant_reduces_to_exact_without_body():
    """The printed source update (Eq. au_ex, 1/(1+kappa) on the first moment only) differs from
    the exact adjoint only through kappa: with gamma = 0 (kappa = 0) the two coincide, and with
    a body they differ."""
    w = CASES["3d_J2"]()
    zero = np.zeros_like(w.gamma)
    _, g0 = oracle.gradient(w.problem, zero, w.motion)
    _, p0 = oracle.gradient_printed(w.problem, zero, w.motion)
    assert np.max(np.abs(p0 - g0)) <= 1e-13 * np.max(np.abs(g0))
    _, g = oracle.gradient(w.problem, w.gamma, w.motion)
    _, p = oracle.gradient_printed(w.problem, w.gamma, w.motion)
    assert np.linalg.norm(p - g) > 1e-3 * np.linalg.norm(g)

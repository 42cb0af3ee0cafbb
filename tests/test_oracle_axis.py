"""Pins of the oracle's rotation about a general 3D axis (Rodrigues' formula).

The z-axis branch is the one the other transfer pins fix; a general axis must agree with it
where the two describe the same motion, carry the design grid onto a permutation of itself for
quarter turns about a coordinate axis, move points rigidly (velocity omega a x r at every design
node, distances kept), and keep the adjoint exact (complex step with a tilted axis).
"""
import math

import numpy as np

import oracle
from paper_2506_23895_gb300 import workloads as W

KMAX, Q = 100.0, 0.1


def _box(n, L, xi_G, axis):
    p = W.periodic_box(3, n, A=0.3, L=L)
    p.xi_G = xi_G
    p.kappa_max, p.q = KMAX, Q
    p.rot_axis = axis
    return p


def _row(theta=0.0, omega=0.0, xG=(0, 0, 0), uG=(0, 0, 0)):
    return np.array([theta, omega, *xG, *uG], dtype=np.float64)


def test_minus_z_axis_equals_z_axis_with_reversed_angle():
    n, L, xiG = (26, 24, 22), (7, 6, 5), (3.0, 2.5, 2.0)
    gam = W.make_gamma(L, 1.0, seed=3)
    xG, uG = (12.3, 11.6, 10.4), (0.01, -0.02, 0.005)
    k1, u1 = oracle.transfer(_box(n, L, xiG, (0.0, 0.0, -1.0)), gam,
                             _row(0.7, 0.05, xG, uG))
    k2, u2 = oracle.transfer(_box(n, L, xiG, (0.0, 0.0, 1.0)), gam,
                             _row(-0.7, -0.05, xG, uG))
    assert np.max(np.abs(k1 - k2)) < 1e-12 * np.max(np.abs(k2))
    assert np.max(np.abs(u1 - u2)) < 1e-14


def test_quarter_turn_about_x_is_a_permutation_of_the_design_grid():
    # R(x, pi/2) d = (dx, -dz, dy): node (i, j, k) lands where node (i, L-1-k, j) of the
    # unrotated grid sits, so gamma'[k'][j'][i] = gamma[L-1-j'][k'][i]
    Lc = 6
    n, L, xiG = (24, 24, 24), (Lc, Lc, Lc), ((Lc - 1) / 2.0,) * 3
    gam = W.make_gamma(L, 1.0, seed=4)
    gp = np.empty_like(gam)
    for kp in range(Lc):
        for jp in range(Lc):
            gp[kp, jp, :] = gam[Lc - 1 - jp, kp, :]
    xG = (11.3, 12.1, 11.7)
    k1, _ = oracle.transfer(_box(n, L, xiG, (1.0, 0.0, 0.0)), gam, _row(math.pi / 2, 0.0, xG))
    k2, _ = oracle.transfer(_box(n, L, xiG, (0.0, 0.0, 1.0)), gp, _row(0.0, 0.0, xG))
    assert np.max(np.abs(k1 - k2)) < 1e-12 * np.max(np.abs(k2))


def test_weights_and_rigid_velocity_for_a_tilted_axis():
    Lc = 7
    n, L, xiG = (30, 30, 30), (Lc, Lc, Lc), ((Lc - 1) / 2.0,) * 3
    axis = np.array(W.unit((1.0, 2.0, 2.0)))
    gam = np.full((Lc, Lc, Lc), 0.5)
    kr = KMAX * Q * 0.5 / (0.5 + Q)
    om, xG, uG = 0.04, (14.4, 15.1, 14.7), np.array([0.003, -0.002, 0.001])
    p = _box(n, L, xiG, tuple(axis))
    row = _row(0.9, om, xG, (0.0, 0.0, 0.0))
    kap, us = oracle.transfer(p, gam, row)
    ones = oracle.transfer_T(p, row, np.ones(kap.shape))
    assert np.allclose(ones, 1.0, atol=1e-13)          # every design node spreads weight 1
    # rotation alone: u_S = omega a x (R m1) is perpendicular to the axis everywhere
    assert np.max(np.abs(np.einsum("a,azyx->zyx", axis, us))) < 1e-16
    pts = [(14, 15, 15), (15, 14, 14), (13, 15, 16)]
    for x, y, z in pts:
        # deep inside, the weights of the rotated lattice sum to one up to the kernel's
        # rotated-lattice error, and u_S follows the rigid field omega a x (x - x_G)
        m0 = kap[z, y, x] / kr
        assert abs(m0 - 1.0) < 5e-3
        ref = om * np.cross(axis, np.array([x, y, z]) - np.array(xG))
        assert np.max(np.abs(us[:, z, y, x] - ref)) < 1e-2 * np.max(np.abs(ref))
    # translation alone: u_S = u_G m0 exactly, with m0 = kappa / kappa_ref for uniform gamma
    kap2, us2 = oracle.transfer(p, gam, _row(0.9, 0.0, xG, tuple(uG)))
    m0 = kap2 / kr
    assert np.max(np.abs(us2 - uG[:, None, None, None] * m0[None])) < 1e-16


def test_adjoint_with_tilted_axis_matches_complex_step():
    w = W.small_duct3d(n_steps=12, rot_axis=W.unit((1.0, 1.0, 3.0)), omega=0.02, trans_amp=0.5)
    J, g = oracle.gradient(w.problem, w.gamma, w.motion)
    wz = W.small_duct3d(n_steps=12, omega=0.02, trans_amp=0.5)
    Jz, _ = oracle.gradient(wz.problem, wz.gamma, wz.motion)
    assert abs(J - Jz) > 1e-8 * abs(Jz)                 # the axis changes the flow
    d = np.random.default_rng(21).standard_normal(g.shape)
    dJ, Jr = oracle.complex_step(w.problem, w.gamma, w.motion, d)
    assert abs(Jr - J) < 1e-14 * abs(J)
    assert abs(dJ - (g * d).sum()) <= 1e-11 * np.abs(g * d).sum()

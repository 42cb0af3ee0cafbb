"""Pins of the oracle's design-to-analysis transfer (Sec. 2.3) and the Brinkman update.

Expected values are hand-computed: the kernel w(r) = (1 + cos(pi r / 2)) / 4 takes the values
1/2 at r = 0, 1/4 at |r| = 1, 0 at |r| = 2, (1 +- sqrt(2)/2) / 4 at |r| = 1/2, 3/2; its
integer-shifted copies sum to one; a counter-clockwise rotation by pi/2 carries the offset
(1, 0) to (0, 1); a rigid rotation moves the point at offset r with velocity omega x r.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W

KMAX, Q = 100.0, 0.1


def _kref(g):
    return KMAX * Q * g / ((1.0 - g) + Q)


def _box(dim, n, L, xi_G):
    p = W.periodic_box(dim, n, A=0.3, L=L)
    p.xi_G = xi_G
    p.kappa_max, p.q = KMAX, Q
    return p


def _row(theta=0.0, omega=0.0, xG=(0, 0, 0), uG=(0, 0, 0)):
    return np.array([theta, omega, *xG, *uG], dtype=np.float64)


@pytest.mark.parametrize("dim", [2, 3])
def test_coincident_grids_give_quarter_half_quarter_filter(dim):
    n = (20, 18, 16 if dim == 3 else 1)
    L = (5, 5, 5 if dim == 3 else 1)
    xi_G = (2.0, 2.0, 2.0 if dim == 3 else 0.0)
    p = _box(dim, n, L, xi_G)
    gam = np.zeros((L[2], L[1], L[0]))
    src = (3, 1, 4 if dim == 3 else 0)          # design node (i, j, k)
    gam[src[2], src[1], src[0]] = 0.5
    xG = (10.0, 9.0, 7.0 if dim == 3 else 0.0)
    kap, _ = oracle.transfer(p, gam, _row(xG=xG))
    tgt = [int(xG[a] + src[a] - xi_G[a]) for a in range(3)]
    expect = np.zeros_like(kap)
    f = {-1: 0.25, 0: 0.5, 1: 0.25}
    K = 100.0 * 0.1 * 0.5 / (1.0 - 0.5 + 0.1)   # = 8.333..., hand value of kappa_ref(0.5)
    for dz in ((-1, 0, 1) if dim == 3 else (0,)):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                w = f[dx] * f[dy] * (f[dz] if dim == 3 else 1.0)
                expect[tgt[2] + dz, tgt[1] + dy, tgt[0] + dx] = K * w
    assert np.max(np.abs(kap - expect)) < 1e-14


def test_half_cell_offset_weights():
    p = _box(2, (20, 18, 1), (5, 5, 1), (2.0, 2.0, 0.0))
    gam = np.zeros((1, 5, 5))
    gam[0, 2, 2] = 0.5
    kap, _ = oracle.transfer(p, gam, _row(xG=(10.5, 9.0, 0.0)))
    K = 100.0 * 0.1 * 0.5 / 0.6
    wn = 0.25 * (1.0 + math.sqrt(2.0) / 2.0)   # |r| = 1/2
    wf = 0.25 * (1.0 - math.sqrt(2.0) / 2.0)   # |r| = 3/2
    row = kap[0, 9, :]
    assert abs(row[10] - K * wn * 0.5) < 1e-14 and abs(row[11] - K * wn * 0.5) < 1e-14
    assert abs(row[9] - K * wf * 0.5) < 1e-14 and abs(row[12] - K * wf * 0.5) < 1e-14
    assert abs(kap.sum() - K) < 1e-13
    assert np.count_nonzero(kap) == 4 * 3


@pytest.mark.parametrize("dim", [2, 3])
def test_partition_of_unity_for_any_rigid_motion(dim):
    n = (40, 38, 30 if dim == 3 else 1)
    L = (9, 8, 7 if dim == 3 else 1)
    xi_G = (4.0, 3.5, 3.0 if dim == 3 else 0.0)
    p = _box(dim, n, L, xi_G)
    gam = W.make_gamma(L, 1.0, seed=2)
    for th in (0.0, 0.37, 1.1, 2.9):
        xG = (19.3, 18.77, 14.61 if dim == 3 else 0.0)
        kap, us = oracle.transfer(p, gam, _row(theta=th, omega=0.0, xG=xG, uG=(0.01, 0.02, 0.03)))
        assert abs(kap.sum() - _kref(gam).sum()) < 1e-12 * _kref(gam).sum()
        # u_S carries u_G with total weight = number of design nodes
        nd = L[0] * L[1] * L[2]
        assert abs(us[0].sum() - 0.01 * nd) < 1e-11
        assert abs(us[1].sum() - 0.02 * nd) < 1e-11


def test_rotation_is_counter_clockwise_about_the_centre():
    p = _box(2, (20, 20, 1), (5, 5, 1), (2.0, 2.0, 0.0))
    gam = np.zeros((1, 5, 5))
    gam[0, 2, 3] = 0.5          # design node at offset (+1, 0) from the centre
    kap, _ = oracle.transfer(p, gam, _row(theta=math.pi / 2.0, xG=(10.0, 10.0, 0.0)))
    K = 100.0 * 0.1 * 0.5 / 0.6
    assert abs(kap[0, 11, 10] - 0.25 * K) < 1e-13   # landed on (10, 11): offset (0, +1)
    assert abs(kap.sum() - K) < 1e-12


def test_rotation_about_z_in_3d_keeps_z():
    p = _box(3, (20, 20, 20), (5, 5, 5), (2.0, 2.0, 2.0))
    gam = np.zeros((5, 5, 5))
    gam[4, 2, 3] = 0.5          # offset (+1, 0, +2)
    kap, _ = oracle.transfer(p, gam, _row(theta=math.pi / 2.0, xG=(10.0, 10.0, 9.0)))
    K = 100.0 * 0.1 * 0.5 / 0.6
    assert abs(kap[11, 11, 10] - 0.125 * K) < 1e-13  # (10, 11, 11)


def test_rigid_velocity_field_on_coincident_grids():
    """Deep inside, the [1/4,1/2,1/4] filter reproduces the affine rigid velocity exactly."""
    p = _box(2, (30, 30, 1), (11, 11, 1), (5.0, 5.0, 0.0))
    gam = np.full((1, 11, 11), 0.3)
    om, uG, xG = 0.07, (0.01, -0.02, 0.0), (15.0, 14.0, 0.0)
    kap, us = oracle.transfer(p, gam, _row(theta=0.0, omega=om, xG=xG, uG=uG))
    for (x, y) in [(15, 14), (13, 17), (18, 11), (12, 12)]:
        rx, ry = x - xG[0], y - xG[1]
        assert abs(us[0, 0, y, x] - (-om * ry + uG[0])) < 1e-15
        assert abs(us[1, 0, y, x] - (om * rx + uG[1])) < 1e-15
        assert abs(kap[0, y, x] - _kref(0.3)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_transposed_transfer_is_the_adjoint(dim):
    n = (30, 28, 22 if dim == 3 else 1)
    L = (7, 6, 5 if dim == 3 else 1)
    xi_G = (3.0, 2.5, 2.0 if dim == 3 else 0.0)
    p = _box(dim, n, L, xi_G)
    gam = W.make_gamma(L, 1.0, seed=9)
    row = _row(theta=0.81, xG=(14.2, 13.6, 10.3 if dim == 3 else 0.0))
    kap, _ = oracle.transfer(p, gam, row)
    e = np.random.default_rng(1).standard_normal(kap.shape)
    te = oracle.transfer_T(p, row, e)
    assert abs((kap * e).sum() - (_kref(gam) * te).sum()) < 1e-12 * np.abs(kap * e).sum()
    # T^T applied to ones gives each design node's total weight, exactly one
    assert np.max(np.abs(oracle.transfer_T(p, row, np.ones_like(e)) - 1.0)) < 1e-14


@pytest.mark.parametrize("dim", [2, 3])
def test_brinkman_update_solves_the_implicit_vpm_relation(dim):
    """With a uniform old state the gather returns u* = U exactly, so after one step the
    interior velocity must satisfy u = u* + F with F = -kappa (u - u_S) (Eqs. u_ex, VPM force)."""
    n = (24, 22, 18 if dim == 3 else 1)
    L = (7, 7, 6 if dim == 3 else 1)
    p = W.periodic_box(dim, n, A=0.3, L=L, n_steps=1)
    p.xi_G = ((L[0] - 1) / 2, (L[1] - 1) / 2, (L[2] - 1) / 2 if dim == 3 else 0.0)
    U = np.array([0.02, -0.01, 0.015 if dim == 3 else 0.0])
    p.u_init = tuple(U)
    gam = W.make_gamma(L, 1.0, seed=4)
    mot = W.motion_table(1, (11.4, 10.7, 8.6 if dim == 3 else 0.0), omega=0.08, theta0=0.5)
    mot[:, 5:8] = (0.005, 0.01, -0.004 if dim == 3 else 0.0)
    kap, us = oracle.transfer(p, gam, mot[1])
    _, fin = oracle.forward(p, gam, mot)
    assert kap.max() > 1.0
    for a in range(dim):
        lhs = fin[1 + a] - U[a]
        rhs = -kap * (fin[1 + a] - us[a])
        assert np.max(np.abs(lhs - rhs)) < 1e-14

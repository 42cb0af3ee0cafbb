"""Pins of the CPU oracle's forward scheme against closed forms and invariants.

Each expected value below is derived by hand from the scheme's definition (Sec. 2.2: the
tau = 1 gather of f^eq with the viscosity term, nu = 1/6 - 2A/9), not by re-running the
oracle's code:

* shear wave u_a = amp*sin(k x_b): the nonlinear terms cancel by the lattice weight identities
  and the scheme multiplies the amplitude by G(k) = 2/3 + cos(k)/3 + (2A/9) sin^2(k) per step,
  for D2Q9 and D3Q15 alike (G ~ 1 - nu k^2, the viscosity relation of Sec. 2.2);
* plane Poiseuille with body force g: u = g y (H - y) / (2 nu) is an exact fixed point when
  the wall gradient is the one-sided second-order difference (u* = u + nu u'' for a parabola);
* plane Couette: u = U y / H is an exact fixed point;
* mass: sum rho* = sum (rho + (2A/3) div u) and the periodic central divergence telescopes,
  so total mass is conserved to rounding for any kappa, u_S (the Brinkman update leaves rho);
* a uniform state with kappa = 0 is invariant, and so is a uniform flow carrying a body that
  translates with it (u_S = u where kappa > 0, by the kernel's partition of unity).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W


def G_factor(k, A):
    return 2.0 / 3.0 + math.cos(k) / 3.0 + (2.0 * A / 9.0) * math.sin(k) ** 2


@pytest.mark.parametrize("dim,comp,axis", [(2, 0, 1), (2, 1, 0), (3, 0, 1), (3, 0, 2),
                                           (3, 1, 0), (3, 1, 2), (3, 2, 0), (3, 2, 1)])
def test_shear_wave_decay_is_exact(dim, comp, axis):
    n = [5, 5, 5] if dim == 3 else [5, 5, 1]
    n[axis] = 24
    A, amp, mode, steps = 0.41, 0.03, 2, 37
    p = W.periodic_box(dim, tuple(n), A=A, n_steps=steps)
    k = 2.0 * math.pi * mode / n[axis]
    coords = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    xb = coords[2 - axis]  # (z, y, x) order
    u = [np.zeros((n[2], n[1], n[0])) for _ in range(3)]
    u[comp] = amp * np.sin(k * xb)
    s0 = W.initial_state(p, u=u)
    _, fin = oracle.forward(p, None, np.zeros((steps + 1, 8)), init_state=s0)
    expect = amp * G_factor(k, A) ** steps * np.sin(k * xb)
    assert np.max(np.abs(fin[1 + comp] - expect)) < 1e-14  # amp 3e-2, ~1e-12 relative
    for a in range(3):
        if a != comp:
            assert np.max(np.abs(fin[1 + a])) < 1e-15
    assert np.max(np.abs(fin[0] - 1.0)) < 1e-13  # rounding of 37 gathers of O(1) terms


def _plates(dim, H, A, top_u=0.0, g=0.0, steps=10):
    n = (4, H + 1, 4 if dim == 3 else 1)
    bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL, W.PERIODIC, W.PERIODIC)
    bcv = ((0, 0, 0, 1),) * 2 + ((0, 0, 0, 1), (top_u, 0, 0, 1)) + ((0, 0, 0, 1),) * 2
    return W.Problem(dim=dim, n=n, L=(0, 0, 0), A=A, bc=bc, bc_val=bcv, body_force=(g, 0, 0),
                     obj_box=(0, 3, 1, H - 1, 0, n[2] - 1), win=(1, steps), n_steps=steps)


@pytest.mark.parametrize("dim", [2, 3])
def test_poiseuille_is_exact_fixed_point(dim):
    H, A, g = 10, 0.3, 1e-5
    p = _plates(dim, H, A, g=g, steps=25)
    nu = 1.0 / 6.0 - 2.0 * A / 9.0
    y = np.arange(H + 1, dtype=np.float64)
    prof = g * y * (H - y) / (2.0 * nu)
    u = [np.broadcast_to(prof[None, :, None], (p.n[2], H + 1, 4)).copy(),
         np.zeros((p.n[2], H + 1, 4)), np.zeros((p.n[2], H + 1, 4))]
    s0 = W.initial_state(p, u=u)
    _, fin = oracle.forward(p, None, np.zeros((26, 8)), init_state=s0)
    # absolute: u* collects sum_i c_i w_i rho, which cancels O(1) terms (rounding ~1e-16)
    assert np.max(np.abs(fin[1] - u[0])) < 1e-14
    assert np.max(np.abs(fin[0] - 1.0)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_poiseuille_from_rest_converges_to_parabola(dim):
    H, A, g, steps = 8, 0.3, 1e-5, 3000
    p = _plates(dim, H, A, g=g, steps=steps)
    p.u_init = (0.0, 0.0, 0.0)
    nu = 1.0 / 6.0 - 2.0 * A / 9.0
    y = np.arange(H + 1, dtype=np.float64)
    prof = g * y * (H - y) / (2.0 * nu)
    _, fin = oracle.forward(p, None, np.zeros((steps + 1, 8)))
    assert np.max(np.abs(fin[1] - prof[None, :, None])) < 1e-10 * prof.max()


@pytest.mark.parametrize("dim", [2, 3])
def test_couette_is_exact_fixed_point_and_attractor(dim):
    H, A, U = 9, 0.5, 0.03
    p = _plates(dim, H, A, top_u=U, steps=40)
    y = np.arange(H + 1, dtype=np.float64)
    prof = U * y / H
    shp = (p.n[2], H + 1, 4)
    u = [np.broadcast_to(prof[None, :, None], shp).copy(), np.zeros(shp), np.zeros(shp)]
    _, fin = oracle.forward(p, None, np.zeros((41, 8)), init_state=W.initial_state(p, u=u))
    assert np.max(np.abs(fin[1] - u[0])) < 1e-14
    p2 = _plates(dim, H, 0.2, top_u=U, steps=2500)  # larger nu: slowest mode decays e^-37
    _, fin2 = oracle.forward(p2, None, np.zeros((2501, 8)))
    assert np.max(np.abs(fin2[1] - prof[None, :, None])) < 1e-11


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_is_conserved_in_periodic_box_with_moving_body(dim):
    if dim == 2:
        n, L, steps = (26, 22, 1), (7, 7, 1), 50
        mot = W.motion_table(steps, (12.3, 10.6, 0.0), omega=0.05, trans_amp=1.5,
                             trans_period=30.0, trans_axis=0, theta0=0.4)
    else:
        n, L, steps = (15, 14, 13), (5, 5, 4), 20
        mot = W.motion_table(steps, (7.2, 6.6, 6.3), omega=0.05, trans_amp=1.0,
                             trans_period=16.0, trans_axis=1, theta0=0.4)
    p = W.periodic_box(dim, n, A=0.35, L=L, n_steps=steps)
    p.xi_G = ((L[0] - 1) / 2.0, (L[1] - 1) / 2.0, (L[2] - 1) / 2.0 if dim == 3 else 0.0)
    gam = W.make_gamma(L, 1.0, seed=5)
    rng = np.random.default_rng(7)
    u = [0.02 * W.gaussian_filter(rng.standard_normal((n[2], n[1], n[0])), 1.5)
         for _ in range(3)]
    if dim == 2:
        u[2][:] = 0.0
    rho = 1.0 + 0.01 * W.gaussian_filter(rng.standard_normal((n[2], n[1], n[0])), 1.5)
    s0 = W.initial_state(p, rho=rho, u=u)
    _, fin = oracle.forward(p, gam, mot, init_state=s0)
    assert abs(fin[0].sum() - rho.sum()) < 1e-13 * rho.sum()
    # the body does act on the flow
    assert np.max(np.abs(fin[1] - u[0])) > 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_flow_invariant_with_and_without_comoving_body(dim):
    U = (0.03, -0.02, 0.01 if dim == 3 else 0.0)
    if dim == 2:
        n, L = (30, 28, 1), (10, 10, 1)
    else:
        n, L = (18, 17, 16), (9, 9, 8)
    steps = 20
    p = W.periodic_box(dim, n, A=0.4, n_steps=steps)
    p.u_init = U
    _, fin = oracle.forward(p, None, np.zeros((steps + 1, 8)))
    for a in range(3):
        assert np.max(np.abs(fin[1 + a] - U[a])) < 1e-15
    # a body translating with the flow; gamma vanishes on a 3-cell rim so m0 = 1 under kappa
    p.L = L
    p.xi_G = ((L[0] - 1) / 2.0, (L[1] - 1) / 2.0, (L[2] - 1) / 2.0 if dim == 3 else 0.0)
    gam = W.make_gamma(L, 1.0, seed=3)
    sl = (slice(None),) if dim == 2 else (slice(3, -3),)
    mask = np.zeros_like(gam)
    if dim == 2:
        mask[:, 3:-3, 3:-3] = 1.0
    else:
        mask[3:-3, 3:-3, 3:-3] = 1.0
    gam = gam * mask
    x0 = np.array([(n[0] - 1) / 2.0 - 3.0, (n[1] - 1) / 2.0 + 2.0, (n[2] - 1) / 2.0])
    if dim == 2:
        x0[2] = 0.0
    mot = np.zeros((steps + 1, 8))
    t = np.arange(steps + 1)
    for a in range(3):
        mot[:, 2 + a] = x0[a] + U[a] * t
        mot[:, 5 + a] = U[a]
    _, fin = oracle.forward(p, gam, mot)
    for a in range(3):
        assert np.max(np.abs(fin[1 + a] - U[a])) < 1e-14
    assert np.max(np.abs(fin[0] - 1.0)) < 1e-13


def test_uniform_inflow_channel_is_steady():
    """Inlet (u prescribed), outlet (rho prescribed, tangential u = 0) and periodic y: a uniform
    stream matching both is a fixed point of the boundary rules."""
    p = W.Problem(dim=2, n=(20, 12, 1), L=(0, 0, 0), A=0.3,
                  bc=(W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC),
                  bc_val=((0.04, 0, 0, 1), (0, 0, 0, 1.0)) + ((0, 0, 0, 1),) * 4,
                  u_init=(0.04, 0, 0), obj_box=(0, 0, 0, 11, 0, 0), win=(1, 30), n_steps=30)
    J, fin = oracle.forward(p, None, np.zeros((31, 8)))
    assert np.max(np.abs(fin[1] - 0.04)) < 1e-15
    assert np.max(np.abs(fin[2])) < 1e-15
    assert np.max(np.abs(fin[0] - 1.0)) < 1e-13
    assert abs(J - (-1.0 / 3.0)) < 1e-14


def test_objective_values_on_uniform_states():
    """J1 = -mean(rho)/3 and J2 = -mean(n.u) over the window (Eqs. objective_1/2)."""
    p = W.periodic_box(3, (6, 5, 7), A=0.3, n_steps=9)
    p.u_init = (0.01, -0.02, 0.025)
    p.rho0 = 1.1
    p.win = (3, 9)
    J1, _ = oracle.forward(p, None, np.zeros((10, 8)))
    assert abs(J1 - (-1.1 / 3.0)) < 1e-13
    p.obj_kind = W.OBJ_VELOCITY
    p.obj_dir = (0.6, 0.0, 0.8)
    p.obj_box = (1, 4, 0, 2, 2, 5)
    J2, _ = oracle.forward(p, None, np.zeros((10, 8)))
    assert abs(J2 - (-(0.6 * 0.01 + 0.8 * 0.025))) < 1e-15

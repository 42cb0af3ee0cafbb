"""Pins of the oracle's boundary rule on edges and corners where faces of different types meet.

The paper prescribes u on no-slip walls and inlets and rho on outlets (Eqs. bc_rho, bc_u) but
leaves the other quantity open.  The reading used on both sides of this repository: a boundary
node copies the unprescribed quantity from the node one step inward along EVERY boundary normal
it lies on (so an edge or corner node copies from the diagonal-inward interior node), and where
faces of different types meet, WALL beats INLET beats OUTLET, ties going to the lower face
index (faces ordered x-, x+, y-, y+, z-, z+).

Each expectation below is written out by hand for one named node: "u is this face's prescribed
velocity" and "rho is the one at that interior node".  The state one step earlier is seeded
noise, so every candidate copy source (the diagonal-inward node, the face-normal neighbours,
the nodes two steps in) carries a different value; a reversed precedence or a copy from a
face-normal neighbour fails at least one assertion.
"""
import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W


def _noisy_state(p, seed):
    nx, ny, nz = p.n
    r = W.splitmix64_uniform(seed, 4 * nx * ny * nz).reshape(4, nz, ny, nx)
    s = np.empty_like(r)
    s[0] = p.rho0 + 0.02 * (r[0] - 0.5)
    for a in range(3):
        s[1 + a] = 0.04 * (r[1 + a] - 0.5)
    if p.dim == 2:
        s[3] = 0.0
    return s


def _one_step(p, seed):
    s0 = _noisy_state(p, seed)
    _, s1 = oracle.forward(p, None, np.zeros((2, 8)), n_steps=1, init_state=s0)
    return s1


def _distinct(values, tol=1e-6):
    v = sorted(values)
    return all(b - a > tol for a, b in zip(v, v[1:]))


# 2D channel: inlet x-, outlet x+, a resting wall y- and a moving lid y+ (distinct velocities)
U_IN, U_LID, RHO_OUT = (0.05, 0.0), (0.02, 0.0), 1.003


def _channel():
    nx, ny = 9, 8
    return W.Problem(
        dim=2, n=(nx, ny, 1), L=(0, 0, 0), A=0.45,
        bc=(W.INLET, W.OUTLET, W.WALL, W.WALL, W.PERIODIC, W.PERIODIC),
        bc_val=((U_IN[0], U_IN[1], 0.0, 1.0), (0.0, 0.0, 0.0, RHO_OUT), (0.0, 0.0, 0.0, 1.0),
                (U_LID[0], U_LID[1], 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0)),
        obj_box=(1, 1, 1, 1, 0, 0), win=(1, 1), n_steps=1)


def test_channel_corner_sources_differ():
    """The interior nodes near the corner (0, 0) hold different densities after the step, and
    the face-normal neighbours (1, 0) and (0, 1) held different ones before it, so the corner
    tests below can tell a copy from the diagonal-inward node from any other source."""
    p = _channel()
    s0 = _noisy_state(p, 71)
    s = _one_step(p, 71)
    rho = s[0, 0]
    assert _distinct([rho[1, 1], rho[2, 1], rho[1, 2], rho[2, 2], RHO_OUT, s0[0, 0, 0, 1],
                      s0[0, 0, 1, 0], s0[0, 0, 1, 1]])


def test_channel_wall_beats_inlet_and_copies_diagonally():
    p = _channel()
    nx, ny = p.n[0], p.n[1]
    s = _one_step(p, 71)
    rho, ux, uy = s[0, 0], s[1, 0], s[2, 0]
    # corner (x=0, y=0): inlet and resting wall meet; the wall wins: u = 0, rho from (1, 1)
    assert (ux[0, 0], uy[0, 0]) == (0.0, 0.0)
    assert rho[0, 0] == rho[1, 1]
    # corner (x=0, y=ny-1): inlet and moving lid; the lid wins: u = U_LID, rho from (1, ny-2)
    assert (ux[ny - 1, 0], uy[ny - 1, 0]) == U_LID
    assert rho[ny - 1, 0] == rho[ny - 2, 1]
    # an inlet node away from the corners: u = U_IN, rho from (1, y)
    assert (ux[3, 0], uy[3, 0]) == U_IN
    assert rho[3, 0] == rho[3, 1]


def test_channel_wall_beats_outlet_and_copies_diagonally():
    p = _channel()
    nx, ny = p.n[0], p.n[1]
    s = _one_step(p, 71)
    rho, ux, uy = s[0, 0], s[1, 0], s[2, 0]
    # corner (x=nx-1, y=0): outlet and resting wall; the wall wins: u = 0, rho from (nx-2, 1)
    assert (ux[0, nx - 1], uy[0, nx - 1]) == (0.0, 0.0)
    assert rho[0, nx - 1] == rho[1, nx - 2]
    assert rho[0, nx - 1] != RHO_OUT
    # corner (x=nx-1, y=ny-1): outlet and lid; the lid wins
    assert (ux[ny - 1, nx - 1], uy[ny - 1, nx - 1]) == U_LID
    assert rho[ny - 1, nx - 1] == rho[ny - 2, nx - 2]
    # an outlet node away from the corners: rho prescribed, normal u copied from (nx-2, y),
    # tangential u prescribed (0)
    assert rho[4, nx - 1] == RHO_OUT
    assert ux[4, nx - 1] == ux[4, nx - 2]
    assert uy[4, nx - 1] == 0.0
    # a wall node away from the corners: u prescribed, rho from the node above it
    assert (ux[0, 4], uy[0, 4]) == (0.0, 0.0)
    assert rho[0, 4] == rho[1, 4]
    assert (ux[ny - 1, 4], uy[ny - 1, 4]) == U_LID
    assert rho[ny - 1, 4] == rho[ny - 2, 4]


# 3D duct along z: walls on all four x/y faces, each with its own tangential velocity (so the
# tie between two walls is visible), inlet z-, outlet z+
WX0, WX1, WY0, WY1 = (0.0, 0.0, 0.011), (0.0, 0.0, -0.007), (0.0, 0.0, 0.023), (0.0, 0.0, 0.031)
U3_IN, RHO3_OUT = (0.0, 0.0, 0.05), 0.998


def _duct():
    nx, ny, nz = 7, 6, 8
    return W.Problem(
        dim=3, n=(nx, ny, nz), L=(0, 0, 0), A=0.4,
        bc=(W.WALL, W.WALL, W.WALL, W.WALL, W.INLET, W.OUTLET),
        bc_val=(WX0 + (1.0,), WX1 + (1.0,), WY0 + (1.0,), WY1 + (1.0,), U3_IN + (1.0,),
                (0.0, 0.0, 0.0, RHO3_OUT)),
        obj_kind=W.OBJ_VELOCITY, obj_box=(2, 2, 2, 2, 3, 3), obj_dir=(0.0, 0.0, 1.0),
        win=(1, 1), n_steps=1)


def _u(s, x, y, z):
    return (s[1, z, y, x], s[2, z, y, x], s[3, z, y, x])


def test_duct_corner_sources_differ():
    """Interior nodes around the corner (0, 0, 0) differ after the step; its boundary
    neighbours differed before it (a copy from one of them reads a value the step has not
    written yet, or the old one)."""
    p = _duct()
    s0 = _noisy_state(p, 72)
    s = _one_step(p, 72)
    r, r0 = s[0], s0[0]
    cands = [r[1, 1, 1], r[2, 1, 1], r[1, 2, 1], r[1, 1, 2], r[2, 2, 2], RHO3_OUT,
             r0[0, 1, 1], r0[1, 0, 1], r0[1, 1, 0], r0[0, 0, 1], r0[0, 1, 0], r0[1, 0, 0]]
    assert _distinct(cands)


def test_duct_edges_and_corners():
    p = _duct()
    nx, ny, nz = p.n
    s = _one_step(p, 72)
    r = s[0]
    z = 4
    # edge x=0, y=0 (two walls tie; the x- face has the lower index): u = WX0, rho from (1,1,z)
    assert _u(s, 0, 0, z) == WX0
    assert r[z, 0, 0] == r[z, 1, 1]
    # edge x=nx-1, y=0: x+ (face 1) beats y- (face 2)
    assert _u(s, nx - 1, 0, z) == WX1
    assert r[z, 0, nx - 1] == r[z, 1, nx - 2]
    # edge x=0, y=ny-1: x- beats y+
    assert _u(s, 0, ny - 1, z) == WX0
    assert r[z, ny - 1, 0] == r[z, ny - 2, 1]
    # edge y=0, z=0 (wall and inlet): the wall wins, rho from (x, 1, 1)
    assert _u(s, 3, 0, 0) == WY0
    assert r[0, 0, 3] == r[1, 1, 3]
    # edge y=ny-1, z=nz-1 (wall and outlet): the wall wins, rho from (x, ny-2, nz-2)
    assert _u(s, 3, ny - 1, nz - 1) == WY1
    assert r[nz - 1, ny - 1, 3] == r[nz - 2, ny - 2, 3]
    assert r[nz - 1, ny - 1, 3] != RHO3_OUT
    # corner (0, 0, 0): x- wall beats the y- wall and the inlet; rho from (1, 1, 1)
    assert _u(s, 0, 0, 0) == WX0
    assert r[0, 0, 0] == r[1, 1, 1]
    # corner (nx-1, ny-1, nz-1): x+ wall beats the y+ wall and the outlet
    assert _u(s, nx - 1, ny - 1, nz - 1) == WX1
    assert r[nz - 1, ny - 1, nx - 1] == r[nz - 2, ny - 2, nx - 2]
    # corner (nx-1, 0, 0)
    assert _u(s, nx - 1, 0, 0) == WX1
    assert r[0, 0, nx - 1] == r[1, 1, nx - 2]


def test_duct_faces_away_from_edges():
    p = _duct()
    nx, ny, nz = p.n
    s = _one_step(p, 72)
    r = s[0]
    x, y, z = 3, 2, 4
    # inlet node: u = U3_IN, rho from one step in z
    assert _u(s, x, y, 0) == U3_IN
    assert r[0, y, x] == r[1, y, x]
    # outlet node: rho prescribed, normal (z) velocity from one step in, tangential 0
    assert r[nz - 1, y, x] == RHO3_OUT
    assert s[3, nz - 1, y, x] == s[3, nz - 2, y, x]
    assert (s[1, nz - 1, y, x], s[2, nz - 1, y, x]) == (0.0, 0.0)
    # wall nodes
    assert _u(s, 0, y, z) == WX0 and r[z, y, 0] == r[z, y, 1]
    assert _u(s, x, ny - 1, z) == WY1 and r[z, ny - 1, x] == r[z, ny - 2, x]


@pytest.mark.parametrize("make", [_channel, _duct])
def test_adjoint_of_corner_rule_matches_complex_step(make):
    """The transposed boundary rule in the adjoint agrees with the forward rule above: the
    gradient of an objective that reads corner and edge nodes through the next step's
    gather matches the complex step of the forward (Sec. 2.4's sensitivity, exact form)."""
    p = make()
    p.n = (12, 11, 1) if p.dim == 2 else (10, 10, 10)
    p.n_steps = 3
    p.win = (2, 3)
    nx, ny, nz = p.n
    LD = 3
    p.L = (LD, LD, LD if p.dim == 3 else 1)
    p.xi_G = ((LD - 1) / 2.0, (LD - 1) / 2.0, (LD - 1) / 2.0 if p.dim == 3 else 0.0)
    # objective region hugging the x- face's interior row, next to the corners
    if p.dim == 2:
        p.obj_box = (1, 1, 1, ny - 2, 0, 0)
    else:
        p.obj_box = (1, 1, 1, ny - 2, 1, nz - 2)
    c = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0 if p.dim == 3 else 0.0)
    m = W.motion_table(p.n_steps, c, omega=0.05, theta0=0.1)
    g = W.make_gamma(p.L, 0.0, seed=5)
    J, grad = oracle.gradient(p, g, m)
    d = W.splitmix64_uniform(9, g.size).reshape(g.shape) - 0.5
    dJ, J2 = oracle.complex_step(p, g, m, d)
    assert abs(J2 - J) <= 1e-14 * abs(J)
    assert abs(float(np.sum(grad * d)) - dJ) <= 1e-11 * max(abs(dJ), 1e-300)

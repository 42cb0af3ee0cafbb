"""Pins of the design-chain oracle (density filter, Heaviside projection, volume constraint).

The filter is checked against a dense matrix built by brute force from its definition (explicit
double loop over node pairs and distances), the projection against its limits and closed
values, the volume constraint against a closed form, and the whole chain around the solver
against central differences of the oracle's objective.
"""
import numpy as np
import pytest

import oracle
from oracle import design_chain as D
from paper_2506_23895_gb300 import workloads as W


def dense_filter(shape, R):
    lz, ly, lx = shape
    idx = [(z, y, x) for z in range(lz) for y in range(ly) for x in range(lx)]
    M = np.zeros((len(idx), len(idx)))
    for a, (z, y, x) in enumerate(idx):
        for b, (z2, y2, x2) in enumerate(idx):
            d = np.sqrt((x - x2) ** 2 + (y - y2) ** 2 + (z - z2) ** 2)
            M[a, b] = max(0.0, R - d)
        M[a] /= M[a].sum()
    return M


@pytest.mark.parametrize("shape,R", [((1, 7, 9), 2.4), ((1, 6, 5), 1.5), ((4, 5, 6), 2.4)])
def test_filter_and_transpose_match_dense_matrix(shape, R):
    M = dense_filter(shape, R)
    rng = np.random.default_rng(3)
    a = rng.random(shape)
    b = rng.standard_normal(shape)
    assert np.allclose(D.density_filter(a, R).ravel(), M @ a.ravel(), rtol=0, atol=1e-14)
    assert np.allclose(D.density_filter_T(b, R).ravel(), M.T @ b.ravel(), rtol=0, atol=1e-14)


def test_filter_hand_values_and_constants():
    # R = 1.5 in 2D: centre 1.5, four axis neighbours 0.5, four diagonals 1.5 - sqrt(2)
    g = np.zeros((1, 5, 5))
    g[0, 2, 2] = 1.0
    wd = 1.5 - np.sqrt(2.0)
    tot = 1.5 + 4 * 0.5 + 4 * wd
    f = D.density_filter(g, 1.5)
    assert abs(f[0, 2, 2] - 1.5 / tot) < 1e-15
    assert abs(f[0, 2, 3] - 0.5 / tot) < 1e-15
    assert abs(f[0, 3, 3] - wd / tot) < 1e-15
    assert f[0, 0, 2] == 0.0
    # constants pass through, also at the grid's edges and corners
    for shape in ((1, 8, 6), (3, 4, 5)):
        c = np.full(shape, 0.37)
        assert np.allclose(D.density_filter(c, 2.4), 0.37, atol=1e-15)


def test_projection_limits_and_values():
    x = np.linspace(0.0, 1.0, 11)
    for beta in (1.0, 8.0, 64.0):
        h = D.project(x, beta)
        assert abs(h[0]) < 1e-15 and abs(h[-1] - 1.0) < 1e-15 and abs(h[5] - 0.5) < 1e-15
        assert np.all(np.diff(h) >= 0) and (beta > 8.0 or np.all(np.diff(h) > 0))
    # beta -> 0: the projection tends to the identity (error O(beta^2))
    e1 = np.max(np.abs(D.project(x, 1e-2) - x))
    e2 = np.max(np.abs(D.project(x, 5e-3) - x))
    assert e1 < 1e-4 and 3.5 < e1 / e2 < 4.5
    # large beta: a step at eta
    h = D.project(np.array([0.45, 0.55]), 400.0)
    assert h[0] < 1e-8 and h[1] > 1 - 1e-8
    # derivative against central differences
    xs = np.array([0.1, 0.4, 0.5, 0.77])
    for beta in (1.0, 8.0):
        fd = (D.project(xs + 1e-6, beta) - D.project(xs - 1e-6, beta)) / 2e-6
        assert np.allclose(D.project_prime(xs, beta), fd, rtol=1e-8)


def test_volume_closed_form_and_gradient():
    shape = (1, 6, 7)
    v, vmax = 0.3, 0.4
    G, dG = D.volume(np.full(shape, v), vmax)
    assert abs(G - (v / vmax - 1.0)) < 1e-15
    assert np.allclose(dG, 1.0 / (vmax * 42))
    # through the chain: a uniform field stays uniform, then projects
    beta = 4.0
    G, dG = D.volume(np.full(shape, v), vmax, R=2.4, beta=beta)
    assert abs(G - (D.project(np.array(v), beta) / vmax - 1.0)) < 1e-14
    g = np.random.default_rng(2).random(shape)
    _, dG = D.volume(g, vmax, R=2.4, beta=beta)
    d = np.random.default_rng(4).standard_normal(shape)
    eps = 1e-6
    fd = (D.volume(g + eps * d, vmax, 2.4, beta)[0] - D.volume(g - eps * d, vmax, 2.4, beta)[0]) / (2 * eps)
    assert abs(fd - (dG * d).sum()) < 1e-8 * abs(fd)


def test_chain_around_the_solver_matches_central_differences():
    w = W.small_channel2d(n_steps=24)
    R, beta = 2.4, 4.0
    gb = D.physical(w.gamma, R, beta)
    _, g_gb = oracle.gradient(w.problem, gb, w.motion)
    g = D.chain_T(w.gamma, g_gb, R, beta)
    flat = g.ravel()
    for c in np.argsort(-np.abs(flat))[:3]:
        gp = w.gamma.copy().ravel()
        gm = gp.copy()
        gp[c] += 1e-5
        gm[c] -= 1e-5
        Jp, _ = oracle.forward(w.problem, D.physical(gp.reshape(g.shape), R, beta), w.motion)
        Jm, _ = oracle.forward(w.problem, D.physical(gm.reshape(g.shape), R, beta), w.motion)
        fd = (Jp - Jm) / 2e-5
        assert abs(fd - flat[c]) <= 1e-6 * abs(flat[c])

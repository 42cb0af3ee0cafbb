"""CPU oracle of the design-grid chain around the solver (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s baselines may import this
module.  Plain numpy in float64, no code shared with the CUDA library.

The paper binarises designs with the Heaviside projection filter it cites (Sec. 1; Sec. 3.1
sets the filter radius R = 2.4 dx and starts the steepness at beta = 1, doubled in
continuation) and constrains the volume with G = int gamma / (V_max int dOmega) - 1
(Eq. constraint, Sec. 2.1).  The paper does not write the filter out; the reading taken is the
usual pair of the cited method:

  density filter   gt_i = sum_j w_ij gamma_j / sum_j w_ij,  w_ij = max(0, R - |xi_i - xi_j|)
                   over the design nodes j of the grid (Euclidean distance in cells);
  projection       gb = [tanh(beta eta) + tanh(beta (gt - eta))] /
                        [tanh(beta eta) + tanh(beta (1 - eta))],  eta = 0.5;

and G is taken on the projected (physical) field gb with unit cell volumes:
G = sum gb / (V_max * n_design) - 1.  The solver sees kappa_ref(gb); dJ/dgamma follows by the
chain rule through the projection and the transposed filter.

Parity status: pinned by tests/test_oracle_design_chain.py (constants, adjointness, limits,
closed forms, finite differences of the composite).
"""
from __future__ import annotations

import itertools

import numpy as np


def _offsets(R: float, dim: int):
    """Integer offsets (dz, dy, dx) with |d| < R and their weights R - |d| (> 0)."""
    r = int(np.ceil(R))
    rng = range(-r, r + 1)
    out = []
    zr = rng if dim == 3 else (0,)
    for dz, dy, dx in itertools.product(zr, rng, rng):
        d = np.sqrt(dx * dx + dy * dy + dz * dz)
        if R - d > 0:
            out.append(((dz, dy, dx), R - d))
    return out


def filter_weights_sum(shape, R: float) -> np.ndarray:
    """W_i = sum_j w_ij over the design nodes j inside the grid (filter normaliser)."""
    dim = 3 if shape[0] > 1 else 2
    W = np.zeros(shape)
    for (dz, dy, dx), w in _offsets(R, dim):
        W += w * _shifted_ones(shape, dz, dy, dx)
    return W


def _shift(a, dz, dy, dx):
    """out_i = a_{i + d} where i + d is inside the grid, else 0."""
    r = max(abs(dz), abs(dy), abs(dx))
    P = np.pad(a, r)
    lz, ly, lx = a.shape
    return P[r + dz:r + dz + lz, r + dy:r + dy + ly, r + dx:r + dx + lx]


def _shifted_ones(shape, dz, dy, dx):
    """1 where node i + d lies inside the grid, else 0."""
    return _shift(np.ones(shape), dz, dy, dx)


def density_filter(gamma: np.ndarray, R: float) -> np.ndarray:
    """gt = F gamma (shape (lz, ly, lx))."""
    dim = 3 if gamma.shape[0] > 1 else 2
    acc = np.zeros_like(gamma, dtype=np.float64)
    for (dz, dy, dx), w in _offsets(R, dim):
        acc += w * _shift(gamma.astype(np.float64), dz, dy, dx)
    return acc / filter_weights_sum(gamma.shape, R)


def density_filter_T(g: np.ndarray, R: float) -> np.ndarray:
    """F^T g: out_j = sum_i w_ij g_i / W_i."""
    dim = 3 if g.shape[0] > 1 else 2
    h = g / filter_weights_sum(g.shape, R)
    acc = np.zeros_like(g, dtype=np.float64)
    for (dz, dy, dx), w in _offsets(R, dim):
        acc += w * _shift(h, dz, dy, dx)   # w_ij symmetric in i - j
    return acc


def project(gt: np.ndarray, beta: float, eta: float = 0.5) -> np.ndarray:
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return (np.tanh(beta * eta) + np.tanh(beta * (gt - eta))) / den


def project_prime(gt: np.ndarray, beta: float, eta: float = 0.5) -> np.ndarray:
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return beta * (1.0 - np.tanh(beta * (gt - eta)) ** 2) / den


def physical(gamma, R, beta, eta=0.5):
    """The field the solver sees: gb = H(F gamma)."""
    return project(density_filter(gamma, R), beta, eta)


def chain_T(gamma, dJ_dgb, R, beta, eta=0.5):
    """dJ/dgamma = F^T (H'(F gamma) * dJ/dgb)."""
    gt = density_filter(gamma, R)
    return density_filter_T(project_prime(gt, beta, eta) * dJ_dgb, R)


def volume(gamma, vmax, R=0.0, beta=1.0, eta=0.5):
    """G of Eq. constraint on the physical field and dG/dgamma."""
    gb = physical(gamma, R, beta, eta) if R > 0 else gamma.astype(np.float64)
    n = gamma.size
    G = gb.sum() / (vmax * n) - 1.0
    d = np.full(gamma.shape, 1.0 / (vmax * n))
    dG = chain_T(gamma, d, R, beta, eta) if R > 0 else d
    return G, dG

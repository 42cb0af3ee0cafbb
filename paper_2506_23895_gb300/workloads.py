"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the CPU oracle.

This module holds no arithmetic of the method itself: it only states problems (grid sizes,
boundary types, objective region, viscosity parameter), draws the design field gamma from a
counter-based generator, and tabulates the prescribed rigid-body schedule
(theta, omega, x_G, u_G per step) that Eqs. rigid_body_position / rigid_body_velocity
(Sec. 2.3) take as given.  Everything the method computes from these inputs lives on the
two independent sides (``oracle/`` and the CUDA library).

Input recipe (stated once here and in the design notes):
  * gamma: SplitMix64 (Steele, Lea & Flood 2014) counter stream -> U[0,1) doubles in C order
    over the design grid, separable Gaussian filter (truncate 4 sigma, half-sample symmetric
    edges), then min-max rescale to [0, 1].
  * motion: rotation at constant omega (theta_n = omega*n, Sec. 3.1/3.3 use 2*pi*t/N_t) plus an
    optional transverse sinusoidal translation of the centre (the 2D pump, Sec. 3.2);
    u_G is the analytic time derivative of x_G.
  * channels (2D) / ducts (3D): uniform inflow on the low face of the flow axis, prescribed
    density on the high face, no-slip walls elsewhere; the design grid is centred.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# face boundary types (faces ordered x-, x+, y-, y+, z-, z+)
PERIODIC, WALL, INLET, OUTLET = 0, 1, 2, 3
# objective kinds (Sec. 2.5): J1 mean pressure over a region, J2 mean directed velocity
OBJ_PRESSURE, OBJ_VELOCITY = 0, 1


@dataclasses.dataclass
class Problem:
    """One forward/adjoint problem: analysis grid, design grid, boundaries, objective.

    Grid nodes are indexed (x, y, z) with x fastest; 2D problems have nz = 1 and lz = 1.
    A design grid with lx == 0 means "no moving body" (kappa = 0, u_S = 0 everywhere).
    """

    dim: int
    n: Tuple[int, int, int]                 # analysis grid nx, ny, nz
    L: Tuple[int, int, int]                 # design grid lx, ly, lz
    A: float                                # viscosity parameter of the LKS equilibrium
    kappa_max: float = 100.0
    q: float = 0.1
    rho0: float = 1.0
    bc: Tuple[int, ...] = (PERIODIC,) * 6
    bc_val: Tuple[Tuple[float, float, float, float], ...] = ((0.0, 0.0, 0.0, 1.0),) * 6
    u_init: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    body_force: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    xi_G: Tuple[float, float, float] = (0.0, 0.0, 0.0)   # rotation centre in design coords
    rot_axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)   # 3D rotation axis (unit vector)
    obj_kind: int = OBJ_PRESSURE
    obj_box: Tuple[int, int, int, int, int, int] = (0, 0, 0, 0, 0, 0)  # inclusive x0,x1,y0,y1,z0,z1
    obj_dir: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    obj_cyl_r: float = 0.0                  # >0: also require (x-cx)^2+(y-cy)^2 <= r^2
    obj_cyl_c: Tuple[float, float] = (0.0, 0.0)
    win: Tuple[int, int] = (1, 1)           # objective window, inclusive step indices
    n_steps: int = 1
    name: str = ""

    @property
    def nodes(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def design_nodes(self) -> int:
        return self.L[0] * self.L[1] * self.L[2] if self.L[0] > 0 else 0

    def nu(self) -> float:
        """Kinematic viscosity implied by A (Sec. 2.2, nu = 1/6 - 2A/9 in lattice units)."""
        return 1.0 / 6.0 - 2.0 * self.A / 9.0


def A_from_nu(nu: float) -> float:
    """Invert nu = 1/6 - 2A/9 (lattice units)."""
    return 4.5 * (1.0 / 6.0 - nu)


# ----------------------------------------------------------------------------- random fields

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """`count` doubles in [0,1) from the SplitMix64 stream started at `seed` (counter form)."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.floor(4.0 * sigma + 0.5))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    return k / k.sum()


def gaussian_filter(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian smoothing, truncated at 4 sigma, half-sample symmetric edges."""
    if sigma <= 0:
        return a.copy()
    k = _gauss_kernel(sigma)
    r = (len(k) - 1) // 2
    out = a.astype(np.float64)
    for ax in range(out.ndim):
        if out.shape[ax] == 1:
            continue
        pad = [(0, 0)] * out.ndim
        pad[ax] = (r, r)
        p = np.pad(out, pad, mode="symmetric")
        acc = np.zeros_like(out)
        for j in range(len(k)):
            sl = [slice(None)] * out.ndim
            sl[ax] = slice(j, j + out.shape[ax])
            acc += k[j] * p[tuple(sl)]
        out = acc
    return out


def make_gamma(L: Sequence[int], sigma: float, seed: int) -> np.ndarray:
    """Design field gamma in [0,1], shape (lz, ly, lx), C order (x fastest)."""
    lx, ly, lz = L
    g = splitmix64_uniform(seed, lx * ly * lz).reshape(lz, ly, lx)
    g = gaussian_filter(g, sigma)
    lo, hi = g.min(), g.max()
    if hi > lo:
        g = (g - lo) / (hi - lo)
    else:
        g = np.zeros_like(g)
    return np.ascontiguousarray(g)


# ----------------------------------------------------------------------------- motion schedules

def motion_table(n_steps: int, x_c: Sequence[float], omega: float = 0.0,
                 trans_amp: float = 0.0, trans_period: float = 1.0, trans_axis: int = 1,
                 theta0: float = 0.0) -> np.ndarray:
    """Rows n = 0..n_steps of (theta, omega, xG[3], uG[3]) for a prescribed rigid motion.

    Rotation at constant rate (theta_n = theta0 + omega*n); the centre x_G oscillates along
    `trans_axis` as x_c + amp*sin(2*pi*n/period) with u_G its exact derivative.
    """
    t = np.arange(n_steps + 1, dtype=np.float64)
    m = np.zeros((n_steps + 1, 8), dtype=np.float64)
    m[:, 0] = theta0 + omega * t
    m[:, 1] = omega
    m[:, 2:5] = np.asarray(x_c, dtype=np.float64)[None, :]
    if trans_amp != 0.0:
        ph = 2.0 * math.pi * t / trans_period
        m[:, 2 + trans_axis] += trans_amp * np.sin(ph)
        m[:, 5 + trans_axis] = trans_amp * (2.0 * math.pi / trans_period) * np.cos(ph)
    return m


# ----------------------------------------------------------------------------- problems

def channel2d(N: int, LD: int, n_steps: int, win: Tuple[int, int], nu: float,
              u_in: float = 0.05, name: str = "") -> Tuple[Problem, float]:
    """2D channel: inlet x=0, outlet x=N-1 (rho=1), walls y=0,N-1; J1 on the inlet face."""
    c = (N - 1) / 2.0
    return Problem(
        dim=2, n=(N, N, 1), L=(LD, LD, 1), A=A_from_nu(nu),
        bc=(INLET, OUTLET, WALL, WALL, PERIODIC, PERIODIC),
        bc_val=((u_in, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0),
                (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0)),
        u_init=(u_in, 0.0, 0.0), xi_G=((LD - 1) / 2.0, (LD - 1) / 2.0, 0.0),
        obj_kind=OBJ_PRESSURE, obj_box=(0, 0, 1, N - 2, 0, 0),
        win=win, n_steps=n_steps, name=name), c


def duct3d(N: int, LD: int, n_steps: int, win: Tuple[int, int], nu: float,
           u_in: float = 0.05, name: str = "") -> Tuple[Problem, float]:
    """3D duct along z: inlet z=0, outlet z=N-1, walls on x and y faces.

    Objective J2: mean +z velocity in a cylinder coaxial with the rotation axis, diameter
    0.25*LD and height 0.12*LD, starting two cells above the design box (scaled from the
    3D rotor's target cylinder, Sec. 3.3)."""
    c = (N - 1) / 2.0
    r = 0.125 * LD
    h = max(1, int(round(0.12 * LD)))
    z0 = int(math.floor(c + (LD - 1) / 2.0)) + 2
    p = Problem(
        dim=3, n=(N, N, N), L=(LD, LD, LD), A=A_from_nu(nu),
        bc=(WALL, WALL, WALL, WALL, INLET, OUTLET),
        bc_val=((0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0),
                (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, u_in, 1.0), (0.0, 0.0, 0.0, 1.0)),
        u_init=(0.0, 0.0, u_in), xi_G=((LD - 1) / 2.0,) * 3,
        obj_kind=OBJ_VELOCITY,
        obj_box=(int(math.floor(c - r)), int(math.ceil(c + r)), int(math.floor(c - r)),
                 int(math.ceil(c + r)), z0, min(N - 2, z0 + h - 1)),
        obj_dir=(0.0, 0.0, 1.0), obj_cyl_r=r, obj_cyl_c=(c, c),
        win=win, n_steps=n_steps, name=name)
    return p, c


@dataclasses.dataclass
class Workload:
    problem: Problem
    gamma: np.ndarray
    motion: np.ndarray


def _last_fraction(n_steps: int, frac: float = 0.1) -> Tuple[int, int]:
    k = max(1, int(round(frac * n_steps)))
    return (n_steps - k + 1, n_steps)


def config(idx: int, n_steps: Optional[int] = None) -> Workload:
    """The named workloads (Sec. 3 example shapes, scaled):

    0: 2D D2Q9 128^2 channel, 48^2 design rotating (rim speed 0.05), sigma 3, 1000 steps,
       J1 averaged over steps 801..1000.
    1: 2D 512^2 channel, 192^2 design, rotation + transverse sinusoid (amp 20, period 2000),
       sigma 4, 20000 steps, window = last 2000 steps.
    3: 3D D3Q15 128^3 duct, 64^3 design rotating about the flow axis, 8000 steps.
    4: 3D 256^3 duct, 96^3 design, rotation + transverse sinusoid, 20000 steps.
    `n_steps` shortens the horizon (window = last 10 %, or 801..1000 scaled for cfg 0)."""
    u = 0.05
    if idx == 0:
        N, LD, steps, sigma = 128, 48, 1000, 3.0
        steps = steps if n_steps is None else n_steps
        win = (801, 1000) if steps == 1000 else _last_fraction(steps, 0.2)
        p, c = channel2d(N, LD, steps, win, nu=u * LD / 100.0, name="cfg0_2d_128")
        m = motion_table(steps, (c, c, 0.0), omega=u / (LD / 2.0))
        g = make_gamma((LD, LD, 1), sigma, seed=0)
    elif idx == 1:
        N, LD, steps, sigma = 512, 192, 20000, 4.0
        steps = steps if n_steps is None else n_steps
        p, c = channel2d(N, LD, steps, _last_fraction(steps), nu=u * LD / 100.0,
                         name="cfg1_2d_512")
        m = motion_table(steps, (c, c, 0.0), omega=u / (LD / 2.0), trans_amp=20.0,
                         trans_period=2000.0, trans_axis=1)
        g = make_gamma((LD, LD, 1), sigma, seed=1)
    elif idx == 3:
        N, LD, steps, sigma = 128, 64, 8000, 3.0
        steps = steps if n_steps is None else n_steps
        p, c = duct3d(N, LD, steps, _last_fraction(steps), nu=u * LD / 100.0,
                      name="cfg3_3d_128")
        m = motion_table(steps, (c, c, c), omega=u / (LD / 2.0))
        g = make_gamma((LD, LD, LD), sigma, seed=3)
    elif idx == 4:
        N, LD, steps, sigma = 256, 96, 20000, 3.0
        steps = steps if n_steps is None else n_steps
        p, c = duct3d(N, LD, steps, _last_fraction(steps), nu=u * LD / 100.0,
                      name="cfg4_3d_256")
        m = motion_table(steps, (c, c, c), omega=u / (LD / 2.0), trans_amp=20.0,
                         trans_period=2000.0, trans_axis=1)
        g = make_gamma((LD, LD, LD), sigma, seed=4)
    else:
        raise ValueError(f"no single-instance workload {idx}")
    return Workload(p, g, m)


def batch_config2(n_inst: int = 64, n_steps: int = 5000, side: Tuple[int, int] = (128, 512),
                  seed: int = 2) -> List[Workload]:
    """The batched 2D workload: n_inst independent channels with square analysis grids of side
    N drawn uniformly from side[0]..side[1], a centred design grid of side round(0.4 N) with its
    own gamma (sigma 3) rotating at a rim speed drawn from U[0.025, 0.1], viscosity from
    Re = 100 on the design side (nu = 0.05 L_D / 100), J1 over the last 10 % of the steps."""
    r = splitmix64_uniform(seed, 2 * n_inst)
    out = []
    for i in range(n_inst):
        N = side[0] + min(side[1] - side[0], int(r[2 * i] * (side[1] - side[0] + 1)))
        LD = max(4, int(round(0.4 * N)))
        rim = 0.025 + 0.075 * r[2 * i + 1]
        p, c = channel2d(N, LD, n_steps, _last_fraction(n_steps), nu=0.05 * LD / 100.0,
                         name=f"batch2d_{i}_{N}")
        m = motion_table(n_steps, (c, c, 0.0), omega=rim / (LD / 2.0))
        g = make_gamma((LD, LD, 1), 3.0, seed=1000 * seed + i)
        out.append(Workload(p, g, m))
    return out


def small_channel2d(nx: int = 24, ny: int = 20, LD: int = 8, n_steps: int = 40,
                    omega: float = 0.02, trans_amp: float = 1.5, seed: int = 11,
                    obj_kind: int = OBJ_PRESSURE, A: float = 0.45) -> Workload:
    """A few-hundred-node 2D channel with a rotating and translating design grid."""
    cx, cy = (nx - 1) / 2.0, (ny - 1) / 2.0
    box = (0, 0, 1, ny - 2, 0, 0) if obj_kind == OBJ_PRESSURE else (nx - 4, nx - 3, 2, ny - 3, 0, 0)
    p = Problem(
        dim=2, n=(nx, ny, 1), L=(LD, LD, 1), A=A,
        bc=(INLET, OUTLET, WALL, WALL, PERIODIC, PERIODIC),
        bc_val=((0.04, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0),
                (0.01, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0)),
        u_init=(0.04, 0.0, 0.0), xi_G=((LD - 1) / 2.0, (LD - 1) / 2.0, 0.0),
        obj_kind=obj_kind, obj_box=box, obj_dir=(1.0, 0.0, 0.0),
        win=(max(1, n_steps // 2), n_steps), n_steps=n_steps, name="small2d")
    m = motion_table(n_steps, (cx, cy, 0.0), omega=omega, trans_amp=trans_amp,
                     trans_period=max(60.0, n_steps / 1.5), trans_axis=1, theta0=0.3)
    g = make_gamma((LD, LD, 1), 1.0, seed)
    return Workload(p, g, m)


def unit(v: Sequence[float]) -> Tuple[float, float, float]:
    """v / |v| as a tuple (a rotation axis)."""
    n = math.sqrt(sum(float(a) * float(a) for a in v))
    return (float(v[0]) / n, float(v[1]) / n, float(v[2]) / n)


def small_duct3d(nx: int = 16, ny: int = 15, nz: int = 16, LD: int = 5, n_steps: int = 24,
                 omega: float = 0.03, trans_amp: float = 1.0, seed: int = 12,
                 obj_kind: int = OBJ_VELOCITY, A: float = 0.45,
                 rot_axis: Tuple[float, float, float] = (0.0, 0.0, 1.0)) -> Workload:
    """A few-thousand-node 3D duct with a design grid rotating about rot_axis (default z) and
    translating in y."""
    cx, cy, cz = (nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0
    if obj_kind == OBJ_VELOCITY:
        box = (int(cx) - 2, int(cx) + 2, int(cy) - 2, int(cy) + 2, nz - 4, nz - 3)
    else:
        box = (1, nx - 2, 1, ny - 2, 0, 0)
    p = Problem(
        dim=3, n=(nx, ny, nz), L=(LD, LD, LD), A=A,
        bc=(WALL, WALL, WALL, WALL, INLET, OUTLET),
        bc_val=((0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.01, 0.0, 1.0),
                (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.04, 1.0), (0.0, 0.0, 0.0, 1.0)),
        u_init=(0.0, 0.0, 0.04), xi_G=((LD - 1) / 2.0,) * 3,
        obj_kind=obj_kind, obj_box=box, obj_dir=(0.0, 0.0, 1.0),
        obj_cyl_r=2.5 if obj_kind == OBJ_VELOCITY else 0.0, obj_cyl_c=(cx, cy),
        win=(max(1, n_steps // 2), n_steps), n_steps=n_steps, name="small3d",
        rot_axis=tuple(rot_axis))
    m = motion_table(n_steps, (cx, cy, cz + 0.25), omega=omega, trans_amp=trans_amp,
                     trans_period=max(40.0, n_steps / 1.5), trans_axis=1, theta0=0.2)
    g = make_gamma((LD, LD, LD), 1.0, seed)
    return Workload(p, g, m)


def periodic_box(dim: int, n: Tuple[int, int, int], A: float = 0.4,
                 L: Tuple[int, int, int] = (0, 0, 0), n_steps: int = 10) -> Problem:
    """Fully periodic box (no walls), used for closed-form and invariant checks."""
    return Problem(dim=dim, n=n, L=L, A=A, bc=(PERIODIC,) * 6,
                   obj_kind=OBJ_PRESSURE, obj_box=(0, n[0] - 1, 0, n[1] - 1, 0, n[2] - 1),
                   win=(1, n_steps), n_steps=n_steps, name="periodic")


def static_box(p: Problem, box: Tuple[int, int, int, int, int, int], kappa: float) -> np.ndarray:
    """Static Brinkman field (nz, ny, nx): kappa on the inclusive box x0,x1,y0,y1,z0,z1."""
    nx, ny, nz = p.n
    k = np.zeros((nz, ny, nx), dtype=np.float64)
    k[box[4]:box[5] + 1, box[2]:box[3] + 1, box[0]:box[1] + 1] = kappa
    return k


def taylor_couette(N: int = 200, r1: float = 45.0, r2: float = 70.0, u_d: float = 0.01,
                   A: float = 0.3, n_steps: int = 12000, kappa_max: float = 100.0) -> Tuple[
                       Workload, np.ndarray]:
    """The appendix's verification case: in a periodic N x N box an inner disk of radius r1
    (a solid design, gamma = 1) rotates at omega = u_d / r1 about the centre inside a fixed
    outer wall, a static solid outside radius r2.  Returns the workload and the static field."""
    LD = int(2 * math.ceil(r1) + 10)
    c = (N - 1) / 2.0
    p = periodic_box(2, (N, N, 1), A=A, L=(LD, LD, 1), n_steps=n_steps)
    p.kappa_max = kappa_max
    p.xi_G = ((LD - 1) / 2.0, (LD - 1) / 2.0, 0.0)
    p.obj_kind = OBJ_VELOCITY
    p.obj_dir = (1.0, 0.0, 0.0)
    p.obj_box = (0, N - 1, 0, N - 1, 0, 0)
    p.win = (n_steps, n_steps)
    p.name = "taylor_couette"
    ii, jj = np.meshgrid(np.arange(LD), np.arange(LD))
    g = ((ii - p.xi_G[0]) ** 2 + (jj - p.xi_G[1]) ** 2 <= r1 * r1).astype(np.float64)[None]
    m = motion_table(n_steps, (c, c, 0.0), omega=u_d / r1)
    xx, yy = np.meshgrid(np.arange(N), np.arange(N))
    ks = np.where((xx - c) ** 2 + (yy - c) ** 2 >= r2 * r2, kappa_max, 0.0)[None]
    return Workload(p, g, m), ks


def initial_state(p: Problem, rho: Optional[np.ndarray] = None,
                  u: Optional[Sequence[np.ndarray]] = None) -> np.ndarray:
    """A state array of shape (4, nz, ny, nx): (rho, ux, uy, uz) planes."""
    nx, ny, nz = p.n
    s = np.zeros((4, nz, ny, nx), dtype=np.float64)
    s[0] = p.rho0 if rho is None else rho
    if u is None:
        for a in range(3):
            s[1 + a] = p.u_init[a]
    else:
        for a in range(3):
            s[1 + a] = u[a]
    return s

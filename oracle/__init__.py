"""CPU oracle: plain single-threaded FP64 C++ restatement of the method (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference arm may
import this package.  It shares no code with the CUDA library and never calls it.

Functions take a problem object with the attributes of ``workloads.Problem`` (duck typed), a
design field gamma of shape (lz, ly, lx) and a motion table of rows
(theta, omega, xG[3], uG[3]) for steps 0..N.

Parity status: every entry point here is pinned by ``tests/test_oracle_*.py`` (closed forms,
invariants, hand-computed transfer weights, complex-step and central differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lks_oracle.cpp")
_SO = os.path.join(_HERE, "liblks_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FP contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_int), ("ly", ctypes.c_int), ("lz", ctypes.c_int),
        ("A", ctypes.c_double), ("kappa_max", ctypes.c_double), ("q", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("bc_val", (ctypes.c_double * 4) * 6),
        ("u_init", ctypes.c_double * 3), ("body_force", ctypes.c_double * 3),
        ("xi_G", ctypes.c_double * 3),
        ("obj_kind", ctypes.c_int),
        ("obj_box", ctypes.c_int * 6),
        ("obj_dir", ctypes.c_double * 3),
        ("obj_cyl_r", ctypes.c_double), ("obj_cyl_c", ctypes.c_double * 2),
        ("win_begin", ctypes.c_int), ("win_end", ctypes.c_int),
        ("rot_axis", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.POINTER(OrcProblem)
            D = ctypes.POINTER(ctypes.c_double)
            lib.orc_forward.argtypes = [P, D, D, ctypes.c_int, D, D, D, D, D]
            lib.orc_gradient.argtypes = [P, D, D, ctypes.c_int, D, D, D, D, D, D]
            lib.orc_gradient_printed.argtypes = [P, D, D, ctypes.c_int, D, D]
            lib.orc_complex_step.argtypes = [P, D, D, ctypes.c_int, D, D, D, ctypes.c_double, D,
                                             D]
            lib.orc_transfer.argtypes = [P, D, D, D, D]
            lib.orc_transfer_T.argtypes = [P, D, D, D]
            lib.orc_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def to_struct(p) -> OrcProblem:
    s = OrcProblem()
    s.dim = p.dim
    s.nx, s.ny, s.nz = p.n
    s.lx, s.ly, s.lz = p.L
    s.A, s.kappa_max, s.q, s.rho0 = p.A, p.kappa_max, p.q, p.rho0
    for f in range(6):
        s.bc[f] = p.bc[f]
        for k in range(4):
            s.bc_val[f][k] = p.bc_val[f][k]
    for a in range(3):
        s.u_init[a] = p.u_init[a]
        s.body_force[a] = p.body_force[a]
        s.xi_G[a] = p.xi_G[a]
        s.obj_dir[a] = p.obj_dir[a]
    s.obj_kind = p.obj_kind
    for k in range(6):
        s.obj_box[k] = p.obj_box[k]
    s.obj_cyl_r = p.obj_cyl_r
    s.obj_cyl_c[0], s.obj_cyl_c[1] = p.obj_cyl_c
    s.win_begin, s.win_end = p.win
    ax = getattr(p, "rot_axis", (0.0, 0.0, 1.0))
    for a in range(3):
        s.rot_axis[a] = ax[a]
    return s


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _check(rc):
    if rc != 0:
        raise RuntimeError("oracle: " + _load().orc_error().decode())


def _gamma_or_empty(p, gamma):
    if gamma is None or p.L[0] == 0:
        return np.zeros(1, dtype=np.float64)
    return _c64(gamma)


def forward(p, gamma, motion, n_steps=None, init_state=None, kstatic=None, lam_term=None):
    """Alg. 1 from the initial state; returns (J, final_state[4, nz, ny, nx]).

    kstatic: static Brinkman coefficient per analysis node (solid at rest), shape
    (nz, ny, nx); lam_term: planes (4, nz, ny, nx) of a terminal term <lam_term, s^N> added
    to J."""
    lib = _load()
    N = p.n_steps if n_steps is None else n_steps
    st = to_struct(p)
    g = _gamma_or_empty(p, gamma)
    m = _c64(motion)
    J = ctypes.c_double(0.0)
    out = np.zeros((4, p.n[2], p.n[1], p.n[0]), dtype=np.float64)
    _check(lib.orc_forward(ctypes.byref(st), _dp(g), _dp(m), N, _dp(_c64(init_state)),
                           _dp(_c64(kstatic)), _dp(_c64(lam_term)), ctypes.byref(J), _dp(out)))
    return J.value, out


def gradient(p, gamma, motion, n_steps=None, init_state=None, kstatic=None, lam_term=None,
             want_lam0=False):
    """Forward plus exact discrete adjoint; returns (J, dJ/dgamma with gamma's shape), plus
    lambda^0 (planes) when want_lam0."""
    lib = _load()
    N = p.n_steps if n_steps is None else n_steps
    st = to_struct(p)
    g = _c64(gamma)
    m = _c64(motion)
    J = ctypes.c_double(0.0)
    out = np.zeros_like(g)
    lam0 = np.zeros((4, p.n[2], p.n[1], p.n[0]), dtype=np.float64) if want_lam0 else None
    _check(lib.orc_gradient(ctypes.byref(st), _dp(g), _dp(m), N, _dp(_c64(init_state)),
                            _dp(_c64(kstatic)), _dp(_c64(lam_term)), ctypes.byref(J), _dp(out),
                            _dp(lam0)))
    return (J.value, out, lam0) if want_lam0 else (J.value, out)


def gradient_printed(p, gamma, motion, n_steps=None):
    """Sec. 2.4's adjoint as printed (not the exact discrete adjoint); returns (J, dJ/dgamma)."""
    lib = _load()
    N = p.n_steps if n_steps is None else n_steps
    st = to_struct(p)
    g = _c64(gamma)
    J = ctypes.c_double(0.0)
    out = np.zeros_like(g)
    _check(lib.orc_gradient_printed(ctypes.byref(st), _dp(g), _dp(_c64(motion)), N,
                                    ctypes.byref(J), _dp(out)))
    return J.value, out


def complex_step(p, gamma, motion, direction, h=1e-30, n_steps=None, kstatic=None,
                 lam_term=None):
    """Directional derivative dJ/dgamma . direction by the complex step; returns (dJ, J)."""
    lib = _load()
    N = p.n_steps if n_steps is None else n_steps
    st = to_struct(p)
    g = _c64(gamma)
    d = _c64(direction)
    m = _c64(motion)
    dJ = ctypes.c_double(0.0)
    J = ctypes.c_double(0.0)
    _check(lib.orc_complex_step(ctypes.byref(st), _dp(g), _dp(m), N, _dp(_c64(kstatic)),
                                _dp(_c64(lam_term)), _dp(d), h, ctypes.byref(dJ),
                                ctypes.byref(J)))
    return dJ.value, J.value


def transfer(p, gamma, motion_row):
    """kappa[nz,ny,nx] and u_S[3,nz,ny,nx] for one motion row."""
    lib = _load()
    st = to_struct(p)
    g = _gamma_or_empty(p, gamma)
    row = _c64(motion_row).reshape(8)
    kap = np.zeros((p.n[2], p.n[1], p.n[0]), dtype=np.float64)
    us = np.zeros((3, p.n[2], p.n[1], p.n[0]), dtype=np.float64)
    _check(lib.orc_transfer(ctypes.byref(st), _dp(g), _dp(row), _dp(kap), _dp(us)))
    return kap, us


def transfer_T(p, motion_row, e):
    """out[lz,ly,lx] = sum_x W(x - x_ref(xi)) e(x)."""
    lib = _load()
    st = to_struct(p)
    row = _c64(motion_row).reshape(8)
    ee = _c64(e)
    lz = 1 if p.dim == 2 else p.L[2]
    out = np.zeros((lz, p.L[1], p.L[0]), dtype=np.float64)
    _check(lib.orc_transfer_T(ctypes.byref(st), _dp(row), _dp(ee), _dp(out)))
    return out

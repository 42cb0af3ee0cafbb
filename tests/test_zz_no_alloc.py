"""The allocation-free step (lks_step_noalloc) against the library's normal forward step and
against the CPU oracle.

lks_step_noalloc exists for callers that cannot allocate device memory when they need a step
(stream capture into a CUDA graph, memory owned by a host framework's pool, loops that must not
block on the allocator).  It keeps its scratch in a static device array, so these tests call it
twice in a row through the C ABI and check both results against the oracle's step from the same
state and against lks_forward(1) of a normal context, within the tolerances the parity tests use
for the precision, with and without a body (kappa_us = NULL).  The file name makes pytest
collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2506_23895_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2506_23895_gb300 import build as B
    B.build()
    from paper_2506_23895_gb300 import lks
    import torch
    assert torch.cuda.is_available()
    lib = lks.load()
    lib.lks_step_noalloc.argtypes = [ctypes.POINTER(lks.LksConfig), ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p,
                                     ctypes.c_size_t]
    lib.lks_step_noalloc.restype = ctypes.c_int
    return lks


def _node_records(planes, rho0, dtype):
    """(rho, ux, uy, uz) planes -> per-node records (rho - rho0, ux, uy, uz)."""
    rec = np.stack([planes[0] - rho0, planes[1], planes[2], planes[3]], axis=-1)
    return np.ascontiguousarray(rec.astype(dtype))


@pytest.mark.parametrize("name,prec", [("2d", 0), ("3d", 0), ("3d", 1)])
def test_noalloc_step_matches_forward_step(L, name, prec):
    import torch

    w = W.small_channel2d() if name == "2d" else W.small_duct3d()
    p = w.problem
    s = L.Solver(p, prec)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    s0 = s.get_state()                 # initial state (boundary values applied)
    kap, us = s.transfer(1)            # kappa and u_S of step 1
    s.forward(1)
    ref = s.get_state()
    s.close()

    dtype = np.float64 if prec == 1 else np.float32
    tdt = torch.float64 if prec == 1 else torch.float32
    st_in = torch.from_numpy(_node_records(s0, p.rho0, dtype)).cuda()
    kus = torch.from_numpy(np.ascontiguousarray(
        np.stack([kap, us[0], us[1], us[2]], axis=-1).astype(dtype))).cuda()
    cfg = L.make_config(p, prec)
    err = ctypes.create_string_buffer(256)
    lib = L.load()
    outs = []
    for _ in range(2):
        out = torch.full_like(st_in, float("nan"))
        torch.cuda.synchronize()
        rc = lib.lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(st_in.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(kus.data_ptr()),
                                  err, 256)
        assert rc == 0, err.value.decode()
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        outs.append(np.stack([o[..., 0] + p.rho0, o[..., 1], o[..., 2], o[..., 3]]))
    _, orc = oracle.forward(p, w.gamma, w.motion, n_steps=1, init_state=s0)
    tol = 1e-11 if prec == 1 else 1e-5
    for o in outs:
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - ref)) <= tol * np.max(np.abs(ref))
        assert np.max(np.abs(o - orc)) <= tol * np.max(np.abs(orc))
    assert np.array_equal(outs[0], outs[1])


def _noalloc(L, cfg, st_in, out, kus):
    err = ctypes.create_string_buffer(256)
    rc = L.load().lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(st_in.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()),
                                   None if kus is None else ctypes.c_void_p(kus.data_ptr()),
                                   err, 256)
    return rc, err.value.decode()


@pytest.mark.parametrize("name,prec", [("2d", 0), ("3d", 0), ("3d", 1)])
def test_noalloc_step_without_body_matches_oracle(L, name, prec):
    """kappa_us = NULL: no body anywhere (kappa = 0); a seeded non-uniform state."""
    import torch

    w = W.small_channel2d() if name == "2d" else W.small_duct3d()
    p = W.Problem(**{**w.problem.__dict__, "L": (0, 0, 0)})
    nx, ny, nz = p.n
    r = W.splitmix64_uniform(77, 4 * nx * ny * nz).reshape(4, nz, ny, nx)
    s0 = np.empty_like(r)
    s0[0] = p.rho0 + 0.01 * (r[0] - 0.5)
    for a in range(3):
        s0[1 + a] = 0.03 * (r[1 + a] - 0.5)
    if p.dim == 2:
        s0[3] = 0.0
    _, orc = oracle.forward(p, None, np.zeros((2, 8)), n_steps=1, init_state=s0)
    dtype = np.float64 if prec == 1 else np.float32
    st_in = torch.from_numpy(_node_records(s0, p.rho0, dtype)).cuda()
    cfg = L.make_config(p, prec)
    tol = 1e-11 if prec == 1 else 1e-5
    outs = []
    for _ in range(2):
        out = torch.full_like(st_in, float("nan"))
        torch.cuda.synchronize()
        rc, msg = _noalloc(L, cfg, st_in, out, None)
        assert rc == 0, msg
        torch.cuda.synchronize()
        o = out.cpu().numpy().astype(np.float64)
        outs.append(np.stack([o[..., 0] + p.rho0, o[..., 1], o[..., 2], o[..., 3]]))
    for o in outs:
        assert np.max(np.abs(o - orc)) <= tol * np.max(np.abs(orc))
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_step_rejects_misaligned_records(L):
    """An address that is not a whole node record is refused before anything is launched."""
    p = W.small_duct3d().problem
    for prec, bad in ((0, 20), (1, 16)):
        cfg = L.make_config(p, prec)
        err = ctypes.create_string_buffer(256)
        lib = L.load()
        rc = lib.lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(bad), ctypes.c_void_p(256),
                                  None, err, 256)
        assert rc == 1 and b"aligned" in err.value
        rc = lib.lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                  ctypes.c_void_p(256 + bad), err, 256)
        assert rc == 1 and b"aligned" in err.value


def test_noalloc_step_rejects_grids_beyond_its_scratch(L):
    p = W.small_duct3d().problem
    big = W.Problem(**{**p.__dict__, "n": (96, 96, 96), "L": (0, 0, 0)})
    cfg = L.make_config(big, 0)
    err = ctypes.create_string_buffer(256)
    rc = L.load().lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                   None, err, 256)
    assert rc == 1
    assert b"limit" in err.value

"""The allocation-free step (lks_step_noalloc) against the library's normal forward step.

lks_step_noalloc exists for callers that cannot allocate device memory when they need a step
(stream capture into a CUDA graph, memory owned by a host framework's pool, loops that must not
block on the allocator).  It keeps its scratch in a static device array, so this test calls it
twice in a row through the C ABI and checks both results against lks_forward(1) of a normal
context, within the tolerances the parity tests use for the precision.  The file name makes
pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

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
    tol = 1e-11 if prec == 1 else 1e-5
    for o in outs:
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - ref)) <= tol * np.max(np.abs(ref))
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_step_rejects_grids_beyond_its_scratch(L):
    p = W.small_duct3d().problem
    big = W.Problem(**{**p.__dict__, "n": (96, 96, 96), "L": (0, 0, 0)})
    cfg = L.make_config(big, 0)
    err = ctypes.create_string_buffer(256)
    rc = L.load().lks_step_noalloc(ctypes.byref(cfg), ctypes.c_void_p(16), ctypes.c_void_p(16),
                                   None, err, 256)
    assert rc == 1
    assert b"limit" in err.value

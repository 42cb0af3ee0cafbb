"""Failure detection without a GPU fault: the failures are made on the host.

* Divergence: an initial state with the fluid at |u| = 0.8 (outside the scheme's low-Mach
  range) or with a patch of NaN must end the forward run with LKS_ERR_DIVERGED; the context stays
  usable, the adjoint refuses to run on the failed forward (LKS_ERR_ORDER), and after the
  initial state is reset and the design set again the next run is bitwise that of a fresh
  context.
* Out of memory: lks_inject_alloc_failure makes one device allocation of the library report
  failure without calling the allocator; each entry point that allocates must return
  LKS_ERR_NOMEM, keep nothing of what it took (the device's free memory is unchanged over many
  failures) and work again on the next call.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_23895_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DIVERGED, ORDER, NOMEM = 5, 2, 3


@pytest.fixture(scope="module")
def L():
    from paper_2506_23895_gb300 import build as B
    B.build()
    from paper_2506_23895_gb300 import lks
    import torch
    assert torch.cuda.is_available()
    return lks


CASES = {
    "3d_fp32": (lambda: W.small_duct3d(nx=34, ny=17, nz=12, n_steps=8), 0),
    "3d_fp64": (lambda: W.small_duct3d(n_steps=8), 1),
    "2d_fp32": (lambda: W.small_channel2d(n_steps=8), 0),
}


def _fresh(L, w, prec):
    s = L.Solver(w.problem, prec)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    return s


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("poison", ["fast", "nan"])
def test_divergence_is_reported_and_the_context_recovers(L, name, poison):
    make, prec = CASES[name]
    w = make()
    p = w.problem
    ref = _fresh(L, w, prec)
    J_ref = ref.forward()
    g_ref = ref.adjoint()
    ref.close()

    s = _fresh(L, w, prec)
    bad = s.get_state()
    nx, ny, nz = p.n
    zc = nz // 2
    patch = (slice(zc, zc + 1), slice(ny // 2 - 2, ny // 2 + 2), slice(nx // 2 - 3, nx // 2 + 3))
    if poison == "fast":
        # the whole fluid at |u| = 0.8: far too fast for the scheme, and still above the
        # check's 0.5 in the core after the few steps of the run
        bad[1][:, 1:ny - 1, 1:nx - 1] = 0.8
    else:
        bad[0][patch] = np.nan
    s.set_initial_state(bad)
    with pytest.raises(L.LksError) as e:
        s.forward()
    assert e.value.status == DIVERGED
    with pytest.raises(L.LksError) as e:
        s.adjoint()
    assert e.value.status == ORDER
    s.set_initial_state(None)
    s.set_design(w.gamma)
    J = s.forward()
    g = s.adjoint()
    s.close()
    assert J == J_ref
    assert np.array_equal(g, g_ref)


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    torch.cuda.empty_cache()   # torch's cached blocks are not the library's
    return torch.cuda.mem_get_info()[0]


def test_allocation_failures_return_nomem_and_leak_nothing(L):
    import torch

    lib = L.load()
    assert lib.lks_inject_alloc_failure(0) == 0
    w = W.small_duct3d(nx=40, ny=40, nz=40, LD=6, n_steps=6)
    cfg = L.make_config(w.problem, L.FP32)
    ws = lib.lks_workspace_bytes(ctypes.byref(cfg))
    assert ws > 4 << 20
    torch.cuda.synchronize()
    free0 = _free_bytes()
    # lks_create without a caller workspace: the library allocates it
    for _ in range(8):
        out = ctypes.c_void_p()
        lib.lks_inject_alloc_failure(1)
        assert lib.lks_create(ctypes.byref(cfg), None, 0, ctypes.byref(out)) == NOMEM
        assert not out.value
    assert lib.lks_inject_alloc_failure(0) == 0
    assert abs(_free_bytes() - free0) < ws // 2
    # a context whose own workspace was allocated, then failures in its temporary buffers
    ctx = ctypes.c_void_p()
    assert lib.lks_create(ctypes.byref(cfg), None, 0, ctypes.byref(ctx)) == 0
    try:
        g = np.ascontiguousarray(w.gamma)
        assert lib.lks_set_design(ctx, g.ctypes.data_as(ctypes.c_void_p), 0) == 0
        rows = np.ascontiguousarray(w.motion)
        m = L.LksMotion(rows.shape[0], rows.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert lib.lks_set_motion(ctx, ctypes.byref(m)) == 0
        nodes = w.problem.nodes
        st = np.zeros(4 * nodes)
        kap = np.zeros(nodes)
        us = np.zeros(3 * nodes)
        D = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        free1 = _free_bytes()
        for _ in range(4):
            lib.lks_inject_alloc_failure(1)
            assert lib.lks_get_state(ctx, D(st)) == NOMEM
            assert b"allocation" in lib.lks_last_error(ctx)
            lib.lks_inject_alloc_failure(1)
            assert lib.lks_transfer(ctx, 2, D(kap), D(us)) == NOMEM
            lib.lks_inject_alloc_failure(1)
            assert lib.lks_set_initial_state(ctx, D(st)) == NOMEM
        assert lib.lks_inject_alloc_failure(0) == 0
        assert abs(_free_bytes() - free1) < 1 << 20
        # everything works again, and the run equals one without the failures
        assert lib.lks_get_state(ctx, D(st)) == 0
        assert lib.lks_set_initial_state(ctx, None) == 0
        J = ctypes.c_double()
        assert lib.lks_forward(ctx, w.problem.n_steps, ctypes.byref(J)) == 0
        s = L.Solver(w.problem, L.FP32)
        s.set_design(w.gamma)
        s.set_motion(w.motion)
        assert s.forward() == J.value
        s.close()
    finally:
        lib.lks_inject_alloc_failure(0)
        lib.lks_destroy(ctx)
    assert abs(_free_bytes() - free0) < ws // 2


def test_batch_create_allocation_failure(L):
    lib = L.load()
    ws = [W.small_channel2d(nx=30 + 4 * i, ny=24, n_steps=6, seed=40 + i) for i in range(3)]
    sol = [L.Solver(w.problem, L.FP32) for w in ws]
    arr = (ctypes.c_void_p * 3)(*[s.ctx.value for s in sol])
    out = ctypes.c_void_p()
    lib.lks_inject_alloc_failure(1)
    try:
        assert lib.lks_batch_create(arr, 3, ctypes.byref(out)) == NOMEM
        assert not out.value
    finally:
        lib.lks_inject_alloc_failure(0)
    assert lib.lks_batch_create(arr, 3, ctypes.byref(out)) == 0
    lib.lks_batch_destroy(out)
    for s in sol:
        s.close()

"""Host-only checks of the C ABI: the library builds and loads, exports every symbol that
include/lks.h declares, sizes workspaces, and its checkpoint schedule reverses every segment
exactly once within the snapshot budget (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2506_23895_gb300 import build as B
from paper_2506_23895_gb300 import lks
from paper_2506_23895_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lks.load()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lks_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lks.EXPORTS)


def test_workspace_bytes_and_invalid_configs(lib):
    w = W.small_duct3d()
    c = lks.make_config(w.problem, lks.FP32)
    n32 = lib.lks_workspace_bytes(ctypes.byref(c))
    c64 = lks.make_config(w.problem, lks.FP64)
    n64 = lib.lks_workspace_bytes(ctypes.byref(c64))
    assert n32 > 0 and n64 > n32
    bad = lks.make_config(w.problem, lks.FP32)
    bad.bc[0] = 0  # periodic on one face only
    assert lib.lks_workspace_bytes(ctypes.byref(bad)) == 0
    bad = lks.make_config(w.problem, lks.FP32)
    bad.nx = 2
    assert lib.lks_workspace_bytes(ctypes.byref(bad)) == 0
    bad = lks.make_config(w.problem, lks.FP32)
    bad.A = 0.8  # non-positive viscosity
    assert lib.lks_workspace_bytes(ctypes.byref(bad)) == 0
    # a checkpoint budget caps the snapshot pool
    big = lks.make_config(W.config(4).problem, lks.FP32)
    full = lib.lks_workspace_bytes(ctypes.byref(big))
    assert full < 100 * 2 ** 30  # two-level minimum, not 20001 snapshots
    big.ckpt_bytes = 8 * 2 ** 30
    assert lib.lks_workspace_bytes(ctypes.byref(big)) < full


def simulate(actions, n_seg, free_slots):
    """Replay a schedule; return the reversed order and the number of segment advances."""
    stored = {0}
    slots = 0
    work = None
    reversed_order = []
    advances = 0
    taped = None
    for kind, a, b in actions:
        if kind == 0:      # restore
            assert a in stored
            work = a
        elif kind == 1:    # advance a -> b
            assert work == a and b > a
            advances += b - a
            work = b
        elif kind == 2:    # store
            assert work == a and a not in stored
            stored.add(a)
            slots += 1
            assert slots <= free_slots
        elif kind == 3:    # free
            stored.remove(a)
            slots -= 1
        elif kind == 4:    # tape segment a
            assert work == a
            advances += 1
            taped = a
            work = a + 1
        elif kind == 5:    # adjoint over segment a
            assert taped == a
            reversed_order.append(a)
            taped = None
    return reversed_order, advances


@pytest.mark.parametrize("n_seg,slots", [(1, 0), (5, 4), (10, 9), (141, 140), (30, 4), (50, 2),
                                         (12, 0), (200, 6)])
def test_checkpoint_schedule_reverses_everything_within_budget(lib, n_seg, slots):
    acts = lks.checkpoint_schedule(n_seg, slots)
    order, adv = simulate(acts, n_seg, slots)
    assert order == list(range(n_seg - 1, -1, -1))
    if slots >= n_seg - 1:
        assert adv == 2 * n_seg - 1 or n_seg == 1  # one extra pass over all but the last
    # binomial bound: with s slots and r sweeps, C(s+r, s) segments need at most r advances each
    from math import comb
    s = slots
    if s > 0:
        r = 1
        while comb(s + r, s) < n_seg:
            r += 1
        assert adv <= (r + 1) * n_seg


def test_rotation_axis_and_transfer_sets_in_the_workspace(lib):
    """A tilted rotation axis adds the cell-list scratch; a non-unit axis is rejected; the z
    axis given explicitly (or as all zeros) sizes like the default; 3D contexts carry a second
    transfer buffer set, 2D ones do not."""
    w = W.small_duct3d()
    base = lib.lks_workspace_bytes(ctypes.byref(lks.make_config(w.problem, lks.FP32)))
    for axis in ((0.0, 0.0, 1.0), (0.0, 0.0, 0.0)):
        w.problem.rot_axis = axis
        assert lib.lks_workspace_bytes(ctypes.byref(lks.make_config(w.problem, lks.FP32))) == base
    w.problem.rot_axis = W.unit((1.0, 2.0, 2.0))
    tilted = lib.lks_workspace_bytes(ctypes.byref(lks.make_config(w.problem, lks.FP32)))
    nodes = w.problem.nodes
    assert tilted >= base + nodes * (4 + 8 * 4)   # cell counts and lists over the whole grid
    w.problem.rot_axis = (0.0, 0.6, 0.6)
    assert lib.lks_workspace_bytes(ctypes.byref(lks.make_config(w.problem, lks.FP32))) == 0
    # the second transfer set of a 3D context holds at least another kappa/u_S box
    w3 = W.small_duct3d()
    c3 = lks.make_config(w3.problem, lks.FP32)
    n3 = lib.lks_workspace_bytes(ctypes.byref(c3))
    c3.lx = c3.ly = c3.lz = 0          # no design grid: no transfer buffers at all
    n3_empty = lib.lks_workspace_bytes(ctypes.byref(c3))
    assert n3 - n3_empty >= 2 * w3.problem.nodes * 16


def test_step_variant_argument_checks(lib):
    lib.lks_step_variant.restype = ctypes.c_int
    v = ctypes.c_int(7)
    assert lib.lks_step_variant(None, 0, ctypes.byref(v)) == 1   # LKS_ERR_ARG without a context
    assert v.value == 7


def test_alloc_failure_injection_on_the_host(lib):
    """The fault-injection countdown: lks_create without a caller workspace fails with
    LKS_ERR_NOMEM at the injected allocation, leaves no context behind, and the countdown
    is consumed (host side only: the injected allocation never reaches the driver)."""
    assert lib.lks_inject_alloc_failure(0) == 0
    w = W.small_duct3d()
    c = lks.make_config(w.problem, lks.FP32)
    out = ctypes.c_void_p(12345)
    assert lib.lks_inject_alloc_failure(1) == 0
    rc = lib.lks_create(ctypes.byref(c), None, 0, ctypes.byref(out))
    assert rc == 3 and not out.value
    assert lib.lks_inject_alloc_failure(0) == 0   # consumed by that allocation
    assert lib.lks_inject_alloc_failure(5) == 0
    assert lib.lks_inject_alloc_failure(0) == 5

"""Fused D2Q9 kernels and batches of contexts (lks_batch_*) on the GPU.

The fused 2D kernels are checked against the plain per-node kernels and the oracle; a batch
must reproduce every member's single-context run bit for bit (same kernels, same arithmetic
per node, only the launch covers all members), whatever the tile shape, with or without CUDA
graphs, and with checkpoint recomputation.
"""
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
    return lks


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def single(L, w, slots=None, flags=0, kernels=None):
    ck = 0 if slots is None else slots * L.state_bytes(w.problem)
    s = L.Solver(w.problem, L.FP32, ckpt_bytes=ck, flags=flags)
    if kernels is not None:
        assert s.kernels == kernels
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    J = s.forward()
    st = s.get_state()
    g = s.adjoint()
    stats = s.stats()
    s.close()
    return J, st, g, stats


CASES = {
    "small2d_J1": lambda: W.small_channel2d(),
    "small2d_J2": lambda: W.small_channel2d(obj_kind=W.OBJ_VELOCITY, n_steps=36, seed=21),
    "ragged2d": lambda: W.small_channel2d(nx=70, ny=45, LD=16, n_steps=60, omega=0.01,
                                          trans_amp=1.5, seed=31),
    "wide2d": lambda: W.small_channel2d(nx=131, ny=66, LD=20, n_steps=40, omega=0.008,
                                        trans_amp=1.0, seed=34),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fused2d_matches_plain_and_oracle(L, name):
    w = CASES[name]()
    Jf, sf, gf, _ = single(L, w, kernels="fused2d")
    Jp, sp, gp, _ = single(L, w, flags=L.FLAG_PLAIN_KERNELS, kernels="plain")
    assert abs(Jf - Jp) <= 2e-6 * abs(Jp)
    assert rel_max(sf, sp) < 1e-5
    assert rel_l2(gf, gp) < 1e-5
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    assert abs(Jf - Jo) <= 1e-5 * abs(Jo)
    assert rel_l2(gf, go) < 1e-4


def test_transfer_tape_matches_transfers_formed_again(L):
    """The adjoint of a taped step reads the step's kappa and u_S from the transfer tape when the
    tape segment fits it (up to max(ceil(sqrt N) + 2, 64) steps), else it forms the transfer
    again: both give the same values, so J, the state and dJ/dgamma are bitwise equal."""
    w = W.small_channel2d(nx=40, ny=30, LD=12, n_steps=150, omega=0.01, seed=31)
    # full history: one tape segment of 150 steps, longer than the transfer tape
    J0, st0, g0, s0 = single(L, w)
    assert s0["tape_steps"] == 150 and s0["recomputed_steps"] == 0
    # 30 snapshot slots: tape segments of 13 steps, recomputed, each within the transfer tape
    J1, st1, g1, s1 = single(L, w, slots=30)
    assert s1["recomputed_steps"] > 0 and s1["tape_steps"] < 64
    assert J0 == J1
    assert np.array_equal(st0, st1)
    assert np.array_equal(g0, g1)


def test_fused2d_periodic_box(L):
    n, Ld, steps = (40, 34, 1), (9, 9, 1), 30
    p = W.periodic_box(2, n, A=0.35, L=Ld, n_steps=steps)
    p.xi_G = (4.0, 4.0, 0.0)
    p.obj_kind = W.OBJ_VELOCITY
    p.obj_dir = (1.0, 0.0, 0.0)
    p.obj_box = (0, 39, 0, 4, 0, 0)
    p.win = (10, 30)
    p.u_init = (0.02, 0.01, 0.0)
    mot = W.motion_table(steps, (19.2, 16.7, 0.0), omega=0.04, trans_amp=1.5, trans_period=60.0,
                         trans_axis=0, theta0=0.3)
    w = W.Workload(p, W.make_gamma(Ld, 1.0, 8), mot)
    Jo, go = oracle.gradient(p, w.gamma, mot)
    J, st, g, _ = single(L, w, kernels="fused2d")
    assert abs(J - Jo) <= 1e-5 * abs(Jo)
    assert rel_l2(g, go) < 1e-4
    assert abs(st[0].sum() - p.nodes) < 1e-4 * p.nodes


def members(n=6, steps=40, side=(20, 70)):
    return W.batch_config2(n_inst=n, n_steps=steps, side=side, seed=5)


def run_batch(L, ws, slots, graphs=True, tiles=(-1, -1)):
    b = L.Batch([w.problem for w in ws], slots)
    b.set_options(graphs, tiles[0], tiles[1])
    for s, w in zip(b.solvers, ws):
        s.set_design(w.gamma)
        s.set_motion(w.motion)
    J = b.forward()
    gs = b.adjoint()
    info = {"tuning": b.tuning(), "stats": b.stats(),
            "recomputed": b.solvers[0].stats()["recomputed_steps"]}
    b.close()
    return J, gs, info


@pytest.mark.parametrize("graphs", [True, False])
def test_batch_members_bitwise_equal_single_runs(L, graphs):
    ws = members()
    slots = 8
    J, gs, info = run_batch(L, ws, slots, graphs=graphs)
    assert info["recomputed"] > 0
    if graphs:
        assert info["stats"]["graphs"] > 0
    for i, w in enumerate(ws):
        Js, _, gsi, _ = single(L, w, slots=slots)
        assert J[i] == Js
        assert np.array_equal(gs[i], gsi)


def test_batch_every_tile_shape_gives_identical_results(L):
    """Every step configuration (tiles, row-marching strips) and every adjoint tile shape gives
    bitwise the same results."""
    ws = members(n=4, steps=24, side=(24, 90))
    ref = None
    for k in range(len(L.tile_shapes())):
        J, gs, info = run_batch(L, ws, 6, tiles=(k, k % 5))
        assert info["tuning"]["step"] == k and info["tuning"]["adjoint"] == k % 5
        if ref is None:
            ref = (J, gs)
        else:
            assert np.array_equal(J, ref[0])
            for a, b in zip(gs, ref[1]):
                assert np.array_equal(a, b)


def test_batch_matches_oracle_and_autotunes(L):
    ws = members(n=3, steps=30, side=(20, 40))
    J, gs, info = run_batch(L, ws, 5)
    t = info["tuning"]
    assert 0 <= t["step"] < len(L.tile_shapes()) and 0 <= t["adjoint"] < len(L.tile_shapes())
    assert min(t["step_ms"]) > 0 and min(t["adjoint_ms"][:5]) > 0
    for i, w in enumerate(ws):
        Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
        assert abs(J[i] - Jo) <= 1e-5 * abs(Jo)
        assert rel_l2(gs[i], go) < 1e-4


def test_batch_full_size_members_short_horizon(L):
    """The 64-instance workload at full grid sizes (128..512), 60 steps: sampled members equal
    their single runs bitwise and the smallest member matches the oracle."""
    ws = W.batch_config2(n_inst=64, n_steps=60)
    J, gs, info = run_batch(L, ws, 12)
    assert info["recomputed"] > 0
    sizes = [w.problem.n[0] for w in ws]
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), 17]
    for i in pick:
        Js, _, gsi, _ = single(L, ws[i], slots=12)
        assert J[i] == Js
        assert np.array_equal(gs[i], gsi)
    i = pick[0]
    Jo, go = oracle.gradient(ws[i].problem, ws[i].gamma, ws[i].motion)
    assert abs(J[i] - Jo) <= 1e-5 * abs(Jo)
    assert rel_l2(gs[i], go) < 1e-4


def test_batch_error_paths(L):
    w = CASES["small2d_J1"]()
    s64 = L.Solver(w.problem, L.FP64)
    import ctypes
    arr = (ctypes.c_void_p * 1)(s64.ctx.value)
    b = ctypes.c_void_p()
    assert L.load().lks_batch_create(arr, 1, ctypes.byref(b)) == 1
    s64.close()
    ws = members(n=2, steps=10)
    bt = L.Batch([x.problem for x in ws], 4)
    with pytest.raises(L.LksError) as e:
        bt.forward()
    assert e.value.status == 2
    with pytest.raises(L.LksError) as e:
        bt.adjoint()
    assert e.value.status == 2
    with pytest.raises(L.LksError) as e:
        bt.set_options(True, 99, 0)
    assert e.value.status == 1
    bt.close()

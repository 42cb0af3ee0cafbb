"""GPU parity: the CUDA library through its C ABI against the CPU oracle on the same seeded
inputs.

Tolerances: the FP64 path matches the oracle to 1e-11 relative (J, final state, dJ/dgamma in
max-norm relative to the largest entry); the FP32 path to 1e-5 relative on J and 1e-4
relative L2 on dJ/dgamma.  Sizes span several tiles with ragged tails; boundary, periodic and
no-body cases are included.
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


def rel_max(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run_gpu(L, w, prec, n=None, ckpt=0, init=None, flags=0, expect_fused=None):
    s = L.Solver(w.problem, prec, ckpt_bytes=ckpt, flags=flags)
    if expect_fused is not None:
        assert s.fused == expect_fused
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    if init is not None:
        s.set_initial_state(init)
    J = s.forward(n)
    st = s.get_state()
    g = s.adjoint()
    stats = s.stats()
    s.close()
    return J, st, g, stats


def corners3d():
    """A duct whose four walls move at four different tangential velocities (inlet z-, outlet
    z+), so every edge and corner rule (wall ties to the lower face, wall over inlet and
    outlet, diagonal-inward density copies) shows in the state; several 32 x 8 tiles with
    ragged tails."""
    w = W.small_duct3d(nx=40, ny=19, nz=14, LD=7, n_steps=16, omega=0.02, trans_amp=0.8,
                       seed=33)
    w.problem.bc_val = ((0.0, 0.0, 0.011, 1.0), (0.0, 0.0, -0.007, 1.0), (0.0, 0.0, 0.023, 1.0),
                        (0.0, 0.0, 0.031, 1.0), (0.0, 0.0, 0.04, 1.0), (0.0, 0.0, 0.0, 0.998))
    return w


def corners2d():
    """A channel with a moving lid and an outlet density off rho0: the corner rules of 2D."""
    w = W.small_channel2d(nx=45, ny=30, LD=10, n_steps=30, omega=0.015, trans_amp=1.0, seed=34)
    w.problem.bc_val = ((0.04, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.003), (0.0, 0.0, 0.0, 1.0),
                        (0.02, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0))
    return w


CASES = {
    "corners3d": corners3d,
    "corners2d": corners2d,
    "small2d_J1": lambda: W.small_channel2d(),
    "small2d_J2": lambda: W.small_channel2d(obj_kind=W.OBJ_VELOCITY, n_steps=36, seed=21),
    "small3d_J2": lambda: W.small_duct3d(),
    "small3d_J1": lambda: W.small_duct3d(obj_kind=W.OBJ_PRESSURE, n_steps=18, seed=22),
    "ragged2d": lambda: W.small_channel2d(nx=70, ny=45, LD=16, n_steps=60, omega=0.01,
                                          trans_amp=1.5, seed=31),
    "ragged3d": lambda: W.small_duct3d(nx=37, ny=29, nz=33, LD=9, n_steps=20, omega=0.01,
                                       trans_amp=1.0, seed=32),
    # nx - 1 and ny - 1 one past a tile (32 x 8): a face in the rim column of a tile and in
    # the rim row of another, next to tiles holding a single face
    "rimface3d": lambda: W.small_duct3d(nx=33, ny=17, nz=13, LD=7, n_steps=14, omega=0.02,
                                        trans_amp=0.8, seed=35),
}


@pytest.mark.parametrize("name", ["small2d_J1", "small3d_J2", "ragged3d"])
def test_transfer_fp64_matches_oracle(L, name):
    w = CASES[name]()
    s = L.Solver(w.problem, L.FP64)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    for n in (1, w.problem.n_steps // 2, w.problem.n_steps):
        k, us = s.transfer(n)
        ko, uso = oracle.transfer(w.problem, w.gamma, w.motion[n])
        assert rel_max(k, ko) < 1e-13
        assert np.max(np.abs(us - uso)) < 1e-13 * max(np.max(np.abs(uso)), 1e-3)
    s.close()


@pytest.mark.parametrize("name", list(CASES))
def test_forward_adjoint_fp64_match_oracle(L, name):
    w = CASES[name]()
    Jo, fo = oracle.forward(w.problem, w.gamma, w.motion)
    Jg, go = oracle.gradient(w.problem, w.gamma, w.motion)
    J, st, g, _ = run_gpu(L, w, L.FP64)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert rel_max(st, fo) < 1e-11
    assert rel_max(g, go) < 1e-11


@pytest.mark.parametrize("name", ["small2d_J1", "small3d_J2", "ragged2d", "ragged3d",
                                  "corners3d", "corners2d"])
def test_forward_adjoint_fp32_within_tolerance(L, name):
    w = CASES[name]()
    Jg, go = oracle.gradient(w.problem, w.gamma, w.motion)
    J, st, g, _ = run_gpu(L, w, L.FP32)
    assert abs(J - Jg) <= 1e-5 * abs(Jg)
    assert rel_l2(g, go) < 1e-4


def test_periodic_box_with_moving_body(L):
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
    Jg, go = oracle.gradient(p, w.gamma, mot)
    J, st, g, _ = run_gpu(L, w, L.FP64)
    assert abs(J - Jg) <= 1e-11 * abs(Jg)
    assert rel_max(g, go) < 1e-11
    # mass conservation carries over to the GPU path
    assert abs(st[0].sum() - p.nodes) < 1e-11 * p.nodes


def test_no_body_plates_match_oracle(L):
    """Walls only, no design grid (kappa = 0 path), 3D Couette start-up."""
    H = 9
    p = W.Problem(dim=3, n=(6, H + 1, 5), L=(0, 0, 0), A=0.3,
                  bc=(W.PERIODIC, W.PERIODIC, W.WALL, W.WALL, W.PERIODIC, W.PERIODIC),
                  bc_val=((0, 0, 0, 1),) * 3 + ((0.03, 0, 0.01, 1),) + ((0, 0, 0, 1),) * 2,
                  obj_kind=W.OBJ_VELOCITY, obj_dir=(1, 0, 0), obj_box=(0, 5, 1, 4, 0, 4),
                  win=(5, 40), n_steps=40)
    w = W.Workload(p, np.zeros((1, 1, 1)), np.zeros((41, 8)))
    Jo, fo = oracle.forward(p, None, w.motion)
    J, st, g, _ = run_gpu(L, w, L.FP64)
    assert abs(J - Jo) <= 1e-11 * abs(Jo)
    assert rel_max(st, fo) < 1e-11


def test_segmented_checkpointing_is_bitwise_equal_to_full_history(L):
    w = CASES["small3d_J2"]()
    _, _, g_full, st_full = run_gpu(L, w, L.FP32)
    assert st_full["recomputed_steps"] == 0
    snap = 4 * 4 * w.problem.nodes
    snap = (snap + 255) // 256 * 256
    for slots in (9, 5):
        _, _, g_seg, st = run_gpu(L, w, L.FP32, ckpt=slots * snap)
        assert st["recomputed_steps"] > 0
        assert np.array_equal(g_seg, g_full)


def test_cfg0_fp64_full_horizon_matches_oracle(L):
    """The 128^2 x 1000-step channel (workload 0) end to end at 1e-11."""
    w = W.config(0)
    Jg, go = oracle.gradient(w.problem, w.gamma, w.motion)
    J, st, g, _ = run_gpu(L, w, L.FP64)
    assert abs(J - Jg) <= 1e-11 * abs(Jg)
    assert rel_max(g, go) < 1e-11
    J32, _, g32, _ = run_gpu(L, w, L.FP32)
    assert abs(J32 - Jg) <= 1e-5 * abs(Jg)
    assert rel_l2(g32, go) < 1e-4


def test_error_paths(L):
    w = CASES["small2d_J1"]()
    s = L.Solver(w.problem, L.FP32)
    with pytest.raises(L.LksError) as e:
        s.forward()
    assert e.value.status == 2
    bad = w.gamma.copy()
    bad[0, 0, 0] = 1.5
    with pytest.raises(L.LksError) as e:
        s.set_design(bad)
    assert e.value.status == 1
    s.set_design(w.gamma)
    far = w.motion.copy()
    far[:, 2] = 2.0  # design centre next to the inlet: footprint leaves the interior
    with pytest.raises(L.LksError) as e:
        s.set_motion(far)
    assert e.value.status == 1
    with pytest.raises(L.LksError) as e:
        s.set_motion(w.motion[:5])
    assert e.value.status == 1
    s.set_motion(w.motion)
    with pytest.raises(L.LksError) as e:
        s.adjoint()
    assert e.value.status == 2
    s.forward()
    s.adjoint()
    s.close()


MID3D = lambda: W.small_duct3d(nx=70, ny=45, nz=52, LD=14, n_steps=30, omega=0.004,
                               trans_amp=2.0, seed=33)


@pytest.mark.parametrize("name", ["small3d_J2", "small3d_J1", "ragged3d", "mid3d",
                                  "corners3d", "rimface3d"])
def test_fused_fp32_step_matches_plain_fp32_and_oracle(L, name):
    w = MID3D() if name == "mid3d" else CASES[name]()
    Jf, sf, gf, _ = run_gpu(L, w, L.FP32, expect_fused=True)
    Jp, sp, gp, _ = run_gpu(L, w, L.FP32, flags=L.FLAG_PLAIN_KERNELS, expect_fused=False)
    assert abs(Jf - Jp) <= 2e-6 * abs(Jp)
    assert rel_max(sf, sp) < 1e-5
    assert rel_l2(gf, gp) < 1e-5
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    assert abs(Jf - Jo) <= 1e-5 * abs(Jo)
    assert rel_l2(gf, go) < 1e-4


@pytest.mark.parametrize("name", ["small3d_J1", "ragged3d", "mid3d", "corners3d", "rimface3d"])
def test_fused_step_variants_agree(L, name):
    """Every variant of the fused 3D forward step (fixed through lks_step_variant) gives the
    same run as variant 0 up to rounding, within the FP32 tolerances of the oracle; the default
    is checked below, and the timed choice picks one of them."""
    w = MID3D() if name == "mid3d" else CASES[name]()
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    res = []
    for v in range(3):
        s = L.Solver(w.problem, L.FP32)
        assert s.step_variant(v) == -1
        s.set_design(w.gamma)
        s.set_motion(w.motion)
        J = s.forward()
        assert s.step_variant() == v
        res.append((J, s.get_state(), s.adjoint()))
        s.close()
    J0, s0, g0 = res[0]
    for J, st, g in res:
        assert abs(J - J0) <= 1e-6 * abs(J0)
        assert rel_max(st, s0) < 1e-6
        assert rel_l2(g, g0) < 1e-6
        assert abs(J - Jo) <= 1e-5 * abs(Jo)
        assert rel_l2(g, go) < 1e-4
    s = L.Solver(w.problem, L.FP32)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    s.forward()
    assert s.step_variant() == 1
    assert s.step_variant(-1) == -1
    s.forward()
    assert s.step_variant() in (0, 1, 2)
    with pytest.raises(L.LksError):
        s.step_variant(3)
    s.close()


def test_kernel_choice_per_context(L):
    w = CASES["small3d_J2"]()
    s = L.Solver(w.problem, L.FP64)
    assert s.kernels == "plain"
    s.close()
    s = L.Solver(w.problem, L.FP32)
    assert s.kernels == "fused3d"
    s.close()
    w2 = CASES["small2d_J1"]()
    s = L.Solver(w2.problem, L.FP32)
    assert s.kernels == "fused2d"
    s.close()
    s = L.Solver(w2.problem, L.FP64)
    assert s.kernels == "plain"
    s.close()
    s = L.Solver(w2.problem, L.FP32, flags=L.FLAG_PAPER_ALKS)
    assert s.kernels == "plain"
    s.close()


def test_full_size_256_cube_two_steps_against_oracle(L):
    """The benchmark's 256^3 grid and 96^3 design (workload 4) in the benchmark's launch
    configuration, over a two-step horizon the oracle can follow: J, the final state and
    dJ/dgamma of the fused FP32 path and the plain FP64 path against the oracle."""
    w = W.config(4, n_steps=2)
    Jo, fo = oracle.forward(w.problem, w.gamma, w.motion)
    Jg, go = oracle.gradient(w.problem, w.gamma, w.motion)
    J64, s64, g64, _ = run_gpu(L, w, L.FP64)
    assert abs(J64 - Jg) <= 1e-11 * abs(Jg)
    assert rel_max(s64, fo) < 1e-11
    assert rel_max(g64, go) < 1e-11
    J32, s32, g32, _ = run_gpu(L, w, L.FP32, expect_fused=True)
    assert abs(J32 - Jg) <= 1e-5 * abs(Jg)
    assert rel_max(s32, fo) < 1e-5
    assert rel_l2(g32, go) < 1e-4


def test_transfer_buffers_do_not_leak_across_runs(L):
    """3D contexts compute the next step's transfer on a side stream into a second buffer set;
    a design change between runs, an explicit lks_transfer in between and a shorter run must
    all give bitwise the results of a fresh context."""
    w = CASES["ragged3d"]()
    g2 = np.clip(w.gamma[::-1].copy() * 0.8 + 0.1, 0.0, 1.0)

    def fresh(gamma, n=None):
        s = L.Solver(w.problem, L.FP32)
        s.set_design(gamma)
        s.set_motion(w.motion)
        J = s.forward(n)
        g = s.adjoint()
        s.close()
        return J, g

    Ja, ga = fresh(w.gamma)
    Jb, gb = fresh(g2)
    Jc, gc = fresh(g2, 11)
    s = L.Solver(w.problem, L.FP32)
    s.set_design(w.gamma)
    s.set_motion(w.motion)
    J1 = s.forward()
    g1 = s.adjoint()
    k_before, _ = s.transfer(5)
    s.set_design(g2)
    k_after, _ = s.transfer(5)
    J2 = s.forward()
    g2_ = s.adjoint()
    J3 = s.forward(11)
    g3 = s.adjoint()
    s.close()
    assert J1 == Ja and np.array_equal(g1, ga)
    assert J2 == Jb and np.array_equal(g2_, gb)
    assert J3 == Jc and np.array_equal(g3, gc)
    assert not np.array_equal(k_before, k_after)


@pytest.mark.parametrize("name", ["small3d_J1", "ragged3d", "mid3d", "corners3d"])
def test_fused_adjoint_variants_agree(L, name):
    """Both schedules of the fused 3D adjoint (two barriers per plane; conversion two planes
    ahead with one barrier) evaluate the same arithmetic in the same order: the gradients are
    bitwise equal, and within the FP32 tolerances of the oracle."""
    w = MID3D() if name == "mid3d" else CASES[name]()
    Jo, go = oracle.gradient(w.problem, w.gamma, w.motion)
    res = []
    for v in range(2):
        s = L.Solver(w.problem, L.FP32)
        assert s.adjoint_variant(v) == v
        s.set_design(w.gamma)
        s.set_motion(w.motion)
        J = s.forward()
        res.append((J, s.adjoint()))
        assert s.adjoint_variant() == v
        s.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    assert rel_l2(res[1][1], go) < 1e-4
    s = L.Solver(w.problem, L.FP32)
    assert s.adjoint_variant() == 1   # the one-barrier schedule is the default
    with pytest.raises(L.LksError):
        s.adjoint_variant(2)
    s.close()

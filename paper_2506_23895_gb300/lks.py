"""Python binding of the C ABI in include/lks.h (argument marshalling only).

Every step of the computation runs in liblks_gb300.so; this module only converts arguments.
PyTorch provides the device workspace (and, optionally, the stream).  If the library is
missing the import of this module's functions raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblks_gb300.so")

FP32, FP64 = 0, 1
STATUS = {0: "LKS_OK", 1: "LKS_ERR_ARG", 2: "LKS_ERR_ORDER", 3: "LKS_ERR_NOMEM",
          4: "LKS_ERR_CUDA", 5: "LKS_ERR_DIVERGED", 6: "LKS_ERR_TIMEOUT"}

# every symbol include/lks.h declares
EXPORTS = ("lks_workspace_bytes", "lks_create", "lks_set_design", "lks_set_motion",
           "lks_set_initial_state", "lks_forward", "lks_adjoint", "lks_get_state",
           "lks_transfer", "lks_uses_fused", "lks_step_variant", "lks_get_stats", "lks_set_timing", "lks_read_timing",
           "lks_checkpoint_schedule", "lks_step_noalloc", "lks_last_error", "lks_destroy",
           "lks_batch_create", "lks_batch_set_options", "lks_batch_forward", "lks_batch_adjoint",
           "lks_batch_tile_shapes", "lks_batch_tuning", "lks_batch_stats",
           "lks_batch_last_error", "lks_batch_destroy", "lks_set_filter", "lks_volume",
           "lks_set_static", "lks_warm_start", "lks_set_adjoint_start", "lks_get_adjoint_state",
           "lks_inject_alloc_failure", "lks_fma_rate", "lks_adjoint_variant")


class LksError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LksConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lx", ctypes.c_int), ("ly", ctypes.c_int), ("lz", ctypes.c_int),
        ("precision", ctypes.c_int), ("max_steps", ctypes.c_int),
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
        ("ckpt_bytes", ctypes.c_size_t),
        ("stream", ctypes.c_void_p),
        ("flags", ctypes.c_int),
        ("rot_axis", ctypes.c_double * 3),
    ]


FLAG_PLAIN_KERNELS = 1
FLAG_PAPER_ALKS = 2


class LksMotion(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int), ("rows", ctypes.POINTER(ctypes.c_double))]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblks_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2506_23895_gb300/build.py")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    lib.lks_workspace_bytes.argtypes = [ctypes.POINTER(LksConfig)]
    lib.lks_workspace_bytes.restype = ctypes.c_size_t
    lib.lks_create.argtypes = [ctypes.POINTER(LksConfig), P, ctypes.c_size_t, ctypes.POINTER(P)]
    lib.lks_set_design.argtypes = [P, P, ctypes.c_int]
    lib.lks_set_motion.argtypes = [P, ctypes.POINTER(LksMotion)]
    lib.lks_set_initial_state.argtypes = [P, D]
    lib.lks_forward.argtypes = [P, ctypes.c_int, D]
    lib.lks_adjoint.argtypes = [P, P, ctypes.c_int]
    lib.lks_get_state.argtypes = [P, D]
    lib.lks_transfer.argtypes = [P, ctypes.c_int, D, D]
    lib.lks_get_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.lks_uses_fused.argtypes = [P]
    lib.lks_uses_fused.restype = ctypes.c_int
    lib.lks_step_variant.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.lks_adjoint_variant.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.lks_adjoint_variant.restype = ctypes.c_int
    lib.lks_set_timing.argtypes = [P, ctypes.c_int]
    lib.lks_read_timing.argtypes = [P, D]
    lib.lks_checkpoint_schedule.argtypes = [ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.lks_checkpoint_schedule.restype = ctypes.c_int
    lib.lks_last_error.argtypes = [P]
    lib.lks_last_error.restype = ctypes.c_char_p
    lib.lks_destroy.argtypes = [P]
    lib.lks_destroy.restype = None
    lib.lks_inject_alloc_failure.argtypes = [ctypes.c_int]
    lib.lks_inject_alloc_failure.restype = ctypes.c_int
    lib.lks_fma_rate.argtypes = [ctypes.c_int, P, D]
    lib.lks_fma_rate.restype = ctypes.c_int
    lib.lks_set_filter.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    lib.lks_set_filter.restype = ctypes.c_int
    lib.lks_volume.argtypes = [P, ctypes.c_double, D, P, ctypes.c_int]
    lib.lks_volume.restype = ctypes.c_int
    lib.lks_set_static.argtypes = [P, D]
    lib.lks_warm_start.argtypes = [P]
    lib.lks_set_adjoint_start.argtypes = [P, ctypes.c_int]
    lib.lks_get_adjoint_state.argtypes = [P, D]
    for name in ("lks_set_static", "lks_warm_start", "lks_set_adjoint_start",
                 "lks_get_adjoint_state"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lks_batch_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(P)]
    lib.lks_batch_set_options.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.lks_batch_forward.argtypes = [P, ctypes.c_int, D]
    lib.lks_batch_adjoint.argtypes = [P, ctypes.POINTER(P), ctypes.c_int]
    lib.lks_batch_tile_shapes.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    lib.lks_batch_tile_shapes.restype = ctypes.c_int
    lib.lks_batch_tuning.argtypes = [P, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_float)]
    lib.lks_batch_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong)]
    lib.lks_batch_last_error.argtypes = [P]
    lib.lks_batch_last_error.restype = ctypes.c_char_p
    lib.lks_batch_destroy.argtypes = [P]
    lib.lks_batch_destroy.restype = None
    for name in ("lks_batch_create", "lks_batch_set_options", "lks_batch_forward",
                 "lks_batch_adjoint", "lks_batch_tuning", "lks_batch_stats"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("lks_create", "lks_set_design", "lks_set_motion", "lks_set_initial_state",
                 "lks_forward", "lks_adjoint", "lks_get_state", "lks_transfer", "lks_get_stats",
                 "lks_set_timing", "lks_read_timing"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def make_config(problem, precision: int = FP32, max_steps: Optional[int] = None,
                ckpt_bytes: int = 0, stream: Optional[int] = None, flags: int = 0) -> LksConfig:
    """lks_config from a workloads.Problem."""
    p = problem
    c = LksConfig()
    c.dim = p.dim
    c.nx, c.ny, c.nz = p.n
    c.lx, c.ly, c.lz = p.L
    c.precision = precision
    c.max_steps = p.n_steps if max_steps is None else max_steps
    c.A, c.kappa_max, c.q, c.rho0 = p.A, p.kappa_max, p.q, p.rho0
    for f in range(6):
        c.bc[f] = p.bc[f]
        for k in range(4):
            c.bc_val[f][k] = p.bc_val[f][k]
    for a in range(3):
        c.u_init[a] = p.u_init[a]
        c.body_force[a] = p.body_force[a]
        c.xi_G[a] = p.xi_G[a]
        c.obj_dir[a] = p.obj_dir[a]
    c.obj_kind = p.obj_kind
    for k in range(6):
        c.obj_box[k] = p.obj_box[k]
    c.obj_cyl_r = p.obj_cyl_r
    c.obj_cyl_c[0], c.obj_cyl_c[1] = p.obj_cyl_c
    c.win_begin, c.win_end = p.win
    c.ckpt_bytes = ckpt_bytes
    c.stream = stream
    c.flags = flags
    ax = getattr(p, "rot_axis", (0.0, 0.0, 1.0))
    for a in range(3):
        c.rot_axis[a] = ax[a]
    return c


def fma_rate(precision: int, stream=None) -> float:
    """Measured FMA throughput of the current device in flop/s (2 per FMA)."""
    lib = load()
    v = ctypes.c_double(0.0)
    s = None if stream is None else int(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                         else stream)
    st = lib.lks_fma_rate(precision, s, ctypes.byref(v))
    if st != 0:
        raise LksError(st, "lks_fma_rate failed")
    return v.value


def checkpoint_schedule(n_segments: int, free_slots: int):
    """The (kind, a, b) actions of the adjoint's checkpoint schedule (host only)."""
    lib = load()
    n = lib.lks_checkpoint_schedule(n_segments, free_slots, None, 0)
    if n < 0:
        raise ValueError("bad schedule arguments")
    buf = (ctypes.c_int * (3 * n))()
    lib.lks_checkpoint_schedule(n_segments, free_slots, buf, n)
    return [tuple(buf[3 * i:3 * i + 3]) for i in range(n)]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Solver:
    """One problem instance on the GPU: set_design, set_motion, forward -> J, adjoint -> dJ/dgamma.

    The device workspace is a torch uint8 tensor owned by this object.
    """

    def __init__(self, problem, precision: int = FP32, max_steps: Optional[int] = None,
                 ckpt_bytes: int = 0, stream=None, flags: int = 0):
        import torch

        self.lib = load()
        self.problem = problem
        self.precision = precision
        s = None if stream is None else int(stream.cuda_stream if hasattr(stream, "cuda_stream")
                                              else stream)
        self.cfg = make_config(problem, precision, max_steps, ckpt_bytes, s, flags)
        nbytes = self.lib.lks_workspace_bytes(ctypes.byref(self.cfg))
        if nbytes == 0:
            raise LksError(1, "invalid configuration")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.ctx = ctypes.c_void_p()
        st = self.lib.lks_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                 nbytes, ctypes.byref(self.ctx))
        if st != 0:
            raise LksError(st, "lks_create failed")
        self._f64 = torch.float64
        self.generation = 0        # counts forward runs
        self.adjoint_ready = False  # a forward run whose adjoint has not been taken yet
        self.nd = problem.design_nodes
        self.design_shape = (1 if problem.dim == 2 else problem.L[2], problem.L[1], problem.L[0])
        self.state_shape = (4, problem.n[2], problem.n[1], problem.n[0])

    def _check(self, st):
        if st != 0:
            raise LksError(st, self.lib.lks_last_error(self.ctx).decode())

    def set_design(self, gamma) -> None:
        if hasattr(gamma, "data_ptr"):  # torch tensor, device or (pinned) host
            g = gamma.detach()
            if g.dtype != self._f64 or not g.is_contiguous():
                g = g.contiguous().double()
            self._keep = g
            self._check(self.lib.lks_set_design(self.ctx, ctypes.c_void_p(g.data_ptr()),
                                                1 if g.is_cuda else 0))
        else:
            g = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
            self._check(self.lib.lks_set_design(self.ctx, g.ctypes.data_as(ctypes.c_void_p), 0))

    def set_filter(self, R: float, beta: float = 1.0, eta: float = 0.5) -> None:
        """Density filter + Heaviside projection in front of the solver (R = 0: off)."""
        self._check(self.lib.lks_set_filter(self.ctx, R, beta, eta))

    def volume(self, vmax: float):
        """(G, dG/dgamma) of the volume constraint on the current design."""
        G = ctypes.c_double(0.0)
        dG = np.zeros(self.design_shape, dtype=np.float64)
        self._check(self.lib.lks_volume(self.ctx, vmax, ctypes.byref(G),
                                        dG.ctypes.data_as(ctypes.c_void_p), 0))
        return G.value, dG

    def set_static(self, kappa_s=None) -> None:
        """Static solid field (nz, ny, nx) of Brinkman coefficients, or None to remove it."""
        if kappa_s is None:
            self._check(self.lib.lks_set_static(self.ctx, None))
        else:
            k = np.ascontiguousarray(np.asarray(kappa_s, dtype=np.float64))
            assert k.size == self.state_shape[1] * self.state_shape[2] * self.state_shape[3]
            self._check(self.lib.lks_set_static(self.ctx, _dptr(k)))

    def warm_start(self) -> None:
        """Initial state := final state of the last forward run."""
        self._check(self.lib.lks_warm_start(self.ctx))

    def set_adjoint_start(self, warm: bool) -> None:
        self._check(self.lib.lks_set_adjoint_start(self.ctx, int(warm)))

    def get_adjoint_state(self) -> np.ndarray:
        s = np.zeros(self.state_shape, dtype=np.float64)
        self._check(self.lib.lks_get_adjoint_state(self.ctx, _dptr(s)))
        return s

    def set_motion(self, rows) -> None:
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, 8))
        m = LksMotion(r.shape[0], _dptr(r))
        self._rows = r
        self._check(self.lib.lks_set_motion(self.ctx, ctypes.byref(m)))

    def set_initial_state(self, state=None) -> None:
        if state is None:
            self._check(self.lib.lks_set_initial_state(self.ctx, None))
        else:
            s = np.ascontiguousarray(np.asarray(state, dtype=np.float64))
            assert s.shape == self.state_shape
            self._check(self.lib.lks_set_initial_state(self.ctx, _dptr(s)))

    def forward(self, n_steps: Optional[int] = None) -> float:
        n = self.problem.n_steps if n_steps is None else n_steps
        J = ctypes.c_double(0.0)
        self.adjoint_ready = False
        self._check(self.lib.lks_forward(self.ctx, n, ctypes.byref(J)))
        self.generation += 1
        self.adjoint_ready = True
        return J.value

    def adjoint(self, out=None):
        """dJ/dgamma into `out` (a contiguous float64 torch tensor, CUDA or host) or a new
        numpy array."""
        if out is not None and hasattr(out, "data_ptr"):
            assert out.element_size() == 8 and out.is_contiguous()
            self.adjoint_ready = False
            self._check(self.lib.lks_adjoint(self.ctx, ctypes.c_void_p(out.data_ptr()),
                                             1 if out.is_cuda else 0))
            return out
        g = np.zeros(self.design_shape, dtype=np.float64)
        self.adjoint_ready = False
        self._check(self.lib.lks_adjoint(self.ctx, g.ctypes.data_as(ctypes.c_void_p), 0))
        return g

    def get_state(self) -> np.ndarray:
        s = np.zeros(self.state_shape, dtype=np.float64)
        self._check(self.lib.lks_get_state(self.ctx, _dptr(s)))
        return s

    def transfer(self, step: int) -> Tuple[np.ndarray, np.ndarray]:
        k = np.zeros(self.state_shape[1:], dtype=np.float64)
        us = np.zeros((3,) + self.state_shape[1:], dtype=np.float64)
        self._check(self.lib.lks_transfer(self.ctx, step, _dptr(k), _dptr(us)))
        return k, us

    @property
    def fused(self) -> bool:
        return bool(self.lib.lks_uses_fused(self.ctx))

    @property
    def kernels(self) -> str:
        """'fused3d', 'fused2d' or 'plain': which kernels run this context's steps."""
        return {1: "fused3d", 2: "fused2d"}.get(self.lib.lks_uses_fused(self.ctx), "plain")

    def step_variant(self, request: int = -2) -> int:
        """Fused 3D step variant: request 0..2 fixes one (1 by default), -1 times them on the
        first step, -2 only reads; returns the variant in use (-1 before the first fused step)."""
        v = ctypes.c_int(-1)
        self._check(self.lib.lks_step_variant(self.ctx, request, ctypes.byref(v)))
        return v.value

    def adjoint_variant(self, request: int = -2) -> int:
        """Fix (0..1) or read (-2) the fused 3D adjoint variant; returns the variant in use."""
        v = ctypes.c_int(-1)
        self._check(self.lib.lks_adjoint_variant(self.ctx, request, ctypes.byref(v)))
        return v.value

    def set_timing(self, stride: int) -> None:
        self._check(self.lib.lks_set_timing(self.ctx, stride))

    def read_timing(self):
        a = (ctypes.c_double * 4)()
        self._check(self.lib.lks_read_timing(self.ctx, a))
        return {"fwd_ms": a[0], "fwd_n": int(a[1]), "adj_ms": a[2], "adj_n": int(a[3])}

    def stats(self):
        a = (ctypes.c_longlong * 5)()
        self._check(self.lib.lks_get_stats(self.ctx, a))
        return {"forward_steps": a[0], "recomputed_steps": a[1], "snapshot_slots": a[2],
                "tape_steps": a[3], "launches": a[4]}

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.lks_destroy(self.ctx)
            self.ctx = None
            self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def state_bytes(problem, precision: int = FP32) -> int:
    """Device bytes of one stored state of a problem (one snapshot slot)."""
    nodes = problem.n[0] * problem.n[1] * problem.n[2]
    return (nodes * 4 * (8 if precision == FP64 else 4) + 255) // 256 * 256


def tile_shapes():
    """Candidate (tx, ty) tile shapes of the fused 2D kernels."""
    lib = load()
    n = lib.lks_batch_tile_shapes(None, 0)
    a = (ctypes.c_int * (2 * n))()
    lib.lks_batch_tile_shapes(a, n)
    return [(a[2 * k], a[2 * k + 1]) for k in range(n)]


class Batch:
    """Many D2Q9 FP32 problems advanced in lock step (lks_batch_*): one launch per phase over
    all members, runs of steps replayed from CUDA graphs, autotuned tile shapes.

    The members are Solvers built with equal max_steps and `slots` snapshot slots each."""

    def __init__(self, problems, slots: int, stream=None, max_steps: Optional[int] = None):
        self.lib = load()
        self.solvers = [Solver(p, FP32, max_steps=max_steps,
                               ckpt_bytes=slots * state_bytes(p, FP32), stream=stream)
                        for p in problems]
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx.value for s in self.solvers])
        self.b = ctypes.c_void_p()
        st = self.lib.lks_batch_create(arr, len(self.solvers), ctypes.byref(self.b))
        if st != 0:
            raise LksError(st, "lks_batch_create failed")

    def _check(self, st):
        if st != 0:
            raise LksError(st, self.lib.lks_batch_last_error(self.b).decode())

    def set_options(self, graphs: bool = True, tile_fwd: int = -1, tile_adj: int = -1) -> None:
        self._check(self.lib.lks_batch_set_options(self.b, int(graphs), tile_fwd, tile_adj))

    def forward(self, n_steps: Optional[int] = None) -> np.ndarray:
        n = self.solvers[0].problem.n_steps if n_steps is None else n_steps
        J = np.zeros(len(self.solvers), dtype=np.float64)
        for s in self.solvers:
            s.adjoint_ready = False
        self._check(self.lib.lks_batch_forward(self.b, n, _dptr(J)))
        return J

    def adjoint(self, outs=None):
        """Per member dJ/dgamma: into `outs` (contiguous float64 torch CUDA tensors) or new
        numpy arrays."""
        B = len(self.solvers)
        if outs is not None:
            ptrs = (ctypes.c_void_p * B)(*[o.data_ptr() for o in outs])
            self._check(self.lib.lks_batch_adjoint(self.b, ptrs, 1))
            return outs
        gs = [np.zeros(s.design_shape, dtype=np.float64) for s in self.solvers]
        ptrs = (ctypes.c_void_p * B)(*[g.ctypes.data for g in gs])
        self._check(self.lib.lks_batch_adjoint(self.b, ptrs, 0))
        return gs

    def tuning(self):
        n = len(tile_shapes())
        ch = (ctypes.c_int * 2)()
        ms = (ctypes.c_float * (2 * n))()
        self._check(self.lib.lks_batch_tuning(self.b, ch, ms))
        return {"step": ch[0], "adjoint": ch[1], "step_ms": list(ms[:n]), "adjoint_ms": list(ms[n:])}

    def stats(self):
        a = (ctypes.c_longlong * 3)()
        self._check(self.lib.lks_batch_stats(self.b, a))
        return {"launches": a[0], "graphs": a[1], "graph_nodes": a[2]}

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.lks_batch_destroy(self.b)
            self.b = None
        for s in getattr(self, "solvers", []):
            s.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Python face of the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never imports the
CUDA package and the CUDA package never imports it.

Every function takes and returns numpy arrays in the canonical layout:
distributions ``A[9, ny, nx]`` (float64), vector fields ``V[2, ny, nx]``,
scalar fields ``[ny, nx]``, masks ``uint8[ny, nx]``.  What each function
computes, with the passage of the paper it follows, is stated in
lbm_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liblbm_oracle.so")
_SOURCES = ["lbm_oracle.c", "lbm_oracle_cs.c", "lbm3_oracle.c"]
_DEPS = _SOURCES + ["lbm_oracle.h", "lbm3_oracle.h", "lattice.inc", "step_body.inc"]

SOLID = 0xFF


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liblbm_oracle.so (gcc, plain C).

    -ffp-contract=off keeps every product and sum rounded on its own, so the
    results do not depend on the host's FMA contraction.  OpenMP only splits
    the per-node loop of the forward step over rows; each node's arithmetic
    is the same whatever the thread count.
    """
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    newest = max(os.path.getmtime(os.path.join(_HERE, s)) for s in _DEPS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
            "-I", _HERE]
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    tmp = _SO + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp"] + srcs + ["-o", tmp, "-lm"],
                       check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + srcs + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("wall_ux", ctypes.c_double * 4), ("wall_uy", ctypes.c_double * 4),
        ("tau", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("rho_w", ctypes.c_double),
        ("open_kind", ctypes.c_int * 4),
        ("open_ux", ctypes.c_double * 4), ("open_uy", ctypes.c_double * 4),
        ("open_rho", ctypes.c_double * 4),
        ("open_val", ctypes.c_void_p * 4),
        ("omega_m", ctypes.c_double),
    ]

OPEN_NONE, OPEN_VELOCITY, OPEN_PRESSURE = 0, 1, 2
SIDES = ("west", "east", "south", "north")


@dataclass
class Setup:
    """One run's geometry and physics (mirrors orc_params)."""
    nx: int
    ny: int
    tau: float
    periodic_x: bool = True
    periodic_y: bool = True
    # wall velocities per side: west, east, south, north
    wall_u: list = field(default_factory=lambda: [(0.0, 0.0)] * 4)
    force: tuple = (0.0, 0.0)
    # open sides: {side index: ("velocity", (ux, uy)) | ("pressure", rho)};
    # the value may also be a per-node array along the side (velocity
    # [2, len], pressure [len])
    open: dict = field(default_factory=dict)
    # two-relaxation-time collision: the magic parameter
    # Lambda = (1/omega - 1/2)(1/omega_m - 1/2) > 0 fixes the odd rate
    # omega_m; 0 = BGK
    trt_magic: float = 0.0

    def omega_m(self) -> float:
        if self.trt_magic <= 0:
            return 0.0
        return 1.0 / (0.5 + self.trt_magic / (self.tau - 0.5))

    def c(self) -> Params:
        p = Params()
        p.nx, p.ny = self.nx, self.ny
        p.periodic_x, p.periodic_y = int(self.periodic_x), int(self.periodic_y)
        for s in range(4):
            p.wall_ux[s], p.wall_uy[s] = self.wall_u[s]
        p.tau = self.tau
        p.fx, p.fy = self.force
        p.rho_w = 1.0
        p.omega_m = self.omega_m()
        self._keep = []
        for s, (kind, val) in self.open.items():
            length = self.ny if s < 2 else self.nx
            p.open_kind[s] = OPEN_VELOCITY if kind == "velocity" else OPEN_PRESSURE
            arr = np.asarray(val, dtype=np.float64)
            if kind == "velocity" and arr.shape == (2,):
                p.open_ux[s], p.open_uy[s] = float(arr[0]), float(arr[1])
            elif kind == "pressure" and arr.shape == ():
                p.open_rho[s] = float(arr)
            else:
                want = (2, length) if kind == "velocity" else (length,)
                assert arr.shape == want, (arr.shape, want)
                arr = np.ascontiguousarray(arr)
                self._keep.append(arr)
                p.open_val[s] = arr.ctypes.data
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        dp = ctypes.c_void_p
        L.orc_lattice.argtypes = [dp, dp, dp, dp]
        L.orc_link_mask.argtypes = [P, dp, dp]
        L.orc_link_mask.restype = ctypes.c_int
        L.orc_tile_map.argtypes = [P, dp, dp, dp, dp]
        L.orc_tile_map.restype = ctypes.c_int
        L.orc_init_equilibrium.argtypes = [P, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [P, dp, dp, dp, dp]
        L.orc_step_cs.argtypes = [P, dp, dp, dp, dp]
        L.orc_run.argtypes = [P, dp, dp, dp, dp, ctypes.c_int]
        L.orc_macros.argtypes = [P, dp, dp, dp, dp, dp, dp]
        L.orc_adjoint_step.argtypes = [P, dp, dp, dp, dp, dp, dp]
        L.orc_macros_adjoint.argtypes = [P, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == tuple(shape), (a.shape, shape)
    return a


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel step loop (for timing it)."""
    lib().orc_set_threads(int(n))


def lattice():
    """(cx, cy, w, opp) as the oracle holds them."""
    cx = np.zeros(9, np.int32)
    cy = np.zeros(9, np.int32)
    w = np.zeros(9, np.float64)
    opp = np.zeros(9, np.int32)
    lib().orc_lattice(_ptr(cx), _ptr(cy), _ptr(w), _ptr(opp))
    return cx, cy, w, opp


def link_mask(s: Setup, solid=None):
    """Per-node link mask (uint8[ny, nx]) and the fluid-node count."""
    mask = np.zeros((s.ny, s.nx), np.uint8)
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
    p = s.c()
    nf = lib().orc_link_mask(ctypes.byref(p), _ptr(sol), _ptr(mask))
    if nf < 0:
        raise ValueError("invalid geometry")
    return mask, nf


def tile_map(s: Setup, mask):
    """(tile_id int32[nty, ntx], nbr int32[ntiles, 9])."""
    T = 16
    ntx, nty = (s.nx + T - 1) // T, (s.ny + T - 1) // T
    tid = np.zeros((nty, ntx), np.int32)
    nbr = np.zeros((ntx * nty, 9), np.int32)
    nt = ctypes.c_int(0)
    p = s.c()
    rc = lib().orc_tile_map(ctypes.byref(p), _ptr(np.ascontiguousarray(mask)), _ptr(tid),
                            _ptr(nbr), ctypes.byref(nt))
    if rc != 0:
        raise ValueError("periodic axis not a multiple of 16")
    return tid, nbr[: nt.value].copy()


def init_equilibrium(s: Setup, mask, rho=None, u=None):
    A = np.zeros((9, s.ny, s.nx))
    rho = _f64(rho, (s.ny, s.nx))
    u = _f64(u, (2, s.ny, s.nx))
    p = s.c()
    lib().orc_init_equilibrium(ctypes.byref(p), _ptr(mask), _ptr(rho),
                               None if u is None else _ptr(u[0]),
                               None if u is None else _ptr(u[1]), _ptr(A))
    return A


def step(s: Setup, mask, A, force=None):
    A = _f64(A, (9, s.ny, s.nx))
    force = _f64(force, (2, s.ny, s.nx))
    B = np.empty_like(A)
    p = s.c()
    lib().orc_step(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(B))
    return B


def step_cs(s: Setup, mask, A, force=None):
    """The step evaluated in complex arithmetic (complex-step derivative)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    assert A.shape == (9, s.ny, s.nx)
    if force is not None:
        force = np.ascontiguousarray(force, dtype=np.complex128)
        assert force.shape == (2, s.ny, s.nx)
    B = np.empty_like(A)
    p = s.c()
    lib().orc_step_cs(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(B))
    return B


def run(s: Setup, mask, A, nsteps: int, force=None):
    A = _f64(A, (9, s.ny, s.nx)).copy()
    force = _f64(force, (2, s.ny, s.nx))
    B = np.empty_like(A)
    p = s.c()
    lib().orc_run(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(B), int(nsteps))
    return A


def macros(s: Setup, mask, A, force=None):
    """(rho [ny, nx], u [2, ny, nx]) of the state A (gathered f', F/2 shift)."""
    A = _f64(A, (9, s.ny, s.nx))
    force = _f64(force, (2, s.ny, s.nx))
    rho = np.empty((s.ny, s.nx))
    u = np.empty((2, s.ny, s.nx))
    p = s.c()
    lib().orc_macros(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(rho),
                     _ptr(u[0]), _ptr(u[1]))
    return rho, u


def _bgk_only(s: Setup, what: str):
    if s.trt_magic > 0:
        raise NotImplementedError("%s: the oracle's adjoint covers the BGK collision only" % what)


def adjoint_step(s: Setup, mask, A, lam_next, force=None, grad_force=None):
    """dL/dA_t from dL/dA_{t+1}; grad_force (2,ny,nx) or (2,) accumulated in place."""
    _bgk_only(s, "adjoint_step")
    A = _f64(A, (9, s.ny, s.nx))
    lam_next = _f64(lam_next, (9, s.ny, s.nx))
    force = _f64(force, (2, s.ny, s.nx))
    lam = np.empty_like(A)
    p = s.c()
    lib().orc_adjoint_step(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(lam_next),
                           _ptr(lam), _ptr(grad_force))
    return lam


def macros_adjoint(s: Setup, mask, A, g_rho, g_u, force=None, lam=None, grad_force=None):
    _bgk_only(s, "macros_adjoint")
    A = _f64(A, (9, s.ny, s.nx))
    force = _f64(force, (2, s.ny, s.nx))
    if lam is None:
        lam = np.zeros_like(A)
    g_rho = _f64(g_rho, (s.ny, s.nx))
    g_u = _f64(g_u, (2, s.ny, s.nx))
    p = s.c()
    lib().orc_macros_adjoint(ctypes.byref(p), _ptr(mask), _ptr(force), _ptr(A), _ptr(g_rho),
                             None if g_u is None else _ptr(g_u[0]),
                             None if g_u is None else _ptr(g_u[1]), _ptr(lam), _ptr(grad_force))
    return lam


# ---- reductions and losses over fluid nodes (plain numpy definitions) ----

def mass(A, mask):
    fl = mask != SOLID
    return float(A[:, fl].sum())


def momentum(A, mask):
    cx, cy, _, _ = lattice()
    fl = mask != SOLID
    a = A[:, fl]
    return float((cx[:, None] * a).sum()), float((cy[:, None] * a).sum())


def loss_mse(u, u_target, mask):
    """L = (1/N_f) sum over fluid nodes of |u - u*|^2."""
    fl = mask != SOLID
    d = (u - u_target)[:, fl]
    return float((d * d).sum() / fl.sum())


def loss_ke(rho, u, mask):
    """L = 1/2 sum over fluid nodes of rho |u|^2."""
    fl = mask != SOLID
    return float(0.5 * (rho[fl] * (u[0][fl] ** 2 + u[1][fl] ** 2)).sum())

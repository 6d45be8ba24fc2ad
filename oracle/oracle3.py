"""Python face of the FP64 CPU oracle of the D3Q19 step (lbm3_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests and the CPU-baseline leg of
``bench.py`` may import this module.  It never imports the CUDA package and
the CUDA package never imports it.

Canonical layouts (numpy, x fastest): distributions ``A[19, nz, ny, nx]``
(float64), vector fields ``V[3, nz, ny, nx]``, scalar fields ``[nz, ny, nx]``,
link masks ``uint32[nz, ny, nx]`` (``SOLID`` for solid nodes).  What each
function computes, with the passage of the paper it follows, is stated in
lbm3_oracle.c.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from oracle import oracle as _orc

SOLID = 0xFFFFFFFF


class Params3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int), ("periodic_z", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("fz", ctypes.c_double),
    ]


@dataclass
class Setup3:
    """One three-dimensional run (mirrors orc3_params); a non-periodic axis
    has stationary half-way bounce-back walls on both faces."""
    nx: int
    ny: int
    nz: int
    tau: float
    periodic: tuple = (True, True, True)
    force: tuple = (0.0, 0.0, 0.0)

    def c(self) -> Params3:
        p = Params3()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        p.periodic_x, p.periodic_y, p.periodic_z = (int(bool(v)) for v in self.periodic)
        p.tau = self.tau
        p.fx, p.fy, p.fz = self.force
        return p

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = _orc.lib()
        P = ctypes.POINTER(Params3)
        vp = ctypes.c_void_p
        L.orc3_lattice.argtypes = [vp, vp, vp]
        L.orc3_link_mask.argtypes = [P, vp, vp]
        L.orc3_link_mask.restype = ctypes.c_long
        L.orc3_init_equilibrium.argtypes = [P, vp, vp, vp, vp]
        L.orc3_step.argtypes = [P, vp, vp, vp]
        L.orc3_run.argtypes = [P, vp, vp, vp, ctypes.c_int]
        L.orc3_macros.argtypes = [P, vp, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def lattice():
    """(c [19, 3] int, w [19] float64, opp [19] int) as the oracle uses them."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19, np.float64)
    opp = np.zeros(19, np.int32)
    lib().orc3_lattice(_p(c), _p(w), _p(opp))
    return c, w, opp


def link_mask(s: Setup3, solid=None):
    """(mask uint32 [nz, ny, nx], fluid node count)."""
    m = np.zeros(s.shape, np.uint32)
    sol = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
    if sol is not None:
        assert sol.shape == s.shape
    p = s.c()
    nf = lib().orc3_link_mask(ctypes.byref(p), _p(sol), _p(m))
    return m, int(nf)


def init_equilibrium(s: Setup3, mask, rho=None, u=None):
    A = np.zeros((19,) + s.shape, np.float64)
    r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    v = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
    p = s.c()
    lib().orc3_init_equilibrium(ctypes.byref(p), _p(np.ascontiguousarray(mask)), _p(r), _p(v), _p(A))
    return A


def step(s: Setup3, mask, A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.empty_like(A)
    p = s.c()
    lib().orc3_step(ctypes.byref(p), _p(np.ascontiguousarray(mask)), _p(A), _p(B))
    return B


def run(s: Setup3, mask, A, nsteps: int):
    A = np.array(A, dtype=np.float64, copy=True, order="C")
    B = np.empty_like(A)
    p = s.c()
    lib().orc3_run(ctypes.byref(p), _p(np.ascontiguousarray(mask)), _p(A), _p(B), int(nsteps))
    return A


def macros(s: Setup3, mask, A):
    rho = np.zeros(s.shape, np.float64)
    u = np.zeros((3,) + s.shape, np.float64)
    p = s.c()
    lib().orc3_macros(ctypes.byref(p), _p(np.ascontiguousarray(mask)), _p(np.ascontiguousarray(A, dtype=np.float64)),
                      _p(rho), _p(u))
    return rho, u


def mass(A, mask):
    """sum over fluid nodes and links of A."""
    fl = mask != SOLID
    return float(A[:, fl].sum())


def momentum(A, mask):
    c, _, _ = lattice()
    fl = mask != SOLID
    return np.array([float((c[:, a, None] * A[:, fl]).sum()) for a in range(3)])

"""Test cases shared by the oracle side and the CUDA side of the parity tests.

A case is plain data (sizes, tau, sides, force, solid mask, initial fields).
`oracle_setup` turns it into the oracle's Setup, `gpu_params` into the keyword
arguments of paper_2108_13241_gb300.lbm.LBM.  Neither side's arithmetic is
here: the fields come from paper_2108_13241_gb300.inputs.
"""
from dataclasses import dataclass, field

import numpy as np

from paper_2108_13241_gb300 import inputs

SIDES = ("west", "east", "south", "north")


@dataclass
class Case:
    name: str
    nx: int
    ny: int
    tau: float
    px: bool = True
    py: bool = True
    walls: dict = field(default_factory=dict)
    force: tuple = (0.0, 0.0)
    solid: np.ndarray = None
    rho0: np.ndarray = None
    u0: np.ndarray = None
    force_field: np.ndarray = None
    # open sides {side name: ("velocity", (ux, uy)) | ("pressure", rho)}, and
    # optional per-node values along a side {side name: array}
    open: dict = field(default_factory=dict)
    open_vals: dict = field(default_factory=dict)


def oracle_setup(orc, c: Case):
    op = {}
    for name, (kind, val) in c.open.items():
        op[SIDES.index(name)] = (kind, c.open_vals.get(name, val))
    return orc.Setup(nx=c.nx, ny=c.ny, tau=c.tau, periodic_x=c.px, periodic_y=c.py,
                     wall_u=[tuple(c.walls.get(s, (0.0, 0.0))) for s in SIDES], force=c.force, open=op)


def gpu_kwargs(c: Case):
    kw = dict(nx=c.nx, ny=c.ny, tau=c.tau, solid=c.solid, force=c.force, periodic_x=c.px,
              periodic_y=c.py, walls=c.walls)
    if c.open:
        kw["open"] = c.open
    return kw


def cavity(n=128, tau=0.6, lid=0.1):
    return Case("cavity%d" % n, n, n, tau, px=False, py=False, walls={"north": (lid, 0.0)})


def porous(nx, ny, frac, seed, tau=0.8, px=True, py=False, force=(2e-5, -1e-5), moving=True, field=False):
    solid = inputs.random_solid(nx, ny, frac, seed)
    walls = {"south": (0.02, 0.0), "north": (-0.03, 0.0)} if moving else {}
    c = Case("porous%dx%d_s%d_f%g" % (nx, ny, seed, frac), nx, ny, tau, px=px, py=py, walls=walls, force=force, solid=solid)
    c.rho0 = 1.0 + 0.01 * inputs.random_field((ny, nx), seed + 1)
    c.u0 = 0.03 * inputs.random_field((2, ny, nx), seed + 2)
    if field:
        c.force_field = 1e-4 * inputs.random_field((2, ny, nx), seed + 3)
    return c


def discs(nx, ny, phi, seed=inputs.GEOMETRY_SEED, tau=0.8, rmin=4.0, rmax=10.0, force=(1e-5, 0.0)):
    solid, achieved, _ = inputs.porous_discs(nx, ny, phi, rmin=rmin, rmax=rmax, seed=seed)
    return Case("discs%dx%d" % (nx, ny), nx, ny, tau, px=True, py=False, force=force, solid=solid)


def rel_l2(a, b, sel=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if sel is not None:
        a = a[..., sel]
        b = b[..., sel]
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))

"""Pins of the oracle's open sides: the constant-velocity and constant-pressure
boundary conditions of Sec. 3 (after Zou & He 1997).

What fixes them, independently of the oracle's own code:
  * uniform flow through a velocity inlet and a pressure outlet is a fixed
    point of the update (every open-side rule returns f^eq of the flow);
  * after one step, a boundary node carries exactly the side's velocity, or
    the side's density with zero tangential velocity (BGK conserves both, so
    the post-collision moments are those the open-side rule imposed);
  * the normal link obeys the bounce-back of the non-equilibrium part that
    defines the rule: f_i - f^eq_i = f_opp(i) - f^eq_opp(i);
  * a pressure-driven channel reaches a steady state whose particle flux
    between neighbouring columns is the same everywhere (discrete mass
    balance) and whose profile satisfies the momentum balance
    nu u'' = c_s^2 (d rho / dx) / rho at mid-channel.
"""
import math

import numpy as np
import pytest

from paper_2108_13241_gb300 import inputs

WEST, EAST, SOUTH, NORTH = 0, 1, 2, 3
TAU_MAGIC = 0.5 + math.sqrt(3.0 / 16.0)


def _feq(orc, s, mask, rho, u):
    return orc.init_equilibrium(s, mask, rho, u)


def _moments(orc, A):
    cx, cy, _, _ = orc.lattice()
    r = A.sum(0)
    return r, np.tensordot(cx, A, 1), np.tensordot(cy, A, 1)


@pytest.mark.parametrize("inlet,outlet,U", [(WEST, EAST, 0.05), (EAST, WEST, -0.04),
                                            (SOUTH, NORTH, 0.03), (NORTH, SOUTH, -0.05)])
@pytest.mark.parametrize("per_node", [False, True])
def test_uniform_flow_is_fixed_point(orc, inlet, outlet, U, per_node):
    nx, ny = 20, 14
    along_x = inlet < 2
    u = (U, 0.0) if along_x else (0.0, U)
    length = ny if along_x else nx
    vin = np.array(u) if not per_node else np.tile(np.array(u)[:, None], (1, length))
    vout = 1.0 if not per_node else np.ones(length)
    s = orc.Setup(nx=nx, ny=ny, tau=0.7, periodic_x=not along_x, periodic_y=along_x,
                  open={inlet: ("velocity", vin), outlet: ("pressure", vout)})
    mask, nf = orc.link_mask(s)
    assert nf == nx * ny
    uf = np.zeros((2, ny, nx))
    uf[0], uf[1] = u
    A0 = _feq(orc, s, mask, np.ones((ny, nx)), uf)
    A = A0.copy()
    for _ in range(25):
        A = orc.step(s, mask, A)
    # round-off only: at most 2 ulp of the largest value per step
    assert np.abs(A - A0).max() <= 25 * 2 * np.finfo(float).eps * np.abs(A0).max()


def _channel(orc, tau=0.8, nx=24, ny=12, seed=5):
    """Walls south/north, per-node velocity profile west, per-node density
    east, perturbed non-equilibrium initial state."""
    y = np.arange(ny)
    prof = np.stack([0.04 * (y + 0.5) * (ny - 0.5 - y) / (ny * ny / 4.0)
                     + 0.002 * inputs.random_field((ny,), seed),
                     0.003 * inputs.random_field((ny,), seed + 1)])
    rho_out = 1.0 + 0.002 * inputs.random_field((ny,), seed + 2)
    s = orc.Setup(nx=nx, ny=ny, tau=tau, periodic_x=False, periodic_y=False,
                  open={WEST: ("velocity", prof), EAST: ("pressure", rho_out)})
    mask, _ = orc.link_mask(s)
    rho0 = 1.0 + 0.01 * inputs.random_field((ny, nx), seed + 3)
    u0 = 0.03 * inputs.random_field((2, ny, nx), seed + 4)
    A = _feq(orc, s, mask, rho0, u0) + 1e-3 * inputs.random_field((9, ny, nx), seed + 5) / 9
    return s, mask, A, prof, rho_out


def test_open_sides_impose_velocity_and_density(orc):
    s, mask, A, prof, rho_out = _channel(orc)
    B = orc.step(s, mask, A)
    r, jx, jy = _moments(orc, B)
    inner = slice(1, s.ny - 1)  # corner nodes also bounce on the walls
    assert np.abs(jx[inner, 0] / r[inner, 0] - prof[0, inner]).max() <= 1e-15
    assert np.abs(jy[inner, 0] / r[inner, 0] - prof[1, inner]).max() <= 1e-15
    assert np.abs(r[inner, -1] - rho_out[inner]).max() <= 1e-14
    assert np.abs(jy[inner, -1]).max() <= 1e-16


def test_normal_link_nonequilibrium_bounces_back(orc):
    s, mask, A, _, _ = _channel(orc)
    B = orc.step(s, mask, A)
    r, jx, jy = _moments(orc, B)
    feq = _feq(orc, s, mask, r, np.stack([jx / r, jy / r]))
    neq = B - feq
    inner = slice(1, s.ny - 1)
    # west: unknown link 1 against its opposite 3; east: unknown 3 against 1
    assert np.abs(neq[1, inner, 0] - neq[3, inner, 0]).max() <= 1e-15
    assert np.abs(neq[3, inner, -1] - neq[1, inner, -1]).max() <= 1e-15


def _column_flux(B, ny):
    """Particles crossing from column x to x+1 minus back (x = 0 .. nx-2);
    diagonal populations of the wall rows bounce and stay in their column."""
    top, bot = np.ones(ny), np.ones(ny)
    top[-1] = 0.0
    bot[0] = 0.0
    R = (B[1] + B[5] * top[:, None] + B[8] * bot[:, None]).sum(0)
    L = (B[3] + B[6] * top[:, None] + B[7] * bot[:, None]).sum(0)
    return R[:-1] - L[1:]


def test_pressure_driven_channel_steady_state(orc):
    """Starting from rest, the density jump at the inlet also excites the
    lattice's staggered mode (j_x alternating in sign from column to column
    and from step to step, uniform in y), which BGK does not damp and the
    pressure sides reflect; the state settles to a period-2 cycle.  The
    average of two consecutive states is steady, and mass balance over the
    two-step period fixes its column flux exactly."""
    nx, ny, drho = 48, 8, 6e-4
    s = orc.Setup(nx=nx, ny=ny, tau=TAU_MAGIC, periodic_x=False, periodic_y=False,
                  open={WEST: ("pressure", 1.0 + drho), EAST: ("pressure", 1.0)})
    mask, _ = orc.link_mask(s)
    A = orc.run(s, mask, _feq(orc, s, mask, None, None), 20000)
    avg = None
    for _ in range(20):
        prev = avg
        A = orc.run(s, mask, A, 2000)
        avg = 0.5 * (A + orc.step(s, mask, A))
        if prev is not None and np.abs(avg - prev).max() < 1e-14:
            break
    assert np.abs(avg - prev).max() < 1e-14, "not steady"
    A = avg
    phi = _column_flux(A, ny)
    assert phi.min() > 0
    assert np.abs(phi - phi.mean()).max() <= 1e-11 * phi.mean()
    rho, u = orc.macros(s, mask, A)
    nu = (TAU_MAGIC - 0.5) / 3.0
    xm = nx // 2
    ux = u[0][:, xm]
    # the profile is a parabola vanishing half a spacing beyond the end rows
    y = np.arange(ny) + 0.5
    shape = y * (ny - y)
    amp = (ux @ shape) / (shape @ shape)
    assert np.abs(ux - amp * shape).max() <= 2e-3 * amp
    # momentum balance at mid-channel: nu u'' = c_s^2 (d rho/dx) / rho
    dpdx = (rho[:, xm + 1] - rho[:, xm - 1]).mean() / 2.0 / 3.0
    curv = -2.0 * amp
    assert curv < 0 and dpdx < 0
    assert abs(nu * curv - dpdx / rho[:, xm].mean()) <= 1e-2 * abs(dpdx)


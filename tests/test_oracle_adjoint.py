"""Pins of the oracle's discrete adjoint.

(i)  <J v, w> = <v, J^T w> for one step, with J v taken by the complex-step
     derivative of the forward step (exact to rounding, no cancellation);
(ii) central finite differences of a final-state loss through T steps and the
     macros, on tiny grids, against the chained adjoint.
"""
import numpy as np
import pytest

from paper_2108_13241_gb300 import inputs

CASES = {
    # name: (nx, ny, periodic_x, periodic_y, walls, solid fraction, per-node force)
    "periodic": (8, 8, True, True, None, 0.0, True),
    "channel": (16, 12, True, False, [(0, 0), (0, 0), (0.0, 0.0), (0.05, 0.0)], 0.15, True),
    "cavity": (12, 10, False, False, [(0, 0), (0, 0), (0, 0), (0.1, 0.0)], 0.1, False),
    # open sides: velocity inlet (per-node profile) and pressure outlet in x
    # with walls in y; pressure inlet and velocity outlet in y, periodic x
    "open_x": (16, 10, False, False, [(0, 0), (0, 0), (0.02, 0.0), (0, 0)], 0.1, True),
    "open_y": (10, 14, True, False, None, 0.1, False),
}
OPEN = {
    "open_x": lambda ny, nx: {0: ("velocity", np.stack([0.03 + 0.01 * inputs.random_field((ny,), 51),
                                                         0.005 * inputs.random_field((ny,), 52)])),
                              1: ("pressure", 1.0 + 0.002 * inputs.random_field((ny,), 53))},
    "open_y": lambda ny, nx: {2: ("pressure", 1.004), 3: ("velocity", (0.01, 0.02))},
}


def _setup(orc, name):
    nx, ny, px, py, walls, frac, field = CASES[name]
    kw = {}
    if walls is not None:
        kw["wall_u"] = walls
    if name in OPEN:
        kw["open"] = OPEN[name](ny, nx)
    s = orc.Setup(nx=nx, ny=ny, tau=0.7, periodic_x=px, periodic_y=py,
                  force=(0.0, 0.0) if field else (2e-4, -1e-4), **kw)
    solid = inputs.random_solid(nx, ny, frac, seed=nx + 3 * ny) if frac else None
    mask, _ = orc.link_mask(s, solid)
    F = 1e-3 * inputs.random_field((2, ny, nx), 17) if field else None
    rho = 1 + 0.02 * inputs.random_field((ny, nx), 18)
    u = 0.05 * inputs.random_field((2, ny, nx), 19)
    A = orc.init_equilibrium(s, mask, rho, u)
    A = A * (1 + 0.01 * inputs.random_field(A.shape, 20))  # off equilibrium
    return s, mask, F, A


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_dot_product_complex_step(orc, name):
    s, mask, F, A = _setup(orc, name)
    fl = (mask != 0xFF)
    vA = inputs.random_field(A.shape, 31) * fl
    wB = inputs.random_field(A.shape, 32) * fl
    h = 1e-30
    if F is not None:
        vF = inputs.random_field(F.shape, 33) * fl
        B = orc.step_cs(s, mask, A + 1j * h * vA, F + 1j * h * vF)
    else:
        vF = None
        B = orc.step_cs(s, mask, A + 1j * h * vA)
    Jv = B.imag / h
    gF = np.zeros_like(F) if F is not None else np.zeros(2)
    lam = orc.adjoint_step(s, mask, A, wB, force=F, grad_force=gF)
    lhs = float((Jv * wB * fl).sum())
    rhs = float((vA * lam).sum())
    if F is not None:
        rhs += float((vF * gF).sum())
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)
    assert np.all(lam[:, ~fl] == 0)
    # the real part of the complex-step run is the ordinary step
    B0 = orc.step(s, mask, A, F)
    assert np.array_equal(B.real, B0)


def _loss_through(orc, s, mask, A0, F, T, u_target):
    A = orc.run(s, mask, A0, T, force=F)
    _, u = orc.macros(s, mask, A, force=F)
    return orc.loss_mse(u, u_target, mask)


def _grad_through(orc, s, mask, A0, F, T, u_target):
    """Chained adjoint: dL/dA0 and dL/dF for L = mean_fluid |u_T - u*|^2."""
    states = [A0]
    for _ in range(T):
        states.append(orc.step(s, mask, states[-1], F))
    fl = mask != 0xFF
    _, u = orc.macros(s, mask, states[-1], force=F)
    g_u = 2.0 * (u - u_target) * fl / fl.sum()
    gF = np.zeros_like(F)
    lam = orc.macros_adjoint(s, mask, states[-1], None, g_u, force=F, grad_force=gF)
    for t in range(T - 1, -1, -1):
        lam = orc.adjoint_step(s, mask, states[t], lam, force=F, grad_force=gF)
    return lam, gF


@pytest.mark.parametrize("name", ["periodic", "channel", "open_x"])
def test_adjoint_matches_central_differences(orc, name):
    s, mask, F, A0 = _setup(orc, name)
    T = 12
    ut = inputs.target_velocity(s.nx, s.ny, (mask == 0xFF).astype(np.uint8), amp=0.05)
    lam, gF = _grad_through(orc, s, mask, A0, F, T, ut)
    rng = inputs.SplitMix64(inputs.FD_SEED)
    fl = np.argwhere(mask != 0xFF)
    for k in range(8):
        y, x = fl[rng.next_u64() % len(fl)]
        c = int(rng.next_u64() % 2)
        i = int(rng.next_u64() % 9)
        # force entry: plateau over a range of step sizes
        fd = []
        for h in (1e-5, 1e-6, 1e-7):
            Fp, Fm = F.copy(), F.copy()
            Fp[c, y, x] += h
            Fm[c, y, x] -= h
            fd.append((_loss_through(orc, s, mask, A0, Fp, T, ut)
                       - _loss_through(orc, s, mask, A0, Fm, T, ut)) / (2 * h))
        g = gF[c, y, x]
        assert min(abs(d - g) for d in fd) <= 1e-7 * abs(g) + 1e-8 * np.abs(gF).max()
        # initial-distribution entry
        fd = []
        for h in (1e-4, 1e-5, 1e-6):
            Ap, Am = A0.copy(), A0.copy()
            Ap[i, y, x] += h
            Am[i, y, x] -= h
            fd.append((_loss_through(orc, s, mask, Ap, F, T, ut)
                       - _loss_through(orc, s, mask, Am, F, T, ut)) / (2 * h))
        g = lam[i, y, x]
        assert min(abs(d - g) for d in fd) <= 1e-7 * abs(g) + 1e-8 * np.abs(lam).max()


def test_uniform_force_gradient_is_sum_of_field_gradient(orc):
    """With F uniform, dL/dF (2-vector) equals the node sum of dL/dF(x)."""
    s, mask, F, A = _setup(orc, "channel")
    lamB = inputs.random_field(A.shape, 40) * (mask != 0xFF)
    Fu = np.zeros_like(F)
    Fu[0], Fu[1] = 3e-4, -2e-4
    g_field = np.zeros_like(F)
    orc.adjoint_step(s, mask, A, lamB, force=Fu, grad_force=g_field)
    s2 = orc.Setup(nx=s.nx, ny=s.ny, tau=s.tau, periodic_x=s.periodic_x,
                   periodic_y=s.periodic_y, wall_u=s.wall_u, force=(3e-4, -2e-4))
    g_uni = np.zeros(2)
    orc.adjoint_step(s2, mask, A, lamB, force=None, grad_force=g_uni)
    assert np.allclose(g_uni, g_field.sum(axis=(1, 2)), rtol=1e-12, atol=1e-15)

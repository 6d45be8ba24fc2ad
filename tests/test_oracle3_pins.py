"""Pins of the D3Q19 FP64 oracle (oracle/lbm3_oracle.c) to facts that do not
come from the oracle itself: the lattice's defining moment identities, the
link mask from its definition by brute force, rest-state invariance, exact
mass conservation, the momentum gain of the Guo force, the viscosity of
Eq. 5 from shear-wave decay along every axis, and the plane Poiseuille
profile between half-way bounce-back walls (exact node by node at the
"magic" relaxation time, quadratic with the analytic curvature at any).
"""
import itertools

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle, oracle3
    oracle.build()
    return oracle3


def test_lattice_is_d3q19_with_isotropic_moments(o3):
    c, w, opp = o3.lattice()
    # the velocity set: every integer vector with components in {-1, 0, 1}
    # and |c|^2 <= 2 (19 of them), each once
    want = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2}
    assert len(want) == 19 and {tuple(v) for v in c} == want
    # weights by speed class: 1/3 rest, 1/18 axis, 1/36 diagonal
    sq = (c * c).sum(axis=1)
    assert np.allclose(w[sq == 0], 1 / 3) and np.allclose(w[sq == 1], 1 / 18) and np.allclose(w[sq == 2], 1 / 36)
    assert (c[opp] == -c).all() and (opp[opp] == np.arange(19)).all()
    d = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib->ab", w, c, c) - d / 3).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, c, c, c)).max() < 1e-15
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c) - iso4).max() < 1e-15


def brute_mask(nx, ny, nz, per, solid, c):
    m = np.zeros((nz, ny, nx), np.int64)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            m[z, y, x] = 0xFFFFFFFF
            continue
        bits = 0
        for i in range(1, 19):
            q = [x - c[i][0], y - c[i][1], z - c[i][2]]
            n = [nx, ny, nz]
            out = False
            for a in range(3):
                if not 0 <= q[a] < n[a]:
                    if per[a]:
                        q[a] %= n[a]
                    else:
                        out = True
            if out or solid[q[2], q[1], q[0]]:
                bits |= 1 << (i - 1)
        m[z, y, x] = bits
    return m


@pytest.mark.parametrize("per", [(True, True, True), (True, False, True), (False, True, False), (False, False, False)])
def test_link_mask_matches_brute_force(o3, per):
    rng = np.random.default_rng(31)
    nx, ny, nz = 7, 5, 6
    solid = (rng.random((nz, ny, nx)) < 0.25).astype(np.uint8)
    s = o3.Setup3(nx, ny, nz, 0.8, periodic=per)
    m, nf = o3.link_mask(s, solid)
    c, _, _ = o3.lattice()
    assert np.array_equal(m.astype(np.int64), brute_mask(nx, ny, nz, per, solid, c))
    assert nf == int((solid == 0).sum())


def porous_box(o3, rng, per=(True, False, True), force=(0.0, 0.0, 0.0)):
    nx, ny, nz = 12, 10, 8
    solid = (rng.random((nz, ny, nx)) < 0.2).astype(np.uint8)
    s = o3.Setup3(nx, ny, nz, 0.7, periodic=per, force=force)
    m, _ = o3.link_mask(s, solid)
    return s, m


def test_rest_state_is_invariant(o3):
    s, m = porous_box(o3, np.random.default_rng(5), per=(False, False, True))
    A0 = o3.init_equilibrium(s, m)
    A = o3.run(s, m, A0, 60)
    fl = m != o3.SOLID
    assert np.abs(A[:, fl] - A0[:, fl]).max() < 1e-15


def test_mass_is_conserved_with_walls_obstacles_and_force(o3):
    rng = np.random.default_rng(6)
    s, m = porous_box(o3, rng, per=(True, False, False), force=(2e-5, -1e-5, 3e-5))
    rho = 1.0 + 0.01 * rng.standard_normal(s.shape)
    u = 0.02 * rng.standard_normal((3,) + s.shape)
    A = o3.init_equilibrium(s, m, rho, u)
    m0 = o3.mass(A, m)
    A = o3.run(s, m, A, 300)
    assert abs(o3.mass(A, m) - m0) / m0 < 1e-13


def test_force_adds_exactly_its_momentum_on_a_periodic_box(o3):
    rng = np.random.default_rng(7)
    F = np.array([3e-5, -2e-5, 1e-5])
    s = o3.Setup3(6, 5, 4, 0.9, force=tuple(F))
    m, nf = o3.link_mask(s)
    A = o3.init_equilibrium(s, m, 1 + 0.01 * rng.standard_normal(s.shape), 0.02 * rng.standard_normal((3,) + s.shape))
    p0 = o3.momentum(A, m)
    steps = 50
    A = o3.run(s, m, A, steps)
    # the Guo source adds (1 - omega/2) F per node and step, the F/2 shift of
    # the velocity the rest: the post-collision momentum grows by exactly F
    assert np.abs(o3.momentum(A, m) - p0 - steps * nf * F).max() < 1e-12


def shear_rate(o3, axis_u, axis_k, n, tau, steps):
    """Measured exponential decay rate of a shear wave u_{axis_u} =
    U sin(2 pi x_{axis_k} / n) on a periodic box n long along axis_k."""
    dims = [4, 4, 4]
    dims[axis_k] = n
    nx, ny, nz = dims
    s = o3.Setup3(nx, ny, nz, tau)
    m, _ = o3.link_mask(s)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coord = (xx, yy, zz)[axis_k]
    prof = np.sin(2 * np.pi * coord / n)
    u = np.zeros((3,) + s.shape)
    u[axis_u] = 1e-4 * prof
    A = o3.init_equilibrium(s, m, None, u)
    amps = []
    for _ in range(2):
        A = o3.run(s, m, A, steps)
        _, v = o3.macros(s, m, A)
        amps.append((v[axis_u] * prof).sum() / (prof * prof).sum())
    return np.log(amps[0] / amps[1]) / steps


@pytest.mark.parametrize("axis_u,axis_k", [(0, 2), (1, 0), (2, 1)])
def test_shear_wave_decays_at_the_viscosity_of_eq5(o3, axis_u, axis_k):
    """nu = (tau - 1/2) / 3 (Eq. 5): the decay rate nu k^2 is matched to
    within the lattice's O(k^2) error, which shrinks as the wave is resolved
    finer (at least 3x from 16 to 32 nodes)."""
    tau = 0.8
    nu = (tau - 0.5) / 3
    errs = []
    for n in (16, 32):
        k = 2 * np.pi / n
        rate = shear_rate(o3, axis_u, axis_k, n, tau, steps=int(0.5 / (nu * k * k)))
        errs.append(abs(rate / (nu * k * k) - 1))
    assert errs[1] < 5e-3 and errs[0] > 3 * errs[1]


def poiseuille_plates(o3, tau, nz, steps, F=1e-6):
    """Walls on the z faces, periodic x and y, force along x; starts from the
    analytic profile and returns (u_x(z), analytic u_x(z))."""
    s = o3.Setup3(4, 4, nz, tau, periodic=(True, True, False), force=(F, 0.0, 0.0))
    m, _ = o3.link_mask(s)
    nu = (tau - 0.5) / 3
    z = np.arange(nz) + 0.5
    ua = F / (2 * nu) * z * (nz - z)  # walls half a spacing outside the outer nodes
    u = np.zeros((3,) + s.shape)
    u[0] = ua[:, None, None]
    A = o3.init_equilibrium(s, m, None, u)
    A = o3.run(s, m, A, steps)
    _, v = o3.macros(s, m, A)
    return v[0][:, 0, 0], ua


def test_poiseuille_between_plates_exact_at_the_magic_tau(o3):
    """Half-way bounce-back puts the wall exactly half a spacing out when
    (tau - 1/2)^2 = 3/16; there the discrete profile is the parabola node by
    node."""
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    ux, ua = poiseuille_plates(o3, tau, 16, 6000)
    assert np.abs(ux / ua - 1).max() < 1e-8


def test_poiseuille_between_plates_quadratic_with_the_analytic_curvature(o3):
    tau, F, nz = 0.8, 1e-6, 16
    ux, _ = poiseuille_plates(o3, tau, nz, 8000, F)
    z = np.arange(nz) + 0.5
    coef = np.polyfit(z, ux, 2)
    assert np.abs(np.polyval(coef, z) - ux).max() < 1e-10 * ux.max()
    nu = (tau - 0.5) / 3
    assert abs(2 * coef[0] / (-F / nu) - 1) < 1e-8

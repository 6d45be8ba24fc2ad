"""GPU parity of the D3Q19 step (lbm3_* of include/lbm.h) with the FP64 CPU
oracle (oracle/lbm3_oracle.c): Algorithm 1 in three dimensions with the
moments of Eq. 2 (Guo F/2 shift), the equilibrium of Eq. 6 with the D3Q19
weights, BGK (Eq. 3-5) and half-way bounce-back.

  * FP64 storage: canonical distributions within 1e-12 relative L2 of the
    oracle after 200 steps, on a periodic box, a porous box with walls on
    two axes and a force, and ragged sizes (nx not a multiple of the block);
  * FP32 storage: velocity within 1e-5 relative L2 of the oracle;
  * macros, get/set of the canonical state, the rest state, argument checks.
"""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle, oracle3
    oracle.build()
    return oracle3


CASES = {
    # name: (nx, ny, nz, tau, periodic, force, solid fraction, seed)
    "periodic_box": (24, 16, 20, 0.8, (True, True, True), (0.0, 0.0, 0.0), 0.0, 301),
    "porous_walls_force": (32, 12, 14, 0.7, (True, False, False), (2e-5, -1e-5, 3e-6), 0.15, 302),
    "ragged_all_walls": (37, 11, 9, 0.9, (False, False, False), (0.0, 1e-5, 0.0), 0.1, 303),
    "wide_rows": (160, 6, 5, 0.6, (True, True, False), (1e-5, 0.0, 0.0), 0.05, 304),
}


def setup(o3, name):
    nx, ny, nz, tau, per, F, frac, seed = CASES[name]
    solid = inputs.random_solid_3d(nx, ny, nz, frac, seed) if frac > 0 else None
    rho = 1.0 + 0.01 * inputs.random_field((nz, ny, nx), seed + 1)
    u = 0.03 * inputs.random_field((3, nz, ny, nx), seed + 2)
    s = o3.Setup3(nx, ny, nz, tau, periodic=per, force=F)
    return s, solid, rho, u


_REF = {}


def oracle_run(o3, name, steps):
    key = (name, steps)
    if key not in _REF:
        s, solid, rho, u = setup(o3, name)
        m, _ = o3.link_mask(s, solid)
        A = o3.run(s, m, o3.init_equilibrium(s, m, rho, u), steps)
        r, v = o3.macros(s, m, A)
        _REF[key] = (A, r, v, m)
    return _REF[key]


def gpu(L, o3, name, steps, precision):
    s, solid, rho, u = setup(o3, name)
    sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, force=s.force, periodic=s.periodic, precision=precision)
    sim.init_equilibrium(rho, u)
    sim.step(steps)
    f = sim.get_f().double().cpu().numpy()
    r, v = sim.macros()
    out = (f, r.double().cpu().numpy(), v.double().cpu().numpy(), sim.fluid_nodes)
    sim.close()
    return out


def rel_l2(a, b, fl):
    return np.linalg.norm((a - b)[..., fl]) / np.linalg.norm(b[..., fl])


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle(L, o3, name):
    A, r_ref, u_ref, m = oracle_run(o3, name, 200)
    f, r, u, nf = gpu(L, o3, name, 200, "f64")
    fl = m != o3.SOLID
    assert nf == int(fl.sum())
    assert rel_l2(f, A, fl) <= 1e-12
    assert rel_l2(u, u_ref, fl) <= 1e-11
    assert np.abs(r - r_ref)[fl].max() <= 1e-12
    # solid nodes: zero macros, canonical state w_i
    if (~fl).any():
        assert (r[~fl] == 0).all() and (u[:, ~fl] == 0).all()
        _, w, _ = o3.lattice()
        assert np.allclose(f[:, ~fl], w[:, None])


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_velocity_matches_oracle(L, o3, name):
    A, _, u_ref, m = oracle_run(o3, name, 200)
    _, _, u, _ = gpu(L, o3, name, 200, "f32")
    assert rel_l2(u, u_ref, m != o3.SOLID) <= 1e-5


def test_set_f_then_step_matches_oracle_step(L, o3):
    """The canonical state goes in and out unchanged (FP64) and one step from
    it is the oracle's step from the same state."""
    s, solid, rho, u = setup(o3, "porous_walls_force")
    m, _ = o3.link_mask(s, solid)
    A0 = o3.run(s, m, o3.init_equilibrium(s, m, rho, u), 7)
    sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, force=s.force, periodic=s.periodic, precision="f64")
    sim.set_f(A0)
    fl = m != o3.SOLID
    back = sim.get_f().cpu().numpy()
    assert np.abs(back - A0)[:, fl].max() <= 1e-15
    sim.step(1)
    B = o3.step(s, m, A0)
    assert rel_l2(sim.get_f().cpu().numpy(), B, fl) <= 1e-13
    assert sim.steps == 1
    sim.close()


def test_rest_state_stays_at_rest(L, o3):
    s, solid, _, _ = setup(o3, "ragged_all_walls")
    sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, periodic=s.periodic, precision="f64")
    sim.init_equilibrium(None, None)
    f0 = sim.get_f().cpu().numpy()
    sim.step(50)
    assert np.abs(sim.get_f().cpu().numpy() - f0).max() < 1e-15
    sim.close()


def test_taylor_green_3d_against_oracle(L, o3):
    """The benchmark's 3-D Taylor-Green field on a 64^3 box, 200 steps (the
    vortex keeps about half its velocity; FP32 storage rounding accumulates
    in absolute terms, so a vortex decayed to a few percent reads a larger
    relative error: 1.1e-5 on 32^3 after 300 steps)."""
    n, steps = 64, 200
    rho, u = inputs.taylor_green_3d(n, n, n, 0.05)
    s = o3.Setup3(n, n, n, 0.8)
    m, _ = o3.link_mask(s)
    A = o3.run(s, m, o3.init_equilibrium(s, m, rho, u), steps)
    _, u_ref = o3.macros(s, m, A)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
        sim = L.LBM3(n, n, n, 0.8, precision=prec)
        sim.init_equilibrium(rho, u)
        sim.step(steps)
        _, v = sim.macros()
        assert rel_l2(v.double().cpu().numpy(), u_ref, m != o3.SOLID) <= tol, prec
        sim.close()


def test_arguments_are_checked(L):
    with pytest.raises(L.LBMError):
        L.LBM3(8, 8, 8, 0.5)
    sim = L.LBM3(8, 8, 8, 0.8)
    with pytest.raises(L.LBMError) as ei:
        sim.step(-1)
    assert ei.value.status == L.LBM_ERR_INVALID
    sim.close()


def test_benchmark_box_one_step_matches_oracle(L, o3):
    """The benchmark's configuration (256^3 periodic 3-D Taylor-Green, FP32,
    the launch bench.py times): one step from the GPU's own state after 10
    steps, against the oracle's step from that state (FP32 storage rounding
    only: 1e-6 relative L2 on f, 1e-5 on u)."""
    n = 256
    rho, u = inputs.taylor_green_3d(n, n, n, 0.05)
    sim = L.LBM3(n, n, n, 0.8, precision="f32")
    sim.init_equilibrium(rho, u)
    del rho, u
    sim.step(10)
    A = sim.get_f().double().cpu().numpy()
    sim.step(1)
    f = sim.get_f().double().cpu().numpy()
    _, v = sim.macros()
    v = v.double().cpu().numpy()
    sim.close()
    s = o3.Setup3(n, n, n, 0.8)
    m, _ = o3.link_mask(s)
    B = o3.step(s, m, A)
    del A
    _, u_ref = o3.macros(s, m, B)
    fl = m != o3.SOLID
    assert rel_l2(f, B, fl) <= 1e-6
    assert rel_l2(v, u_ref, fl) <= 1e-5


@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
def test_porous_spheres_benchmark_box_one_step_matches_oracle(L, o3, pattern):
    """The benchmark's porous configuration (256^3 random spheres, porosity
    0.5, force along x, FP32; two lattices on the dense grid, AA over the
    node list -- the launches bench.py times): one step from the GPU's own
    state after 10 steps from a Taylor-Green velocity field, against the
    oracle's step from that state (FP32 storage rounding only: 1e-6
    relative L2 on f, 1e-5 on u, fluid nodes)."""
    n = 256
    solid, _ = inputs.porous_spheres_3d(n, 0.5)
    rho, u = inputs.taylor_green_3d(n, n, n, 0.05)
    sim = L.LBM3(n, n, n, 0.8, solid=solid, force=(1e-6, 0.0, 0.0), precision="f32", pattern=pattern)
    assert (sim.list_nodes > 0) == (pattern == "aa")
    sim.init_equilibrium(rho, u)
    del rho, u
    sim.step(10)
    A = sim.get_f().double().cpu().numpy()
    sim.step(1)
    f = sim.get_f().double().cpu().numpy()
    _, v = sim.macros()
    v = v.double().cpu().numpy()
    sim.close()
    s = o3.Setup3(n, n, n, 0.8, force=(1e-6, 0.0, 0.0))
    m, _ = o3.link_mask(s, solid)
    B = o3.step(s, m, A)
    del A
    _, u_ref = o3.macros(s, m, B)
    fl = m != o3.SOLID
    assert rel_l2(f, B, fl) <= 1e-6
    assert rel_l2(v, u_ref, fl) <= 1e-5


def test_box_beyond_32_bit_slot_offsets_equals_its_tiled_period(L):
    """640^3 nodes (19 x 640^3 > 2^32 values a lattice: 64-bit slot offsets,
    40 GB of FP32 lattices): a 3-D Taylor-Green field of period 64 tiled ten
    times along each axis evolves exactly like the 64^3 box it tiles -- every
    node does the same arithmetic on the same neighbour values, so the two
    agree bit for bit after 20 steps."""
    p, reps, steps = 64, 10, 20
    rho, u = inputs.taylor_green_3d(p, p, p, 0.05)
    r_s = torch.as_tensor(rho, dtype=torch.float32, device="cuda")
    u_s = torch.as_tensor(u, dtype=torch.float32, device="cuda")
    small = L.LBM3(p, p, p, 0.8, precision="f32")
    small.init_equilibrium(r_s, u_s)
    small.step(steps)
    _, v_small = small.macros()
    small.close()
    n = p * reps
    big = L.LBM3(n, n, n, 0.8, precision="f32")
    assert 19 * n ** 3 > 2 ** 32
    big.init_equilibrium(r_s.repeat(reps, reps, reps), u_s.repeat(1, reps, reps, reps))
    big.step(steps)
    _, v_big = big.macros()
    big.close()
    del big
    tiled = v_small.repeat(1, reps, reps, reps)
    assert torch.equal(v_big, tiled)


def test_fp16s_storage_taylor_green_and_porous_against_oracle(L, o3):
    """FP16-shifted storage ((f - w) 2^10 in binary16, stochastic rounding,
    FP32 arithmetic): the 3-D Taylor-Green velocity within 1e-3 relative L2
    of the FP64 oracle after 200 steps on 64^3 (the precision target of the
    two-dimensional configurations); on the porous, walled, forced box --
    whose random initial field decays to a small velocity, against which
    binary16's 11-bit mantissa reads larger -- within 1e-2; and bit-for-bit
    reproducible (counter-based random bits)."""
    n, steps = 64, 200
    rho, u = inputs.taylor_green_3d(n, n, n, 0.05)
    s = o3.Setup3(n, n, n, 0.8)
    m, _ = o3.link_mask(s)
    A = o3.run(s, m, o3.init_equilibrium(s, m, rho, u), steps)
    _, u_ref = o3.macros(s, m, A)
    runs = []
    for _ in range(2):
        sim = L.LBM3(n, n, n, 0.8, precision="f16s")
        sim.init_equilibrium(rho, u)
        sim.step(steps)
        _, v = sim.macros()
        runs.append(v.double().cpu().numpy())
        sim.close()
    assert np.array_equal(runs[0], runs[1])
    assert rel_l2(runs[0], u_ref, m != o3.SOLID) <= 1e-3
    A, _, u_ref, m = oracle_run(o3, "porous_walls_force", 200)
    _, _, v, _ = gpu(L, o3, "porous_walls_force", 200, "f16s")
    assert rel_l2(v, u_ref, m != o3.SOLID) <= 1e-2


def test_fp16s_needs_even_nx(L):
    with pytest.raises(L.LBMError) as ei:
        L.LBM3(37, 8, 8, 0.8, precision="f16s")
    assert ei.value.status == L.LBM_ERR_INVALID


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("steps", [1, 2, 7])
@pytest.mark.parametrize("name", ["porous_walls_force", "periodic_box", "ragged_all_walls"])
def test_aa_pattern_equals_two_lattice(L, o3, name, steps, precision):
    """The in-place AA pattern (one lattice, alternating gather/scatter and
    local steps) gives the two-lattice step's state bit for bit after odd
    and even step counts, and the same macros; it needs half the memory."""
    s, solid, rho, u = setup(o3, name)
    out = {}
    for pattern in ("two_lattice", "aa"):
        sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, force=s.force, periodic=s.periodic,
                     precision=precision, pattern=pattern)
        sim.init_equilibrium(rho, u)
        sim.step(steps)
        r, v = sim.macros()
        out[pattern] = (sim.get_f().cpu().numpy(), r.cpu().numpy(), v.cpu().numpy(), sim.workspace.numel())
        sim.close()
    m, _ = o3.link_mask(s, solid)
    fl = m != o3.SOLID
    f2, r2, u2, b2 = out["two_lattice"]
    fa, ra, ua, ba = out["aa"]
    assert np.array_equal(fa[:, fl], f2[:, fl])
    assert np.array_equal(ra, r2) and np.array_equal(ua, u2)
    assert ba < 0.6 * b2


def test_aa_set_f_and_fp16s_refused(L, o3):
    s, solid, rho, u = setup(o3, "porous_walls_force")
    m, _ = o3.link_mask(s, solid)
    A0 = o3.run(s, m, o3.init_equilibrium(s, m, rho, u), 3)
    sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, force=s.force, periodic=s.periodic,
                 precision="f64", pattern="aa")
    sim.set_f(A0)
    sim.step(3)
    B = o3.run(s, m, A0, 3)
    assert rel_l2(sim.get_f().cpu().numpy(), B, m != o3.SOLID) <= 1e-13
    sim.close()
    with pytest.raises(L.LBMError) as ei:
        L.LBM3(16, 8, 8, 0.8, precision="f16s", pattern="aa")
    assert ei.value.status == L.LBM_ERR_UNSUPPORTED


def test_porous_spheres_crop_matches_oracle(L, o3):
    """A 48^3 crop of the benchmark's 3-D porous medium (random spheres,
    porosity 0.5), walls on the z faces, force along x: FP64 within 1e-12 of
    the oracle on f, FP32 within 1e-5 on u, two-lattice and AA, 60 steps."""
    solid_full, _ = inputs.porous_spheres_3d(256, 0.5)
    solid = np.ascontiguousarray(solid_full[:48, :48, :48])
    s = o3.Setup3(48, 48, 48, 0.8, periodic=(True, True, False), force=(1e-5, 0.0, 0.0))
    m, _ = o3.link_mask(s, solid)
    A = o3.run(s, m, o3.init_equilibrium(s, m), 60)
    _, u_ref = o3.macros(s, m, A)
    fl = m != o3.SOLID
    for prec in ("f64", "f32"):
        for pattern in ("two_lattice", "aa"):
            sim = L.LBM3(48, 48, 48, 0.8, solid=solid, force=s.force, periodic=s.periodic, precision=prec,
                         pattern=pattern)
            sim.init_equilibrium(None, None)
            sim.step(60)
            f = sim.get_f().double().cpu().numpy()
            _, v = sim.macros()
            sim.close()
            if prec == "f64":
                assert rel_l2(f, A, fl) <= 1e-12, pattern
            assert rel_l2(v.double().cpu().numpy(), u_ref, fl) <= 1e-5, (prec, pattern)


def listed_count(solid, shape, precision, pattern):
    """Entries the node list should hold: fluid nodes and, with two lattices,
    the solid nodes sharing a 32-byte sector (4 FP64 / 8 FP32 nodes of
    consecutive index) with a fluid node."""
    n = int(np.prod(shape))
    fl = np.ones(n, bool) if solid is None else ~np.asarray(solid, bool).reshape(-1)
    if pattern == "aa":
        return int(fl.sum())
    g = 4 if precision == "f64" else 8
    pad = np.zeros(-(-n // g) * g, bool)
    pad[:n] = fl
    any_fluid = np.repeat(pad.reshape(-1, g).any(1), g)[:n]
    return int(any_fluid.sum())


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
@pytest.mark.parametrize("name", ["porous_walls_force", "ragged_all_walls", "spheres_crop"])
def test_node_list_equals_dense_grid(L, o3, name, pattern, precision):
    """The listed step (one thread per listed node, coordinates from the
    node index) gives the dense grid's state and macros bit for bit after
    odd and even step counts, on ragged boxes and a crop of the porous
    spheres; the list holds the fluid nodes and, with two lattices, the
    solid nodes sharing a sector with them."""
    if name == "spheres_crop":
        solid_full, _ = inputs.porous_spheres_3d(256, 0.5)
        solid = np.ascontiguousarray(solid_full[:40, :36, :44])
        s = o3.Setup3(44, 36, 40, 0.8, periodic=(True, True, False), force=(1e-5, 2e-6, 0.0))
        rho = 1.0 + 0.01 * inputs.random_field((40, 36, 44), 401)
        u = 0.03 * inputs.random_field((3, 40, 36, 44), 402)
    else:
        s, solid, rho, u = setup(o3, name)
    m, _ = o3.link_mask(s, solid)
    fl = m != o3.SOLID
    for steps in (5, 6):
        out = {}
        for mode in ("never", "always"):
            sim = L.LBM3(s.nx, s.ny, s.nz, s.tau, solid=solid, force=s.force, periodic=s.periodic,
                         precision=precision, pattern=pattern, node_list=mode)
            if mode == "never":
                assert sim.list_nodes == 0
            else:
                assert sim.list_nodes == listed_count(solid, (s.nz, s.ny, s.nx), precision, pattern)
            sim.init_equilibrium(rho, u)
            sim.step(steps)
            r, v = sim.macros()
            out[mode] = (sim.get_f().cpu().numpy(), r.cpu().numpy(), v.cpu().numpy())
            sim.close()
        fd, rd, ud = out["never"]
        fs, rs, us = out["always"]
        assert np.array_equal(fs[:, fl], fd[:, fl]), steps
        assert np.array_equal(rs, rd) and np.array_equal(us, ud), steps


def test_node_list_chosen_on_sparse_boxes_only(L):
    """auto: a list for the AA pattern when it holds at most 90% of the
    nodes (the porous spheres), the dense grid with two lattices and on a
    box with walls only; FP16s storage always runs its dense pair kernel."""
    solid_full, _ = inputs.porous_spheres_3d(256, 0.5)
    solid = np.ascontiguousarray(solid_full[:32, :32, :32])
    sim = L.LBM3(32, 32, 32, 0.8, solid=solid, precision="f32", pattern="aa")
    assert 0 < sim.list_nodes < 0.9 * 32 ** 3
    sim.close()
    sim = L.LBM3(32, 32, 32, 0.8, solid=solid, precision="f32")
    assert sim.list_nodes == 0
    sim.close()
    sim = L.LBM3(32, 32, 32, 0.8, periodic=(True, True, False), precision="f32", pattern="aa")
    assert sim.list_nodes == 0
    sim.close()
    sim = L.LBM3(32, 32, 32, 0.8, solid=solid, precision="f16s", node_list="always")
    assert sim.list_nodes == 0
    sim.close()

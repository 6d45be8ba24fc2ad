"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances:
  * FP64 storage: canonical distributions within 1e-12 relative L2 of the
    oracle after the run (the GPU computes in shifted variables with FMA
    contraction, the oracle unshifted without: only rounding differs);
  * FP32 storage: velocity within 1e-5 relative L2 after 1000 steps;
  * FP16-shifted storage: the velocity error against the oracle is measured
    and bounded (binary16 keeps 11 bits of f_i - w_i);
  * integer tables (link mask, tile map): bit-exact;
  * FP64 variants that feed the same collision the same operands (dense vs
    tiled, two-lattice vs AA) agree bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs
from tests import cases as C

pytestmark = pytest.mark.gpu

VARIANTS = [("dense", "two_lattice"), ("dense", "aa"), ("sparse", "two_lattice"), ("sparse", "aa")]


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def run_gpu(L, case, steps, precision="f64", layout="dense", pattern="two_lattice"):
    sim = L.LBM(precision=precision, layout=layout, pattern=pattern, **C.gpu_kwargs(case))
    if case.force_field is not None:
        sim.set_force(case.force_field)
    sim.init_equilibrium(case.rho0, case.u0)
    sim.step(steps)
    f = sim.get_f().double().cpu().numpy()
    rho, u = sim.macros()
    torch.cuda.synchronize()
    out = dict(f=f, rho=rho.double().cpu().numpy(), u=u.double().cpu().numpy(), sim=sim)
    return out


def run_oracle(orc, case, steps):
    s = C.oracle_setup(orc, case)
    mask, nf = orc.link_mask(s, case.solid)
    A = orc.init_equilibrium(s, mask, case.rho0, case.u0)
    A = orc.run(s, mask, A, steps, force=case.force_field)
    rho, u = orc.macros(s, mask, A, force=case.force_field)
    return dict(f=A, rho=rho, u=u, mask=mask, nf=nf, setup=s)


_ORACLE_CACHE = {}


def oracle_cached(orc, case, steps):
    key = (case.name, case.tau, steps, case.px, case.py, tuple(sorted(case.walls.items())), case.force)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = run_oracle(orc, case, steps)
    return _ORACLE_CACHE[key]


# ------------------------------------------------------------------ FP64 parity

@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_cavity_fp64_matches_oracle(L, orc, layout, pattern):
    """Lid-driven cavity 128^2, tau 0.6, lid 0.1, 1000 steps, FP64."""
    case = C.cavity(128)
    o = oracle_cached(orc, case, 1000)
    g = run_gpu(L, case, 1000, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    err = C.rel_l2(g["f"], o["f"], fl)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None]
    dev = C.rel_l2(g["f"][:, fl] - w, o["f"][:, fl] - w)
    assert err <= 1e-12, err
    assert dev <= 1e-10, dev
    assert C.rel_l2(g["u"], o["u"], fl) <= 1e-11


@pytest.mark.parametrize("layout,pattern", VARIANTS)
@pytest.mark.parametrize("steps", [1, 2, 101])
def test_porous_ragged_fp64_matches_oracle(L, orc, layout, pattern, steps):
    """48 x 37 (ragged last tile row), 25% random solids, periodic x, moving
    walls in y, uniform Guo force, random initial state; odd and even step
    counts exercise both AA steps."""
    case = C.porous(48, 37, 0.25, seed=101)
    o = oracle_cached(orc, case, steps)
    g = run_gpu(L, case, steps, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12
    assert C.rel_l2(g["u"], o["u"], fl) <= 1e-11


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_periodic_force_field_fp64_matches_oracle(L, orc, layout, pattern):
    """Fully periodic 64 x 32 with obstacles and a per-node force field."""
    case = C.porous(64, 32, 0.2, seed=202, py=True, moving=False, field=True, force=(0.0, 0.0))
    o = oracle_cached(orc, case, 60)
    g = run_gpu(L, case, 60, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12


def test_all_walls_moving_fp64(L, orc):
    """Every side a moving wall (tangential), corners by the y-first rule."""
    case = C.Case("box", 32, 24, 0.7, px=False, py=False,
                  walls={"west": (0.0, 0.03), "east": (0.0, -0.02), "south": (0.04, 0.0), "north": (-0.05, 0.0)})
    o = oracle_cached(orc, case, 300)
    for layout, pattern in VARIANTS:
        g = run_gpu(L, case, 300, "f64", layout, pattern)
        fl = o["mask"] != 0xFF
        assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12, (layout, pattern)


def test_fp64_variants_bitwise_identical(L):
    """Dense/tiled x two-lattice/AA feed the same collision the same operands."""
    case = C.porous(48, 37, 0.25, seed=101)
    ref = None
    for layout, pattern in VARIANTS:
        for steps in (7, 8):
            g = run_gpu(L, case, steps, "f64", layout, pattern)
            key = steps
            if ref is None:
                ref = {}
            if key not in ref:
                ref[key] = g["f"]
            else:
                assert np.array_equal(g["f"], ref[key]), (layout, pattern, steps)


@pytest.mark.parametrize("precision", ["f32", "f16s"])
def test_low_precision_variants_bitwise_identical(L, precision):
    case = C.porous(64, 48, 0.3, seed=303)
    ref = None
    for layout, pattern in VARIANTS:
        g = run_gpu(L, case, 9, precision, layout, pattern)
        if ref is None:
            ref = g["f"]
        else:
            assert np.array_equal(g["f"], ref), (layout, pattern)


# ------------------------------------------------------------------ FP32 / FP16s

@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_cavity_fp32_velocity_within_1e5(L, orc, layout, pattern):
    case = C.cavity(128)
    o = oracle_cached(orc, case, 1000)
    g = run_gpu(L, case, 1000, "f32", layout, pattern)
    fl = o["mask"] != 0xFF
    err = C.rel_l2(g["u"], o["u"], fl)
    assert err <= 1e-5, err


@pytest.mark.parametrize("layout,pattern", [("dense", "two_lattice"), ("sparse", "aa")])
def test_cavity_fp16s_velocity_error_bounded(L, orc, layout, pattern):
    case = C.cavity(128)
    o = oracle_cached(orc, case, 1000)
    g = run_gpu(L, case, 1000, "f16s", layout, pattern)
    fl = o["mask"] != 0xFF
    err = C.rel_l2(g["u"], o["u"], fl)
    print("fp16s cavity rel L2 u error:", err)
    assert err <= 1e-2, err


# ------------------------------------------------------------------ other entry points

def test_macros_reduce_and_loss_match_oracle(L, orc):
    case = C.porous(64, 40, 0.2, seed=404)
    o = oracle_cached(orc, case, 33)
    for layout, pattern in VARIANTS:
        g = run_gpu(L, case, 33, "f64", layout, pattern)
        fl = o["mask"] != 0xFF
        assert np.abs(g["rho"][fl] - o["rho"][fl]).max() < 1e-13
        assert np.abs(g["u"][:, fl] - o["u"][:, fl]).max() < 1e-13
        assert np.all(g["rho"][~fl] == 1) and np.all(g["u"][:, ~fl] == 0)
        sim = g["sim"]
        mass, mom = sim.reduce()
        assert abs(mass - orc.mass(o["f"], o["mask"])) < 1e-10
        om = orc.momentum(o["f"], o["mask"])
        assert abs(mom[0] - om[0]) < 1e-12 and abs(mom[1] - om[1]) < 1e-12
        ut = inputs.target_velocity(case.nx, case.ny, case.solid)
        assert abs(sim.loss_mse(ut) - orc.loss_mse(o["u"], ut, o["mask"])) < 1e-14
        assert abs(sim.loss_ke() - orc.loss_ke(o["rho"], o["u"], o["mask"])) < 1e-12


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_get_set_roundtrip_and_resume(L, orc, layout, pattern):
    """set_f(A) then get_f gives A back (canonical layout, any pattern); a run
    resumed from an exported state continues exactly."""
    case = C.porous(48, 32, 0.2, seed=505)
    g = run_gpu(L, case, 5, "f64", layout, pattern)
    sim = g["sim"]
    f5 = sim.get_f()
    sim.step(4)
    f9 = sim.get_f().cpu().numpy()
    sim2 = L.LBM(precision="f64", layout=layout, pattern=pattern, **C.gpu_kwargs(case))
    sim2.set_f(f5)
    back = sim2.get_f()
    fl = sim.link_mask() != 0xFF
    assert torch.allclose(back[:, torch.as_tensor(fl).cuda()], f5[:, torch.as_tensor(fl).cuda()], rtol=0, atol=1e-16)
    sim2.step(4)
    # get_f returns w_i + stored value and set_f stores f_i - w_i: one rounding each way
    assert C.rel_l2(sim2.get_f().cpu().numpy(), f9, fl) <= 1e-15


def test_tables_from_context_match_oracle(L, orc):
    case = C.porous(80, 53, 0.4, seed=606)
    s = C.oracle_setup(orc, case)
    omask, _ = orc.link_mask(s, case.solid)
    otid, onbr = orc.tile_map(s, omask)
    sim = L.LBM(precision="f32", layout="sparse", **C.gpu_kwargs(case))
    assert np.array_equal(sim.link_mask(), omask)
    tid, nbr = sim.tile_map()
    assert np.array_equal(tid, otid) and np.array_equal(nbr, onbr)


def test_all_solid_and_tiny_domains(L):
    solid = np.ones((20, 32), np.uint8)
    for layout in ("dense", "sparse"):
        sim = L.LBM(32, 20, 0.8, solid=solid, periodic_y=False, precision="f32", layout=layout)
        sim.step(3)
        mass, _ = sim.reduce()
        assert mass == 0.0 and sim.fluid_nodes == 0
    sim = L.LBM(16, 1, 0.8, precision="f64")  # one periodic row
    sim.step(5)
    mass, _ = sim.reduce()
    assert abs(mass - 16) < 1e-12


def test_step_count_and_zero_steps(L):
    sim = L.LBM(32, 16, 0.8, precision="f32")
    f0 = sim.get_f()
    sim.step(0)
    assert torch.equal(sim.get_f(), f0) and sim.steps == 0
    sim.step(3)
    assert sim.steps == 3


@pytest.mark.parametrize("layout,pattern", VARIANTS)
@pytest.mark.parametrize("steps", [1, 2, 41])
def test_wall_rows_fp64_matches_oracle(L, orc, layout, pattern, steps):
    """Periodic x, moving walls in y, no obstacle (small grid: one masked
    launch)."""
    nx, ny = 64, 24
    case = C.Case("wallrows%dx%d" % (nx, ny), nx, ny, 0.7, px=True, py=False,
                  walls={"south": (0.03, 0.0), "north": (-0.02, 0.0)}, force=(1e-5, -2e-6))
    case.rho0 = 1.0 + 0.01 * inputs.random_field((ny, nx), 711)
    case.u0 = 0.03 * inputs.random_field((2, ny, nx), 712)
    o = oracle_cached(orc, case, steps)
    g = run_gpu(L, case, steps, "f64", layout, pattern)
    assert C.rel_l2(g["f"], o["f"]) <= 1e-12
    assert C.rel_l2(g["u"], o["u"]) <= 1e-11


@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
@pytest.mark.parametrize("steps", [1, 2])
@pytest.mark.parametrize("sides", ["walls", "open"])
def test_wall_rows_split_fp64_large_grid(L, orc, pattern, steps, sides):
    """2048 x 2056 (> 2^21 nodes), periodic x, moving walls (or velocity
    inlet and pressure outlet) in y, force: the dense layout runs the two
    boundary rows with the masked kernel and the other rows with the unmasked
    one; every node against the oracle."""
    nx, ny = 2048, 2056
    case = C.Case("wallrows_large_" + sides, nx, ny, 0.7, px=True, py=False,
                  walls={"south": (0.03, 0.0), "north": (-0.02, 0.0)}, force=(1e-5, -2e-6))
    if sides == "open":
        case.walls = {}
        case.open = {"south": ("velocity", (0.01, 0.02)), "north": ("pressure", 1.0)}
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    case.rho0 = 1.0 + 0.01 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    case.u0 = np.stack([0.03 * np.cos(2 * np.pi * y / ny) + 0 * x, 0.02 * np.sin(2 * np.pi * x / nx) + 0 * y])
    o = run_oracle(orc, case, steps)
    g = run_gpu(L, case, steps, "f64", "dense", pattern)
    assert C.rel_l2(g["f"], o["f"]) <= 1e-12
    ref = run_gpu(L, case, steps, "f64", "sparse", pattern)
    assert np.array_equal(g["f"], ref["f"])


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f16s", 5e-3)])
def test_wall_rows_low_precision(L, orc, precision, tol):
    nx, ny = 128, 64
    fx, rho, u = inputs.poiseuille(nx, ny, 0.8, 0.05)
    case = C.Case("pois%dx%d" % (nx, ny), nx, ny, 0.8, px=True, py=False, force=(fx, 0.0))
    case.rho0, case.u0 = rho, u + 0.01 * inputs.random_field((2, ny, nx), 713)
    o = oracle_cached(orc, case, 300)
    for layout, pattern in VARIANTS:
        g = run_gpu(L, case, 300, precision, layout, pattern)
        err = C.rel_l2(g["u"], o["u"])
        assert err <= tol, (layout, pattern, err)


def _active_vector_fraction(solid):
    """2-node vectors along tile rows that hold a fluid node, over all
    vectors of the 16x16 tiles that hold one (the tiled step switches to its
    vector list below 0.67 / 0.85 of this)."""
    ny, nx = solid.shape
    pad = np.ones(((ny + 15) // 16 * 16, nx), np.uint8)
    pad[:ny] = solid
    fl = pad == 0
    tiles = fl.reshape(fl.shape[0] // 16, 16, nx // 16, 16).any(axis=(1, 3))
    return fl.reshape(fl.shape[0], nx // 2, 2).any(axis=2).sum() / (tiles.sum() * 128)


@pytest.mark.parametrize("layout,pattern", VARIANTS)
@pytest.mark.parametrize("steps", [1, 2, 33])
def test_low_porosity_vector_list_fp64_matches_oracle(L, orc, layout, pattern, steps):
    """Discs r in [4, 10] at porosity 0.3 on 256 x 200 (ragged last tile
    row): under half of the kept tiles' vectors hold fluid, so the tiled
    step runs over its vector list in every step kind."""
    case = C.discs(256, 200, 0.3, seed=inputs.GEOMETRY_SEED + 5, rmin=4.0, rmax=10.0)
    assert _active_vector_fraction(case.solid) < 0.6
    case.rho0 = 1.0 + 0.01 * inputs.random_field((case.ny, case.nx), 811)
    case.u0 = 0.02 * inputs.random_field((2, case.ny, case.nx), 812)
    o = oracle_cached(orc, case, steps)
    g = run_gpu(L, case, steps, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
def test_low_porosity_vector_list_bitwise_equals_dense(L, precision):
    case = C.discs(256, 200, 0.3, seed=inputs.GEOMETRY_SEED + 5, rmin=4.0, rmax=10.0)
    case.rho0 = 1.0 + 0.01 * inputs.random_field((case.ny, case.nx), 811)
    case.u0 = 0.02 * inputs.random_field((2, case.ny, case.nx), 812)
    ref = None
    for layout, pattern in VARIANTS:
        g = run_gpu(L, case, 9, precision, layout, pattern)
        if ref is None:
            ref = g["f"]
        else:
            assert np.array_equal(g["f"], ref), (precision, layout, pattern)


# ------------------------------------------------- the porous-medium workload

@pytest.mark.parametrize("phi", [0.2, 0.5, 0.8])
@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
def test_porous_workload_512_matches_oracle_200_steps(L, orc, phi, pattern):
    """The benchmark's porous medium at 512^2 with its own generator
    parameters (seeded non-overlapping discs r in [8, 32], force (1e-6, 0),
    periodic x, walls y, tau 0.8, from rest), tiled layout, 200 steps: FP64
    distributions within 1e-12 of the oracle, FP32 velocity within 1e-5."""
    solid, _, _ = inputs.porous_discs(512, 512, phi, rmin=8, rmax=32)
    case = C.Case("porous_workload512_%g" % phi, 512, 512, 0.8, px=True, py=False, force=(1e-6, 0.0), solid=solid)
    o = oracle_cached(orc, case, 200)
    fl = o["mask"] != 0xFF
    g = run_gpu(L, case, 200, "f64", "sparse", pattern)
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12
    g32 = run_gpu(L, case, 200, "f32", "sparse", pattern)
    assert C.rel_l2(g32["u"], o["u"], fl) <= 1e-5

"""GPU parity of the open sides (constant velocity / constant pressure, Sec. 3)
against the FP64 oracle, through the C ABI, in every layout and pattern."""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs
from tests import cases as C
from tests.test_gpu_parity import VARIANTS, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def channel(nx=48, ny=37, frac=0.15, seed=611, per_node=True, force=(1e-5, 0.0)):
    """West velocity inlet (per-node profile), east pressure outlet (per-node
    densities), moving south wall, resting north wall, random solids away from
    the open columns, uniform force, random initial state; ny ragged for the
    tiles."""
    solid = inputs.random_solid(nx, ny, frac, seed)
    solid[:, :2] = 0
    solid[:, -2:] = 0
    y = np.arange(ny)
    prof = np.stack([0.04 * (y + 0.5) * (ny - 0.5 - y) / (ny * ny / 4.0)
                     + 0.002 * inputs.random_field((ny,), seed + 1),
                     0.003 * inputs.random_field((ny,), seed + 2)])
    rho_out = 1.0 + 0.002 * inputs.random_field((ny,), seed + 3)
    c = C.Case("openchan%dx%d_s%d" % (nx, ny, seed), nx, ny, 0.7, px=False, py=False,
               walls={"south": (0.02, 0.0)}, force=force, solid=solid,
               open={"west": ("velocity", (0.03, 0.0)), "east": ("pressure", 1.001)})
    if per_node:
        c.open_vals = {"west": prof, "east": rho_out}
    c.rho0 = 1.0 + 0.01 * inputs.random_field((ny, nx), seed + 4)
    c.u0 = 0.03 * inputs.random_field((2, ny, nx), seed + 5)
    return c


def vertical(nx=32, ny=48, seed=622):
    """South velocity inlet, north pressure outlet, periodic x."""
    c = C.Case("openvert%dx%d" % (nx, ny), nx, ny, 0.8, px=True, py=False,
               open={"south": ("velocity", (0.01, 0.04)), "north": ("pressure", 0.999)})
    c.solid = inputs.random_solid(nx, ny, 0.1, seed)
    c.solid[:2] = 0
    c.solid[-2:] = 0
    c.rho0 = 1.0 + 0.01 * inputs.random_field((ny, nx), seed + 1)
    c.u0 = 0.02 * inputs.random_field((2, ny, nx), seed + 2)
    return c


def run_gpu(L, case, steps, precision="f64", layout="dense", pattern="two_lattice"):
    sim = L.LBM(precision=precision, layout=layout, pattern=pattern, **C.gpu_kwargs(case))
    for side, vals in case.open_vals.items():
        sim.set_side_values(side, vals)
    sim.init_equilibrium(case.rho0, case.u0)
    sim.step(steps)
    f = sim.get_f().double().cpu().numpy()
    rho, u = sim.macros()
    torch.cuda.synchronize()
    return dict(f=f, rho=rho.double().cpu().numpy(), u=u.double().cpu().numpy(), sim=sim)


@pytest.mark.parametrize("layout,pattern", VARIANTS)
@pytest.mark.parametrize("steps", [1, 2, 57])
def test_open_channel_fp64_matches_oracle(L, orc, layout, pattern, steps):
    case = channel()
    o = run_oracle(orc, case, steps)
    g = run_gpu(L, case, steps, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12
    assert C.rel_l2(g["u"], o["u"], fl) <= 1e-11
    assert np.abs(g["rho"][fl] - o["rho"][fl]).max() <= 1e-13


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_open_vertical_uniform_values_fp64_matches_oracle(L, orc, layout, pattern):
    case = vertical()
    o = run_oracle(orc, case, 80)
    g = run_gpu(L, case, 80, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12


def test_open_variants_bitwise_identical(L):
    case = channel()
    for precision in ("f64", "f32", "f16s"):
        ref = None
        for layout, pattern in VARIANTS:
            g = run_gpu(L, case, 9, precision, layout, pattern)
            if ref is None:
                ref = g["f"]
            else:
                assert np.array_equal(g["f"], ref), (precision, layout, pattern)


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f16s", 5e-3)])
def test_open_channel_low_precision_velocity(L, orc, precision, tol):
    case = channel(nx=96, ny=64, frac=0.1)
    o = run_oracle(orc, case, 400)
    g = run_gpu(L, case, 400, precision, "dense", "two_lattice")
    fl = o["mask"] != 0xFF
    err = C.rel_l2(g["u"], o["u"], fl)
    print(precision, "open channel rel L2 u error:", err)
    assert err <= tol, err


def test_uniform_flow_fixed_point_fp64(L):
    nx, ny, U = 64, 32, 0.05
    sim = L.LBM(nx=nx, ny=ny, tau=0.7, periodic_x=False, periodic_y=True, precision="f64",
                open={"west": ("velocity", (U, 0.0)), "east": ("pressure", 1.0)})
    u = torch.zeros((2, ny, nx), dtype=torch.float64, device="cuda")
    u[0] = U
    sim.init_equilibrium(None, u)
    f0 = sim.get_f()
    sim.step(100)
    assert (sim.get_f() - f0).abs().max().item() <= 100 * 2 * 2.2e-16 * f0.abs().max().item()


def test_velocity_side_macros_report_the_profile(L):
    case = channel(per_node=True, force=(0.0, 0.0))
    g = run_gpu(L, case, 5, "f64")
    inner = slice(1, case.ny - 1)
    prof = case.open_vals["west"]
    assert np.abs(g["u"][0][inner, 0] - prof[0][inner]).max() <= 1e-14
    assert np.abs(g["u"][1][inner, 0] - prof[1][inner]).max() <= 1e-14
    assert np.abs(g["rho"][inner, -1] - case.open_vals["east"][inner]).max() <= 1e-14


def test_side_values_need_an_open_side(L):
    sim = L.LBM(nx=32, ny=16, tau=0.8, precision="f64")
    with pytest.raises(RuntimeError):
        L.lbm_set_side_values(sim.ctx, 0, None)


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_open_y_sides_without_obstacles_fp64(L, orc, layout, pattern):
    """Velocity inlet south, pressure outlet north, periodic x, no obstacle:
    the dense layout splits the open rows from the rest."""
    c = vertical()
    c.solid = None
    c.name = "openvert_free"
    o = run_oracle(orc, c, 61)
    g = run_gpu(L, c, 61, "f64", layout, pattern)
    assert C.rel_l2(g["f"], o["f"]) <= 1e-12


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_open_sides_over_low_porosity_fp64(L, orc, layout, pattern):
    """Velocity inlet and pressure outlet across a low-porosity disc medium
    (the tiled step runs over its vector list with the open-side rule)."""
    solid, _, _ = inputs.porous_discs(256, 160, 0.35, rmin=4, rmax=10, seed=inputs.GEOMETRY_SEED + 9)
    solid[:, :2] = 0
    solid[:, -2:] = 0
    c = C.Case("openporous", 256, 160, 0.75, px=False, py=False, solid=solid,
               open={"west": ("velocity", (0.02, 0.0)), "east": ("pressure", 1.0)})
    c.rho0 = 1.0 + 0.005 * inputs.random_field((160, 256), 901)
    c.u0 = 0.01 * inputs.random_field((2, 160, 256), 902)
    o = run_oracle(orc, c, 45)
    g = run_gpu(L, c, 45, "f64", layout, pattern)
    fl = o["mask"] != 0xFF
    assert C.rel_l2(g["f"], o["f"], fl) <= 1e-12

"""Two-relaxation-time collision on the GPU (lbm_params.collision = LBM_TRT)
against the FP64 oracle's TRT step, in every layout and pattern:

  * FP64 storage: canonical distributions within 1e-12 relative L2 of the
    oracle (cavity with a moving lid, porous ragged box with moving walls and
    a force, open sides);
  * FP32 storage: velocity within 1e-5 relative L2 after 1000 steps;
  * the tiled and listed / staged steps equal the dense step bit for bit;
  * Lambda = 3/16 makes the half-way bounce-back channel exact at tau = 0.6,
    on the GPU as in the oracle;
  * the adjoint calls refuse TRT (their transpose covers BGK).
"""
import math

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
    return lbm


def run_gpu(L, case, magic, steps, precision, layout, pattern):
    sim = L.LBM(precision=precision, layout=layout, pattern=pattern, collision="trt", magic=magic,
                **C.gpu_kwargs(case))
    sim.init_equilibrium(case.rho0, case.u0)
    sim.step(steps)
    f = sim.get_f().double().cpu().numpy()
    _, u = sim.macros()
    out = f, u.double().cpu().numpy()
    sim.close()
    return out


_CACHE = {}


def run_oracle(orc, case, magic, steps):
    key = (case.name, magic, steps)
    if key not in _CACHE:
        s = C.oracle_setup(orc, case)
        s.trt_magic = magic
        mask, _ = orc.link_mask(s, case.solid)
        A = orc.run(s, mask, orc.init_equilibrium(s, mask, case.rho0, case.u0), steps)
        _, u = orc.macros(s, mask, A)
        _CACHE[key] = (A, u, mask)
    return _CACHE[key]


def open_case():
    nx, ny = 64, 40
    solid = inputs.random_solid(nx, ny, 0.1, 77)
    solid[:, :2] = 0
    solid[:, -2:] = 0
    c = C.Case("trt_open", nx, ny, 0.7, px=False, py=False, walls={"north": (0.01, 0.0)}, solid=solid,
               open={"west": ("velocity", (0.03, 0.0)), "east": ("pressure", 1.0)})
    c.rho0 = 1.0 + 0.005 * inputs.random_field((ny, nx), 78)
    c.u0 = 0.02 * inputs.random_field((2, ny, nx), 79)
    return c


CASES = {
    "cavity": (lambda: C.cavity(128), 3.0 / 16.0, 200),
    "porous_ragged": (lambda: C.porous(48, 37, 0.25, seed=101), 0.1, 101),
    "open_sides": (open_case, 0.25, 60),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_trt_fp64_matches_oracle(L, orc, name, layout, pattern):
    make, magic, steps = CASES[name]
    case = make()
    A, u_ref, mask = run_oracle(orc, case, magic, steps)
    f, u = run_gpu(L, case, magic, steps, "f64", layout, pattern)
    fl = mask != 0xFF
    assert C.rel_l2(f, A, fl) <= 1e-12
    assert C.rel_l2(u, u_ref, fl) <= 1e-10


@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_trt_fp32_cavity_velocity_within_1e5(L, orc, layout, pattern):
    case = C.cavity(128)
    _, u_ref, mask = run_oracle(orc, case, 3.0 / 16.0, 1000)
    _, u = run_gpu(L, case, 3.0 / 16.0, 1000, "f32", layout, pattern)
    fl = mask != 0xFF
    assert C.rel_l2(u, u_ref, fl) <= 1e-5


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
def test_trt_layouts_bitwise_identical(L, precision):
    """Porous discs at porosity 0.35 (FP32 takes the staged tiled step, FP64
    and FP16s the listed one) and at 0.85 (FP16s staged): every layout and
    pattern equals the dense two-lattice run bit for bit."""
    for phi in (0.35, 0.85):
        solid, _, _ = inputs.porous_discs(192, 144, phi, rmin=4.0, rmax=9.0, seed=905)
        case = C.Case("trt_discs", 192, 144, 0.7, px=True, py=False, walls={"south": (0.02, 0.0)},
                      force=(1e-5, -2e-6), solid=solid)
        case.rho0 = 1.0 + 0.01 * inputs.random_field((144, 192), 906)
        case.u0 = 0.02 * inputs.random_field((2, 144, 192), 907)
        ref = None
        for layout, pattern in VARIANTS:
            f, _ = run_gpu(L, case, 0.2, 9, precision, layout, pattern)
            if ref is None:
                ref = f
            else:
                assert np.array_equal(f[:, solid == 0], ref[:, solid == 0]), (phi, layout, pattern)


def test_trt_magic_3_16_channel_exact_on_gpu(L):
    """Channel of 32 rows, walls half a spacing outside the first and last,
    Guo force, tau = 0.6 (where BGK is not exact): with Lambda = 3/16 the
    steady FP64 profile is the parabola F/(2 nu) (y + 1/2)(ny - 1/2 - y)."""
    nx, ny, tau = 16, 32, 0.6
    fx, rho, u = inputs.poiseuille(nx, ny, tau, 0.01)
    sim = L.LBM(nx, ny, tau, force=(fx, 0.0), periodic_y=False, precision="f64", collision="trt",
                magic=3.0 / 16.0)
    sim.init_equilibrium(rho, u)
    sim.step(int(4 * ny * ny / ((tau - 0.5) / 3)))
    _, uu = sim.macros()
    prof = uu[0].double().cpu().numpy()[:, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    exact = fx / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(prof - exact).max() <= 1e-8 * exact.max()


def test_trt_equal_rates_is_bgk(L):
    """Lambda = (tau - 1/2)^2 (odd rate = even rate) runs BGK up to rounding."""
    case = C.porous(48, 37, 0.25, seed=101)
    tau = case.tau
    ft, _ = run_gpu(L, case, (tau - 0.5) ** 2, 40, "f64", "dense", "two_lattice")
    sim = L.LBM(precision="f64", **C.gpu_kwargs(case))
    sim.init_equilibrium(case.rho0, case.u0)
    sim.step(40)
    fb = sim.get_f().cpu().numpy()
    fl = case.solid == 0
    assert np.abs(ft[:, fl] - fb[:, fl]).max() < 1e-14


def test_adjoint_refuses_trt(L):
    sim = L.LBM(32, 16, 0.8, precision="f64", collision="trt", magic=3.0 / 16.0)
    lam = torch.zeros((9, 16, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LBMError) as e:
        sim.macros_backward(None, torch.zeros((2, 16, 32), dtype=torch.float64, device="cuda"), lam, None)
    assert e.value.status == L.LBM_ERR_UNSUPPORTED

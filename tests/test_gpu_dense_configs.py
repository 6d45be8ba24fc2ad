"""GPU parity on the dense throughput configurations as configured, and on
the paper's sparse benchmark geometries.

Dense (the benchmark's Taylor-Green and body-force Poiseuille boxes at
1024^2, tau 0.8, peak velocity 0.05, 1000 steps; Algorithm 1 with the moments
of Eq. 2, the equilibrium of Eq. 6, BGK of Eq. 3-4 and, for Poiseuille, the
Guo force with half-way walls):
  * FP64 storage, dense and tiled, two-lattice and AA: canonical
    distributions within 1e-12 relative L2 of the FP64 oracle;
  * FP32 storage, every variant: velocity within 1e-5 relative L2 of the
    oracle.

Sparse geometries of Sec. 4.2.2 (a 512^2 crop of the 4096^2 geometry, periodic
x, walls y, F = (1e-6, 0), tau 0.8, from rest, 100 steps): the random discs
with r in [8, 256] and the regular 8 x 8 disc array, tiled layout and dense
layout with the per-node link mask: FP64 within 1e-12 of the oracle, FP32
velocity within 1e-5.
"""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs
from tests import cases as C

pytestmark = pytest.mark.gpu

VARIANTS = [("dense", "two_lattice"), ("dense", "aa"), ("sparse", "two_lattice"), ("sparse", "aa")]
N, STEPS, TAU, U = 1024, 1000, 0.8, 0.05


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def tgv_case():
    c = C.Case("tgv%d" % N, N, N, TAU)
    c.rho0, c.u0 = inputs.taylor_green(N, N, U)
    return c


def poiseuille_case():
    fx, rho, u = inputs.poiseuille(N, N, TAU, U)
    c = C.Case("poiseuille%d" % N, N, N, TAU, px=True, py=False, force=(fx, 0.0))
    c.rho0, c.u0 = rho, u
    return c


def sparse_crop(kind):
    """512^2 crop (rows and columns 0..511) of the 4096^2 geometry."""
    if kind == "random_r8_256":
        solid, phi, _ = inputs.porous_discs(4096, 4096, 0.3, rmin=8, rmax=256)
    else:
        solid, phi, _ = inputs.circle_array(4096, 4096, 0.4, 8)
    crop = np.ascontiguousarray(solid[:512, :512])
    assert 0 < crop.sum() < crop.size
    return C.Case("crop512_" + kind, 512, 512, TAU, px=True, py=False, force=(1e-6, 0.0), solid=crop)


_CACHE = {}


def oracle(orc, case, steps):
    key = (case.name, steps)
    if key not in _CACHE:
        s = C.oracle_setup(orc, case)
        mask, _ = orc.link_mask(s, case.solid)
        A = orc.init_equilibrium(s, mask, case.rho0, case.u0)
        A = orc.run(s, mask, A, steps)
        _, u = orc.macros(s, mask, A)
        _CACHE[key] = (A, u, mask)
    return _CACHE[key]


def gpu(L, case, steps, precision, layout, pattern):
    sim = L.LBM(precision=precision, layout=layout, pattern=pattern, **C.gpu_kwargs(case))
    sim.init_equilibrium(case.rho0, case.u0)
    sim.step(steps)
    _, u = sim.macros()
    f = sim.get_f().double().cpu().numpy() if precision == "f64" else None
    u = u.double().cpu().numpy()
    sim.close()
    return f, u


W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None]


@pytest.mark.parametrize("make", [tgv_case, poiseuille_case], ids=["taylor_green", "poiseuille"])
@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_dense_config_fp64_1000_steps_matches_oracle(L, orc, make, layout, pattern):
    case = make()
    A, u_ref, mask = oracle(orc, case, STEPS)
    f, u = gpu(L, case, STEPS, "f64", layout, pattern)
    fl = mask != 0xFF
    err = C.rel_l2(f, A, fl)
    dev = C.rel_l2(f[:, fl] - W, A[:, fl] - W)
    print("%s %s/%s FP64: rel L2 f %.3e, of f - w %.3e" % (case.name, layout, pattern, err, dev))
    assert err <= 1e-12, err
    assert dev <= 1e-10, dev
    assert C.rel_l2(u, u_ref, fl) <= 1e-10


@pytest.mark.parametrize("make", [tgv_case, poiseuille_case], ids=["taylor_green", "poiseuille"])
@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_dense_config_fp32_1000_steps_velocity_within_1e5(L, orc, make, layout, pattern):
    case = make()
    _, u_ref, mask = oracle(orc, case, STEPS)
    _, u = gpu(L, case, STEPS, "f32", layout, pattern)
    fl = mask != 0xFF
    err = C.rel_l2(u, u_ref, fl)
    print("%s %s/%s FP32: rel L2 u %.3e" % (case.name, layout, pattern, err))
    assert err <= 1e-5, err


@pytest.mark.parametrize("kind", ["random_r8_256", "array_8x8"])
@pytest.mark.parametrize("layout,pattern", VARIANTS)
def test_sparse_benchmark_geometry_crop_matches_oracle(L, orc, kind, layout, pattern):
    case = _CACHE.get(("geom", kind))
    if case is None:
        case = _CACHE[("geom", kind)] = sparse_crop(kind)
    A, u_ref, mask = oracle(orc, case, 100)
    fl = mask != 0xFF
    f, _ = gpu(L, case, 100, "f64", layout, pattern)
    assert C.rel_l2(f, A, fl) <= 1e-12
    _, u32 = gpu(L, case, 100, "f32", layout, pattern)
    assert C.rel_l2(u32, u_ref, fl) <= 1e-5

"""Field arguments in pinned host memory: lbm_init_equilibrium reads them and
lbm_macros writes them directly through the device's mapping of pinned host
memory (no staging copy).  The results must equal the device-buffer path bit
for bit, in FP64 and FP32, dense and tiled."""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs
from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    return lbm


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("layout", ["dense", "sparse"])
def test_pinned_host_fields_equal_device_fields(L, precision, layout):
    case = C.porous(64, 48, 0.2, seed=515)
    dt = torch.float64 if precision == "f64" else torch.float32
    rho_h = torch.as_tensor(case.rho0, dtype=dt).pin_memory()
    u_h = torch.as_tensor(case.u0, dtype=dt).pin_memory()
    out = []
    for host in (True, False):
        sim = L.LBM(precision=precision, layout=layout, **C.gpu_kwargs(case))
        if host:
            L.lbm_init_equilibrium(sim.ctx, rho_h, u_h)
        else:
            sim.init_equilibrium(rho_h.cuda(), u_h.cuda())
        sim.step(11)
        if host:
            r = torch.empty((case.ny, case.nx), dtype=dt).pin_memory()
            u = torch.empty((2, case.ny, case.nx), dtype=dt).pin_memory()
            L.lbm_macros(sim.ctx, r, u)
            torch.cuda.synchronize()
        else:
            r, u = sim.macros()
        out.append((sim.get_f().cpu(), r.cpu(), u.cpu()))
        sim.close()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


def test_pageable_host_fields_are_refused(L):
    sim = L.LBM(32, 16, 0.8, precision="f32")
    with pytest.raises(ValueError):
        L.lbm_init_equilibrium(sim.ctx, torch.ones((16, 32)), None)

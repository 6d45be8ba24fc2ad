"""lbm_reduce_f_noalloc: the reduction for callers that cannot allocate device
memory when they need it (stream capture, host-owned buffers).  It is checked
through the C ABI against the context-based lbm_reduce on the same states, on
two calls in a row (the shared static scratch must not carry anything over).
Kept in a file collected last so that a stop-at-first-failure run has already
run every other test."""
import numpy as np
import pytest
import torch

from tests import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    return lbm


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_noalloc_reduce_matches_lbm_reduce_on_two_calls(L, precision, tol):
    case = C.porous(80, 53, 0.3, seed=777)
    sim = L.LBM(precision=precision, **C.gpu_kwargs(case))
    sim.init_equilibrium(case.rho0, case.u0)
    mask = torch.as_tensor(sim.link_mask(), device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(7 + call)
        mass, mom = sim.reduce()
        f = sim.get_f()
        L.lbm_reduce_f_noalloc(precision, f, mask, case.nx, case.ny, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) <= tol * abs(mass), (call, got[0], mass)
        assert abs(got[1] - mom[0]) <= tol * abs(mass), (call, got[1], mom[0])
        assert abs(got[2] - mom[1]) <= tol * abs(mass), (call, got[2], mom[1])
        out.fill_(float("nan"))


def test_noalloc_rejects_rows_beyond_its_scratch(L):
    f = torch.zeros(9 * 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f, None, 1, L.NOALLOC_MAX_ROWS + 1, out)
    # the C entry point itself refuses too (no device work is issued)
    st = L._load().lbm_reduce_f_noalloc(L.LBM_F64, f.data_ptr(), None, 1, L.NOALLOC_MAX_ROWS + 1,
                                        out.data_ptr(), None)
    assert st == L.LBM_ERR_INVALID

"""lbm_reduce_f_noalloc: the reduction for callers that cannot allocate device
memory when they need it (stream capture, host-owned buffers).  It is checked
through the C ABI on two calls in a row (the shared static scratch must not
carry anything over) against
  * the oracle's mass and momentum (plain numpy sums over fluid nodes) of the
    very array it was given, and of the oracle's own FP64 run of the case;
  * the context-based lbm_reduce on the same state.
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


# FP16s exports FP32 values, so its sums are as exact as FP32's; the physics
# tolerance against the oracle's FP64 run is the precision's own error
@pytest.mark.parametrize("precision,phys_tol", [("f64", 1e-12), ("f32", 1e-5), ("f16s", 1e-3)])
def test_noalloc_reduce_matches_oracle_and_lbm_reduce_on_two_calls(L, orc, precision, phys_tol):
    case = C.porous(80, 53, 0.3, seed=777)
    s = C.oracle_setup(orc, case)
    omask, _ = orc.link_mask(s, case.solid)
    A = orc.init_equilibrium(s, omask, case.rho0, case.u0)
    sim = L.LBM(precision=precision, **C.gpu_kwargs(case))
    sim.init_equilibrium(case.rho0, case.u0)
    mask = torch.as_tensor(sim.link_mask(), device="cuda")
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    done = 0
    for call in range(2):
        n = 7 + call
        sim.step(n)
        A = orc.run(s, omask, A, n)
        done += n
        f = sim.get_f()
        L.lbm_reduce_f_noalloc(precision, f, mask, case.nx, case.ny, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        fh = f.double().cpu().numpy()
        # the sums of the array it was given, in FP64 (each node's 9 values
        # are summed in FP64 on both sides; only the order differs)
        m_ref = orc.mass(fh, omask)
        px, py = orc.momentum(fh, omask)
        assert abs(got[0] - m_ref) <= 1e-12 * abs(m_ref), (call, got[0], m_ref)
        assert abs(got[1] - px) <= 1e-12 * abs(m_ref), (call, got[1], px)
        assert abs(got[2] - py) <= 1e-12 * abs(m_ref), (call, got[2], py)
        # the oracle's own FP64 run of the same steps
        mo = orc.mass(A, omask)
        ox, oy = orc.momentum(A, omask)
        assert abs(got[0] - mo) <= phys_tol * abs(mo), (call, got[0], mo)
        assert abs(got[1] - ox) <= phys_tol * abs(mo) and abs(got[2] - oy) <= phys_tol * abs(mo)
        # the context's reduction of the same state
        mass, mom = sim.reduce()
        assert abs(got[0] - mass) <= 1e-5 * abs(mass) and abs(got[1] - mom[0]) <= 1e-5 * abs(mass)
        out.fill_(float("nan"))
    assert done == 15


def test_noalloc_without_mask_on_a_side_stream(L, orc):
    """Fully periodic all-fluid box (mask NULL: every node counts), called
    twice on a stream other than the current one."""
    nx, ny = 64, 48
    from paper_2108_13241_gb300 import inputs
    rho, u = inputs.taylor_green(nx, ny, 0.05)
    side = torch.cuda.Stream()
    sim = L.LBM(nx, ny, 0.8, precision="f64")
    sim.init_equilibrium(rho, u)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(5)
        f = sim.get_f()
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            L.lbm_reduce_f_noalloc("f64", f, None, nx, ny, out, stream=side.cuda_stream)
        side.synchronize()
        fh = f.cpu().numpy()
        allm = np.zeros((ny, nx), np.uint8)
        m_ref = orc.mass(fh, allm)
        px, py = orc.momentum(fh, allm)
        got = out.cpu().numpy()
        assert abs(got[0] - m_ref) <= 1e-12 * m_ref, (call, got[0], m_ref)
        assert abs(got[1] - px) <= 1e-12 * m_ref and abs(got[2] - py) <= 1e-12 * m_ref, (call, got, px, py)
        out.fill_(float("nan"))


def test_noalloc_rejects_bad_arguments(L):
    f = torch.zeros(9 * 16, dtype=torch.float64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f, None, 1, L.NOALLOC_MAX_ROWS + 1, out)
    # the C entry point itself refuses too (no device work is issued)
    st = L._load().lbm_reduce_f_noalloc(L.LBM_F64, f.data_ptr(), None, 1, L.NOALLOC_MAX_ROWS + 1,
                                        out.data_ptr(), None)
    assert st == L.LBM_ERR_INVALID
    # the binding checks dtype, sizes and placement before any device work
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f32", f, None, 4, 4, out)          # float64 given for f32
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f, None, 4, 5, out)          # 9*4*5 > 144 values
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f, torch.zeros(3, dtype=torch.uint8, device="cuda"), 4, 4, out)
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f, None, 4, 4, torch.zeros(3, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        L.lbm_reduce_f_noalloc("f64", f.cpu(), None, 4, 4, out)

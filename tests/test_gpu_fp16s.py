"""FP16-shifted storage: properties of its rounding that hold at any size.

The time step stores (f_i - w_i) * 2^10 in binary16 with stochastic rounding
(13 random bits added below the kept mantissa before truncation, two values
per conversion instruction), so the
storage error has zero mean, and the collision's odd part carries its
constant as a float pair: a uniform flow, a fixed point of the update, keeps
the mean momentum of its initial state up to zero-mean noise.  The rounding
is also deterministic: the same run gives the same bits.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    return lbm


def _uniform(L, n, u0, pattern):
    sim = L.LBM(n, n, 0.8, precision="f16s", pattern=pattern)
    u = torch.zeros((2, n, n), dtype=torch.float32, device="cuda")
    u[0], u[1] = u0
    sim.init_equilibrium(None, u)
    return sim


@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
def test_uniform_flow_mean_momentum_is_unbiased(L, pattern):
    """The initial state is rounded to nearest, identically at every node, so
    its momentum is off u0 by up to binary16's step; the time steps must then
    leave that momentum alone up to the zero-mean noise of their rounding
    (a rounded constant or a biased rounding would move it by ~1e-7 of |u|
    per step, ~1e-4 over the run)."""
    n, u0 = 512, (0.0123, -0.0071)
    sim = _uniform(L, n, u0, pattern)
    _, u = sim.macros()
    start = u.double().mean(dim=(1, 2)).cpu().numpy()
    means = []
    for _ in range(40):
        sim.step(25)
        _, u = sim.macros()
        means.append(u.double().mean(dim=(1, 2)).cpu().numpy())
    m = np.mean(means, axis=0)
    rel = np.abs(m - start) / np.linalg.norm(u0)
    assert rel.max() <= 3e-5, rel


def test_stochastic_rounding_is_deterministic(L):
    n = 128
    out = []
    for _ in range(2):
        sim = _uniform(L, n, (0.02, 0.01), "two_lattice")
        sim.step(17)
        out.append(sim.get_f())
        del sim
    assert torch.equal(out[0], out[1])

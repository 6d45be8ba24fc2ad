"""Parity at the benchmark's full size and launch configuration.

Dense periodic Taylor-Green 4096^2 (tau 0.8, U 0.05) -- the workload
bench.py times -- in FP32 (two-lattice and AA) and FP16s: the GPU state after
k steps is exported, the FP64 oracle takes one step from exactly that state
on the whole grid, and the GPU's own next step must match it to the rounding
of one step in the storage precision.  Mass is conserved to FP64 round-off
over the run (a property that holds at any size).
"""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs

pytestmark = pytest.mark.gpu

N = 4096


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    return lbm


@pytest.fixture(scope="module")
def tgv():
    rho, u = inputs.taylor_green(N, N, 0.05)
    return rho, u


@pytest.mark.parametrize("precision,pattern,tol", [("f32", "two_lattice", 1e-5), ("f32", "aa", 1e-5),
                                                   ("f16s", "two_lattice", 2e-3)])
def test_one_step_from_gpu_state_matches_oracle_full_size(L, orc, tgv, precision, pattern, tol):
    rho, u = tgv
    sim = L.LBM(N, N, 0.8, precision=precision, pattern=pattern)
    sim.init_equilibrium(rho, u)
    sim.step(7)
    m0, _ = sim.reduce()
    A = sim.get_f().double().cpu().numpy()
    sim.step(1)
    B = sim.get_f().double().cpu().numpy()
    s = orc.Setup(nx=N, ny=N, tau=0.8)
    mask, _ = orc.link_mask(s)
    ref = orc.step(s, mask, A)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    # error relative to the deviation from rest (what the storage holds); the
    # canonical export w_i + stored value rounds once more in FP32
    err = np.linalg.norm(B - ref) / np.linalg.norm(ref - w)
    assert err <= tol, err
    sim.step(100)
    m1, _ = sim.reduce()
    # FP32 storage keeps mass to ~1e-9 relative over 100 steps; binary16
    # storage rounds each of the 9 stored values independently (half an ulp
    # of f_i - w_i, ~4e-6), so mass performs a small random walk
    assert abs(m1 - m0) <= (1e-9 if precision == "f32" else 1e-5) * m0


def test_full_size_aa_equals_two_lattice_fp32(L, tgv):
    rho, u = tgv
    out = []
    for pattern in ("two_lattice", "aa"):
        sim = L.LBM(N, N, 0.8, precision="f32", pattern=pattern)
        sim.init_equilibrium(rho, u)
        sim.step(11)
        out.append(sim.get_f())
        del sim
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("phi", [0.2, 0.8])
@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
def test_porous_full_size_one_step_matches_oracle(L, orc, phi, pattern):
    """The 4096^2 porous medium (discs r in [8, 32], force 1e-6, periodic x,
    walls y) in the tiled FP32 layout, as bench.py times it: one GPU step from
    the GPU's own state against one oracle step from the same state, every
    fluid node."""
    solid, _, _ = inputs.porous_discs(N, N, phi, rmin=8, rmax=32)
    sim = L.LBM(N, N, 0.8, solid=solid, force=(1e-6, 0.0), periodic_y=False, precision="f32",
                layout="sparse", pattern=pattern)
    # deviations from rest of order 1e-2, so that the FP32 export w_i + (f_i -
    # w_i) rounds far below the tolerance (as in the Taylor-Green case)
    rho, u = inputs.taylor_green(N, N, 0.05)
    sim.init_equilibrium(rho, u)
    sim.step(5)
    A = sim.get_f().double().cpu().numpy()
    sim.step(1)
    B = sim.get_f().double().cpu().numpy()
    s = orc.Setup(nx=N, ny=N, tau=0.8, periodic_x=True, periodic_y=False, force=(1e-6, 0.0))
    mask, nf = orc.link_mask(s, solid)
    assert nf == sim.fluid_nodes
    ref = orc.step(s, mask, A)
    fl = mask != 0xFF
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None]
    err = np.linalg.norm(B[:, fl] - ref[:, fl]) / np.linalg.norm(ref[:, fl] - w)
    assert err <= 1e-5, err


def test_maximum_size_sampled_nodes_match_oracle(L, orc):
    """The largest grid the 32-bit element indices allow (9 nx ny < 2^32:
    21760 x 21920, 477M nodes, 34 GB of FP32 lattices), periodic, smooth
    seeded field: one GPU step against the oracle at sampled nodes, each
    recomputed by the oracle on a 3 x 3 periodic patch cut from the GPU's
    state around it (the node's update depends on nothing else), and mass
    conserved over the step."""
    nx, ny = 21760, 21920
    assert 9 * nx * ny < 2 ** 32 <= 9 * nx * (ny + 16)
    sim = L.LBM(nx, ny, 0.8, precision="f32")
    y = torch.arange(ny, dtype=torch.float32, device="cuda")[:, None]
    x = torch.arange(nx, dtype=torch.float32, device="cuda")[None, :]
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    u = torch.stack([-0.05 * torch.cos(kx * x) * torch.sin(ky * y), 0.05 * torch.sin(kx * x) * torch.cos(ky * y)])
    rho = 1.0 + 0.01 * torch.cos(kx * x) * torch.cos(ky * y)
    sim.init_equilibrium(rho, u)
    del u, rho
    m0, _ = sim.reduce()
    A = sim.get_f()
    sim.step(1)
    m1, _ = sim.reduce()
    B = sim.get_f()
    assert abs(m1 - m0) <= 1e-9 * m0
    rng = inputs.SplitMix64(inputs.FD_SEED)
    pts = [(0, 0), (ny - 1, nx - 1), (ny // 2, nx // 3)]
    pts += [(int(rng.next_u64() % ny), int(rng.next_u64() % nx)) for _ in range(29)]
    s = orc.Setup(nx=3, ny=3, tau=0.8)
    mask, _ = orc.link_mask(s)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    for (py, px) in pts:
        ys = torch.tensor([(py - 1) % ny, py, (py + 1) % ny], device="cuda")
        xs = torch.tensor([(px - 1) % nx, px, (px + 1) % nx], device="cuda")
        patch = A[:, ys][:, :, xs].double().cpu().numpy()
        ref = orc.step(s, mask, patch)[:, 1, 1]
        got = B[:, py, px].double().cpu().numpy()
        err = np.abs(got - ref).max() / np.abs(ref - w).max()
        assert err <= 1e-5, ((py, px), err)
    del A, B
    sim.close()
    torch.cuda.empty_cache()

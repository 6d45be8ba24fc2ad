"""CUDA-graph replay of lbm_step, lbm_forward_states and lbm_backward.

A graph replays the same kernels with the same arguments as the direct
launches (the FP16s steps read their time-step index from a device counter),
so every result must be bitwise equal to the same run with graphs off: over
both patterns, all three precisions, dense, tiled and listed layouts, walls,
obstacles, force fields, open sides and the split wall-row launch; across a
change of the force after a graph was recorded; and through the adjoint's
recompute and backward sweep.
"""
import pytest
import torch

from paper_2108_13241_gb300 import inputs
from tests import cases as C

pytestmark = pytest.mark.gpu

STEPS = 70  # two 32-step replays and six direct steps


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import autograd, lbm
    return lbm, autograd


def _run(lbm, graphs, kw, precision, pattern, layout, steps, field=None, rho_u=None):
    sim = lbm.LBM(precision=precision, pattern=pattern, layout=layout, **kw)
    sim.set_graphs(graphs)
    if field is not None:
        sim.set_force(torch.as_tensor(field, dtype=sim.dtype, device="cuda"))
    rho, u = rho_u if rho_u is not None else (None, None)
    sim.init_equilibrium(rho, u)
    for n in steps:
        sim.step(n)
    f = sim.get_f()
    count = sim.steps
    sim.close()
    return f, count


def _configs():
    n = 96
    tg = inputs.taylor_green(n, n, 0.05)
    por = C.porous(n, 64, 0.3, 11, field=True)
    disc = C.discs(128, 128, 0.3)
    return {
        "tgv_periodic": (dict(nx=n, ny=n, tau=0.8), None, tg),
        "cavity": (C.gpu_kwargs(C.cavity(64)), None, None),
        "porous_walls_field": (C.gpu_kwargs(por), por.force_field, (por.rho0, por.u0)),
        "discs_list": (C.gpu_kwargs(disc), None, None),
        "open_channel": (dict(nx=96, ny=32, tau=0.8, periodic_x=False, periodic_y=False,
                              open={"west": ("velocity", (0.04, 0.0)), "east": ("pressure", 1.0)}), None, None),
    }


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("pattern", ["two_lattice", "aa"])
@pytest.mark.parametrize("layout", ["dense", "sparse"])
def test_graph_replay_is_bitwise_equal_to_direct_launches(L, precision, pattern, layout):
    lbm, _ = L
    for name, (kw, field, rho_u) in _configs().items():
        if name == "open_channel" and layout == "sparse":
            continue
        # 33 leaves the other lattice parity, whose graph the 45 records
        a, na = _run(lbm, True, kw, precision, pattern, layout, [STEPS, 33, 45], field, rho_u)
        b, nb = _run(lbm, False, kw, precision, pattern, layout, [STEPS, 33, 45], field, rho_u)
        assert na == nb == STEPS + 33 + 45
        assert torch.equal(a, b), name


def test_graph_replay_split_wall_rows(L):
    """A dense grid above 2^21 nodes with walls only in y runs two launches
    per step (masked wall rows, unmasked interior); both go into the graph."""
    lbm, _ = L
    kw = dict(nx=2048, ny=1040, tau=0.8, periodic_y=False, force=(1e-6, 0.0),
              walls={"north": (0.02, 0.0)})
    out = []
    for graphs in (True, False):
        sim = lbm.LBM(precision="f32", **kw)
        sim.set_graphs(graphs)
        assert sim.launches_per_step == 2
        sim.init_equilibrium(None, None)
        sim.step(64)
        out.append(sim.get_f())
        sim.close()
    assert torch.equal(out[0], out[1])


def test_graph_rerecorded_after_force_change(L):
    lbm, _ = L
    c = C.porous(64, 48, 0.2, 5, field=True)
    out = []
    for graphs in (True, False):
        sim = lbm.LBM(precision="f32", **C.gpu_kwargs(c))
        sim.set_graphs(graphs)
        sim.set_force(torch.as_tensor(c.force_field, dtype=sim.dtype, device="cuda"))
        sim.init_equilibrium(torch.as_tensor(c.rho0, dtype=sim.dtype, device="cuda"),
                             torch.as_tensor(c.u0, dtype=sim.dtype, device="cuda"))
        sim.step(64)
        # a new force tensor (another pointer), then the uniform force only
        sim.set_force(torch.as_tensor(-2 * c.force_field, dtype=sim.dtype, device="cuda"))
        sim.step(64)
        sim.set_force(None)
        sim.step(64)
        out.append(sim.get_f())
        sim.close()
    assert torch.equal(out[0], out[1])


def test_step_launch_count(L):
    lbm, _ = L
    sim = lbm.LBM(96, 96, 0.8)
    assert sim.step_launches(70) == 70 + 1 + 2
    assert sim.step_launches(31) == 31
    sim.set_graphs(False)
    assert sim.step_launches(70) == 70
    sim.close()


def test_adjoint_graphs_bitwise_equal_to_direct(L):
    """Recompute (lbm_forward_states) and backward sweep (lbm_backward) as
    replayed graphs: segments of 12 steps over T = 40 (three full segments
    replay one recording, the last, shorter one records its own)."""
    lbm, ag = L
    nx, ny = 64, 48
    solid, _ = inputs.channel_cylinders(nx, ny, count=3, rmin=3, rmax=5, clearance=2, seed=inputs.GEOMETRY_SEED)
    F0 = 1e-4 * inputs.random_field((2, ny, nx), 7)
    ut = 0.01 * inputs.random_field((2, ny, nx), 8)
    grads = []
    for graphs in (True, False):
        sim = lbm.LBM(nx, ny, 0.8, solid=solid, periodic_y=False, walls={"north": (0.01, 0.0)}, precision="f32")
        sim.set_graphs(graphs)
        F = torch.as_tensor(F0, dtype=sim.dtype, device="cuda").requires_grad_(True)
        rho, u = ag.simulate(sim, 40, None, F, K=12)
        loss = ((u - torch.as_tensor(ut, dtype=sim.dtype, device="cuda")) ** 2).sum()
        loss.backward()
        grads.append((float(loss), F.grad.clone()))
        sim.close()
    assert grads[0][0] == grads[1][0]
    assert torch.equal(grads[0][1], grads[1][1])
    assert torch.isfinite(grads[0][1]).all() and grads[0][1].abs().max() > 0

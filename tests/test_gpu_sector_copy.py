"""lbm_sector_copy, the measurement aid that moves a step's DRAM sectors
without the step's arithmetic: it copies exactly the 32-byte sectors that
hold a fluid node, in all nine slots, from the current lattice into the
other one, leaves the state A_t untouched, and reports 2 * 9 * 32 bytes per
such sector.  White-box: the test reads the two lattices out of the caller's
workspace, where lbm_create places them (lattice 0 at offset 0, lattice 1 at
the next 256-byte boundary after it; dense f[i][y][x], tiled
f[tile][i][256])."""
import numpy as np
import pytest
import torch

from paper_2108_13241_gb300 import inputs

pytestmark = pytest.mark.gpu

ES = {"f64": 8, "f32": 4, "f16s": 2}


@pytest.fixture(scope="module")
def L():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm
    return lbm


def slot_mask(sim, layout):
    """Link mask in the lattice's slot order: canonical [ny][nx] (dense) or
    [tile][16][16] (tiled, 0xFF outside the grid)."""
    m = sim.link_mask()
    if layout == "dense":
        return m.reshape(-1)
    tid, nbr = sim.tile_map()
    out = np.full((nbr.shape[0], 16, 16), 0xFF, np.uint8)
    pad = np.full((tid.shape[0] * 16, tid.shape[1] * 16), 0xFF, np.uint8)
    pad[: m.shape[0], : m.shape[1]] = m
    for ty in range(tid.shape[0]):
        for tx in range(tid.shape[1]):
            if tid[ty, tx] >= 0:
                out[tid[ty, tx]] = pad[16 * ty: 16 * ty + 16, 16 * tx: 16 * tx + 16]
    return out.reshape(-1)


@pytest.mark.parametrize("precision", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("layout", ["dense", "sparse"])
def test_sector_copy_moves_exactly_the_fluid_sectors(L, precision, layout):
    nx, ny = 192, 80
    solid, _, _ = inputs.porous_discs(nx, ny, 0.4, rmin=4.0, rmax=9.0, seed=77)
    sim = L.LBM(nx, ny, 0.8, solid=solid, force=(1e-5, 0.0), periodic_y=False, precision=precision,
                layout=layout, pattern="two_lattice")
    sim.init_equilibrium(None, None)
    sim.step(4)  # even: lattice 0 holds A_t
    torch.cuda.synchronize()
    es = ES[precision]
    m = slot_mask(sim, layout)
    nslot = m.size
    lat = 9 * nslot * es
    off1 = (lat + 255) // 256 * 256
    ws = sim.workspace
    ws[off1: off1 + lat].fill_(0xAB)
    f_before = sim.get_f().cpu().numpy()
    nbytes = sim.sector_copy(3)
    torch.cuda.synchronize()
    e = 32 // es
    # lattice blocks: the whole slot (dense f[i][y][x]) or one tile
    # (tiled f[tile][i][256]); sectors of e nodes within a block's slot
    nblk = 1 if layout == "dense" else nslot // 256
    fluid_sec = (m.reshape(nblk, -1, e) != 0xFF).any(axis=2)  # [block][sector]
    assert nbytes == 2 * 9 * 32 * int(fluid_sec.sum())
    a = ws[:lat].cpu().numpy().reshape(nblk, 9, -1, 32)
    b = ws[off1: off1 + lat].cpu().numpy().reshape(nblk, 9, -1, 32)
    sel = np.broadcast_to(fluid_sec[:, None, :], a.shape[:3])
    assert np.array_equal(b[sel], a[sel])
    assert (b[~sel] == 0xAB).all()
    # the state is untouched and the next step overwrites the copy
    assert np.array_equal(sim.get_f().cpu().numpy(), f_before)
    ref = L.LBM(nx, ny, 0.8, solid=solid, force=(1e-5, 0.0), periodic_y=False, precision=precision,
                layout=layout, pattern="two_lattice")
    ref.init_equilibrium(None, None)
    ref.step(4)
    sim.step(3)
    ref.step(3)
    fl = solid == 0
    assert np.array_equal(sim.get_f().cpu().numpy()[:, fl], ref.get_f().cpu().numpy()[:, fl])
    sim.close()
    ref.close()


def test_sector_copy_all_fluid_box_copies_every_sector(L):
    sim = L.LBM(64, 32, 0.8, precision="f32", layout="dense", pattern="two_lattice")
    assert sim.sector_copy(1) == 2 * 9 * 64 * 32 * 4
    sim.close()


def test_sector_copy_refuses_aa_and_negative_counts(L):
    sim = L.LBM(64, 32, 0.8, precision="f32", layout="dense", pattern="aa")
    with pytest.raises(L.LBMError) as ei:
        sim.sector_copy(1)
    assert ei.value.status == L.LBM_ERR_UNSUPPORTED
    sim.close()
    sim = L.LBM(64, 32, 0.8, precision="f32", layout="dense", pattern="two_lattice")
    with pytest.raises(L.LBMError) as ei:
        sim.sector_copy(-1)
    assert ei.value.status == L.LBM_ERR_INVALID
    sim.close()

"""Host-side checks of the CUDA library that need no GPU: the shared library
builds, loads and exports every function include/lbm.h declares; parameter
validation; the host-built link mask and tile tables match the oracle bit for
bit."""
import numpy as np
import pytest

from paper_2108_13241_gb300 import inputs
from tests.cases import SIDES


@pytest.fixture(scope="module")
def lbm():
    from paper_2108_13241_gb300 import build
    build.build()
    from paper_2108_13241_gb300 import lbm as L
    return L


def test_library_exports_every_declared_symbol(lbm):
    L = lbm._load()
    syms = lbm.header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(L, s)]
    assert missing == []


def test_status_strings(lbm):
    for s in range(7):
        assert lbm.lbm_status_string(s)


@pytest.mark.parametrize("bad", [
    dict(nx=24), dict(nx=0), dict(ny=0), dict(tau=0.5), dict(tau=float("nan")),
    dict(periodic_mismatch=True), dict(sparse_periodic_ny=True),
    dict(nx=21760, ny=21936),  # 9 nx ny >= 2^32: beyond 32-bit element indices
])
def test_invalid_parameters_rejected(lbm, bad):
    nx, ny, tau = bad.get("nx", 32), bad.get("ny", 16), bad.get("tau", 0.8)
    p, _ = lbm.make_params(nx, ny, tau, stream=0)
    if bad.get("periodic_mismatch"):
        p.east.periodic = 0
    if bad.get("sparse_periodic_ny"):
        p.ny = 20
        p.layout = lbm.LBM_SPARSE_TILE16
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_workspace_bytes(p)
    assert e.value.status == lbm.LBM_ERR_INVALID


def test_workspace_bytes_counts_lattices(lbm):
    for prec, s in (("f64", 8), ("f32", 4), ("f16s", 2)):
        for pat, nl in (("two_lattice", 2), ("aa", 1)):
            p, _ = lbm.make_params(64, 48, 0.8, precision=prec, pattern=pat, stream=0)
            b = lbm.lbm_workspace_bytes(p)
            lat = 9 * 64 * 48 * s
            assert nl * lat <= b <= nl * lat + 64 * 1024


@pytest.mark.parametrize("shape", [(16, 16), (48, 32), (37, 48), (20, 64)])
@pytest.mark.parametrize("px,py", [(1, 1), (1, 0), (0, 1), (0, 0)])
def test_geometry_tables_match_oracle(lbm, orc, shape, px, py):
    ny, nx = shape
    sparse_ok = not (py and ny % 16)
    for frac, seed in [(0.0, 1), (0.3, 2), (0.9, 3)]:
        solid = inputs.random_solid(nx, ny, frac, seed=seed + nx * ny)
        solid[: min(16, ny), :16] = 1
        s = orc.Setup(nx=nx, ny=ny, tau=0.8, periodic_x=bool(px), periodic_y=bool(py))
        omask, onf = orc.link_mask(s, solid)
        layout = "sparse" if sparse_ok else "dense"
        p, keep = lbm.make_params(nx, ny, 0.8, solid=solid, periodic_x=bool(px), periodic_y=bool(py),
                                  layout=layout, stream=0)
        mask, tid, nbr, nf = lbm.lbm_geometry(p)
        assert np.array_equal(mask, omask)
        assert nf == onf
        if sparse_ok:
            otid, onbr = orc.tile_map(s, omask)
            assert np.array_equal(tid, otid)
            assert np.array_equal(nbr, onbr)


def test_geometry_porous_generator_tables(lbm, orc):
    solid, phi, nd = inputs.porous_discs(256, 128, 0.5, rmin=8, rmax=32, seed=inputs.GEOMETRY_SEED)
    assert abs(phi - 0.5) < 0.05 and nd > 5
    s = orc.Setup(nx=256, ny=128, tau=0.8, periodic_x=True, periodic_y=False)
    omask, onf = orc.link_mask(s, solid)
    otid, onbr = orc.tile_map(s, omask)
    p, keep = lbm.make_params(256, 128, 0.8, solid=solid, periodic_y=False, layout="sparse", stream=0)
    mask, tid, nbr, nf = lbm.lbm_geometry(p)
    assert np.array_equal(mask, omask) and nf == onf
    assert np.array_equal(tid, otid) and np.array_equal(nbr, onbr)


def test_sides_order_matches_header(lbm):
    p, _ = lbm.make_params(32, 16, 0.8, periodic_x=False, periodic_y=False,
                           walls={"west": (1, 2), "east": (3, 4), "south": (5, 6), "north": (7, 8)}, stream=0)
    got = [(getattr(p, s).ux, getattr(p, s).uy) for s in SIDES]
    assert got == [(1, 2), (3, 4), (5, 6), (7, 8)]


@pytest.mark.parametrize("bad", ["adjacent", "periodic", "rho", "speed"])
def test_invalid_open_sides_rejected(lbm, bad):
    kw = dict(periodic_x=False, periodic_y=False)
    if bad == "adjacent":
        kw["open"] = {"west": ("velocity", (0.05, 0.0)), "north": ("pressure", 1.0)}
    elif bad == "periodic":
        kw = dict(periodic_x=True, periodic_y=False, open={"west": ("velocity", (0.05, 0.0))})
    elif bad == "rho":
        kw["open"] = {"east": ("pressure", 0.0)}
    else:
        kw["open"] = {"west": ("velocity", (-1.5, 0.0))}
    p, _ = lbm.make_params(32, 16, 0.8, stream=0, **kw)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_workspace_bytes(p)
    assert e.value.status == lbm.LBM_ERR_INVALID


@pytest.mark.parametrize("sides", [("west", "east"), ("south", "north"), ("east", None)])
def test_geometry_with_open_sides_matches_oracle(lbm, orc, sides):
    """Links across an open side are marked like links across a wall; the
    mask and the tile tables match the oracle's."""
    nx, ny = 48, 32
    solid = inputs.random_solid(nx, ny, 0.2, seed=77)
    along_x = sides[0] in ("west", "east")
    op = {sides[0]: ("velocity", (0.02, 0.01))}
    if sides[1]:
        op[sides[1]] = ("pressure", 1.0)
    s = orc.Setup(nx=nx, ny=ny, tau=0.8, periodic_x=not along_x, periodic_y=along_x,
                  open={SIDES.index(k): v for k, v in op.items()})
    omask, onf = orc.link_mask(s, solid)
    otid, onbr = orc.tile_map(s, omask)
    p, keep = lbm.make_params(nx, ny, 0.8, solid=solid, periodic_x=not along_x, periodic_y=along_x,
                              layout="sparse", stream=0, open=op)
    mask, tid, nbr, nf = lbm.lbm_geometry(p)
    assert np.array_equal(mask, omask) and nf == onf
    assert np.array_equal(tid, otid) and np.array_equal(nbr, onbr)


def _p3(lbm, nx=24, ny=10, nz=8, precision="f32", pattern="two_lattice", periodic=(1, 1, 1), solid=None, tau=0.8):
    import ctypes
    p = lbm.lbm3_params()
    p.nx, p.ny, p.nz = nx, ny, nz
    keep = None
    if solid is not None:
        keep = np.ascontiguousarray(solid, dtype=np.uint8)
        p.solid = keep.ctypes.data_as(ctypes.c_void_p)
    p.tau = tau
    p.periodic_x, p.periodic_y, p.periodic_z = periodic
    p.precision = lbm.PRECISIONS[precision]
    p.pattern = lbm.PATTERNS[pattern]
    return p, keep


def _ws3(lbm, p):
    import ctypes
    n = ctypes.c_size_t(0)
    st = lbm._load().lbm3_workspace_bytes(ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_d3q19_workspace_counts_lattices_and_mask(lbm):
    """Two lattices or one (AA) of 19 values a node, plus a 32-bit link mask
    only when some link bounces (a wall axis or a solid node)."""
    def al(b):
        return (b + 255) // 256 * 256
    nx, ny, nz = 24, 10, 8
    N = nx * ny * nz
    for prec, s in (("f64", 8), ("f32", 4), ("f16s", 2)):
        for pat, nl in (("two_lattice", 2), ("aa", 1)):
            if prec == "f16s" and pat == "aa":
                continue
            p, _ = _p3(lbm, nx, ny, nz, prec, pat)
            st, b = _ws3(lbm, p)
            assert st == lbm.LBM_OK and b == nl * al(19 * N * s)
            p, _ = _p3(lbm, nx, ny, nz, prec, pat, periodic=(1, 0, 1))
            st, b = _ws3(lbm, p)
            assert st == lbm.LBM_OK and b == nl * al(19 * N * s) + al(4 * N)
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[3, 4, 5] = 1
    p, keep = _p3(lbm, nx, ny, nz, "f32", solid=solid)
    st, b = _ws3(lbm, p)
    assert st == lbm.LBM_OK and b == 2 * al(19 * N * 4) + al(4 * N)


@pytest.mark.parametrize("bad", [dict(ny=65536), dict(nz=0), dict(tau=0.5), dict(precision="f16s", nx=25),
                                 dict(nx=2048, ny=2048, nz=1024)])
def test_d3q19_invalid_parameters_rejected(lbm, bad):
    kw = dict(nx=24, ny=10, nz=8, precision="f32", tau=0.8)
    kw.update(bad)
    p, _ = _p3(lbm, kw["nx"], kw["ny"], kw["nz"], kw["precision"], tau=kw["tau"])
    st, _ = _ws3(lbm, p)
    assert st == lbm.LBM_ERR_INVALID


def test_d3q19_workspace_holds_the_node_list(lbm):
    """The node list (8 bytes an entry: node index, link mask) joins the
    workspace with the AA pattern when it holds at most 90% of the nodes
    (auto), always with node_list = 2, never with 1 or for FP16s; two
    lattices list the solid nodes that share a 32-byte sector with a fluid
    node (used with node_list = 2 only), AA only the fluid nodes."""
    def al(b):
        return (b + 255) // 256 * 256
    nx, ny, nz = 24, 10, 8
    N = nx * ny * nz
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:, :, 3:20] = 1            # x = 0..2 and 20..23 fluid: 7 of 24 a row
    fl = (solid.reshape(-1) == 0)
    for prec, s, g in (("f64", 8, 4), ("f32", 4, 8)):
        for pat, nl in (("two_lattice", 2), ("aa", 1)):
            if pat == "aa":
                n_list = int(fl.sum())
            else:
                n_list = int(np.repeat(fl.reshape(-1, g).any(1), g).sum())
            base = nl * al(19 * N * s) + al(4 * N)
            for mode, want in ((0, n_list if pat == "aa" else 0), (1, 0), (2, n_list)):
                p, keep = _p3(lbm, nx, ny, nz, prec, pat, solid=solid)
                p.node_list = mode
                st, b = _ws3(lbm, p)
                assert st == lbm.LBM_OK and b == base + al(8 * want), (prec, pat, mode)
    # walls only: every node would be listed -- auto keeps the dense grid
    p, _ = _p3(lbm, nx, ny, nz, "f32", periodic=(1, 0, 1))
    st, b = _ws3(lbm, p)
    assert st == lbm.LBM_OK and b == 2 * al(19 * N * 4) + al(4 * N)
    p.node_list = 2
    st, b = _ws3(lbm, p)
    assert st == lbm.LBM_OK and b == 2 * al(19 * N * 4) + al(4 * N) + al(8 * N)
    # FP16s runs its dense pair kernel
    p, keep = _p3(lbm, nx, ny, nz, "f16s", solid=solid)
    p.node_list = 2
    st, b = _ws3(lbm, p)
    assert st == lbm.LBM_OK and b == 2 * al(19 * N * 2) + al(4 * N)
    p.node_list = 3
    assert _ws3(lbm, p)[0] == lbm.LBM_ERR_INVALID


def test_d3q19_binding_rejects_unknown_node_list_mode(lbm):
    with pytest.raises(ValueError):
        lbm.LBM3(8, 8, 8, 0.8, node_list="sometimes")

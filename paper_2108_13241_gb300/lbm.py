"""ctypes binding of the C ABI in include/lbm.h (argument marshalling only).

Every function named ``lbm_*`` here calls the C function of the same name in
``_lib/liblbm.so``; every step of the computation runs in that library's CUDA
kernels.  PyTorch supplies device memory (tensors) and the stream.  There is
no CPU fallback: if the library is missing, importing the binding raises.

``LBM`` wraps one context: it allocates the workspace as a torch tensor,
keeps the tensors the library holds pointers to alive, and converts between
tensors and the canonical layouts of lbm.h.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbm.h")

LBM_OK, LBM_ERR_INVALID, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_DIVERGED, LBM_ERR_TIMEOUT, \
    LBM_ERR_UNSUPPORTED = range(7)
LBM_F64, LBM_F32, LBM_F16S = 0, 1, 2
LBM_DENSE, LBM_SPARSE_TILE16 = 0, 1
LBM_TWO_LATTICE, LBM_AA = 0, 1

PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S}
LAYOUTS = {"dense": LBM_DENSE, "sparse": LBM_SPARSE_TILE16}
PATTERNS = {"two_lattice": LBM_TWO_LATTICE, "aa": LBM_AA}
LBM_BGK, LBM_TRT = 0, 1
COLLISIONS = {"bgk": LBM_BGK, "trt": LBM_TRT}
STORAGE_BYTES = {LBM_F64: 8, LBM_F32: 4, LBM_F16S: 2}


class LBMError(RuntimeError):
    def __init__(self, fn: str, status: int, detail: str = ""):
        self.status = status
        super().__init__("%s failed: %s%s" % (fn, _status_name(status), (" (" + detail + ")") if detail else ""))


class lbm_side(ctypes.Structure):
    _fields_ = [("periodic", ctypes.c_int), ("ux", ctypes.c_double), ("uy", ctypes.c_double),
                ("kind", ctypes.c_int), ("rho", ctypes.c_double)]


LBM_SIDE_WALL, LBM_SIDE_VELOCITY, LBM_SIDE_PRESSURE = 0, 1, 2
SIDES = ("west", "east", "south", "north")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("solid", ctypes.c_void_p),
        ("tau", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("west", lbm_side), ("east", lbm_side), ("south", lbm_side), ("north", lbm_side),
        ("precision", ctypes.c_int), ("layout", ctypes.c_int), ("pattern", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("collision", ctypes.c_int), ("magic", ctypes.c_double),
    ]


class lbm3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("solid", ctypes.c_void_p),
        ("tau", ctypes.c_double),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double), ("fz", ctypes.c_double),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int), ("periodic_z", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("pattern", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("node_list", ctypes.c_int),
    ]


NODE_LISTS = {"auto": 0, "never": 1, "always": 2}


_lib = None
_P = ctypes.POINTER(lbm_params)
_vp = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is not built (%s); run paper_2108_13241_gb300.build.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "lbm_workspace_bytes": ([_P, ctypes.POINTER(ctypes.c_size_t)], st),
        "lbm_create": ([_P, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)], st),
        "lbm_destroy": ([_vp], st),
        "lbm_set_force": ([_vp, _vp], st),
        "lbm_set_side_values": ([_vp, ctypes.c_int, _vp], st),
        "lbm_init_equilibrium": ([_vp, _vp, _vp], st),
        "lbm_step": ([_vp, ctypes.c_int], st),
        "lbm_macros": ([_vp, _vp, _vp], st),
        "lbm_get_f": ([_vp, _vp], st),
        "lbm_set_f": ([_vp, _vp], st),
        "lbm_reduce": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], st),
        "lbm_loss": ([_vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)], st),
        "lbm_state_bytes": ([_vp, ctypes.POINTER(ctypes.c_size_t)], st),
        "lbm_save_state": ([_vp, _vp], st),
        "lbm_load_state": ([_vp, _vp], st),
        "lbm_forward_states": ([_vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_longlong], st),
        "lbm_backward": ([_vp, ctypes.POINTER(_vp), ctypes.c_int, _vp, _vp, _vp], st),
        "lbm_macros_backward": ([_vp, _vp, _vp, _vp, _vp], st),
        "lbm_link_mask": ([_vp, _vp], st),
        "lbm_tile_map": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int)], st),
        "lbm_geometry": ([_P, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_longlong)], st),
        "lbm_reduce_f_noalloc": ([ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp], st),
        "lbm_fluid_nodes": ([_vp], ctypes.c_longlong),
        "lbm_step_count": ([_vp], ctypes.c_longlong),
        "lbm_launches_per_step": ([_vp], ctypes.c_int),
        "lbm_set_graphs": ([_vp, ctypes.c_int], st),
        "lbm_sector_copy": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)], st),
        "lbm_step_launches": ([_vp, ctypes.c_int], ctypes.c_longlong),
        "lbm_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "lbm_last_error": ([_vp], ctypes.c_char_p),
        "lbm3_workspace_bytes": ([ctypes.POINTER(lbm3_params), ctypes.POINTER(ctypes.c_size_t)], st),
        "lbm3_create": ([ctypes.POINTER(lbm3_params), _vp, ctypes.c_size_t, ctypes.POINTER(_vp)], st),
        "lbm3_destroy": ([_vp], st),
        "lbm3_init_equilibrium": ([_vp, _vp, _vp], st),
        "lbm3_step": ([_vp, ctypes.c_int], st),
        "lbm3_macros": ([_vp, _vp, _vp], st),
        "lbm3_get_f": ([_vp, _vp], st),
        "lbm3_set_f": ([_vp, _vp], st),
        "lbm3_fluid_nodes": ([_vp], ctypes.c_longlong),
        "lbm3_list_nodes": ([_vp], ctypes.c_longlong),
        "lbm3_step_count": ([_vp], ctypes.c_longlong),
        "lbm3_last_error": ([_vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def header_symbols(path: str = HEADER) -> list:
    """Names of the functions include/lbm.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm3?_[a-z0-9_]+)\s*\(", text)))


def _status_name(s: int) -> str:
    try:
        return _load().lbm_status_string(s).decode()
    except Exception:  # noqa: BLE001 - only used to format messages
        return "status %d" % s


def _check(fn: str, status: int, ctx=None):
    if status != LBM_OK:
        detail = ""
        if ctx:
            detail = (_load().lbm_last_error(ctx) or b"").decode()
        raise LBMError(fn, status, detail)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C names

def lbm_workspace_bytes(p: lbm_params) -> int:
    n = ctypes.c_size_t(0)
    _check("lbm_workspace_bytes", _load().lbm_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
    return n.value


def lbm_create(p: lbm_params, workspace: torch.Tensor):
    ctx = ctypes.c_void_p()
    _check("lbm_create", _load().lbm_create(ctypes.byref(p), _ptr(workspace), workspace.numel(),
                                            ctypes.byref(ctx)))
    return ctx


def lbm_destroy(ctx):
    _check("lbm_destroy", _load().lbm_destroy(ctx))


def lbm_set_side_values(ctx, side: int, values: Optional[torch.Tensor]):
    _check("lbm_set_side_values", _load().lbm_set_side_values(ctx, int(side), _ptr(values)), ctx)


def lbm_set_force(ctx, force: Optional[torch.Tensor]):
    _check("lbm_set_force", _load().lbm_set_force(ctx, _ptr(force)), ctx)


def _field(t: Optional[torch.Tensor]):
    """A field argument: a CUDA tensor, or a pinned host tensor the device
    maps (the kernel then reads or writes host memory directly)."""
    if t is not None and not t.is_cuda and not t.is_pinned():
        raise ValueError("field tensors must be on the GPU or in pinned host memory")
    return _ptr(t)


def lbm_init_equilibrium(ctx, rho: Optional[torch.Tensor], u: Optional[torch.Tensor]):
    _check("lbm_init_equilibrium", _load().lbm_init_equilibrium(ctx, _field(rho), _field(u)), ctx)


def lbm_step(ctx, n: int):
    _check("lbm_step", _load().lbm_step(ctx, int(n)), ctx)


def lbm_set_graphs(ctx, enable: bool):
    _check("lbm_set_graphs", _load().lbm_set_graphs(ctx, int(bool(enable))), ctx)


def lbm_sector_copy(ctx, n: int) -> int:
    """Launches n sector copies (measurement aid); returns the bytes of one."""
    b = ctypes.c_longlong(0)
    _check("lbm_sector_copy", _load().lbm_sector_copy(ctx, int(n), ctypes.byref(b)), ctx)
    return int(b.value)


def lbm_step_launches(ctx, n: int) -> int:
    return _load().lbm_step_launches(ctx, int(n))


def lbm_macros(ctx, rho: Optional[torch.Tensor], u: Optional[torch.Tensor]):
    _check("lbm_macros", _load().lbm_macros(ctx, _field(rho), _field(u)), ctx)


def lbm_get_f(ctx, f: torch.Tensor):
    _check("lbm_get_f", _load().lbm_get_f(ctx, _ptr(f)), ctx)


def lbm_set_f(ctx, f: torch.Tensor):
    _check("lbm_set_f", _load().lbm_set_f(ctx, _ptr(f)), ctx)


def lbm_reduce(ctx):
    m = ctypes.c_double(0)
    mom = (ctypes.c_double * 2)()
    _check("lbm_reduce", _load().lbm_reduce(ctx, ctypes.byref(m), mom), ctx)
    return m.value, (mom[0], mom[1])


def lbm_loss(ctx, kind: int, target: Optional[torch.Tensor] = None) -> float:
    out = ctypes.c_double(0)
    _check("lbm_loss", _load().lbm_loss(ctx, int(kind), _ptr(target), ctypes.byref(out)), ctx)
    return out.value


def lbm_state_bytes(ctx) -> int:
    n = ctypes.c_size_t(0)
    _check("lbm_state_bytes", _load().lbm_state_bytes(ctx, ctypes.byref(n)), ctx)
    return n.value


def lbm_save_state(ctx, dst: torch.Tensor):
    _check("lbm_save_state", _load().lbm_save_state(ctx, _ptr(dst)), ctx)


def lbm_load_state(ctx, src: torch.Tensor):
    _check("lbm_load_state", _load().lbm_load_state(ctx, _ptr(src)), ctx)


def _ptr_array(ts: Sequence[torch.Tensor]):
    arr = (ctypes.c_void_p * max(1, len(ts)))()
    for k, t in enumerate(ts):
        arr[k] = t.data_ptr()
    return arr


def lbm_forward_states(ctx, states: Sequence[torch.Tensor], t0: int = 0):
    """states[0] holds A_t0; fills states[1..n] (n = len(states) - 1)."""
    _check("lbm_forward_states",
           _load().lbm_forward_states(ctx, _ptr_array(states), len(states) - 1, int(t0)), ctx)


def lbm_backward(ctx, states: Sequence[torch.Tensor], lam: torch.Tensor, lam_tmp: torch.Tensor,
                 grad_force: torch.Tensor):
    _check("lbm_backward", _load().lbm_backward(ctx, _ptr_array(states), len(states), _ptr(lam),
                                                _ptr(lam_tmp), _ptr(grad_force)), ctx)


def lbm_macros_backward(ctx, g_rho: Optional[torch.Tensor], g_u: Optional[torch.Tensor],
                        lam: torch.Tensor, grad_force: Optional[torch.Tensor]):
    _check("lbm_macros_backward", _load().lbm_macros_backward(ctx, _ptr(g_rho), _ptr(g_u), _ptr(lam),
                                                              _ptr(grad_force)), ctx)


def lbm_link_mask(ctx, ny: int, nx: int) -> np.ndarray:
    m = np.zeros((ny, nx), np.uint8)
    _check("lbm_link_mask", _load().lbm_link_mask(ctx, m.ctypes.data_as(ctypes.c_void_p)), ctx)
    return m


def lbm_tile_map(ctx, ny: int, nx: int):
    nt = ctypes.c_int(0)
    _check("lbm_tile_map", _load().lbm_tile_map(ctx, None, None, ctypes.byref(nt)), ctx)
    tid = np.zeros(((ny + 15) // 16, (nx + 15) // 16), np.int32)
    nbr = np.zeros((nt.value, 9), np.int32)
    _check("lbm_tile_map", _load().lbm_tile_map(ctx, tid.ctypes.data_as(ctypes.c_void_p),
                                                nbr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nt)), ctx)
    return tid, nbr


def lbm_geometry(p: lbm_params):
    """Host-only tables: (mask [ny,nx], tile_id or None, nbr or None, nfluid)."""
    nx, ny = p.nx, p.ny
    mask = np.zeros((ny, nx), np.uint8)
    nt = ctypes.c_int(0)
    nf = ctypes.c_longlong(0)
    sparse = p.layout == LBM_SPARSE_TILE16
    tid = np.zeros(((ny + 15) // 16, (nx + 15) // 16), np.int32) if sparse else None
    nbr = np.zeros((tid.size, 9), np.int32) if sparse else None
    _check("lbm_geometry", _load().lbm_geometry(
        ctypes.byref(p), mask.ctypes.data_as(ctypes.c_void_p),
        None if tid is None else tid.ctypes.data_as(ctypes.c_void_p),
        None if nbr is None else nbr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nt), ctypes.byref(nf)))
    if sparse:
        nbr = nbr[: nt.value].copy()
    return mask, tid, nbr, nf.value


NOALLOC_MAX_ROWS = 16384  # LBM_NOALLOC_MAX_ROWS of lbm.h


def lbm_reduce_f_noalloc(precision, f: torch.Tensor, mask: Optional[torch.Tensor], nx: int, ny: int,
                         out: torch.Tensor, stream=None):
    """Mass and momentum of canonical f [9, ny, nx] into out (3 doubles, on the
    device) without any allocation in the library (see lbm.h); only pointers
    are passed, nothing is allocated here either.  The tensors are checked
    before any device work: a wrong dtype or a short buffer would make the
    kernel read past its end."""
    if ny > NOALLOC_MAX_ROWS:
        raise ValueError("lbm_reduce_f_noalloc: ny = %d exceeds LBM_NOALLOC_MAX_ROWS = %d (the size of its "
                         "static scratch)" % (ny, NOALLOC_MAX_ROWS))
    if nx < 1 or ny < 1:
        raise ValueError("lbm_reduce_f_noalloc: nx and ny must be >= 1")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if prec not in STORAGE_BYTES:
        raise ValueError("lbm_reduce_f_noalloc: unknown precision %r" % (precision,))
    want = torch.float64 if prec == LBM_F64 else torch.float32
    dev = torch.device("cuda", torch.cuda.current_device())

    def on_device(name, t):
        if t.device != dev:
            raise ValueError("lbm_reduce_f_noalloc: %s is on %s, not on the current device %s"
                             % (name, t.device, dev))
        if not t.is_contiguous():
            raise ValueError("lbm_reduce_f_noalloc: %s must be contiguous" % name)

    on_device("f", f)
    if f.dtype != want:
        raise ValueError("lbm_reduce_f_noalloc: f must be %s for precision %r, got %s" % (want, precision, f.dtype))
    if f.numel() < 9 * nx * ny:
        raise ValueError("lbm_reduce_f_noalloc: f holds %d values, needs 9*nx*ny = %d" % (f.numel(), 9 * nx * ny))
    if mask is not None:
        on_device("mask", mask)
        if mask.dtype != torch.uint8 or mask.numel() < nx * ny:
            raise ValueError("lbm_reduce_f_noalloc: mask must be uint8 with at least nx*ny entries")
    on_device("out", out)
    if out.dtype != torch.float64 or out.numel() < 3:
        raise ValueError("lbm_reduce_f_noalloc: out must be float64 with at least 3 entries")
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    _check("lbm_reduce_f_noalloc", _load().lbm_reduce_f_noalloc(prec, _ptr(f), _ptr(mask), int(nx), int(ny),
                                                                _ptr(out), stream or None))


def lbm_fluid_nodes(ctx) -> int:
    return _load().lbm_fluid_nodes(ctx)


def lbm_step_count(ctx) -> int:
    return _load().lbm_step_count(ctx)


def lbm_status_string(s: int) -> str:
    return _load().lbm_status_string(s).decode()


def lbm_last_error(ctx) -> str:
    return (_load().lbm_last_error(ctx) or b"").decode()


# ------------------------------------------------------------------ helpers

def make_params(nx: int, ny: int, tau: float, solid: Optional[np.ndarray] = None,
                force=(0.0, 0.0), periodic_x: bool = True, periodic_y: bool = True,
                walls=None, precision="f32", layout="dense", pattern="two_lattice",
                stream=None, open=None, collision="bgk", magic=0.0):
    """lbm_params from Python values.  walls: {"west"|"east"|"south"|"north":
    (ux, uy)} velocities of wall sides (axes not periodic).  open: {side name:
    ("velocity", (ux, uy)) | ("pressure", rho)} open sides.  collision: "bgk"
    or "trt" (magic: the TRT magic parameter, 0 = 3/16).  Returns
    (params, keepalive) -- keepalive holds the solid array while params is used."""
    p = lbm_params()
    p.nx, p.ny = int(nx), int(ny)
    keep = None
    if solid is not None:
        keep = np.ascontiguousarray(solid, dtype=np.uint8)
        assert keep.shape == (ny, nx)
        p.solid = keep.ctypes.data_as(ctypes.c_void_p)
    p.tau = float(tau)
    p.fx, p.fy = float(force[0]), float(force[1])
    walls = walls or {}
    for name, per in (("west", periodic_x), ("east", periodic_x), ("south", periodic_y), ("north", periodic_y)):
        s = getattr(p, name)
        s.periodic = int(bool(per))
        s.ux, s.uy = walls.get(name, (0.0, 0.0))
    for name, (kind, val) in (open or {}).items():
        s = getattr(p, name)
        if kind == "velocity":
            s.kind = LBM_SIDE_VELOCITY
            s.ux, s.uy = float(val[0]), float(val[1])
        elif kind == "pressure":
            s.kind = LBM_SIDE_PRESSURE
            s.rho = float(val)
        else:
            raise ValueError("open side kind must be 'velocity' or 'pressure'")
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.layout = LAYOUTS[layout] if isinstance(layout, str) else int(layout)
    p.pattern = PATTERNS[pattern] if isinstance(pattern, str) else int(pattern)
    p.collision = COLLISIONS[collision] if isinstance(collision, str) else int(collision)
    p.magic = float(magic)
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream().cuda_stream
    p.stream = stream or None
    return p, keep


class LBM:
    """One simulation context on the current CUDA device and stream."""

    def __init__(self, nx: int, ny: int, tau: float, solid=None, force=(0.0, 0.0),
                 periodic_x: bool = True, periodic_y: bool = True, walls=None,
                 precision="f32", layout="dense", pattern="two_lattice", device="cuda", open=None,
                 collision="bgk", magic=0.0):
        self.nx, self.ny = int(nx), int(ny)
        self.params, keep = make_params(nx, ny, tau, solid, force, periodic_x, periodic_y, walls,
                                        precision, layout, pattern, open=open, collision=collision,
                                        magic=magic)
        self.precision = self.params.precision
        self.dtype = torch.float64 if self.precision == LBM_F64 else torch.float32
        self.device = torch.device(device)
        nbytes = lbm_workspace_bytes(self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lbm_create(self.params, self.workspace)
        del keep
        self.params.solid = None
        self._force = None
        self._side_vals = [None] * 4

    # resources -------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    # state -------------------------------------------------------------------
    @property
    def fluid_nodes(self) -> int:
        return lbm_fluid_nodes(self.ctx)

    @property
    def steps(self) -> int:
        return lbm_step_count(self.ctx)

    @property
    def launches_per_step(self) -> int:
        return _load().lbm_launches_per_step(self.ctx)

    def step_launches(self, n: int) -> int:
        """Kernel launches that step(n) makes (graph nodes included)."""
        return lbm_step_launches(self.ctx, n)

    def sector_copy(self, n: int = 1) -> int:
        """n copies of the lattice's fluid-holding DRAM sectors into the
        other lattice (lbm_sector_copy); returns the bytes of one copy."""
        return lbm_sector_copy(self.ctx, n)

    def set_graphs(self, enable: bool):
        """Replay CUDA graphs for long step runs (default) or launch every
        kernel from the host."""
        lbm_set_graphs(self.ctx, enable)

    def _t(self, a, shape):
        t = torch.as_tensor(a, dtype=self.dtype, device=self.device).contiguous()
        assert tuple(t.shape) == tuple(shape), (t.shape, shape)
        return t

    def set_side_values(self, side, values=None):
        """Per-node values of an open side (velocity [2, len], pressure
        [len]); None returns to the uniform value."""
        k = SIDES.index(side) if isinstance(side, str) else int(side)
        if values is None:
            self._side_vals[k] = None
        else:
            length = self.ny if k < 2 else self.nx
            kind = getattr(self.params, SIDES[k]).kind
            shape = (2, length) if kind == LBM_SIDE_VELOCITY else (length,)
            self._side_vals[k] = self._t(values, shape)
        lbm_set_side_values(self.ctx, k, self._side_vals[k])

    def set_force(self, force=None):
        self._force = None if force is None else self._t(force, (2, self.ny, self.nx))
        lbm_set_force(self.ctx, self._force)

    def init_equilibrium(self, rho=None, u=None):
        r = None if rho is None else self._t(rho, (self.ny, self.nx))
        v = None if u is None else self._t(u, (2, self.ny, self.nx))
        lbm_init_equilibrium(self.ctx, r, v)

    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def macros(self):
        rho = torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        u = torch.empty((2, self.ny, self.nx), dtype=self.dtype, device=self.device)
        lbm_macros(self.ctx, rho, u)
        return rho, u

    def get_f(self) -> torch.Tensor:
        f = torch.empty((9, self.ny, self.nx), dtype=self.dtype, device=self.device)
        lbm_get_f(self.ctx, f)
        return f

    def set_f(self, f):
        t = self._t(f, (9, self.ny, self.nx))
        lbm_set_f(self.ctx, t)

    def reduce(self):
        return lbm_reduce(self.ctx)

    def loss_mse(self, target) -> float:
        t = self._t(target, (2, self.ny, self.nx))
        return lbm_loss(self.ctx, 0, t)

    def loss_ke(self) -> float:
        return lbm_loss(self.ctx, 1, None)

    def link_mask(self) -> np.ndarray:
        return lbm_link_mask(self.ctx, self.ny, self.nx)

    def tile_map(self):
        return lbm_tile_map(self.ctx, self.ny, self.nx)

    # checkpoints and adjoint -------------------------------------------------
    @property
    def state_bytes(self) -> int:
        return lbm_state_bytes(self.ctx)

    def new_state(self) -> torch.Tensor:
        return torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)

    def save_state(self, dst: Optional[torch.Tensor] = None) -> torch.Tensor:
        dst = self.new_state() if dst is None else dst
        lbm_save_state(self.ctx, dst)
        return dst

    def load_state(self, src: torch.Tensor):
        lbm_load_state(self.ctx, src)

    def forward_states(self, states: Sequence[torch.Tensor], t0: int = 0):
        lbm_forward_states(self.ctx, states, t0)

    def backward(self, states: Sequence[torch.Tensor], lam: torch.Tensor, lam_tmp: torch.Tensor,
                 grad_force: torch.Tensor):
        lbm_backward(self.ctx, states, lam, lam_tmp, grad_force)

    def macros_backward(self, g_rho, g_u, lam: torch.Tensor, grad_force: Optional[torch.Tensor]):
        gr = None if g_rho is None else self._t(g_rho, (self.ny, self.nx))
        gu = None if g_u is None else self._t(g_u, (2, self.ny, self.nx))
        lbm_macros_backward(self.ctx, gr, gu, lam, grad_force)


# ------------------------------------------------------------ D3Q19 (lbm3_*)

def _check3(fn: str, status: int, ctx=None):
    if status != LBM_OK:
        detail = ""
        if ctx:
            detail = (_load().lbm3_last_error(ctx) or b"").decode()
        raise LBMError(fn, status, detail)


class LBM3:
    """One D3Q19 context (lbm3_* of include/lbm.h) on the current CUDA device
    and stream: dense, two lattices, stationary half-way bounce-back walls on
    the faces of non-periodic axes and on solid nodes, uniform Guo force.
    Canonical arrays: f [19, nz, ny, nx], u [3, nz, ny, nx], rho [nz, ny, nx].
    node_list: "auto" (a node list for the AA pattern on sparse geometries),
    "never" (the dense grid) or "always" (whenever a link bounces); FP64 /
    FP32 only."""

    def __init__(self, nx: int, ny: int, nz: int, tau: float, solid=None, force=(0.0, 0.0, 0.0),
                 periodic=(True, True, True), precision="f32", device="cuda", pattern="two_lattice",
                 node_list="auto"):
        if isinstance(node_list, str) and node_list not in NODE_LISTS:
            raise ValueError("node_list must be one of %s" % sorted(NODE_LISTS))
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        p = lbm3_params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        keep = None
        if solid is not None:
            keep = np.ascontiguousarray(solid, dtype=np.uint8)
            assert keep.shape == (nz, ny, nx)
            p.solid = keep.ctypes.data_as(ctypes.c_void_p)
        p.tau = float(tau)
        p.fx, p.fy, p.fz = (float(v) for v in force)
        p.periodic_x, p.periodic_y, p.periodic_z = (int(bool(v)) for v in periodic)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.precision = prec
        p.pattern = PATTERNS[pattern] if isinstance(pattern, str) else int(pattern)
        p.stream = torch.cuda.current_stream().cuda_stream or None
        p.node_list = NODE_LISTS[node_list] if isinstance(node_list, str) else int(node_list)
        self.dtype = torch.float64 if prec == LBM_F64 else torch.float32
        self.device = torch.device(device)
        n = ctypes.c_size_t(0)
        _check3("lbm3_workspace_bytes", _load().lbm3_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device=self.device)
        ctx = ctypes.c_void_p()
        _check3("lbm3_create", _load().lbm3_create(ctypes.byref(p), _ptr(self.workspace), self.workspace.numel(),
                                                   ctypes.byref(ctx)))
        self.ctx = ctx
        del keep

    def close(self):
        if getattr(self, "ctx", None):
            _load().lbm3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def fluid_nodes(self) -> int:
        return _load().lbm3_fluid_nodes(self.ctx)

    @property
    def list_nodes(self) -> int:
        """Entries of the node list the step runs over (0: the dense grid)."""
        return _load().lbm3_list_nodes(self.ctx)

    @property
    def steps(self) -> int:
        return _load().lbm3_step_count(self.ctx)

    def _t(self, t, shape):
        t = torch.as_tensor(t, dtype=self.dtype, device=self.device).contiguous()
        if tuple(t.shape) != tuple(shape):
            raise ValueError("expected shape %s, got %s" % (tuple(shape), tuple(t.shape)))
        return t

    def init_equilibrium(self, rho=None, u=None):
        r = None if rho is None else self._t(rho, self.shape)
        v = None if u is None else self._t(u, (3,) + self.shape)
        _check3("lbm3_init_equilibrium", _load().lbm3_init_equilibrium(self.ctx, _ptr(r), _ptr(v)), self.ctx)
        torch.cuda.current_stream().synchronize()

    def step(self, n: int = 1):
        _check3("lbm3_step", _load().lbm3_step(self.ctx, int(n)), self.ctx)

    def macros(self):
        rho = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        u = torch.empty((3,) + self.shape, dtype=self.dtype, device=self.device)
        _check3("lbm3_macros", _load().lbm3_macros(self.ctx, _ptr(rho), _ptr(u)), self.ctx)
        return rho, u

    def get_f(self) -> torch.Tensor:
        f = torch.empty((19,) + self.shape, dtype=self.dtype, device=self.device)
        _check3("lbm3_get_f", _load().lbm3_get_f(self.ctx, _ptr(f)), self.ctx)
        return f

    def set_f(self, f):
        t = self._t(f, (19,) + self.shape)
        _check3("lbm3_set_f", _load().lbm3_set_f(self.ctx, _ptr(t)), self.ctx)
        torch.cuda.current_stream().synchronize()

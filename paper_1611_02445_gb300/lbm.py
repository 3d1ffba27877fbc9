"""Thin ctypes binding of ``liblbm_gb300.so`` (C ABI in ``include/lbm.h``).

Functions keep the C names and only marshal arguments: every step of the computation
runs in the library's CUDA kernels. There is no CPU fallback: if the library is not
built, ``load()`` raises. Host arrays are numpy arrays; device arrays are torch CUDA
tensors (passed by ``data_ptr()``); streams are torch streams or raw ``cudaStream_t``
integers.
"""
from __future__ import annotations

import ctypes as ct
import os
import re

import numpy as np

from . import build as _build

LBM_F64, LBM_F32, LBM_F16S, LBM_F64_NATIVE, LBM_F16S_SR = 0, 1, 2, 3, 4
DTYPES = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "f64n": LBM_F64_NATIVE, "f16sr": LBM_F16S_SR}
SOLID, FLUID, INLET, OUTLET = 0, 1, 2, 3
PERIODIC_X, PERIODIC_Y, PERIODIC_Z = 1, 2, 4
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSUPPORTED",
          5: "LBM_ESTATE", 6: "LBM_ENONFINITE", 7: "LBM_ETIMEOUT", 8: "LBM_EINTERNAL"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")
TESTING_HEADER = os.path.join(os.path.dirname(HEADER), "lbm_testing.h")


class LBMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path() -> str:
    """The library this process loads: the normal build, or the checked build
    (LBM_CHECKED, see include/lbm_testing.h) when the environment sets LBM_CHECKED=1."""
    return _build.LIB_CHECKED if os.environ.get("LBM_CHECKED") == "1" else _build.LIB


def load():
    """Load the CUDA library and declare its signatures; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build(); "
                           "this package has no CPU fallback")
    L = ct.CDLL(path)
    vp, i, u, d, i64 = ct.c_void_p, ct.c_int, ct.c_uint, ct.c_double, ct.c_int64
    pd = ct.POINTER(ct.c_double)
    L.lbm_create.argtypes = [vp, i, i, i, i, i, i, u, vp, ct.POINTER(vp)]
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [vp]
    L.lbm_last_error.restype = ct.c_char_p
    L.lbm_set_stream.argtypes = [vp, vp]
    L.lbm_set_params.argtypes = [vp, d, pd, vp, i, pd, d]
    L.lbm_init_equilibrium.argtypes = [vp, d, pd]
    L.lbm_set_model.argtypes = [vp, i, i, pd]
    L.lbm_set_lid.argtypes = [vp, i, pd]
    L.lbm_set_bc.argtypes = [vp, i, i, i]
    L.lbm_step.argtypes = [vp, i]
    L.lbm_step_kernel.argtypes = [vp, i, i]
    L.lbm_macroscopic.argtypes = [vp, vp, vp, i, i]
    L.lbm_reduce.argtypes = [vp, pd, pd]
    L.lbm_get_f_box.argtypes = [vp, i, i, i, i, i, i, vp]
    L.lbm_get_f.argtypes = [vp, vp]
    L.lbm_set_f.argtypes = [vp, vp]
    L.lbm_get_tiles.argtypes = [vp, vp, vp, ct.POINTER(i64)]
    L.lbm_get_info.argtypes = [vp, ct.POINTER(i64), ct.POINTER(i64), ct.POINTER(i64)]
    L.lbm_save_state.argtypes = [vp, vp, ct.POINTER(ct.c_size_t)]
    L.lbm_load_state.argtypes = [vp, vp, ct.c_size_t]
    L.lbm_adjoint.argtypes = [vp, i, i, i, pd, vp, i, pd]
    L.lbm_build_tiles_noalloc.argtypes = [vp, i, i, i, vp, vp, ct.POINTER(i64), vp]
    pi = ct.POINTER(ct.c_int)
    L.lbm_partition_z.argtypes = [vp, i, i, i, i, pi]
    L.lbm_slab_geometry.argtypes = [vp, i, i, i, u, i, i, vp, pi, pi, pi]
    L.lbm_create_slab.argtypes = [vp, i, i, i, i, i, u, i, i, vp, ct.POINTER(vp)]
    L.lbm_halo_bytes.argtypes = [vp, i, i, ct.POINTER(ct.c_size_t)]
    L.lbm_halo_pack.argtypes = [vp, i, vp]
    L.lbm_halo_unpack.argtypes = [vp, i, vp]
    L.lbm_testing_live_allocations.argtypes = []
    L.lbm_testing_live_allocations.restype = i64
    L.lbm_testing_fail_allocation.argtypes = [i64]
    L.lbm_testing_fail_allocation.restype = None
    L.lbm_testing_checked_build.argtypes = []
    L.lbm_testing_plant_check.argtypes = [vp, ct.c_uint64]
    for name in header_functions() + header_functions(TESTING_HEADER):
        getattr(L, name)   # every declared entry point must be exported
    _lib = L
    return L


def header_functions(header: str = HEADER):
    """Names of the functions declared in include/lbm.h (or another of the headers)."""
    text = open(header).read()
    return re.findall(r"^\s*(?:lbm_status|void|int|int64_t|const char\s*\*)\s*\**\s*(lbm_\w+)\s*\(", text, re.M)


def _ptr(x):
    """Address of a numpy array, a torch tensor or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _on_device(x) -> int:
    return int(hasattr(x, "is_cuda") and bool(x.is_cuda))


def _d3(v):
    if v is None:
        return None
    a = (ct.c_double * 3)(*[float(t) for t in v])
    return a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(status, ctx=None):
    if status != 0:
        msg = load().lbm_last_error(ctx)
        raise LBMError(status, msg.decode() if msg else "")


# ------------------------------------------------------------------ C entry points
def lbm_create(node_type, nx, ny, nz, tile=4, dtype=LBM_F64, periodic=0, stream=None):
    L = load()
    if isinstance(node_type, np.ndarray):
        node_type = np.ascontiguousarray(node_type, dtype=np.uint8)
    out = ct.c_void_p()
    st = L.lbm_create(_ptr(node_type), _on_device(node_type), int(nx), int(ny), int(nz), int(tile),
                      int(dtype), int(periodic), _stream(stream), ct.byref(out))
    _check(st, None)
    return out.value


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_last_error(ctx=None) -> str:
    m = load().lbm_last_error(ctx)
    return m.decode() if m else ""


def lbm_set_stream(ctx, stream):
    _check(load().lbm_set_stream(ctx, _stream(stream)), ctx)


def lbm_set_params(ctx, tau, g=None, g_field=None, u_in=None, rho_out=1.0):
    if isinstance(g_field, np.ndarray):
        g_field = np.ascontiguousarray(g_field, dtype=np.float64)
    _check(load().lbm_set_params(ctx, float(tau), _d3(g), _ptr(g_field), _on_device(g_field), _d3(u_in),
                                 float(rho_out)), ctx)
    return g_field


def lbm_set_model(ctx, equilibrium=0, collision=0, rates=None):
    r = None
    if rates is not None:
        r = (ct.c_double * 5)(*[float(x) for x in rates])
    _check(load().lbm_set_model(ctx, int(equilibrium), int(collision), r), ctx)


def lbm_set_bc(ctx, scheme=0, inlet_face=0, outlet_face=1):
    _check(load().lbm_set_bc(ctx, int(scheme), int(inlet_face), int(outlet_face)), ctx)


def lbm_set_lid(ctx, face=-1, u=None):
    _check(load().lbm_set_lid(ctx, int(face), _d3(u)), ctx)


def lbm_init_equilibrium(ctx, rho0=1.0, u0=None):
    _check(load().lbm_init_equilibrium(ctx, float(rho0), _d3(u0)), ctx)


def lbm_step(ctx, n=1):
    _check(load().lbm_step(ctx, int(n)), ctx)


KERNEL_FULL, KERNEL_PROPAGATE, KERNEL_RW = 0, 1, 2
EQ_QCOMPR, EQ_INCOMPR = 0, 1
COLL_BGK, COLL_MRT = 0, 1
BC_EQUILIBRIUM, BC_ZOU_HE = 0, 1


def lbm_step_kernel(ctx, kind, n=1):
    _check(load().lbm_step_kernel(ctx, int(kind), int(n)), ctx)


def lbm_macroscopic(ctx, rho, u, out_f64=True):
    """rho, u: numpy arrays (host) or torch CUDA tensors (device) of the dense sizes."""
    _check(load().lbm_macroscopic(ctx, _ptr(rho), _ptr(u), int(bool(out_f64)), _on_device(rho)), ctx)


def lbm_reduce(ctx):
    m = ct.c_double()
    p = (ct.c_double * 3)()
    _check(load().lbm_reduce(ctx, ct.byref(m), p), ctx)
    return m.value, np.array(list(p))


def lbm_get_f_box(ctx, x0, y0, z0, bx, by, bz):
    out = np.empty((19, bz, by, bx), np.float64)
    _check(load().lbm_get_f_box(ctx, int(x0), int(y0), int(z0), int(bx), int(by), int(bz), _ptr(out)), ctx)
    return out


def lbm_get_f(ctx, shape):
    nz, ny, nx = shape
    out = np.empty((19, nz, ny, nx), np.float64)
    _check(load().lbm_get_f(ctx, _ptr(out)), ctx)
    return out


def lbm_set_f(ctx, f_dense):
    f = np.ascontiguousarray(f_dense, dtype=np.float64)
    _check(load().lbm_set_f(ctx, _ptr(f)), ctx)


def lbm_get_info(ctx):
    a, b, c = ct.c_int64(), ct.c_int64(), ct.c_int64()
    _check(load().lbm_get_info(ctx, ct.byref(a), ct.byref(b), ct.byref(c)), ctx)
    return a.value, b.value, c.value


def lbm_get_tiles(ctx, tile_grid):
    """Returns (tile_map [Tz, Ty, Tx] int32, non_empty uint32[n_tiles])."""
    n = ct.c_int64()
    _check(load().lbm_get_tiles(ctx, None, None, ct.byref(n)), ctx)
    tm = np.empty(tile_grid, np.int32)
    ne = np.empty(max(n.value, 1), np.uint32)
    _check(load().lbm_get_tiles(ctx, _ptr(tm), _ptr(ne), ct.byref(n)), ctx)
    return tm, ne[:n.value].copy()


def lbm_save_state(ctx) -> bytes:
    n = ct.c_size_t()
    _check(load().lbm_save_state(ctx, None, ct.byref(n)), ctx)
    buf = ct.create_string_buffer(n.value)
    _check(load().lbm_save_state(ctx, buf, ct.byref(n)), ctx)
    return buf.raw[:n.value]


def lbm_load_state(ctx, blob: bytes):
    _check(load().lbm_load_state(ctx, blob, len(blob)), ctx)


def lbm_adjoint(ctx, T, ckpt_every, plane_x, dL_dg=None, want_dtau=True):
    """Outlet-flux loss after T steps and, when dL_dg (a host numpy array or a device
    tensor of nx*ny*nz doubles) or want_dtau is given, its gradients. Returns
    (L, dL/dtau or None)."""
    loss = ct.c_double()
    dtau = ct.c_double()
    if isinstance(dL_dg, np.ndarray):
        assert dL_dg.dtype == np.float64 and dL_dg.flags.c_contiguous
    _check(load().lbm_adjoint(ctx, int(T), int(ckpt_every), int(plane_x), ct.byref(loss), _ptr(dL_dg),
                              _on_device(dL_dg), ct.byref(dtau) if want_dtau else None), ctx)
    return loss.value, (dtau.value if want_dtau else None)


NOALLOC_MAX_TILES = 1 << 22


def _noalloc_buffer(name, x, dtypes, need):
    """A device tensor the allocation-free builder may read or write: CUDA, one of the
    given dtypes, contiguous and at least ``need`` elements. The C entry point takes raw
    device pointers and cannot check their extent, so the binding checks it before any
    launch."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise ValueError(f"lbm_build_tiles_noalloc: {name} must be a CUDA tensor (a host array "
                         "would be read through a device pointer)")
    if x.dtype not in dtypes:
        raise ValueError(f"lbm_build_tiles_noalloc: {name} must have dtype "
                         f"{' or '.join(str(d) for d in dtypes)}, not {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"lbm_build_tiles_noalloc: {name} must be contiguous")
    if x.numel() < need:
        raise ValueError(f"lbm_build_tiles_noalloc: {name} has {x.numel()} elements, needs {need}")


def lbm_build_tiles_noalloc(node_type, nx, ny, nz, tile_map, non_empty, stream=None):
    """Tile map into caller-owned device buffers, without any device allocation.

    For callers that cannot allocate device memory themselves (their framework's
    allocator owns it, or allocation is forbidden after start-up): node_type (uint8,
    nx*ny*nz), tile_map (int32, one entry per tile of the grid) and non_empty (32-bit,
    as many entries) are contiguous CUDA tensors the caller already holds; their dtype
    and size are checked here, before any launch. Returns the number of kept tiles."""
    import torch
    nx, ny, nz = int(nx), int(ny), int(nz)
    if min(nx, ny, nz) < 1:
        raise ValueError("lbm_build_tiles_noalloc: dimensions must be >= 1")
    n_grid = ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 3) // 4)
    if n_grid <= NOALLOC_MAX_TILES:
        _noalloc_buffer("node_type", node_type, (torch.uint8,), nx * ny * nz)
        _noalloc_buffer("tile_map", tile_map, (torch.int32,), n_grid)
        _noalloc_buffer("non_empty", non_empty, (torch.int32, torch.uint32), n_grid)
    # larger grids are refused by the library before it touches any buffer
    n = ct.c_int64()
    st = load().lbm_build_tiles_noalloc(_ptr(node_type), nx, ny, nz, _ptr(tile_map),
                                        _ptr(non_empty), ct.byref(n), _stream(stream))
    if st != 0:
        hint = {4: f"the tile grid exceeds {NOALLOC_MAX_TILES} tiles held by the static scratch; "
                   "use lbm_create", 1: "invalid arguments or node types outside 0..3"}.get(st, "")
        raise LBMError(st, f"lbm_build_tiles_noalloc: {hint}")
    return n.value


# ------------------------------------------------------------ slabs and their halos
def lbm_partition_z(node_type, nranks: int) -> np.ndarray:
    """Tile-plane bounds of nranks z-slabs with about equal non-solid node counts (host)."""
    nt = np.ascontiguousarray(node_type, dtype=np.uint8)
    nz, ny, nx = nt.shape
    out = (ct.c_int * (nranks + 1))()
    st = load().lbm_partition_z(nt.ctypes.data, nx, ny, nz, int(nranks), out)
    if st != 0:
        raise LBMError(st, load().lbm_last_error(None).decode())
    return np.array(out[:], dtype=np.int64)


def lbm_slab_geometry(node_type, periodic: int, plane_begin: int, plane_end: int):
    """The node types of a slab's box and its ghost planes (host): (sub, ghost_lo, ghost_hi)."""
    nt = np.ascontiguousarray(node_type, dtype=np.uint8)
    nz, ny, nx = nt.shape
    nzs, gl, gh = ct.c_int(), ct.c_int(), ct.c_int()
    L = load()
    st = L.lbm_slab_geometry(nt.ctypes.data, nx, ny, nz, int(periodic), int(plane_begin), int(plane_end), None,
                             ct.byref(nzs), ct.byref(gl), ct.byref(gh))
    if st != 0:
        raise LBMError(st, L.lbm_last_error(None).decode())
    sub = np.empty((nzs.value, ny, nx), np.uint8)
    L.lbm_slab_geometry(nt.ctypes.data, nx, ny, nz, int(periodic), int(plane_begin), int(plane_end),
                        sub.ctypes.data, ct.byref(nzs), ct.byref(gl), ct.byref(gh))
    return sub, gl.value, gh.value


def lbm_create_slab(node_type, dtype, periodic, plane_begin, plane_end, stream=None):
    nt = np.ascontiguousarray(node_type, dtype=np.uint8)
    nz, ny, nx = nt.shape
    out = ct.c_void_p()
    L = load()
    st = L.lbm_create_slab(nt.ctypes.data, nx, ny, nz, 4, int(dtype), int(periodic), int(plane_begin),
                           int(plane_end), _stream(stream), ct.byref(out))
    if st != 0:
        raise LBMError(st, L.lbm_last_error(None).decode())
    return out.value


def lbm_halo_bytes(ctx, side: int, pack: bool) -> int:
    n = ct.c_size_t()
    _check(load().lbm_halo_bytes(ctx, int(side), int(bool(pack)), ct.byref(n)), ctx)
    return n.value


def _halo_buffer(ctx, side: int, pack: bool, buf):
    """A halo buffer is device memory of at least lbm_halo_bytes bytes: the library copies
    into or out of it with device-to-device copies and cannot check it, so the binding
    refuses anything else before the call."""
    import torch
    need = lbm_halo_bytes(ctx, side, pack)
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("halo buffers must be contiguous CUDA tensors")
    if buf.numel() * buf.element_size() < need:
        raise ValueError(f"halo buffer of {buf.numel() * buf.element_size()} bytes, needs {need}")


def lbm_halo_pack(ctx, side: int, buf):
    if lbm_halo_bytes(ctx, side, True):
        _halo_buffer(ctx, side, True, buf)
    _check(load().lbm_halo_pack(ctx, int(side), _ptr(buf)), ctx)


def lbm_halo_unpack(ctx, side: int, buf):
    if lbm_halo_bytes(ctx, side, False):
        _halo_buffer(ctx, side, False, buf)
    _check(load().lbm_halo_unpack(ctx, int(side), _ptr(buf)), ctx)


# ------------------------------------------------------------------ test hooks
def testing_live_allocations() -> int:
    """Device buffers the library holds now (include/lbm_testing.h)."""
    return int(load().lbm_testing_live_allocations())


def testing_fail_allocation(k: int):
    """Make the k-th device allocation from now on fail as out of memory (k < 0: none)."""
    load().lbm_testing_fail_allocation(int(k))


def testing_checked_build() -> bool:
    return bool(load().lbm_testing_checked_build())


def testing_plant_check(ctx, word: int):
    _check(load().lbm_testing_plant_check(ctx, int(word)), ctx)


# ------------------------------------------------------------------ convenience class
class Lattice:
    """One geometry on the GPU: owns an lbm_ctx and releases it on close()."""

    def __init__(self, node_type, dtype="f64", periodic=0, stream=None):
        shape = tuple(node_type.shape)
        self.shape = shape
        nz, ny, nx = shape
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.ctx = lbm_create(node_type, nx, ny, nz, 4, self.dtype, periodic, stream)
        self.tile_grid = ((nz + 3) // 4, (ny + 3) // 4, (nx + 3) // 4)
        self._keep = None

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, tau, g=None, g_field=None, u_in=None, rho_out=1.0):
        self._keep = lbm_set_params(self.ctx, tau, g, g_field, u_in, rho_out)

    def set_model(self, equilibrium=EQ_QCOMPR, collision=COLL_BGK, rates=None):
        lbm_set_model(self.ctx, equilibrium, collision, rates)

    def set_bc(self, scheme=BC_EQUILIBRIUM, inlet_face=0, outlet_face=1):
        lbm_set_bc(self.ctx, scheme, inlet_face, outlet_face)

    def set_lid(self, face=-1, u=None):
        lbm_set_lid(self.ctx, face, u)

    def init_equilibrium(self, rho0=1.0, u0=None):
        lbm_init_equilibrium(self.ctx, rho0, u0)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def step_kernel(self, kind, n=1):
        lbm_step_kernel(self.ctx, kind, n)

    def set_stream(self, stream):
        lbm_set_stream(self.ctx, stream)

    def reduce(self):
        return lbm_reduce(self.ctx)

    def macroscopic(self, out_f64=True):
        nz, ny, nx = self.shape
        dt = np.float64 if out_f64 else np.float32
        rho = np.empty((nz, ny, nx), dt)
        u = np.empty((3, nz, ny, nx), dt)
        lbm_macroscopic(self.ctx, rho, u, out_f64)
        return rho, u

    def get_f(self):
        return lbm_get_f(self.ctx, self.shape)

    def get_f_box(self, x0, y0, z0, bx, by, bz):
        return lbm_get_f_box(self.ctx, x0, y0, z0, bx, by, bz)

    def set_f(self, f):
        lbm_set_f(self.ctx, f)

    def tiles(self):
        return lbm_get_tiles(self.ctx, self.tile_grid)

    def info(self):
        n_tiles, n_nonsolid, copy_bytes = lbm_get_info(self.ctx)
        return {"n_tiles": n_tiles, "n_nonsolid": n_nonsolid, "copy_bytes": copy_bytes,
                "eta_t": n_nonsolid / (64 * n_tiles) if n_tiles else 0.0}

    def adjoint(self, T, ckpt_every, plane_x, grads=True):
        """(L, dL/dF_x dense numpy array or None, dL/dtau or None) after T steps."""
        dg = np.zeros(self.shape, np.float64) if grads else None
        L, dtau = lbm_adjoint(self.ctx, T, ckpt_every, plane_x, dg, grads)
        return L, dg, dtau

    def save_state(self) -> bytes:
        return lbm_save_state(self.ctx)

    def load_state(self, blob: bytes):
        lbm_load_state(self.ctx, blob)

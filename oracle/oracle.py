"""ctypes front end of the FP64 oracle (``oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the benchmark's
CPU-baseline leg; the CUDA library never touches it.

Arrays: node types ``nt`` are uint8 ``[nz, ny, nx]``; populations are float64
``[19, nz, ny, nx]`` (x fastest); solid nodes hold NaN. ``periodic`` is a bit mask
(1: x, 2: y, 4: z).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

Q = 19
_lib = None


def load(path):
    """Open an oracle shared library and declare its C signatures."""
    L = ct.CDLL(path)
    d = ct.POINTER(ct.c_double)
    u8 = ct.POINTER(ct.c_uint8)
    i32 = ct.POINTER(ct.c_int32)
    u32 = ct.POINTER(ct.c_uint32)
    ci, cl, cu, cd = ct.c_int, ct.c_long, ct.c_uint, ct.c_double
    L.oracle_version.restype = ci
    L.oracle_lattice.argtypes = [i32, d, i32]
    L.oracle_collide.argtypes = [d, ci, cd, d, d, cd, d]
    L.oracle_step.argtypes = [d, d, u8, ci, ci, ci, cu, cd, d, d, d, cd, ci]
    L.oracle_init.argtypes = [d, u8, cl, cd, d]
    L.oracle_macroscopic.argtypes = [d, u8, cl, d, d, d, d]
    L.oracle_reduce.argtypes = [d, u8, cl, d, d, d]
    L.oracle_tiling.argtypes = [u8, ci, ci, ci, ci, i32, u32]
    L.oracle_tiling.restype = cl
    L.oracle_to_tiles.argtypes = [d, u8, ci, ci, ci, u32, cl, d, u8]
    L.oracle_from_tiles.argtypes = [d, ci, ci, ci, u32, cl, d]
    L.oracle_step_tiled.argtypes = [d, d, u8, i32, u32, cl, ci, ci, ci, cu, cd, d, d, d, cd]
    L.oracle_step_tl.argtypes = [d, d, d, d, u8, ci, ci, ci, cu, cd, cd, d, d, d, d, d, cd]
    L.oracle_collide_adj.argtypes = [d, ci, cd, d, d, cd, d, d, d, d]
    L.oracle_step_adj.argtypes = [d, d, d, u8, ci, ci, ci, cu, cd, d, d, d, cd, d, d, d]
    L.oracle_mrt_matrix.argtypes = [d]
    L.oracle_collide_m.argtypes = [d, ci, cd, d, d, cd, ci, ci, d, d]
    L.oracle_step_m.argtypes = [d, d, u8, ci, ci, ci, cu, cd, d, d, d, cd, ci, ci, d, ci, d, ci, ci, ci, ci]
    L.oracle_zou_he.argtypes = [d, ci, ci, ci, d, cd, d]
    L.oracle_macroscopic_m.argtypes = [d, u8, cl, d, d, ci, d, d]
    L.oracle_loss.argtypes = [d, u8, ci, ci, ci, ci, d, d, d, d, d]
    L.oracle_loss.restype = cd
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _p(a, t=ct.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ct.POINTER(t))


def _d3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def lattice():
    c = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q, np.float64)
    op = np.zeros(Q, np.int32)
    lib().oracle_lattice(_p(c, ct.c_int32), _p(w), _p(op, ct.c_int32))
    return c, w, op


def collide(f, node_type, tau, F=(0, 0, 0), u_in=(0, 0, 0), rho_out=1.0):
    f = _f64(f).reshape(Q)
    out = np.zeros(Q)
    Fa, ui = _d3(F), _d3(u_in)
    lib().oracle_collide(_p(f), int(node_type), float(tau), _p(Fa), _p(ui), float(rho_out), _p(out))
    return out


def collide_adj(f, node_type, tau, lam, F=(0, 0, 0), u_in=(0, 0, 0), rho_out=1.0):
    f = _f64(f).reshape(Q)
    lam = _f64(lam).reshape(Q)
    mu = np.zeros(Q)
    Fb = np.zeros(3)
    tb = np.zeros(1)
    Fa, ui = _d3(F), _d3(u_in)
    lib().oracle_collide_adj(_p(f), int(node_type), float(tau), _p(Fa), _p(ui), float(rho_out),
                             _p(lam), _p(mu), _p(Fb), _p(tb))
    return mu, Fb, float(tb[0])


def init(nt, rho0=1.0, u0=(0, 0, 0)):
    nt = _u8(nt)
    f = np.zeros((Q,) + nt.shape)
    lib().oracle_init(_p(f), _p(nt, ct.c_uint8), nt.size, float(rho0), _p(_d3(u0)))
    return f


def step(A, nt, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0), rho_out=1.0,
         nthreads=1, out=None):
    nt = _u8(nt)
    A = _f64(A)
    nz, ny, nx = nt.shape
    B = A.copy() if out is None else out
    gf = None if g_field is None else _f64(g_field)
    lib().oracle_step(_p(A), _p(B), _p(nt, ct.c_uint8), nx, ny, nz, int(periodic), float(tau),
                      _p(_d3(g)), _p(gf), _p(_d3(u_in)), float(rho_out), int(nthreads))
    return B


def run(f, nt, steps, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0), rho_out=1.0,
        nthreads=1):
    """``steps`` fused steps with A/B ping-pong; returns the final state."""
    A = _f64(f).copy()
    B = A.copy()
    for _ in range(steps):
        step(A, nt, periodic, tau, g, g_field, u_in, rho_out, nthreads, out=B)
        A, B = B, A
    return A


def macroscopic(f, nt, g=(0, 0, 0), g_field=None):
    nt = _u8(nt)
    f = _f64(f)
    rho = np.zeros(nt.shape)
    u = np.zeros((3,) + nt.shape)
    gf = None if g_field is None else _f64(g_field)
    lib().oracle_macroscopic(_p(f), _p(nt, ct.c_uint8), nt.size, _p(_d3(g)), _p(gf), _p(rho), _p(u))
    return rho, u


def reduce(f, nt, g=(0, 0, 0), g_field=None):
    nt = _u8(nt)
    f = _f64(f)
    out = np.zeros(4)
    gf = None if g_field is None else _f64(g_field)
    lib().oracle_reduce(_p(f), _p(nt, ct.c_uint8), nt.size, _p(_d3(g)), _p(gf), _p(out))
    return float(out[0]), out[1:].copy()


def tiling(nt, a=4):
    """Algorithm 1. Returns (tile_map [Tz, Ty, Tx] int32, non_empty uint32[n_tiles])."""
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    T = ((nz + a - 1) // a, (ny + a - 1) // a, (nx + a - 1) // a)
    tm = np.zeros(T, np.int32)
    ne = np.zeros(int(np.prod(T)), np.uint32)
    n = lib().oracle_tiling(_p(nt, ct.c_uint8), nx, ny, nz, a, _p(tm, ct.c_int32), _p(ne, ct.c_uint32))
    return tm, ne[:n].copy()


def to_tiles(f, nt, non_empty):
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    k = len(non_empty)
    ne = np.ascontiguousarray(non_empty, dtype=np.uint32)
    ft = None if f is None else np.zeros((k, Q, 64))
    ntt = np.zeros((k, 64), np.uint8)
    lib().oracle_to_tiles(_p(None if f is None else _f64(f)), _p(nt, ct.c_uint8), nx, ny, nz,
                          _p(ne, ct.c_uint32), k, _p(ft), _p(ntt, ct.c_uint8))
    return ft, ntt


def from_tiles(ft, shape, non_empty):
    nz, ny, nx = shape
    ne = np.ascontiguousarray(non_empty, dtype=np.uint32)
    f = np.zeros((Q, nz, ny, nx))
    lib().oracle_from_tiles(_p(_f64(ft)), nx, ny, nz, _p(ne, ct.c_uint32), len(ne), _p(f))
    return f


def step_tiled(At, ntt, tile_map, non_empty, shape, periodic, tau, g=(0, 0, 0), g_field_t=None,
               u_in=(0, 0, 0), rho_out=1.0):
    nz, ny, nx = shape
    At = _f64(At)
    Bt = At.copy()
    tm = np.ascontiguousarray(tile_map, dtype=np.int32)
    ne = np.ascontiguousarray(non_empty, dtype=np.uint32)
    gf = None if g_field_t is None else _f64(g_field_t)
    lib().oracle_step_tiled(_p(At), _p(Bt), _p(_u8(ntt), ct.c_uint8), _p(tm, ct.c_int32),
                            _p(ne, ct.c_uint32), len(ne), nx, ny, nz, int(periodic), float(tau),
                            _p(_d3(g)), _p(gf), _p(_d3(u_in)), float(rho_out))
    return Bt


def step_tl(A, dA, nt, periodic, tau, dtau=0.0, g=(0, 0, 0), dg=(0, 0, 0), g_field=None,
            dg_field=None, u_in=(0, 0, 0), rho_out=1.0):
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    A, dA = _f64(A), _f64(dA)
    B, dB = A.copy(), np.zeros_like(dA)
    gf = None if g_field is None else _f64(g_field)
    dgf = None if dg_field is None else _f64(dg_field)
    lib().oracle_step_tl(_p(A), _p(dA), _p(B), _p(dB), _p(nt, ct.c_uint8), nx, ny, nz,
                         int(periodic), float(tau), float(dtau), _p(_d3(g)), _p(_d3(dg)), _p(gf),
                         _p(dgf), _p(_d3(u_in)), float(rho_out))
    return B, dB


def step_adj(A, lam_next, nt, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0),
             rho_out=1.0, gbar_field=None, gbar=None, taubar=None):
    """One adjoint step; accumulates into gbar_field (dense, optional), gbar[3], taubar[1]."""
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    lam = np.zeros_like(_f64(lam_next))
    gbar = np.zeros(3) if gbar is None else gbar
    taubar = np.zeros(1) if taubar is None else taubar
    gf = None if g_field is None else _f64(g_field)
    lib().oracle_step_adj(_p(_f64(A)), _p(_f64(lam_next)), _p(lam), _p(nt, ct.c_uint8), nx, ny, nz,
                          int(periodic), float(tau), _p(_d3(g)), _p(gf), _p(_d3(u_in)),
                          float(rho_out), _p(gbar_field), _p(gbar), _p(taubar))
    return lam


def loss(f, nt, plane_x, g=(0, 0, 0), g_field=None, gbar_field=None, gbar=None):
    """Outlet-flux loss and its seed adjoint; returns (L, lam)."""
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    lam = np.zeros((Q,) + nt.shape)
    gbar = np.zeros(3) if gbar is None else gbar
    gf = None if g_field is None else _f64(g_field)
    L = lib().oracle_loss(_p(_f64(f)), _p(nt, ct.c_uint8), nx, ny, nz, int(plane_x), _p(_d3(g)),
                          _p(gf), _p(lam), _p(gbar_field), _p(gbar))
    return L, lam


def adjoint(nt, T, plane_x, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0),
            rho_out=1.0, f0=None):
    """Loss after T steps from f0 (equilibrium rho=1, u=0 by default) and its gradients.

    Forward stores every state (small boxes only); the reverse sweep applies the
    adjoint step T times. Returns (L, dL/dg_field dense or None, dL/dg[3], dL/dtau).
    """
    nt = _u8(nt)
    A = init(nt) if f0 is None else _f64(f0).copy()
    states = [A]
    for _ in range(T):
        states.append(step(states[-1], nt, periodic, tau, g, g_field, u_in, rho_out))
    gbar_field = None if g_field is None else np.zeros(nt.shape)
    gbar = np.zeros(3)
    taubar = np.zeros(1)
    L, lam = loss(states[T], nt, plane_x, g, g_field, gbar_field, gbar)
    for t in range(T - 1, -1, -1):
        lam = step_adj(states[t], lam, nt, periodic, tau, g, g_field, u_in, rho_out,
                       gbar_field, gbar, taubar)
    return L, gbar_field, gbar, float(taubar[0])


def forward_loss(nt, T, plane_x, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0),
                 rho_out=1.0, f0=None):
    A = init(nt) if f0 is None else _f64(f0)
    A = run(A, nt, T, periodic, tau, g, g_field, u_in, rho_out)
    return loss(A, nt, plane_x, g, g_field)[0]


def nonsolid(nt):
    return np.asarray(nt) != 0


def default_threads():
    return os.cpu_count() or 1


# ------------------------------------------------------------------ collision models
EQ_QCOMPR, EQ_INCOMPR = 0, 1
COLL_BGK, COLL_MRT = 0, 1


def mrt_matrix():
    """The D3Q19 moment matrix M[k, i] (d'Humieres et al. 2002 basis)."""
    M = np.zeros((Q, Q))
    lib().oracle_mrt_matrix(_p(M))
    return M


def mrt_rates(tau, s_e=1.19, s_eps=1.4, s_q=1.2, s_pi=1.4, s_m=1.98):
    """The 19 relaxation rates in moment order; the viscous moments relax with 1/tau.
    Defaults: the rates d'Humieres et al. (2002) suggest for D3Q19; the conserved
    moments' rates are 1 (they do not enter the update)."""
    s_nu = 1.0 / tau
    return np.array([1.0, s_e, s_eps, 1.0, s_q, 1.0, s_q, 1.0, s_q, s_nu, s_pi, s_nu, s_pi,
                     s_nu, s_nu, s_nu, s_m, s_m, s_m])


def _rates(rates):
    if rates is None:
        return np.zeros(Q)
    r = _f64(rates).reshape(Q)
    return r


def collide_m(f, node_type, tau, F=(0, 0, 0), u_in=(0, 0, 0), rho_out=1.0, eq=EQ_QCOMPR, coll=COLL_BGK,
              rates=None):
    f = _f64(f).reshape(Q)
    out = np.zeros(Q)
    r = _rates(rates)
    lib().oracle_collide_m(_p(f), int(node_type), float(tau), _p(_d3(F)), _p(_d3(u_in)), float(rho_out),
                           int(eq), int(coll), _p(r), _p(out))
    return out


def step_m(A, nt, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0), rho_out=1.0, eq=EQ_QCOMPR,
           coll=COLL_BGK, rates=None, nthreads=1, out=None, lid_face=-1, lid_u=(0, 0, 0), bc=0, in_face=0,
           out_face=1):
    nt = _u8(nt)
    A = _f64(A)
    nz, ny, nx = nt.shape
    B = A.copy() if out is None else out
    gf = None if g_field is None else _f64(g_field)
    r = _rates(rates)
    lib().oracle_step_m(_p(A), _p(B), _p(nt, ct.c_uint8), nx, ny, nz, int(periodic), float(tau), _p(_d3(g)),
                        _p(gf), _p(_d3(u_in)), float(rho_out), int(eq), int(coll), _p(r), int(lid_face),
                        _p(_d3(lid_u)), int(bc), int(in_face), int(out_face), int(nthreads))
    return B


def run_m(f, nt, steps, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0), rho_out=1.0, eq=EQ_QCOMPR,
          coll=COLL_BGK, rates=None, nthreads=1, lid_face=-1, lid_u=(0, 0, 0), bc=0, in_face=0, out_face=1):
    """``steps`` fused steps of the chosen collision model (and moving wall); returns the
    final state."""
    A = _f64(f).copy()
    B = A.copy()
    for _ in range(steps):
        step_m(A, nt, periodic, tau, g, g_field, u_in, rho_out, eq, coll, rates, nthreads, out=B,
               lid_face=lid_face, lid_u=lid_u, bc=bc, in_face=in_face, out_face=out_face)
        A, B = B, A
    return A


def macroscopic_m(f, nt, g=(0, 0, 0), g_field=None, eq=EQ_QCOMPR):
    nt = _u8(nt)
    nz, ny, nx = nt.shape
    N = nx * ny * nz
    rho = np.zeros((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    gf = None if g_field is None else _f64(g_field)
    lib().oracle_macroscopic_m(_p(_f64(f)), _p(nt, ct.c_uint8), N, _p(_d3(g)), _p(gf), int(eq), _p(rho), _p(u))
    return rho, u


BC_EQUILIBRIUM, BC_ZOU_HE = 0, 1


def zou_he(f, face, kind, eq=EQ_QCOMPR, u_b=(0, 0, 0), rho_b=1.0):
    """Complete the populations of a boundary node on box face ``face`` (Zou-He):
    kind 0 velocity u_b, kind 1 pressure (density rho_b)."""
    f = _f64(f).reshape(Q)
    out = np.zeros(Q)
    lib().oracle_zou_he(_p(f), int(face), int(kind), int(eq), _p(_d3(u_b)), float(rho_b), _p(out))
    return out

"""The z-slab decomposition with halo exchange, on CPU ranks over gloo.

The planner (lbm_partition_z) and the slab boxes (lbm_slab_geometry) are the library's
host code; the exchange schedule (partition.halo_exchange) is the binding's, with host
tensors in place of device buffers. Each rank steps its slab's box with the FP64 oracle
and exchanges, before every step, the five populations per node that cross each cut
(partition.DIRS_UP / DIRS_DOWN) of its boundary tile planes. After the steps every
rank's own nodes equal the single-domain oracle bit for bit (the per-node arithmetic is
the same; only the data's origin differs), and the FP64 all-reduce of the slabs' mass
equals the single-domain mass to rounding.
"""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1611_02445_gb300 import build as B
from paper_1611_02445_gb300 import lbm
from paper_1611_02445_gb300 import partition as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    lbm.load()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _geometry(case):
    from paper_1611_02445_gb300 import inputs as I
    nx, ny, nz, periodic, seed = case
    return I.random_box(nx, ny, nz, p_solid=0.3, seed=seed), periodic


# ------------------------------------------------------------------ host pieces
def test_partition_covers_every_plane_in_balanced_slabs():
    from paper_1611_02445_gb300 import inputs as I
    nt = I.sphere_pack(64, 8.0, 0.35, I.SEED_POROUS_256)
    per_plane = (nt != 0).reshape(16, 4, 64, 64).sum(axis=(1, 2, 3))
    for world in (1, 2, 3, 5, 16):
        pb = lbm.lbm_partition_z(nt, world)
        assert pb[0] == 0 and pb[-1] == 16 and np.all(np.diff(pb) >= 1)
        loads = [per_plane[pb[r]:pb[r + 1]].sum() for r in range(world)]
        # each cut sits within one plane of the ideal share
        ideal = per_plane.sum() / world
        assert max(loads) <= ideal + per_plane.max() + 1, (world, loads)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_partition_z(nt, 17)                    # more slabs than tile planes


@pytest.mark.parametrize("periodic", [0, 0b100, 0b111])
def test_slab_box_is_the_wrapped_slice_with_ghost_planes(periodic):
    from paper_1611_02445_gb300 import inputs as I
    nt = I.random_box(12, 8, 30 if not periodic & 4 else 32, p_solid=0.4, seed=9)
    nz = nt.shape[0]
    Tz = (nz + 3) // 4
    pb = lbm.lbm_partition_z(nt, 3)
    for r in range(3):
        b, e = int(pb[r]), int(pb[r + 1])
        sub, gl, gh = lbm.lbm_slab_geometry(nt, periodic, b, e)
        assert gl == int(b > 0 or bool(periodic & 4)) and gh == int(e < Tz or bool(periodic & 4))
        z = 4 * (b - gl) + np.arange(sub.shape[0])
        z = z % nz if periodic & 4 else z
        inside = z < nz
        assert np.array_equal(sub[inside], nt[z[inside]]) and not sub[~inside].any()
    sub, gl, gh = lbm.lbm_slab_geometry(nt, periodic, 0, Tz)      # the whole domain: no ghosts
    assert gl == gh == 0 and np.array_equal(sub[:nz], nt)


def test_neighbours_and_errors():
    assert P.neighbours(0, 1, True) == (None, None)
    assert P.neighbours(0, 3, False) == (None, 1) and P.neighbours(2, 3, False) == (1, None)
    assert P.neighbours(0, 3, True) == (2, 1) and P.neighbours(2, 3, True) == (1, 0)
    assert P.neighbours(1, 2, True) == (0, 0)
    nt = np.ones((8, 8, 8), np.uint8)
    for b, e in ((1, 1), (-1, 1), (0, 3)):
        with pytest.raises(lbm.LBMError):
            lbm.lbm_slab_geometry(nt, 0, b, e)


# ----------------------------------------------------------- gloo ranks, oracle slabs
def _rank_main(rank, world, port, case, steps, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_1611_02445_gb300 import inputs as I
    from paper_1611_02445_gb300 import lbm as Lb
    from paper_1611_02445_gb300 import partition as Pt
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        nt, periodic = _geometry(case)
        nz = nt.shape[0]
        tau, g = 0.8, (1e-5, -3e-6, 2e-6)
        f0 = I.random_populations(nt, 0.05, seed=5)
        pb = Lb.lbm_partition_z(nt, world)
        b, e = int(pb[rank]), int(pb[rank + 1])
        sub, gl, gh = Lb.lbm_slab_geometry(nt, periodic, b, e)
        nzs = sub.shape[0]
        z = 4 * (b - gl) + np.arange(nzs)
        z = z % nz if periodic & 4 else z
        f = np.full((19,) + sub.shape, np.nan)
        inside = z < nz
        f[:, inside] = f0[:, z[inside]]
        f[:, sub == 0] = np.nan
        up, down = list(Pt.DIRS_UP), list(Pt.DIRS_DOWN)
        lo_own = slice(4 * gl, 4 * gl + 4)                 # lowest own tile plane
        hi_own = slice(nzs - 4 * gh - 4, nzs - 4 * gh)     # highest own tile plane
        for _ in range(steps):
            send_lo = torch.from_numpy(np.ascontiguousarray(f[down][:, lo_own])) if gl else None
            send_hi = torch.from_numpy(np.ascontiguousarray(f[up][:, hi_own])) if gh else None
            recv_lo = torch.empty((5, 4) + sub.shape[1:], dtype=torch.float64) if gl else None
            recv_hi = torch.empty((5, 4) + sub.shape[1:], dtype=torch.float64) if gh else None
            Pt.halo_exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, bool(periodic & 4))
            if gl:
                f[up, 0:4] = recv_lo.numpy()
            if gh:
                f[down, nzs - 4:] = recv_hi.numpy()
            f = O.step(f, sub, periodic & 0b011, tau, g)
        own = slice(4 * gl, nzs - 4 * gh)
        own_nt = sub[own]
        mass = float(np.nansum(f[:, own][:, own_nt != 0]))
        total = Pt.global_sums([mass])[0]
        q.put((rank, z[own], f[:, own], total))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run_ranks(world, case, steps):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, case, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world,case", [(2, (12, 8, 32, 0b111, 3)), (2, (12, 8, 32, 0b011, 4)),
                                        (3, (8, 12, 30, 0b011, 6)), (3, (8, 8, 40, 0b100, 7))])
def test_slabs_on_gloo_ranks_equal_the_single_domain_oracle(world, case):
    from oracle import oracle as O
    from paper_1611_02445_gb300 import inputs as I
    steps = 6
    nt, periodic = _geometry(case)
    f0 = I.random_populations(nt, 0.05, seed=5)
    fo = O.run(f0, nt, steps, periodic, 0.8, (1e-5, -3e-6, 2e-6))
    out = _run_ranks(world, case, steps)
    covered = np.zeros(nt.shape[0], bool)
    for rank, zs, f_own, total in out:
        real = zs < nt.shape[0]
        zr = zs[real]
        assert not covered[zr].any()
        covered[zr] = True
        m = nt[zr] != 0
        assert np.array_equal(f_own[:, real][:, m], fo[:, zr][:, m]), rank   # bit for bit
        mo = O.reduce(fo, nt, (1e-5, -3e-6, 2e-6))[0]
        assert abs(total - mo) <= 1e-12 * mo
    assert covered.all()

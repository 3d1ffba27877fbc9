"""Domain decomposition into z-slabs with a halo exchange between ranks.

The paper runs one GPU and names multi-GPU execution as future work (Sec. 5); the step
itself (Sec. 3.4, Algorithm 2) is unchanged here. Each rank owns a contiguous range of
tile planes along z (``lbm_partition_z``: about equal non-solid node counts) and keeps
one ghost tile plane on each side where the domain continues (``lbm_create_slab``).
Before every step the populations that cross a cut -- the five directions with
c_z = -1 (read from the slab above) or c_z = +1 (read from the slab below) -- of the
boundary tiles are packed on the device, exchanged with torch.distributed
point-to-point operations and unpacked into the neighbours' ghost planes. Global mass
and momentum are an FP64 all-reduce of the slabs' own sums.

The transport (``halo_exchange``) takes plain tensors, so the same schedule runs over
NCCL with device buffers and over gloo with host buffers.
"""
from __future__ import annotations

import numpy as np

from . import lbm

# Directions whose populations cross a z cut, in the order the library packs them.
DIRS_DOWN = (6, 12, 14, 16, 18)   # c_z = -1: what a slab's top plane reads from the slab above
DIRS_UP = (5, 11, 13, 15, 17)     # c_z = +1: what a slab's bottom plane reads from the slab below


def neighbours(rank: int, world: int, periodic_z: bool):
    """(rank below, rank above) of a slab, or None where the domain ends."""
    if world < 2:
        return None, None
    lo = rank - 1 if rank > 0 else (world - 1 if periodic_z else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic_z else None)
    return lo, hi


def halo_exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic_z: bool, group=None):
    """Swap boundary data with the slabs below and above.

    send_lo / send_hi: this slab's packed bottom / top boundary (for the slab below /
    above); recv_lo / recv_hi: buffers for the ghost planes at the bottom / top (None
    where there is none). Two phases -- upward (top boundaries to the slab above), then
    downward -- so that two slabs that are each other's neighbour on both sides (two
    ranks on a periodic axis) still match every message with the right buffer.
    """
    import torch.distributed as dist
    lo, hi = neighbours(rank, world, periodic_z)
    for snd, dst, rcv, src in ((send_hi, hi, recv_lo, lo), (send_lo, lo, recv_hi, hi)):
        ops = []
        if snd is not None and dst is not None:
            ops.append(dist.P2POp(dist.isend, snd, dst, group))
        if rcv is not None and src is not None:
            ops.append(dist.P2POp(dist.irecv, rcv, src, group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


def global_sums(values, group=None, device=None):
    """FP64 sum of per-rank values over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64), dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class SlabLattice:
    """One rank's slab of a domain decomposed along z, on the current CUDA device.

    Every rank passes the whole domain's node types; the slab bounds come from
    ``lbm_partition_z`` unless ``plane_begin`` is given. ``step(n)`` exchanges the halo
    before each of the n steps; ``reduce()`` returns the global FP64 mass and momentum.
    """

    def __init__(self, node_type, dtype="f64", periodic=0, rank=0, world=1, plane_begin=None, stream=None,
                 group=None):
        import torch
        self.rank, self.world, self.group = rank, world, group
        self.periodic_z = bool(periodic & lbm.PERIODIC_Z)
        self.dtype = lbm.DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        pb = lbm.lbm_partition_z(node_type, world) if plane_begin is None else np.asarray(plane_begin)
        self.planes = (int(pb[rank]), int(pb[rank + 1]))
        self.ctx = lbm.lbm_create_slab(node_type, self.dtype, periodic, *self.planes, stream)
        _, self.ghost_lo, self.ghost_hi = lbm.lbm_slab_geometry(node_type, periodic, *self.planes)
        dev = torch.device("cuda", torch.cuda.current_device())

        def buf(side, pack):
            n = lbm.lbm_halo_bytes(self.ctx, side, pack)
            has = self.ghost_lo if side == 0 else self.ghost_hi
            return torch.empty(n, dtype=torch.uint8, device=dev) if has else None

        self.send = [buf(0, True), buf(1, True)]
        self.recv = [buf(0, False), buf(1, False)]
        self.device = dev

    def close(self):
        if self.ctx:
            lbm.lbm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, tau, g=None, u_in=None, rho_out=1.0):
        lbm.lbm_set_params(self.ctx, tau, g, None, u_in, rho_out)

    def init_equilibrium(self, rho0=1.0, u0=None):
        lbm.lbm_init_equilibrium(self.ctx, rho0, u0)

    def exchange(self):
        import torch
        for side in (0, 1):
            if self.send[side] is not None:
                lbm.lbm_halo_pack(self.ctx, side, self.send[side])
        torch.cuda.current_stream(self.device).synchronize()
        halo_exchange(self.send[0], self.send[1], self.recv[0], self.recv[1], self.rank, self.world,
                      self.periodic_z, self.group)
        for side in (0, 1):
            if self.recv[side] is not None:
                lbm.lbm_halo_unpack(self.ctx, side, self.recv[side])

    def step(self, n=1):
        for _ in range(n):
            self.exchange()
            lbm.lbm_step(self.ctx, 1)

    def reduce(self):
        mass, mom = lbm.lbm_reduce(self.ctx)
        s = global_sums([mass, *mom], self.group, self.device)
        return float(s[0]), s[1:4]

    def info(self):
        n_t, n_ns, nbytes = lbm.lbm_get_info(self.ctx)
        return {"n_tiles": n_t, "n_nonsolid": n_ns, "copy_bytes": nbytes}

"""The z-slab decomposition on the GPU: slab contexts (lbm_create_slab) exchanging their
halos through lbm_halo_pack / lbm_halo_unpack against one whole-domain context.

The ranks are emulated in one process on one GPU, strictly in sequence: every slab packs
its boundary planes into device buffers, then every slab unpacks its neighbours' buffers
into its ghost planes, then every slab steps (no kernel waits on another). The transport
between processes (partition.halo_exchange over NCCL or gloo) is covered on CPU ranks
in test_partition.py. The per-node arithmetic of a slab equals the whole domain's, so
the own nodes must agree bit for bit in every storage format.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02445_gb300 import build as B
from paper_1611_02445_gb300 import inputs as I
from paper_1611_02445_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    lbm.load()


def _slab_f(f0, nt, periodic, b, gl, nzs):
    nz = nt.shape[0]
    z = 4 * (b - gl) + np.arange(nzs)
    z = z % nz if periodic & 4 else z
    f = np.full((19, nzs) + nt.shape[1:], np.nan)
    inside = z < nz
    f[:, inside] = f0[:, z[inside]]
    return f, z


def _run_slabs(nt, f0, dtype, periodic, world, steps, tau, g):
    import torch
    pb = lbm.lbm_partition_z(nt, world)
    slabs = []
    for r in range(world):
        b, e = int(pb[r]), int(pb[r + 1])
        sub, gl, gh = lbm.lbm_slab_geometry(nt, periodic, b, e)
        ctx = lbm.lbm_create_slab(nt, lbm.DTYPES[dtype], periodic, b, e)
        lbm.lbm_set_params(ctx, tau, g)
        fs, z = _slab_f(f0, nt, periodic, b, gl, sub.shape[0])
        lbm.lbm_set_f(ctx, fs)
        slabs.append(dict(ctx=ctx, sub=sub, gl=gl, gh=gh, z=z))
    lo = [(r - 1) % world if (r > 0 or periodic & 4) else None for r in range(world)]
    hi = [(r + 1) % world if (r < world - 1 or periodic & 4) else None for r in range(world)]
    for _ in range(steps):
        packs = []
        for s in slabs:
            p = {}
            for side, has in ((0, s["gl"]), (1, s["gh"])):
                if has:
                    p[side] = torch.empty(lbm.lbm_halo_bytes(s["ctx"], side, True), dtype=torch.uint8, device="cuda")
                    lbm.lbm_halo_pack(s["ctx"], side, p[side])
            packs.append(p)
        torch.cuda.synchronize()
        for r, s in enumerate(slabs):
            if s["gl"]:   # the slab below packed its top plane (its side 1)
                buf = packs[lo[r]][1]
                assert buf.numel() == lbm.lbm_halo_bytes(s["ctx"], 0, False)
                lbm.lbm_halo_unpack(s["ctx"], 0, buf)
            if s["gh"]:
                buf = packs[hi[r]][0]
                assert buf.numel() == lbm.lbm_halo_bytes(s["ctx"], 1, False)
                lbm.lbm_halo_unpack(s["ctx"], 1, buf)
        torch.cuda.synchronize()
        for s in slabs:
            lbm.lbm_step(s["ctx"], 1)
    out = []
    for s in slabs:
        f = lbm.lbm_get_f(s["ctx"], s["sub"].shape)
        mass, mom = lbm.lbm_reduce(s["ctx"])
        rho = np.zeros(s["sub"].shape)
        u = np.zeros((3,) + s["sub"].shape)
        lbm.lbm_macroscopic(s["ctx"], rho, u, out_f64=True)
        own = slice(4 * s["gl"], s["sub"].shape[0] - 4 * s["gh"])
        out.append((s["z"][own], f[:, own], mass, mom, rho[own], u[:, own],
                    lbm.lbm_get_info(s["ctx"])[1]))
        lbm.lbm_destroy(s["ctx"])
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
@pytest.mark.parametrize("world,periodic", [(2, 0b111), (3, 0b011), (4, 0b111), (2, 0b100)])
def test_slab_contexts_equal_the_whole_domain(dtype, world, periodic):
    nt = I.sphere_pack(48, 6.0, 0.4, 161102450)
    if not periodic & 0b011:
        nt = nt.copy()
        nt[:, 0, :] = 0                                         # walls where x, y do not wrap
        nt[:, :, 0] = 0
    f0 = I.random_populations(nt, 0.05, seed=51)
    tau, g, steps = 0.8, (1e-5, 2e-6, -1e-6), 7
    with lbm.Lattice(nt, dtype, periodic) as L:
        L.set_params(tau, g)
        L.set_f(f0)
        L.step(steps)
        fg = L.get_f()
        mass_w, mom_w = L.reduce()
        rho_w, u_w = L.macroscopic()
        n_w = L.info()["n_nonsolid"]
    out = _run_slabs(nt, f0, dtype, periodic, world, steps, tau, g)
    covered = np.zeros(nt.shape[0], bool)
    mass, mom, n_own = 0.0, np.zeros(3), 0
    for z, f, m, p, rho, u, n in out:
        real = z < nt.shape[0]
        zr = z[real]
        assert not covered[zr].any()
        covered[zr] = True
        solid = nt[zr] == 0
        assert np.array_equal(f[:, real], fg[:, zr], equal_nan=True)            # bit for bit
        assert np.array_equal(rho[real][~solid], rho_w[zr][~solid])
        assert np.array_equal(u[:, real][:, ~solid], u_w[:, zr][:, ~solid])
        mass += m
        mom += p
        n_own += n
    assert covered.all() and n_own == n_w
    assert abs(mass - mass_w) <= 1e-12 * mass_w
    assert np.abs(mom - mom_w).max() <= 1e-12 * mass_w
    if dtype == "f64":
        fo = O.run(f0, nt, steps, periodic, tau, g)
        m = nt != 0
        _, W, _ = O.lattice()
        assert float((np.abs(fg[:, m] - fo[:, m]) / W[:, None]).max()) <= 1e-12


def test_halo_calls_need_a_ghost_plane():
    nt = I.random_box(8, 8, 16, p_solid=0.2, seed=3)
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(0.8)
        L.init_equilibrium()
        assert lbm.lbm_halo_bytes(L.ctx, 0, True) == 0
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_halo_pack(L.ctx, 0, np.zeros(1))
        assert e.value.status == 5                                # LBM_ESTATE
    ctx = lbm.lbm_create_slab(nt, lbm.DTYPES["f64"], 0b011, 0, 2)  # bottom slab, z not periodic
    try:
        import torch
        lbm.lbm_set_params(ctx, 0.8)
        lbm.lbm_init_equilibrium(ctx)
        n = lbm.lbm_halo_bytes(ctx, 1, True)
        assert n > 0
        for bad in (np.zeros(n, np.uint8), torch.zeros(n, dtype=torch.uint8),
                    torch.zeros(n - 1, dtype=torch.uint8, device="cuda")):
            with pytest.raises(ValueError):                       # refused before the call
                lbm.lbm_halo_pack(ctx, 1, bad)
        lbm.lbm_set_params(ctx, 0.8)
        lbm.lbm_init_equilibrium(ctx)
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_halo_unpack(ctx, 0, np.zeros(1))              # no slab below
        assert e.value.status == 5
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_adjoint(ctx, 4, 2, 1)
        assert e.value.status == 4                                # LBM_EUNSUPPORTED
    finally:
        lbm.lbm_destroy(ctx)

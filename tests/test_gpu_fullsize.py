"""Full-size parity of every instantiation of the step kernel (Sec. 3.4, Algorithm 2).

The step kernel is persistent: each CTA walks work groups b, b + G, b + 2G, ... through
rings of staging slots (headers, neighbour records and words, gathered data) that only
wrap when a CTA walks more than one group. The small-box parity tests have fewer groups
than resident CTAs, so they never reach that regime. Here every storage format,
collision model and boundary scheme runs on a 256^3-class geometry in the launch
configuration of the benchmark, where every CTA walks tens of groups.

Method (as for the FP64 LBGK case in test_gpu_parity): after some steps from a flow
with u ~ 0.05 (far from rest, so every term of the collision matters), 10^3 boxes are
exported before and after one more step. The oracle steps each box as its own
non-periodic problem; nodes whose 19 sources lie inside the box (the interior, plus the
box faces that are domain faces: a moving lid, an inlet or outlet plane) have the same
update there as in the full problem, and are compared.

Bars, per population, relative to the lattice weight w_i:
  - FP64 storage (hybrid and all-FP64 arithmetic, every model): 1e-12;
  - FP32 storage: 1e-6. The step stores h = f - w in FP32 and computes on h in FP32;
    each result carries ~3 roundings of 2^-24 relative of terms no larger than ~0.4 w
    (the equilibrium part w(drho + 3 c.j) at u ~ 0.05), about 1e-7 w. Zou-He boundary
    nodes: 4e-6 (the bar of the small-box Zou-He tests). The completion forms rho and
    the unknown populations from sums of known ones, terms of order 1 in f, so its
    roundings are ~1e-7 absolute, a few 1e-6 of the diagonal weight 1/36;
  - FP16 storage: the rounding of the stored value itself, in spacings of binary16 at
    h_oracle * 2^12: stochastic rounding, which picks either neighbour, one spacing;
    round-to-nearest half a spacing, except that the rounding carries the node's mass
    and momentum residues into directions 1-6 (each takes half its axis' residue: at most
    S / 2, S the sum of all 19 half spacings) and 0 (the mass residue: at most 2 S); plus
    the FP32 arithmetic bound above;
  - the calibration kernels (propagation only, read/write only): bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02445_gb300 import build as B
from paper_1611_02445_gb300 import inputs as I
from paper_1611_02445_gb300 import lbm

pytestmark = pytest.mark.gpu

_, W, _ = O.lattice()
F64_TOL = 1e-12
F32_TOL = 1e-6
ZOU_HE_F32_TOL = 4e-6
U0 = (0.05, -0.02, 0.03)     # initial uniform velocity: bounce-back makes it non-equilibrium
N = 256


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    lbm.load()


@pytest.fixture(scope="module")
def pack():
    return I.sphere_pack(N, 8.0, 0.35, I.SEED_POROUS_256)


def _corners(n, dims, seed):
    rng = np.random.default_rng(seed)
    out = [tuple(int(rng.integers(0, d)) for d in dims) for _ in range(n)]
    return out + [tuple(d - 6 for d in dims), (0, 0, 0)]   # two across the periodic seams


def _crop(a, x0, y0, z0, sx, sy, sz, wrap=True):
    """a[..., z, y, x] over the box, indices wrapped (periodic) or clipped."""
    nz, ny, nx = a.shape[-3:]
    zi, yi, xi = np.arange(z0, z0 + sz), np.arange(y0, y0 + sy), np.arange(x0, x0 + sx)
    if wrap:
        zi, yi, xi = zi % nz, yi % ny, xi % nx
    return a[..., zi[:, None, None], yi[None, :, None], xi[None, None, :]]


def _f16_bound(fo, w):
    """Half a binary16 spacing of h * 2^12 (in f units) per element, h = f - w."""
    x = np.abs((fo - w) * 4096.0)
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -14)))
    return 0.5 * 2.0 ** (e - 10) / 4096.0


def _check(dtype, Bg, Bo, f32_tol=F32_TOL):
    w = W[:, None]
    err = np.abs(Bg - Bo)
    if dtype in ("f64", "f64n"):
        worst = float((err / w).max())
        assert worst <= F64_TOL, worst
    elif dtype == "f32":
        worst = float((err / w).max())
        assert worst <= f32_tol, worst
    else:
        half = _f16_bound(Bo, w)
        if dtype == "f16sr":
            bound = 2.0 * half                        # one spacing: either neighbour
        else:
            S = half.sum(axis=0)                      # per node: all 19 half spacings
            bound = half.copy()
            bound[1:7] += 0.5 * S                     # half an axis' residue each
            bound[0] += 2.0 * S                       # the mass residue
        bound = bound + F32_TOL * w
        worst = float((err / bound).max())
        assert worst <= 1.0, worst
    return worst


def _sampled(L, boxes, oracle_step, dtype, steps_before=12, f32_tol=F32_TOL):
    """boxes: list of (x0, y0, z0, sx, sy, sz, inner) with inner a boolean [sz, sy, sx]
    mask of the compared nodes (before the solid mask)."""
    L.step(steps_before)
    before = [L.get_f_box(*b[:6]) for b in boxes]
    L.step(1)
    after = [L.get_f_box(*b[:6]) for b in boxes]
    worst, compared = 0.0, 0
    for b, A, Bg in zip(boxes, before, after):
        Bo = oracle_step(A, b)
        m = b[6] & np.isfinite(A[0])
        if m.any():
            worst = max(worst, _check(dtype, Bg[:, m], Bo[:, m], f32_tol))
            compared += int(m.sum())
    assert compared > 1000, compared
    return worst


def _interior(s=10):
    m = np.zeros((s, s, s), bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def _periodic_boxes(dims, seed, n=12):
    return [(x - 1, y - 1, z - 1, 10, 10, 10, _interior()) for (x, y, z) in _corners(n, dims, seed)]


# ------------------------------------------------ porous pack, every storage format
@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32", "f16s", "f16sr"])
def test_porous_256_every_format(pack, dtype):
    """FP64 hybrid and all-FP64 arithmetic, FP32, FP16 round-to-nearest and stochastic
    rounding, LBGK + Guo with a force that has y and z components (for FP64 storage the
    general form of the hybrid collision; test_gpu_parity's full-size FP64 test runs the
    form for a force along x)."""
    tau, g = 0.7, (1e-5, 2e-6, -1e-6)
    with lbm.Lattice(pack, dtype, 0b111) as L:
        L.set_params(tau, g)
        L.init_equilibrium(1.0, U0)
        worst = _sampled(L, _periodic_boxes(pack.shape[::-1], 1),
                         lambda A, b: O.step(A, _crop(pack, *b[:6]), 0, tau, g), dtype)
    print(f"porous 256^3 {dtype}: worst {worst:.3e} of the bar")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_porous_256_per_node_force(pack, dtype):
    """A per-node x force field (the force is staged per node by the kernel)."""
    tau, g = 0.8, (0.0, 1e-6, 0.0)
    rng = np.random.default_rng(7)
    gf = 1e-5 + 1e-6 * rng.standard_normal(pack.shape)
    with lbm.Lattice(pack, dtype, 0b111) as L:
        L.set_params(tau, g, gf)
        L.init_equilibrium(1.0, U0)
        worst = _sampled(L, _periodic_boxes(pack.shape[::-1], 2),
                         lambda A, b: O.step(A, _crop(pack, *b[:6]), 0, tau, g, _crop(gf, *b[:6])), dtype)
    print(f"porous 256^3 per-node force {dtype}: worst {worst:.3e} of the bar")


@pytest.mark.parametrize("dtype", ["f64", "f64n", "f32", "f16s"])
@pytest.mark.parametrize("eq,coll", [(O.EQ_INCOMPR, O.COLL_BGK), (O.EQ_QCOMPR, O.COLL_MRT),
                                     (O.EQ_INCOMPR, O.COLL_MRT)])
def test_porous_256_collision_models(pack, eq, coll, dtype):
    """The incompressible equilibrium (Eq. 4) and the MRT collision (Eq. 8)."""
    tau, g = 0.7, (1e-5, 0.0, 0.0)
    rates = O.mrt_rates(tau) if coll == O.COLL_MRT else None
    with lbm.Lattice(pack, dtype, 0b111) as L:
        L.set_params(tau, g)
        L.set_model(eq, coll)
        L.init_equilibrium(1.0, U0)
        worst = _sampled(L, _periodic_boxes(pack.shape[::-1], 3),
                         lambda A, b: O.step_m(A, _crop(pack, *b[:6]), 0, tau, g, eq=eq, coll=coll, rates=rates),
                         dtype)
    print(f"porous 256^3 eq {eq} coll {coll} {dtype}: worst {worst:.3e} of the bar")


# ------------------------------------------------------ dense cavity with moving lid
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cavity_256_moving_lid(dtype):
    """Dense 256^3 closed box (no dropped tiles, every group full), the face z = nz moving
    along x and y: boxes in the bulk and boxes whose top face is the lid."""
    nt = np.ones((N, N, N), np.uint8)
    tau, u_lid = 0.6, (0.08, 0.03, 0.0)
    top = np.zeros((10, 10, 10), bool)
    top[1:, 1:-1, 1:-1] = True                      # bottom halo row excluded, lid row kept
    boxes = [b for b in _periodic_boxes((N, N, N), 4) if 0 < b[2] and b[2] + 10 <= N and
             0 < b[0] and b[0] + 10 <= N and 0 < b[1] and b[1] + 10 <= N]
    boxes += [(x, y, N - 10, 10, 10, 10, top) for (x, y) in ((5, 7), (N // 2 - 8, 3 * N // 4), (N - 11, 3))]
    with lbm.Lattice(nt, dtype, 0) as L:
        L.set_params(tau)
        L.set_lid(5, u_lid)
        L.init_equilibrium(1.0, U0)

        def ostep(A, b):
            lid = 5 if b[2] + b[5] == N else -1
            return O.step_m(A, _crop(nt, *b[:6], wrap=False), 0, tau, lid_face=lid, lid_u=u_lid)

        worst = _sampled(L, boxes, ostep, dtype)
    print(f"cavity 256^3 lid {dtype}: worst {worst:.3e} of the bar")


# ------------------------------------- a context beyond the 32-bit gather indices
def test_cavity_512_fp64_with_64bit_gather_indices():
    """Dense 512^3 closed box with the lid, FP64 (41 GB for the two copies): 134 M nodes in
    full groups, so a copy has 512^3 * 19 > 2^31 elements and the step forms its gather
    indices in 64 bits (the instantiation every smaller context leaves unused)."""
    n = 512
    assert n ** 3 * 19 >= 2 ** 31
    nt = np.ones((n, n, n), np.uint8)
    tau, u_lid = 0.6, (0.08, 0.03, 0.0)
    top = np.zeros((10, 10, 10), bool)
    top[1:, 1:-1, 1:-1] = True
    boxes = [b for b in _periodic_boxes((n, n, n), 5) if 0 < b[2] and b[2] + 10 <= n and
             0 < b[0] and b[0] + 10 <= n and 0 < b[1] and b[1] + 10 <= n]
    boxes += [(x, y, n - 10, 10, 10, 10, top) for (x, y) in ((5, 7), (n // 2 - 8, 3 * n // 4), (n - 11, 3))]
    # a box in the last tiles of the copy, where the 64-bit indices are largest
    boxes += [(n - 11, n - 11, n - 21, 10, 10, 10, _interior())]
    with lbm.Lattice(nt, "f64", 0) as L:
        assert L.info()["n_nonsolid"] == n ** 3
        L.set_params(tau)
        L.set_lid(5, u_lid)
        L.init_equilibrium(1.0, U0)

        def ostep(A, b):
            lid = 5 if b[2] + b[5] == n else -1
            return O.step_m(A, _crop(nt, *b[:6], wrap=False), 0, tau, lid_face=lid, lid_u=u_lid)

        worst = _sampled(L, boxes, ostep, "f64", steps_before=4)
    print(f"cavity 512^3 lid f64 (64-bit gather indices): worst {worst:.3e} of the bar")


# ----------------------------------------------- Zou-He duct longer than the grid
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_zou_he_duct_many_groups(dtype):
    """A 256 x 64 x 64 duct (16 384 tiles: many work groups per CTA) with walls at y = 0,
    ny - 1, periodic in z, Zou-He velocity inlet at x = 0 and pressure outlet at
    x = nx - 1; boxes at the inlet, in the bulk and at the outlet."""
    nx, ny, nz = 256, 64, 64
    nt = np.ones((nz, ny, nx), np.uint8)
    nt[:, 0, :] = 0
    nt[:, ny - 1, :] = 0
    nt[:, 1:ny - 1, 0] = 2
    nt[:, 1:ny - 1, nx - 1] = 3
    tau, u_in, rho_out = 0.7, (0.04, 0.0, 0.0), 1.0
    inlet = np.zeros((10, 10, 10), bool)
    inlet[1:-1, 1:-1, :-1] = True                   # x = 0 face kept, far halo dropped
    outlet = np.zeros((10, 10, 10), bool)
    outlet[1:-1, 1:-1, 1:] = True
    boxes = [(0, 20, 30, 10, 10, 10, inlet), (0, 0, 60, 10, 10, 10, inlet),
             (nx - 10, 40, 5, 10, 10, 10, outlet), (nx - 10, 54, 62, 10, 10, 10, outlet),
             (100, 10, 20, 10, 10, 10, _interior()), (200, 50, 60, 10, 10, 10, _interior())]
    with lbm.Lattice(nt, dtype, 0b100) as L:
        L.set_params(tau, None, None, u_in, rho_out)
        L.set_bc(lbm.BC_ZOU_HE, 0, 1)
        L.init_equilibrium(1.0, (0.04, 0.0, 0.0))

        def ostep(A, b):
            # inlet boxes start at x = 0 and outlet boxes end at x = nx - 1: the box's own
            # faces 0 and 1 are the domain's inlet and outlet planes
            return O.step_m(A, _crop(nt, *b[:6]), 0, tau, u_in=u_in, rho_out=rho_out, bc=O.BC_ZOU_HE,
                            in_face=0, out_face=1)

        worst = _sampled(L, boxes, ostep, dtype, steps_before=30, f32_tol=ZOU_HE_F32_TOL)
    print(f"Zou-He duct {dtype}: worst {worst:.3e} of the bar")


# ------------------------------------------------------- calibration kernels
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_calibration_kernels_full_size(pack, dtype):
    """Propagation only equals the oracle's streaming with bounce-back (tau = inf, no
    force) bit for bit; read/write only leaves every node's values as they were."""
    import math
    with lbm.Lattice(pack, dtype, 0b111) as L:
        L.set_params(0.7, (1e-5, 0, 0))
        L.init_equilibrium(1.0, U0)
        L.step(8)
        boxes = _periodic_boxes(pack.shape[::-1], 5)
        before = [L.get_f_box(*b[:6]) for b in boxes]
        L.step_kernel(lbm.KERNEL_PROPAGATE, 1)
        after = [L.get_f_box(*b[:6]) for b in boxes]
        for b, A, Bg in zip(boxes, before, after):
            Bo = O.step(A, _crop(pack, *b[:6]), 0, math.inf)
            m = b[6] & np.isfinite(A[0])
            assert np.array_equal(Bg[:, m], Bo[:, m])
        L.step_kernel(lbm.KERNEL_RW, 3)
        again = [L.get_f_box(*b[:6]) for b in boxes]
        for Bg, Bh in zip(after, again):
            assert np.array_equal(Bg, Bh, equal_nan=True)

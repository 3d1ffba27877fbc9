"""GPU parity: the CUDA library, called through its C ABI, against the FP64 oracle.

Bars
  - tile map and nonEmptyTiles: bit-exact (integer work);
  - FP64 storage: max over non-solid nodes and directions of |f_gpu - f_oracle| / w_i
    <= 1e-12 after the stated number of steps (the fused kernel contracts multiply-adds
    and sums in a different order, so results are not bit-identical);
  - FP32 / FP16-shifted storage: bounds derived from the storage rounding (see each test).
Sizes span several tiles, ragged (padded) tails, every periodic mask, inlet and outlet
nodes and per-node forces.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    lbm.load()


def rel_err(fg, fo, nt):
    m = nt != 0
    if not m.any():
        return 0.0
    return float((np.abs(fg[:, m] - fo[:, m]) / W[:, None]).max())


def run_pair(nt, f0, steps, periodic, tau, g=(0, 0, 0), g_field=None, u_in=(0, 0, 0), rho_out=1.0,
             dtype="f64"):
    with lbm.Lattice(nt, dtype, periodic) as L:
        L.set_params(tau, g, g_field, u_in, rho_out)
        L.set_f(f0)
        L.step(steps)
        fg = L.get_f()
        red = L.reduce()
        rho_g, u_g = L.macroscopic()
    fo = O.run(f0, nt, steps, periodic, tau, g, g_field, u_in, rho_out)
    return fg, fo, red, (rho_g, u_g)


# ------------------------------------------------------------------- tile builder
@pytest.mark.parametrize("shape,p_solid,seed", [
    ((8, 8, 8), 0.5, 0), ((13, 9, 11), 0.9, 1), ((33, 17, 5), 0.97, 2), ((1, 1, 1), 0.0, 3),
    ((64, 32, 48), 0.995, 4), ((7, 40, 3), 0.8, 5)])
def test_tile_map_bit_exact(shape, p_solid, seed):
    nx, ny, nz = shape
    nt = I.random_box(nx, ny, nz, p_solid=p_solid, seed=seed, boundary=True)
    tm_o, ne_o = O.tiling(nt)
    with lbm.Lattice(nt, "f64", 0) as L:
        tm_g, ne_g = L.tiles()
        info = L.info()
    assert np.array_equal(tm_g, tm_o)
    assert np.array_equal(ne_g, ne_o)
    assert info["n_tiles"] == len(ne_o)
    assert info["n_nonsolid"] == int(np.count_nonzero(nt))


def test_tile_map_all_solid_and_all_fluid():
    nt = np.zeros((12, 8, 16), np.uint8)
    with lbm.Lattice(nt, "f64", 0b111) as L:
        tm, ne = L.tiles()
        assert len(ne) == 0 and (tm == -1).all()
        L.set_params(0.8)
        L.init_equilibrium()
        L.step(3)
        assert L.reduce()[0] == 0.0
    nt = I.dense_box(16, 8, 12)
    tm_o, ne_o = O.tiling(nt)
    with lbm.Lattice(nt, "f64", 0) as L:
        tm, ne = L.tiles()
    assert np.array_equal(tm, tm_o) and np.array_equal(ne, ne_o)


def test_tile_map_vessel_shape():
    nt = I.vessel_tree(128, 64, 64, seed=3, root_radius=6.0, length_factor=4.0)
    tm_o, ne_o = O.tiling(nt)
    with lbm.Lattice(nt, "f32", 0) as L:
        tm, ne = L.tiles()
    assert np.array_equal(tm, tm_o) and np.array_equal(ne, ne_o)


# ------------------------------------------------------------------ FP64 step
FP64_MODES = ["f64", "f64n"]


@pytest.mark.parametrize("dtype", FP64_MODES)
@pytest.mark.parametrize("periodic", [0b000, 0b111, 0b101, 0b010])
@pytest.mark.parametrize("g", [(1e-5, 2e-6, -3e-6), (1e-5, 0.0, 0.0)])
def test_f64_step_random_box(periodic, dtype, g):
    """A per-node x force with a uniform y, z force, or none (the hybrid FP64 collision's
    form for a force along x)."""
    rng = np.random.default_rng(periodic)
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=periodic + 50, boundary=True)
    nt[:4, :4, :4] = I.SOLID
    f0 = I.random_populations(nt, 0.05, seed=periodic)
    gf = 1e-5 * (1 + 0.1 * rng.standard_normal(nt.shape))
    fg, fo, red, _ = run_pair(nt, f0, 100, periodic, 0.7, g, gf, (0.05, 0.01, 0.0), 1.0, dtype=dtype)
    assert rel_err(fg, fo, nt) <= F64_TOL
    # solid nodes stay NaN in the export
    assert np.isnan(fg[:, nt == 0]).all()


@pytest.mark.parametrize("dtype", FP64_MODES)
@pytest.mark.parametrize("g", [(1e-5, 2e-6, -3e-6), (1e-5, 0.0, 0.0)])
def test_f64_step_populations_outside_fast_conversion_range(dtype, g):
    """At 40 % of the nodes three diagonal populations are set between -0.05 w and 0.5 w,
    below 2^-6 and some negative: the hybrid collision then forms the node's moments
    with its fallback conversion, in the first steps until the collision has relaxed
    them; the velocity stays small, so the rest of its arithmetic is unchanged."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=77, boundary=True)
    f0 = I.random_populations(nt, 0.05, seed=77)
    rng = np.random.default_rng(77)
    pick = (rng.random(nt.shape) < 0.4) & (nt != 0)
    for i in (9, 14, 18):
        f0[i][pick] = W[i] * rng.uniform(-0.05, 0.5, size=int(pick.sum()))
    assert (f0[:, nt != 0] < 2.0 ** -6).any() and (f0[:, nt != 0] < 0).any()
    for steps in (1, 20):
        fg, fo, _, _ = run_pair(nt, f0, steps, 0b111, 0.7, g, dtype=dtype)
        assert rel_err(fg, fo, nt) <= F64_TOL


@pytest.mark.parametrize("dtype", FP64_MODES)
@pytest.mark.parametrize("shape", [(13, 9, 11), (5, 6, 7), (4, 4, 4), (21, 3, 9)])
def test_f64_step_ragged_nonperiodic(shape, dtype):
    nx, ny, nz = shape
    nt = I.random_box(nx, ny, nz, p_solid=0.2, seed=nx, boundary=False)
    f0 = I.random_populations(nt, 0.05, seed=1)
    fg, fo, _, _ = run_pair(nt, f0, 60, 0, 0.9, (2e-5, 0, 0), dtype=dtype)
    assert rel_err(fg, fo, nt) <= F64_TOL


@pytest.mark.parametrize("dtype", FP64_MODES)
def test_f64_poiseuille_1000_steps(dtype):
    nt = I.poiseuille_channel(32, 32, 32)
    f0 = O.init(nt)
    fg, fo, red, (rho_g, u_g) = run_pair(nt, f0, 1000, 0b101, 0.8, (1e-6, 0, 0), dtype=dtype)
    assert rel_err(fg, fo, nt) <= F64_TOL
    m0 = np.count_nonzero(nt)
    assert abs(red[0] - m0) / m0 <= 1e-12
    rho_o, u_o = O.macroscopic(fo, nt, g=(1e-6, 0, 0))
    assert np.abs(u_g - u_o).max() <= 1e-12
    assert np.abs(rho_g - rho_o).max() <= 1e-12


@pytest.mark.parametrize("dtype,tol", [("f64n", 1e-15), ("f64", 1e-13)])
def test_f64_equilibrium_fixed_point(dtype, tol):
    """FP64 arithmetic keeps the rest state to rounding (1e-15). The double-float
    equilibrium term carries ~2^-45 relative error per step, and (1 - 1/tau) f + Y maps
    it to a fixed point within ~2^-45 (3e-14) of w; the bound is tol * w_i."""
    nt = I.random_box(16, 12, 8, p_solid=0.4, seed=9)
    with lbm.Lattice(nt, dtype, 0b011) as L:
        L.set_params(0.65)
        L.init_equilibrium(1.0)
        f0 = L.get_f()
        L.step(100)
        f1 = L.get_f()
    m = nt != 0
    assert (np.abs(f1[:, m] - f0[:, m]) / W[:, None]).max() <= tol


def test_f64_reduce_and_macroscopic_match_oracle():
    rng = np.random.default_rng(3)
    nt = I.random_box(16, 12, 20, p_solid=0.3, seed=77, boundary=True)
    f0 = I.random_populations(nt, 0.05, seed=4)
    gf = 1e-4 * (1 + 0.1 * rng.standard_normal(nt.shape))
    g = (0.0, 1e-5, 2e-5)
    fg, fo, (mass, mom), (rho_g, u_g) = run_pair(nt, f0, 10, 0b111, 0.8, g, gf, (0.03, 0, 0), 1.0)
    m_o, p_o = O.reduce(fo, nt, g, gf)
    assert abs(mass - m_o) <= 1e-12 * abs(m_o)
    assert np.abs(mom - p_o).max() <= 1e-12 * abs(m_o)
    rho_o, u_o = O.macroscopic(fo, nt, g, gf)
    assert np.abs(rho_g - rho_o).max() <= 1e-12
    assert np.abs(u_g - u_o).max() <= 1e-12
    # float output path
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(0.8, g, gf, (0.03, 0, 0))
        L.set_f(fo)
        rho32, u32 = L.macroscopic(out_f64=False)
    assert rho32.dtype == np.float32
    assert np.abs(rho32 - rho_o).max() <= 1e-6 and np.abs(u32 - u_o).max() <= 1e-7


def test_mass_conservation_gpu():
    nt = I.random_box(24, 16, 20, p_solid=0.3, seed=12)
    with lbm.Lattice(nt, "f64", 0b101) as L:
        L.set_params(0.7, (1e-4, 0, 0))
        L.init_equilibrium()
        m0, _ = L.reduce()
        L.step(200)
        m1, _ = L.reduce()
    assert abs(m1 - m0) / m0 <= 1e-12


# ----------------------------------------------------------- reduced precision
@pytest.mark.parametrize("dtype,tol", [("f32", 1e-6), ("f16s", 2e-3), ("f16sr", 2e-3)])
def test_reduced_precision_step(dtype, tol):
    """Both reduced formats store and compute h = f - w, of size ~0.05 w here. FP32 rounds
    each of the ~3 operations behind an output to 2^-24 relative of at most ~0.3 w, about
    5e-8 w a step; FP16 storage rounds h to 2^-11 relative. Over 20 steps the bounds are
    20 * 5e-8 = 1e-6 (f32) and 20 * 0.05 * 4.9e-4 ~ 5e-4 (f16s), with a safety factor."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=5, boundary=True)
    f0 = I.random_populations(nt, 0.05, seed=2)
    fg, fo, _, _ = run_pair(nt, f0, 20, 0b111, 0.8, (1e-5, 0, 0), None, (0.05, 0, 0), 1.0, dtype=dtype)
    err = rel_err(fg, fo, nt)
    print(f"{dtype}: max |f - f_oracle| / w = {err:.3e}")
    assert err <= tol


# ------------------------------------------------------------------ edge cases
def test_single_node_box_bounces_everything():
    nt = np.ones((1, 1, 1), np.uint8)
    f0 = I.random_populations(nt, 0.1, seed=8)
    fg, fo, _, _ = run_pair(nt, f0, 7, 0, 0.8, (1e-5, 0, 0))
    assert rel_err(fg, fo, nt) <= F64_TOL


def test_state_roundtrip_and_mismatch():
    nt = I.random_box(8, 8, 8, p_solid=0.3, seed=2)
    with lbm.Lattice(nt, "f32", 0b111) as L:
        L.set_params(0.8)
        L.init_equilibrium()
        L.step(5)
        blob = L.save_state()
        f5 = L.get_f()
        L.step(5)
        L.load_state(blob)
        assert np.array_equal(L.get_f(), f5, equal_nan=True)
        bad = bytearray(blob)
        bad[-1] ^= 0xFF
        with pytest.raises(lbm.LBMError) as e:
            L.load_state(bytes(bad))
        assert e.value.status == 5
    nt2 = nt.copy()
    nt2[0, 0, 0] = 1 - min(nt2[0, 0, 0], 1)
    with lbm.Lattice(nt2, "f32", 0b111) as L2:
        with pytest.raises(lbm.LBMError) as e:
            L2.load_state(blob)
        assert e.value.status == 5


def _padded_lanes(nt, ne, max_tiles):
    """Padded lane of every (tile, slot) in the grouped layout the library documents: kept
    tiles in rank order cut greedily into groups of at most max_tiles tiles and 256
    non-solid nodes, a tile's nodes on consecutive lanes in slot order; -1 for solid and
    padding slots."""
    nz, ny, nx = nt.shape
    Tx, Ty = (nx + 3) // 4, (ny + 3) // 4
    s = np.arange(64)
    t = ne.astype(np.int64)[:, None]
    x = 4 * (t % Tx) + (s & 3)
    y = 4 * ((t // Tx) % Ty) + ((s >> 2) & 3)
    z = 4 * (t // (Tx * Ty)) + (s >> 4)
    inside = (x < nx) & (y < ny) & (z < nz)
    nonsolid = np.zeros_like(inside)
    nonsolid[inside] = nt[z[inside], y[inside], x[inside]] != 0
    lanes = -np.ones(nonsolid.shape, np.int64)
    group, used, tiles = 0, 0, 0
    for k in range(len(ne)):
        cnt = int(nonsolid[k].sum())
        if tiles == max_tiles or used + cnt > 256:
            group, used, tiles = group + 1, 0, 0
        lanes[k, nonsolid[k]] = 256 * group + used + np.arange(cnt)
        used += cnt
        tiles += 1
    return lanes, group + 1, (x, y, z)


@pytest.mark.parametrize("dtype", ["f32", "f64", "f16s"])
def test_grouped_layout_and_padding_lanes(dtype):
    """The raw copy (the payload of a saved state) is laid out as documented: storage group
    g holds one 256-lane data block per direction, f_i of the node on padded lane P at
    (P // 256, i, P % 256). Every non-solid node's value there is the one lbm_get_f exports,
    and after any number of steps, single launches or graph replays, the padding lanes of
    the groups still hold the zeros they were created with: the step writes only its
    nodes' lanes."""
    nt = I.random_box(13, 10, 9, p_solid=0.45, seed=11)          # ragged: padding slots too
    elem, uint = {"f32": (np.float32, np.uint32), "f64": (np.float64, np.uint64),
                  "f16s": (np.float16, np.uint16)}[dtype]
    with lbm.Lattice(nt, dtype, 0) as L:                          # ragged axes cannot be periodic
        L.set_params(0.7, g=(1e-5, 0.0, 0.0))
        L.init_equilibrium()
        _, ne = L.tiles()
        lanes, n_groups, (x, y, z) = _padded_lanes(nt, ne, 16 if dtype == "f64" else 8)
        assert (lanes >= 0).any() and (lanes < 0).any()
        assert L.info()["copy_bytes"] == n_groups * 19 * 256 * np.dtype(elem).itemsize
        for steps in (1, 1, 2, 16, 17):
            L.step(steps)
            blob = L.save_state()
            size = n_groups * 19 * 256 * np.dtype(elem).itemsize
            f = np.frombuffer(blob[len(blob) - size:], dtype=elem).reshape(n_groups, 19, 256)
            flat = f.transpose(0, 2, 1).reshape(n_groups * 256, 19)      # [padded lane][direction]
            used = np.zeros(n_groups * 256, bool)
            used[lanes[lanes >= 0]] = True
            assert (flat[~used].view(uint) == 0).all()
            assert np.isfinite(flat[used]).all()
            if dtype == "f64":
                fd = L.get_f()
                m = lanes >= 0
                assert np.array_equal(flat[lanes[m]], fd[:, z[m], y[m], x[m]].T)


def test_argument_errors():
    nt = np.ones((8, 8, 8), np.uint8)
    with lbm.Lattice(nt, "f64", 0) as L:
        with pytest.raises(lbm.LBMError) as e:
            L.set_params(0.5)
        assert e.value.status == 1
        with pytest.raises(lbm.LBMError) as e:
            L.step(1)
        assert e.value.status == 5          # no parameters and state yet
        L.set_params(0.8)
        L.init_equilibrium()
        L.step(1)                            # the context still works after argument errors
    bad = np.ones((8, 8, 8), np.uint8)
    bad[3, 3, 3] = 7
    with pytest.raises(lbm.LBMError) as e:
        lbm.Lattice(bad, "f64", 0)
    assert e.value.status == 1


# --------------------------------------------------- full size, sampled outputs
def _box(nt, x0, y0, z0, b):
    nz, ny, nx = nt.shape
    zi = np.arange(z0, z0 + b) % nz
    yi = np.arange(y0, y0 + b) % ny
    xi = np.arange(x0, x0 + b) % nx
    return nt[np.ix_(zi, yi, xi)]


def test_full_size_porous_sampled():
    """Porous 256^3 sphere pack (radius 8, porosity 0.35), FP64, in the benchmark's
    configuration: after 20 steps, boxes of 10^3 nodes (with a one-node halo) are
    exported before and after one more step; the oracle steps each box and the interior
    8^3 nodes are compared. Gathers of interior nodes stay inside the box, so the box
    problem equals the full periodic problem there."""
    nt = I.sphere_pack(256, 8.0, 0.35, I.SEED_POROUS_256)
    tau, g = 0.7, (1e-5, 0.0, 0.0)
    rng = np.random.default_rng(0)
    corners = [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(6)] + [(250, 250, 250), (0, 0, 0)]
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(tau, g)
        L.init_equilibrium()
        L.step(20)
        before = [L.get_f_box(x - 1, y - 1, z - 1, 10, 10, 10) for (x, y, z) in corners]
        L.step(1)
        after = [L.get_f_box(x - 1, y - 1, z - 1, 10, 10, 10) for (x, y, z) in corners]
    for (x, y, z), A, Bg in zip(corners, before, after):
        ntb = _box(nt, x - 1, y - 1, z - 1, 10)
        Bo = O.step(A, ntb, 0, tau, g)
        inner = np.zeros_like(ntb, dtype=bool)
        inner[1:-1, 1:-1, 1:-1] = ntb[1:-1, 1:-1, 1:-1] != 0
        err = float((np.abs(Bg[:, inner] - Bo[:, inner]) / W[:, None]).max()) if inner.any() else 0.0
        assert err <= F64_TOL


@pytest.mark.parametrize("dtype", FP64_MODES)
def test_vessel_crop_inlet_outlet_parity(dtype):
    """A small seeded vessel tree with the inlet velocity 0.05 and outlets, FP64."""
    nt = I.vessel_tree(96, 48, 48, seed=11, root_radius=5.0, length_factor=4.0)
    assert (nt == I.INLET).any() and (nt == I.OUTLET).any()
    f0 = O.init(nt)
    fg, fo, _, _ = run_pair(nt, f0, 100, 0, 0.6, (0, 0, 0), None, (0.05, 0, 0), 1.0, dtype=dtype)
    assert rel_err(fg, fo, nt) <= F64_TOL


# ------------------------------------------------- calibration kernels (Sec. 4.1)
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_propagation_only_kernel_is_pure_streaming(dtype):
    """With the collision left out the step is the streaming permutation with halfway
    bounce-back: the oracle's step with tau = inf and F = 0, bit for bit (on values already
    representable in the storage format). Fluid and solid nodes only: the oracle applies
    the inlet/outlet closures whatever tau is."""
    import math
    nt = I.random_box(12, 8, 16, p_solid=0.35, seed=31, boundary=False)
    f0 = I.random_populations(nt, 0.05, seed=32)
    with lbm.Lattice(nt, dtype, 0b101) as L:
        L.set_params(0.8)
        L.set_f(f0)
        f_in = L.get_f()                     # f0 rounded to the storage format
        L.step_kernel(lbm.KERNEL_PROPAGATE, 3)
        fg = L.get_f()
    fo = O.run(f_in, nt, 3, 0b101, math.inf)
    m = nt != 0
    assert np.array_equal(fg[:, m], fo[:, m])


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_read_write_only_kernel_is_identity(dtype):
    nt = I.random_box(12, 8, 16, p_solid=0.35, seed=33)
    f0 = I.random_populations(nt, 0.05, seed=34)
    with lbm.Lattice(nt, dtype, 0b111) as L:
        L.set_params(0.8)
        L.set_f(f0)
        f_in = L.get_f()
        L.step_kernel(lbm.KERNEL_RW, 5)
        fg = L.get_f()
    assert np.array_equal(fg, f_in, equal_nan=True)


def test_graph_replay_matches_single_launches():
    """lbm_step(n) replays a captured graph of 16 steps; the result equals n single steps."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=41)
    f0 = I.random_populations(nt, 0.05, seed=42)
    outs = []
    for chunk in (1, 37):
        with lbm.Lattice(nt, "f64", 0b111) as L:
            L.set_params(0.8, (1e-5, 0, 0))
            L.set_f(f0)
            for _ in range(37 // chunk):
                L.step(chunk)
            L.set_params(0.75, (1e-5, 0, 0))   # a parameter change drops the graphs
            L.step(33)
            outs.append(L.get_f())
    assert np.array_equal(outs[0], outs[1], equal_nan=True)

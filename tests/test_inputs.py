"""The seeded synthetic inputs: deterministic, shaped like the workloads they stand for,
and free of lattice-Boltzmann arithmetic (they serve both the oracle and the CUDA path).

The counts pinned here are the workload statistics the benchmark lines and the design
notes quote (non-solid nodes, kept 4^3 tiles, eta_t); a change to a generator or a seed
shows up here before it silently changes a benchmark.
"""
import ast
import os

import numpy as np
import pytest

from paper_1611_02445_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def kept_tiles(nt):
    """Number of 4^3 tiles (padded with solid nodes) holding a non-solid node."""
    nz, ny, nx = nt.shape
    pad = np.zeros(((nz + 3) // 4 * 4, (ny + 3) // 4 * 4, (nx + 3) // 4 * 4), np.uint8)
    pad[:nz, :ny, :nx] = nt
    Z, Y, X = (s // 4 for s in pad.shape)
    return int(pad.reshape(Z, 4, Y, 4, X, 4).any(axis=(1, 3, 5)).sum())


@pytest.mark.parametrize("n, seed, nonsolid, tiles", [
    (256, I.SEED_POROUS_256, 5_871_741, 167_327),     # the benchmark workload
    (128, I.SEED_POROUS_256, 732_512, 20_981),        # its 128^3 version (ncu captures)
])
def test_sphere_pack_statistics(n, seed, nonsolid, tiles):
    nt = I.sphere_pack(n, 8.0, 0.35, seed)
    assert nt.shape == (n, n, n) and nt.dtype == np.uint8
    assert set(np.unique(nt)) <= {I.SOLID, I.FLUID}
    assert int(np.count_nonzero(nt)) == nonsolid
    assert kept_tiles(nt) == tiles
    porosity = nonsolid / nt.size
    assert 0.345 <= porosity <= 0.35            # spheres are added until it first drops to 0.35
    assert 0.54 <= nonsolid / (64 * tiles) <= 0.55
    assert np.array_equal(nt, I.sphere_pack(n, 8.0, 0.35, seed))


def test_adjoint_pack_statistics():
    nt = I.sphere_pack(128, 8.0, 0.4, I.SEED_POROUS_128)      # the adjoint workload
    assert int(np.count_nonzero(nt)) == 837_863
    assert 0.395 <= np.count_nonzero(nt) / nt.size <= 0.4


def test_sphere_pack_is_periodic_and_seeded():
    a = I.sphere_pack(64, 8.0, 0.35, seed=5)
    b = I.sphere_pack(64, 8.0, 0.35, seed=6)
    assert not np.array_equal(a, b)
    # minimum-image spheres: solid regions wrap across every face, so opposite faces share
    # solid nodes in proportion to the solid fraction
    for ax in range(3):
        lo = np.take(a, 0, axis=ax) == I.SOLID
        hi = np.take(a, -1, axis=ax) == I.SOLID
        assert (lo & hi).mean() > 0.3


def test_vessel_tree_statistics():
    nt = I.vessel_tree(1024, 512, 512)
    assert nt.shape == (512, 512, 1024)
    assert int(np.count_nonzero(nt)) == 1_706_485
    assert kept_tiles(nt) == 34_709
    assert abs(np.count_nonzero(nt) / nt.size - 0.00636) < 5e-5
    inlet = nt == I.INLET
    assert inlet.any() and (nt == I.OUTLET).any()
    assert inlet[:, :, 1:].sum() == 0                 # inlets only on the x = 0 face
    # the root enters at the centre of the x = 0 face
    zs, ys = np.nonzero(inlet[:, :, 0])
    assert abs(zs.mean() - 256) < 2 and abs(ys.mean() - 256) < 2
    assert np.array_equal(nt, I.vessel_tree(1024, 512, 512))


def test_poiseuille_channel_and_random_box():
    ch = I.poiseuille_channel(32, 32, 32)
    assert (ch[:, 0, :] == I.SOLID).all() and (ch[:, -1, :] == I.SOLID).all()
    assert (ch[:, 1:-1, :] == I.FLUID).all()
    rb = I.random_box(13, 10, 9, p_solid=0.45, seed=11)
    assert rb.shape == (9, 10, 13)
    assert np.array_equal(rb, I.random_box(13, 10, 9, p_solid=0.45, seed=11))
    big = I.random_box(64, 64, 64, p_solid=0.3, seed=3)
    assert abs((big == I.SOLID).mean() - 0.3) < 0.01
    bc = I.random_box(16, 16, 16, p_solid=0.2, seed=4, boundary=True)
    assert (bc == I.INLET).any() and (bc == I.OUTLET).any()


def test_random_fields():
    nt = I.random_box(8, 8, 8, p_solid=0.3, seed=1)
    f = I.random_populations(nt, 0.05, seed=1)
    assert f.shape == (19, 8, 8, 8)
    assert np.isnan(f[:, nt == I.SOLID]).all()
    w = f[:, nt != I.SOLID]
    ref = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None]
    assert (np.abs(w / ref - 1.0) <= 0.05).all()
    g = I.body_force_field(I.sphere_pack(64, 8.0, 0.35, seed=2), 1e-5, 1e-7)
    assert abs(g.mean() - 1e-5) < 1e-9 and abs(g.std() - 1e-7) < 2e-9
    assert np.array_equal(g, I.body_force_field(I.sphere_pack(64, 8.0, 0.35, seed=2), 1e-5, 1e-7))


def test_inputs_module_holds_no_method_code():
    """The generators import nothing from the oracle or the CUDA binding."""
    tree = ast.parse(open(os.path.join(ROOT, "paper_1611_02445_gb300", "inputs.py")).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            names.add(node.module or "")
    assert names <= {"__future__", "math", "numpy"}, names

"""The allocation-free tile-map builder, checked against lbm_create's tile map.

lbm_build_tiles_noalloc is for callers that cannot allocate device memory -- code running
under a framework whose allocator already owns the GPU memory, or hosts that forbid
allocation once they have started. Such callers pass their own input and output
buffers; the builder's temporary storage comes from a static device array. This file
is collected last so that, if it fails, a run stopping at the first failure has already
run every other test. It passes alone in a fresh process and after the other tests.
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


def _grid(nt):
    nz, ny, nx = nt.shape
    return ((nz + 3) // 4, (ny + 3) // 4, (nx + 3) // 4)


def _noalloc(nt):
    import torch
    nz, ny, nx = nt.shape
    T = int(np.prod(_grid(nt)))
    d_nt = torch.from_numpy(np.ascontiguousarray(nt, dtype=np.uint8).reshape(-1)).cuda()
    tm = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    ne = torch.full((T,), -7, dtype=torch.int32, device="cuda")
    n = lbm.lbm_build_tiles_noalloc(d_nt, nx, ny, nz, tm, ne)
    torch.cuda.synchronize()
    return tm.cpu().numpy().reshape(_grid(nt)), ne.cpu().numpy().view(np.uint32)[:n].copy()


def _with_lbm_create(nt):
    with lbm.Lattice(nt, "f64", 0) as L:
        return L.tiles()


def test_noalloc_tiles_match_lbm_create_on_two_calls_in_a_row():
    big = I.random_box(37, 29, 23, p_solid=0.9, seed=1, boundary=True)
    small = I.random_box(13, 9, 11, p_solid=0.5, seed=2)
    # larger grid first: the second call starts from the scratch the first one left
    for nt in (big, small, small):
        tm, ne = _noalloc(nt)
        tm_ref, ne_ref = _with_lbm_create(nt)
        assert np.array_equal(tm, tm_ref)      # integer work: bit-exact
        assert np.array_equal(ne, ne_ref)
        tm_o, ne_o = O.tiling(nt)              # and against the oracle's Algorithm 1 directly
        assert np.array_equal(tm, tm_o) and np.array_equal(ne, ne_o)


def test_noalloc_error_flag_is_cleared_between_calls():
    import torch
    bad = np.ones((8, 8, 8), np.uint8)
    bad[5, 2, 1] = 9
    d_bad = torch.from_numpy(bad.reshape(-1)).cuda()
    tm = torch.empty(8, dtype=torch.int32, device="cuda")
    ne = torch.empty(8, dtype=torch.int32, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tiles_noalloc(d_bad, 8, 8, 8, tm, ne)
    assert e.value.status == 1
    good = I.random_box(8, 8, 8, p_solid=0.3, seed=4)
    tm_g, ne_g = _noalloc(good)
    tm_ref, ne_ref = _with_lbm_create(good)
    assert np.array_equal(tm_g, tm_ref) and np.array_equal(ne_g, ne_ref)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    import torch
    d = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    # 1028^3 nodes -> 257^3 tiles > 2^22: rejected before any device work
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_build_tiles_noalloc(d, 1028, 1028, 1028, out, out)
    assert e.value.status == 4
    assert "static scratch" in str(e.value)

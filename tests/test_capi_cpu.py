"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every entry
point declared in include/lbm.h, and rejects invalid arguments before touching the GPU."""
import ctypes as ct
import re

import numpy as np
import pytest

from paper_1611_02445_gb300 import build as B
from paper_1611_02445_gb300 import lbm


@pytest.fixture(scope="module")
def L():
    B.build()
    return lbm.load()


def test_header_declares_the_boundary():
    names = set(lbm.header_functions())
    for n in ("lbm_create", "lbm_destroy", "lbm_set_params", "lbm_init_equilibrium", "lbm_step",
              "lbm_macroscopic", "lbm_reduce", "lbm_get_f", "lbm_set_f", "lbm_get_f_box",
              "lbm_get_tiles", "lbm_get_info", "lbm_save_state", "lbm_load_state", "lbm_last_error",
              "lbm_set_stream"):
        assert n in names


def test_every_declared_symbol_is_exported(L):
    raw = ct.CDLL(lbm.library_path())
    for n in lbm.header_functions() + lbm.header_functions(lbm.TESTING_HEADER):
        assert hasattr(raw, n), n


def test_checked_library_builds_and_exports_the_same_symbols():
    path = B.build(checked=True)
    raw = ct.CDLL(path)
    for n in lbm.header_functions() + lbm.header_functions(lbm.TESTING_HEADER):
        assert hasattr(raw, n), n
    raw.lbm_testing_checked_build.restype = ct.c_int
    assert raw.lbm_testing_checked_build() == 1
    assert L_checked_flag(lbm.load()) == 0


def L_checked_flag(L):
    return int(L.lbm_testing_checked_build())


def test_injected_allocation_failure_reports_enomem_and_leaks_nothing(L):
    """The host-side hook fails the next device allocation the way cudaMalloc does when
    memory runs out: lbm_create releases what it holds and returns LBM_ENOMEM."""
    nt = np.ones((8, 8, 8), np.uint8)
    live = lbm.testing_live_allocations()
    lbm.testing_fail_allocation(0)
    try:
        st, ctx = _create(L, nt, (8, 8, 8))
    finally:
        lbm.testing_fail_allocation(-1)
    assert st == 2 and ctx is None                            # LBM_ENOMEM, no context
    assert "memory" in L.lbm_last_error(None).decode()
    assert lbm.testing_live_allocations() == live


def test_build_targets_sm_103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _create(L, nt, dims, tile=4, dtype=0, periodic=0):
    out = ct.c_void_p()
    st = L.lbm_create(nt.ctypes.data if nt is not None else None, 0, *dims, tile, dtype, periodic, None,
                      ct.byref(out))
    return st, out.value


def test_argument_validation_without_gpu(L):
    nt = np.ones((8, 8, 8), np.uint8)
    assert _create(L, nt, (8, 8, 8), tile=5)[0] == 4          # LBM_EUNSUPPORTED
    assert "4x4x4" in L.lbm_last_error(None).decode()
    assert _create(L, nt, (0, 8, 8))[0] == 1                   # LBM_EINVAL
    assert _create(L, nt, (6, 8, 8), periodic=1)[0] == 1        # periodic axis not a multiple of 4
    assert _create(L, nt, (8, 8, 8), dtype=7)[0] == 1
    assert _create(L, nt, (8, 8, 8), periodic=8)[0] == 1
    assert _create(L, None, (8, 8, 8))[0] == 1
    out = ct.c_void_p()
    assert L.lbm_create(nt.ctypes.data, 0, 8, 8, 8, 4, 0, 0, None, None) == 1
    assert L.lbm_step(None, 1) == 1
    assert L.lbm_last_error(None) is not None
    L.lbm_destroy(None)


def test_axis_near_int_max_is_rejected_before_any_device_work(L):
    """Tile counts are formed in 64 bits: an axis of INT_MAX nodes must not wrap to a
    negative tile count and reach a launch."""
    big = 2 ** 31 - 1
    nt = np.ones(8, np.uint8)
    assert _create(L, nt, (big, big, big))[0] == 1                 # LBM_EINVAL: > 2^31 tiles
    assert "2^31" in L.lbm_last_error(None).decode()
    n = ct.c_int64(-5)
    for dims in ((big, 1, 1), (1, big, 1), (big, big, big)):
        st = L.lbm_build_tiles_noalloc(nt.ctypes.data, *dims, nt.ctypes.data, nt.ctypes.data, ct.byref(n), None)
        assert st == 4                                           # LBM_EUNSUPPORTED, before device work
    assert n.value == -5


def test_noalloc_binding_checks_buffers_before_the_call():
    """The C entry point takes raw device pointers; the binding refuses host arrays, CPU
    tensors, wrong dtypes and undersized buffers before anything is launched."""
    import torch
    nx, ny, nz = 9, 8, 8                                          # 3 x 2 x 2 = 12 tiles
    nt = torch.ones(nx * ny * nz, dtype=torch.uint8)
    tm = torch.zeros(12, dtype=torch.int32)
    ne = torch.zeros(12, dtype=torch.int32)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lbm.lbm_build_tiles_noalloc(nt.numpy(), nx, ny, nz, tm, ne)
    with pytest.raises(ValueError, match="CUDA tensor"):
        lbm.lbm_build_tiles_noalloc(nt, nx, ny, nz, tm, ne)
    with pytest.raises(ValueError, match="dimensions"):
        lbm.lbm_build_tiles_noalloc(nt, 0, ny, nz, tm, ne)


def test_noalloc_buffer_checks_on_fake_device_tensors(monkeypatch):
    """Dtype, contiguity and size checks, with is_cuda faked (no GPU here): every case
    raises in the binding, so the library is never called."""
    import torch
    monkeypatch.setattr(torch.Tensor, "is_cuda", property(lambda self: True))
    monkeypatch.setattr(lbm, "load", lambda: pytest.fail("the library was called"))
    nt = torch.ones(9 * 8 * 8, dtype=torch.uint8)                # 3 x 2 x 2 = 12 tiles
    tm = torch.zeros(12, dtype=torch.int32)
    cases = (((nt[1:], tm, tm), "node_type has 575 elements, needs 576"),
             ((nt.to(torch.int32), tm, tm), "node_type must have dtype"),
             ((nt, tm[1:], tm), "tile_map has 11 elements, needs 12"),
             ((nt, tm.to(torch.int64), tm), "tile_map must have dtype"),
             ((nt, tm, torch.zeros(24, dtype=torch.int32)[::2]), "non_empty must be contiguous"),
             ((nt, tm, tm[1:]), "non_empty has 11 elements, needs 12"))
    for (a, b, c), msg in cases:
        with pytest.raises(ValueError, match=msg):
            lbm.lbm_build_tiles_noalloc(a, 9, 8, 8, b, c)

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
    for n in lbm.header_functions():
        assert hasattr(raw, n), n


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

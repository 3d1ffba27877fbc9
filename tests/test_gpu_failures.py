"""Failure detection, tested without a GPU fault: the failures are made on the host (a
fake out-of-memory from the allocation hook, a NaN put into the state through the API,
a record planted where a failed device-side check would leave it). See
include/lbm_testing.h for the hooks and the checked build (LBM_CHECKED)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02445_gb300 import build as B
from paper_1611_02445_gb300 import inputs as I
from paper_1611_02445_gb300 import lbm

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_, W, _ = O.lattice()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()
    lbm.load()


def _err(fg, fo, nt):
    m = nt != 0
    return float((np.abs(fg[:, m] - fo[:, m]) / W[:, None]).max())


@pytest.fixture(autouse=True)
def _no_injection_left():
    yield
    lbm.testing_fail_allocation(-1)


def test_nan_in_the_state_trips_the_mass_watchdog():
    """lbm_reduce returns LBM_ENONFINITE when a population is NaN, before and after it
    has been streamed and collided; the context still works afterwards."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=81)
    f0 = I.random_populations(nt, 0.05, seed=82)
    z, y, x = (int(v[0]) for v in np.nonzero(nt == 1))
    bad = f0.copy()
    bad[7, z, y, x] = np.nan
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(0.8)
        L.set_f(bad)
        for steps in (0, 3):
            L.step(steps)
            with pytest.raises(lbm.LBMError) as e:
                L.reduce()
            assert e.value.status == 6                        # LBM_ENONFINITE
        L.set_f(f0)                                            # not sticky: a clean state works
        L.step(5)
        fg = L.get_f()
    assert _err(fg, O.run(f0, nt, 5, 0b111, 0.8), nt) <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16sr"])
def test_every_allocation_of_create_can_fail_without_leaking(dtype):
    """Fail the k-th device allocation of lbm_create for k = 0, 1, ... until it needs
    fewer: each failure returns LBM_ENOMEM and leaves no buffer behind; the context built
    afterwards steps like the oracle."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=83, boundary=True)
    live0 = lbm.testing_live_allocations()
    for k in range(200):
        lbm.testing_fail_allocation(k)
        try:
            L = lbm.Lattice(nt, dtype, 0b110)
        except lbm.LBMError as e:
            assert e.status == 2, (k, str(e))                   # LBM_ENOMEM
            assert lbm.testing_live_allocations() == live0, k
            continue
        finally:
            lbm.testing_fail_allocation(-1)
        break
    assert k >= 10, k                                           # lbm_create makes many allocations
    f0 = I.random_populations(nt, 0.05, seed=84)
    with L:
        L.set_params(0.8, (1e-5, 0, 0), None, (0.03, 0, 0), 1.0)
        L.set_f(f0)
        L.step(10)
        fg = L.get_f()
    assert lbm.testing_live_allocations() == live0
    if dtype == "f64":
        assert _err(fg, O.run(f0, nt, 10, 0b110, 0.8, (1e-5, 0, 0), None, (0.03, 0, 0), 1.0), nt) <= 1e-12


def test_adjoint_out_of_memory_leaves_the_state_unchanged():
    """lbm_adjoint allocates its checkpoints before any work: a failure there returns
    LBM_ENOMEM (not sticky), frees what it took and leaves the state as it was."""
    nt = I.random_box(12, 8, 16, p_solid=0.3, seed=85)
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(0.8, (1e-5, 0, 0))
        L.init_equilibrium()
        L.step(3)
        blob = L.save_state()
        live0 = lbm.testing_live_allocations()
        failures = 0
        for k in range(8):
            lbm.testing_fail_allocation(k)
            try:
                L.adjoint(8, 4, 5)
            except lbm.LBMError as e:
                assert e.status == 2, str(e)
                failures += 1
                assert lbm.testing_live_allocations() == live0
                assert L.save_state() == blob
                continue
            finally:
                lbm.testing_fail_allocation(-1)
            break
        assert failures >= 1
        L.load_state(blob)
        loss, dg, dtau = L.adjoint(8, 4, 5)
        L.load_state(blob)
        loss2, dg2, dtau2 = L.adjoint(8, 4, 5)
        assert loss == loss2 and dtau == dtau2 and np.array_equal(dg, dg2)
        assert lbm.testing_live_allocations() == live0


def test_field_allocation_failure_is_sticky_and_teardown_is_clean():
    """An allocation failure inside a call that changes device state (the force field of
    lbm_set_params) makes the context fail for good (LBM_ENOMEM is sticky); destroying it
    still frees everything."""
    nt = I.random_box(8, 8, 8, p_solid=0.2, seed=86)
    live0 = lbm.testing_live_allocations()
    L = lbm.Lattice(nt, "f32", 0b111)
    gf = np.full(nt.shape, 1e-5)
    lbm.testing_fail_allocation(0)
    with pytest.raises(lbm.LBMError) as e:
        L.set_params(0.8, None, gf)
    lbm.testing_fail_allocation(-1)
    assert e.value.status == 2
    with pytest.raises(lbm.LBMError) as e:
        L.step(1)
    assert e.value.status == 2
    L.close()
    assert lbm.testing_live_allocations() == live0


def test_checked_build_is_silent_and_matches_the_oracle():
    """The LBM_CHECKED library (every index the step kernel takes from its tables is
    tested before use) on small boxes of every format and on the porous 256^3 pack: no
    check fires, results within the parity bars; a planted record fails the next step
    with LBM_EINTERNAL. Run in a child process, which loads the checked library."""
    env = dict(os.environ, LBM_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_runner.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]

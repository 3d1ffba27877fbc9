"""Run in a child process with LBM_CHECKED=1 (the checked library, include/lbm_testing.h):
small random boxes of every storage format and the porous 256^3 pack, checked against the
oracle; the index checks must stay silent. Then a planted record must make the next step
fail with LBM_EINTERNAL. Prints "checked ok" at the end; any failure raises."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1611_02445_gb300 import build as B  # noqa: E402
from paper_1611_02445_gb300 import inputs as I  # noqa: E402
from paper_1611_02445_gb300 import lbm  # noqa: E402

_, W, _ = O.lattice()
# bars of the small-box parity tests (20 steps): FP64 1e-12 of w, FP32 4e-6, FP16 3e-3
BARS = {"f64": 1e-12, "f64n": 1e-12, "f32": 4e-6, "f16s": 3e-3}


def small_boxes():
    rng = np.random.default_rng(20)
    for n in range(12):
        nx, ny, nz = (int(v) for v in rng.integers(4, 13, 3))
        periodic = int(rng.integers(0, 8))
        for a, d in enumerate((nx, ny, nz)):
            if d % 4:
                periodic &= ~(1 << a)          # a periodic axis must be a multiple of 4
        yield n, I.random_box(nx, ny, nz, p_solid=0.3, seed=100 + n, boundary=True), periodic


def main():
    assert os.environ.get("LBM_CHECKED") == "1"
    B.build(checked=True)
    assert lbm.testing_checked_build()
    tau, g, u_in = 0.8, (1e-5, -2e-6, 0.0), (0.04, 0.0, 0.0)
    for n, nt, periodic in small_boxes():
        f0 = I.random_populations(nt, 0.05, seed=200 + n)
        fo = O.run(f0, nt, 20, periodic, tau, g, None, u_in, 1.0)
        m = nt != 0
        for dtype, bar in BARS.items():
            with lbm.Lattice(nt, dtype, periodic) as L:
                L.set_params(tau, g, None, u_in, 1.0)
                L.set_f(f0)
                L.step(20)                       # raises LBM_EINTERNAL if a check failed
                fg = L.get_f()
            err = float((np.abs(fg[:, m] - fo[:, m]) / W[:, None]).max()) if m.any() else 0.0
            assert err <= bar, (n, dtype, err)
    # full size: every CTA walks many work groups
    pack = I.sphere_pack(256, 8.0, 0.35, I.SEED_POROUS_256)
    for dtype in ("f64", "f32", "f16s"):
        with lbm.Lattice(pack, dtype, 0b111) as L:
            L.set_params(0.7, (1e-5, 0.0, 0.0))
            L.init_equilibrium(1.0, (0.05, 0.0, 0.0))
            L.step(40)
            L.step_kernel(lbm.KERNEL_PROPAGATE, 2)
            L.step_kernel(lbm.KERNEL_RW, 2)
            mass, _ = L.reduce()
            assert np.isfinite(mass)
    # the host side: a planted record (code 3: gather source, value 77) fails the next
    # step with LBM_EINTERNAL, and the context stays failed
    nt = I.random_box(8, 8, 8, p_solid=0.2, seed=7)
    with lbm.Lattice(nt, "f64", 0b111) as L:
        L.set_params(0.8)
        L.init_equilibrium()
        L.step(2)
        lbm.testing_plant_check(L.ctx, (3 << 56) | 77)
        try:
            L.step(1)
            raise AssertionError("a planted check record did not fail the step")
        except lbm.LBMError as e:
            assert e.status == 8 and "gather source" in str(e) and "value 77" in str(e), str(e)
        try:
            L.reduce()
            raise AssertionError("the context did not stay failed")
        except lbm.LBMError as e:
            assert e.status == 8
    print("checked ok")


if __name__ == "__main__":
    main()

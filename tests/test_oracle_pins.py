"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests runs the CUDA library. Each pins a part of the oracle to
something other than the oracle itself: values printed in the paper (golden
fixtures), lattice identities, moment identities of the collision, exact
conservation laws, permutation properties of streaming, a dense-versus-tiled brute
force, and the plane-Poiseuille closed form.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02445_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# --------------------------------------------------------------------------- lattice
def test_lattice_matches_paper_constants():
    g = golden("paper_lattice.json")
    c, w, op = O.lattice()
    assert math.isclose(w[0], g["weights"]["rest"][0] / g["weights"]["rest"][1], rel_tol=0, abs_tol=0)
    for i in g["axis_indices"]:
        assert w[i] == 1.0 / 18.0
        assert np.abs(c[i]).sum() == 1
    for i in g["diagonal_indices"]:
        assert w[i] == 1.0 / 36.0
        assert np.abs(c[i]).sum() == 2
    assert list(c[3]) == g["e3"]
    # 19 distinct velocities, opposites pair up
    assert len({tuple(v) for v in c}) == 19
    for i in range(19):
        assert list(c[op[i]]) == list(-c[i])
        assert op[op[i]] == i


def test_lattice_isotropy():
    """Moment identities of D3Q19 with c_s^2 = 1/3 (Sec. 2.2)."""
    c, w, _ = O.lattice()
    c = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ c).max() < 1e-16
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.abs(second - np.eye(3) / 3.0).max() <= 4 * np.finfo(float).eps
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.abs(third).max() <= 4 * np.finfo(float).eps
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    assert np.abs(fourth - iso).max() <= 4 * np.finfo(float).eps


# ------------------------------------------------------------------------- collision
def _rand_f(rng, amp=0.1):
    _, w, _ = O.lattice()
    return w * (1.0 + amp * (2 * rng.random(19) - 1))


@pytest.mark.parametrize("seed", range(5))
def test_collision_moments_fluid(seed):
    """BGK + Guo: mass is kept, momentum gains F, the second moment relaxes to
    rho/3 I + rho u u with rate 1/tau and gains (1 - 1/(2 tau))(u F + F u)."""
    rng = np.random.default_rng(seed)
    c, w, _ = O.lattice()
    c = c.astype(np.float64)
    f = _rand_f(rng)
    tau = 0.5 + rng.random() * 1.5
    F = 1e-3 * (2 * rng.random(3) - 1)
    out = O.collide(f, I.FLUID, tau, F)
    rho = f.sum()
    j = c.T @ f
    u = (j + 0.5 * F) / rho
    assert abs(out.sum() - rho) < 1e-15
    assert np.abs(c.T @ out - (j + F)).max() < 1e-16
    Pi = np.einsum("i,ia,ib->ab", f, c, c)
    Pi_out = np.einsum("i,ia,ib->ab", out, c, c)
    Pi_eq = rho * np.eye(3) / 3.0 + rho * np.outer(u, u)
    beta = 1.0 - 0.5 / tau
    expect = (1 - 1 / tau) * Pi + Pi_eq / tau + beta * (np.outer(u, F) + np.outer(F, u))
    assert np.abs(Pi_out - expect).max() < 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_collision_single_relaxation_rate(seed):
    """Without force every moment relaxes towards the equilibrium at the one rate 1/tau
    (Eq. 2): out(tau) - f^eq = (1 - 1/tau)(f - f^eq), with f^eq = out(tau = 1); and
    f^eq has the moments rho, rho u, rho/3 I + rho u u (Eq. 3 with c_s^2 = 1/3)."""
    rng = np.random.default_rng(seed)
    c, w, _ = O.lattice()
    c = c.astype(np.float64)
    f = _rand_f(rng)
    feq = O.collide(f, I.FLUID, 1.0)
    rho = f.sum()
    u = (c.T @ f) / rho
    assert abs(feq.sum() - rho) < 1e-15
    assert np.abs(c.T @ feq - rho * u).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", feq, c, c) - (rho * np.eye(3) / 3 + rho * np.outer(u, u))).max() < 1e-15
    for tau in (0.55, 0.8, 1.7):
        out = O.collide(f, I.FLUID, tau)
        assert np.abs((out - feq) - (1 - 1 / tau) * (f - feq)).max() < 1e-16
    again = O.collide(feq, I.FLUID, 0.7)
    assert np.abs(again - feq).max() < 1e-16


def test_collision_boundary_closures():
    """Inlet returns the equilibrium with the inlet velocity and the local density;
    outlet the equilibrium with the outlet density and the local velocity (Sec. 2.2)."""
    rng = np.random.default_rng(7)
    c, w, _ = O.lattice()
    c = c.astype(np.float64)
    f = _rand_f(rng)
    uin = np.array([0.05, 0.01, -0.02])
    out = O.collide(f, I.INLET, 0.6, (0, 0, 0), uin, 1.0)
    assert abs(out.sum() - f.sum()) < 1e-15
    assert np.abs(c.T @ out - f.sum() * uin).max() < 1e-16
    F = np.array([1e-4, 0, 0])
    out = O.collide(f, I.OUTLET, 0.6, F, uin, 1.02)
    u = (c.T @ f + 0.5 * F) / f.sum()
    assert abs(out.sum() - 1.02) < 1e-15
    assert np.abs(c.T @ out - 1.02 * u).max() < 1e-16


# ---------------------------------------------------------------------------- tiling
def _channel_tiles(side, ox, oy, a=4, box=16, nz=8):
    nt = np.zeros((nz, box, box), np.uint8)
    nt[:, oy:oy + side, ox:ox + side] = I.FLUID
    tm, ne = O.tiling(nt, a)
    return nt, tm, ne


def test_tiling_channel8_golden():
    g = golden("channel8_tiling.json")
    counts = {}
    etas = []
    for oy in range(4):
        for ox in range(4):
            nt, tm, ne = _channel_tiles(g["side"], ox, oy)
            per_section = len(ne) // (nt.shape[0] // g["tile"])
            eta = np.count_nonzero(nt) / (len(ne) * 64)
            counts[per_section] = counts.get(per_section, 0) + 1
            assert round(eta, 2) == g["eta_t_rounded_2"][str(per_section)]
            etas.append(eta)
    assert {str(k): v for k, v in counts.items()} == g["tiles_per_cross_section_count"]
    assert round(float(np.mean(etas)), 2) == g["mean_eta_t_rounded_2"]


def test_tiling_side_a_plus_one_constant():
    """A channel one node wider than a tile needs the same number of tiles for every
    tiling (Sec. 3.3)."""
    counts = {len(_channel_tiles(5, ox, oy)[2]) for oy in range(4) for ox in range(4)}
    assert len(counts) == 1


def test_tiling_aligned_4x4_channel_full():
    nt, tm, ne = _channel_tiles(4, 0, 0)
    assert np.count_nonzero(nt) == len(ne) * 64


def test_tiling_dense_and_empty():
    for b in (1, 4, 5, 9, 12):
        tm, ne = O.tiling(I.dense_box(b, b, b))
        assert len(ne) == math.ceil(b / 4) ** 3
    tm, ne = O.tiling(np.zeros((8, 8, 8), np.uint8))
    assert len(ne) == 0 and (tm == -1).all()


@pytest.mark.parametrize("seed", range(4))
def test_tiling_brute_force(seed):
    """Algorithm 1 against a vectorised restatement: keep a tile iff any node is not
    solid, rank tiles in z-y-x order."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = rng.integers(1, 23, size=3)
    nt = I.random_box(int(nx), int(ny), int(nz), p_solid=0.97, seed=seed, boundary=True)
    tm, ne = O.tiling(nt)
    Tz, Ty, Tx = tm.shape
    pad = np.zeros((Tz * 4, Ty * 4, Tx * 4), np.uint8)
    pad[:nz, :ny, :nx] = nt
    keep = (pad.reshape(Tz, 4, Ty, 4, Tx, 4) != 0).any(axis=(1, 3, 5)).reshape(-1)
    rank = np.cumsum(keep) - 1
    assert np.array_equal(tm.reshape(-1), np.where(keep, rank, -1))
    assert np.array_equal(ne, np.nonzero(keep)[0].astype(np.uint32))


# ---------------------------------------------------------------------- step: exact
def test_equilibrium_fixed_point_with_walls():
    nt = I.random_box(12, 8, 8, p_solid=0.3, seed=3)
    f0 = O.init(nt, 1.0)
    f = O.run(f0, nt, 100, periodic=0b101, tau=0.7)
    m = nt != 0
    assert np.abs(f[:, m] - f0[:, m]).max() <= 1e-15


def test_uniform_flow_fixed_point_periodic():
    nt = I.dense_box(8, 8, 8)
    f0 = O.init(nt, 1.02, (0.03, -0.01, 0.02))
    f = O.run(f0, nt, 100, periodic=0b111, tau=0.9)
    assert np.abs(f - f0).max() <= 1e-15


@pytest.mark.parametrize("force", [0.0, 1e-4])
def test_mass_conservation(force):
    nt = I.random_box(12, 12, 8, p_solid=0.3, seed=11)
    f0 = I.random_populations(nt, 0.05, seed=2)
    m0 = O.reduce(f0, nt)[0]
    f = O.run(f0, nt, 100, periodic=0b011, tau=0.8, g=(force, -0.5 * force, 0.2 * force))
    m1 = O.reduce(f, nt, g=(force, -0.5 * force, 0.2 * force))[0]
    assert abs(m1 - m0) / m0 <= 1e-12


def test_momentum_closed_form():
    """Fully periodic, no solids, uniform F: total momentum grows by n F per step."""
    nt = I.dense_box(8, 4, 4)
    n = nt.size
    F = np.array([1e-4, -2e-5, 3e-5])
    f = I.random_populations(nt, 0.05, seed=5)
    # P(0) of the random state with the same F convention
    P0 = O.reduce(f, nt, g=F)[1]
    for t in range(1, 21):
        f = O.step(f, nt, 0b111, 0.75, g=F)
        P = O.reduce(f, nt, g=F)[1]
        assert np.abs(P - (P0 + t * n * F)).max() <= 1e-12 * n * (np.abs(F).max() * t + 0.05)


def test_uniform_acceleration_closed_form():
    """A uniform periodic fluid at rest under a uniform force F: the velocity used in
    the collision of step t is (t - 1/2) F / rho, and it is what the macroscopic export
    and the momentum reduction report from the stored post-collision populations."""
    nt = I.dense_box(4, 4, 8)
    F = np.array([2e-5, -1e-5, 3e-6])
    f = O.init(nt, 1.0)
    for t in range(1, 11):
        f = O.step(f, nt, 0b111, 0.9, g=F)
        rho, u = O.macroscopic(f, nt, g=F)
        m, P = O.reduce(f, nt, g=F)
        expect = (t - 0.5) * F
        # u comes from sums of O(1/36) populations: rounding ~1e-17 per node
        assert np.abs(u.reshape(3, -1) - expect[:, None]).max() <= 1e-15
        assert np.abs(P - nt.size * expect).max() <= 1e-15 * nt.size
        assert abs(m - nt.size) <= 1e-12 * nt.size


def test_streaming_is_shift_when_collision_off():
    """With tau = inf and F = 0 the step is pure pull streaming: in a fully periodic box
    f_i(x) <- f_i(x - c_i), a cyclic shift."""
    c, _, _ = O.lattice()
    nt = I.dense_box(5, 6, 7)
    A = I.random_populations(nt, 0.5, seed=9)
    B = O.step(A, nt, 0b111, math.inf)
    for i in range(19):
        assert np.array_equal(B[i], np.roll(A[i], shift=(c[i][2], c[i][1], c[i][0]), axis=(0, 1, 2)))


def test_streaming_time_reversal_with_walls():
    """Halfway bounce-back streaming is time reversible: reversing all velocities,
    streaming, and reversing again undoes a streaming step (R S R S = identity)."""
    _, _, op = O.lattice()
    nt = I.random_box(9, 7, 8, p_solid=0.35, seed=4)
    A = I.random_populations(nt, 0.5, seed=6)
    B = O.step(A, nt, 0b010, math.inf)
    C = O.step(B[op], nt, 0b010, math.inf)[op]
    m = nt != 0
    assert np.array_equal(C[:, m], A[:, m])
    # and the step is a permutation of the populations
    assert np.array_equal(np.sort(B[:, m], axis=None), np.sort(A[:, m], axis=None))


@pytest.mark.parametrize("periodic", [0b000, 0b111, 0b101])
def test_dense_and_tiled_bit_identical(periodic):
    rng = np.random.default_rng(periodic)
    nt = I.random_box(12, 8, 16, p_solid=0.4, seed=periodic + 20, boundary=True)
    nt[:4, :4, :4] = I.SOLID          # an all-solid tile
    f = I.random_populations(nt, 0.05, seed=periodic)
    gfield = 1e-5 * (1 + 0.1 * rng.standard_normal(nt.shape))
    kw = dict(tau=0.7, g=(1e-5, 2e-6, -3e-6), u_in=(0.05, 0, 0), rho_out=1.0)
    tm, ne = O.tiling(nt)
    ft, ntt = O.to_tiles(f, nt, ne)
    gft, _ = O.to_tiles(np.broadcast_to(gfield, (19,) + nt.shape), nt, ne)
    A = f
    At = ft
    for _ in range(5):
        A = O.step(A, nt, periodic, g_field=gfield, **kw)
        At = O.step_tiled(At, ntt, tm, ne, nt.shape, periodic, g_field_t=gft[:, 0, :], **kw)
    back = O.from_tiles(At, nt.shape, ne)
    m = nt != 0
    assert np.array_equal(back[:, m], A[:, m])


# ----------------------------------------------------------------- plane Poiseuille
def _poiseuille(steps, tau=0.8, g=1e-6, ny=32):
    nt = I.poiseuille_channel(4, ny, 4)
    f = O.run(O.init(nt), nt, steps, periodic=0b101, tau=tau, g=(g, 0, 0))
    rho, u = O.macroscopic(f, nt, g=(g, 0, 0))
    return nt, u


def test_poiseuille_closed_form():
    """Steady plane Poiseuille flow between halfway walls at y = 1/2 and y = ny - 3/2:
    u_x = g/(2 nu) (y - 1/2)(ny - 3/2 - y), nu = (tau - 1/2)/3."""
    tau, g, ny = 0.8, 1e-6, 32
    nt, u = _poiseuille(12000, tau, g, ny)
    nu = (tau - 0.5) / 3.0
    y = np.arange(1, ny - 1, dtype=np.float64)
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    ux = u[0][:, 1:ny - 1, :]
    err = np.sqrt(((ux - exact[None, :, None]) ** 2).sum() / (np.broadcast_to(exact[None, :, None], ux.shape) ** 2).sum())
    assert err <= 1e-3
    yc = (ny - 1) / 2.0
    assert abs(g / (2 * nu) * (yc - 0.5) * (ny - 1.5 - yc) - 1.125e-3) < 1e-15   # u_max = g H^2 / (8 nu)
    # transverse velocity vanishes by symmetry; what remains is accumulated rounding
    assert np.abs(u[1]).max() <= 1e-10 * 1.125e-3 and np.abs(u[2]).max() <= 1e-10 * 1.125e-3


def test_poiseuille_bulk_curvature():
    """At steady state the discrete profile is a parabola: its second difference is
    -g/nu at every interior node."""
    tau, g, ny = 0.8, 1e-6, 32
    nt, u = _poiseuille(30000, tau, g, ny)
    nu = (tau - 0.5) / 3.0
    ux = u[0][0, :, 0]
    # interior rows y = 2 .. ny-3, whose neighbours y-1, y+1 are both fluid
    d2 = ux[3:ny - 1] - 2 * ux[2:ny - 2] + ux[1:ny - 3]
    assert np.abs(d2 / (-g / nu) - 1).max() <= 1e-8


def test_shear_wave_decay_rate():
    """A sinusoidal shear wave decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3."""
    ny, tau, u0 = 64, 0.8, 1e-4
    c, w, _ = O.lattice()
    nt = I.dense_box(4, ny, 4)
    y = np.arange(ny)
    ux = u0 * np.sin(2 * np.pi * y / ny)
    cu = c[:, 0][:, None] * ux[None, :]
    f = (w[:, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * ux[None, :] ** 2))
    f = np.broadcast_to(f[:, None, :, None], (19, 4, ny, 4)).copy()

    def amp(state):
        _, u = O.macroscopic(state, nt)
        return 2 * (u[0][0, :, 0] * np.sin(2 * np.pi * y / ny)).mean()

    f = O.run(f, nt, 200, 0b111, tau)
    a1 = amp(f)
    f = O.run(f, nt, 400, 0b111, tau)
    a2 = amp(f)
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / ny
    rate = -np.log(a2 / a1) / 400
    assert abs(rate / (nu * k * k) - 1) < 2e-3

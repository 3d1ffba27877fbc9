"""Pins of the oracle's collision models beyond quasi-compressible LBGK: the
incompressible equilibrium (Eq. 4 with the velocity of Eq. 6) and the MRT collision
(Eq. 8) in the D3Q19 moment basis of d'Humieres et al. (2002).

What pins them, other than the code itself:
  - the basis: orthogonal rows with the normalisations d'Humieres et al. list for D3Q19
    (19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8);
  - the equilibrium moments m^eq = M f^eq against the closed forms of the same paper
    (e = -11 rho + 19 j.j / rho, eps = 3 rho - 11/2 j.j / rho, q = -2/3 j, 3 p_xx = (3 j_x^2 -
    j.j) / rho, 3 pi_xx = -1/2 3 p_xx, p_ww = (j_y^2 - j_z^2) / rho, pi_ww = -1/2 p_ww, p_xy =
    j_x j_y / rho, m = 0; rho_0 = 1 in place of rho for the incompressible model);
  - MRT with every rate 1/tau is LBGK;
  - a perturbation along one basis vector relaxes by exactly its own rate;
  - mass is conserved and momentum grows by the force, for any rates;
  - plane Poiseuille with halfway bounce-back is exact to rounding when the two-relaxation
    combination Lambda = (1/s_even - 1/2)(1/s_odd - 1/2) is 3/16 (Ginzburg & d'Humieres,
    PRE 68, 2003): LBGK at tau = 1/2 + sqrt(3)/4, and MRT run as two rates with
    s_odd = 1 / (1/2 + (3/16) / (tau - 1/2));
  - the incompressible model: the moments of its equilibrium, momentum P(t) = P(0) + t n F
    in a periodic box, and the exact Poiseuille profile at the same Lambda.
"""
import numpy as np
import pytest

from oracle import oracle as O

C, W, OPP = O.lattice()
Q = 19


def test_basis_orthogonal_with_published_norms():
    M = O.mrt_matrix()
    G = M @ M.T
    assert np.array_equal(G, np.diag(np.diag(G)))
    assert np.diag(G).tolist() == [19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8]
    # rows 0, 3, 5, 7 are the conserved moments rho, j_x, j_y, j_z
    assert np.array_equal(M[0], np.ones(Q))
    assert np.array_equal(M[3], C[:, 0]) and np.array_equal(M[5], C[:, 1]) and np.array_equal(M[7], C[:, 2])


def _feq(rho, u, eq):
    cu = C @ u
    uu = u @ u
    if eq == O.EQ_QCOMPR:
        return W * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
    return W * (rho + 3 * cu + 4.5 * cu * cu - 1.5 * uu)


@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
def test_equilibrium_moments_match_published_closed_forms(eq):
    """The oracle's equilibrium (collide_m at tau = 1 with F = 0 returns f^eq) projected on
    the basis, against d'Humieres et al.'s equilibrium moments."""
    M = O.mrt_matrix()
    rng = np.random.default_rng(3)
    for _ in range(5):
        rho = 1 + 0.1 * rng.standard_normal()
        u = 0.05 * rng.standard_normal(3)
        f = W * (rho + 0.01 * rng.standard_normal(Q))
        # shift f so that its moments are rho and j with j = rho u (eq 0) or u (eq 1)
        j = rho * u if eq == O.EQ_QCOMPR else u
        f = f + W * (rho - f.sum()) + 3 * W * (C @ (j - C.T @ f))
        assert f.sum() == pytest.approx(rho, abs=1e-14)
        feq = O.collide_m(f, 1, 1.0, eq=eq)
        m = M @ feq
        r0 = rho if eq == O.EQ_QCOMPR else 1.0
        jj = j @ j
        want = np.zeros(Q)
        want[0] = rho
        want[1] = -11 * rho + 19 * jj / r0
        want[2] = 3 * rho - 5.5 * jj / r0
        want[3], want[5], want[7] = j
        want[4], want[6], want[8] = -2.0 / 3.0 * j
        want[9] = (3 * j[0] ** 2 - jj) / r0
        want[10] = -0.5 * want[9]
        want[11] = (j[1] ** 2 - j[2] ** 2) / r0
        want[12] = -0.5 * want[11]
        want[13] = j[0] * j[1] / r0
        want[14] = j[1] * j[2] / r0
        want[15] = j[0] * j[2] / r0
        assert np.allclose(m, want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
def test_mrt_with_equal_rates_is_lbgk(eq):
    rng = np.random.default_rng(5)
    for tau in (0.55, 0.8, 1.3):
        for _ in range(4):
            f = W * (1 + 0.05 * rng.standard_normal(Q))
            F = 1e-4 * rng.standard_normal(3)
            a = O.collide_m(f, 1, tau, F, eq=eq, coll=O.COLL_BGK)
            b = O.collide_m(f, 1, tau, F, eq=eq, coll=O.COLL_MRT, rates=np.full(Q, 1.0 / tau))
            assert np.abs(a - b).max() <= 4e-15


def test_lbgk_incompressible_from_collide_m_matches_definition():
    """LBGK with Eq. 4 / Eq. 6: f* = f - (f - f^eq)/tau + (1 - 1/2tau) G at u = j + F/2."""
    rng = np.random.default_rng(6)
    f = W * (1 + 0.05 * rng.standard_normal(Q))
    F = 1e-4 * rng.standard_normal(3)
    tau = 0.7
    u = C.T @ f + 0.5 * F
    G = W * (3 * (C @ F - u @ F) + 9 * (C @ u) * (C @ F))
    want = f - (f - _feq(f.sum(), u, O.EQ_INCOMPR)) / tau + (1 - 0.5 / tau) * G
    got = O.collide_m(f, 1, tau, F, eq=O.EQ_INCOMPR)
    assert np.abs(got - want).max() <= 1e-16


@pytest.mark.parametrize("k", [1, 2, 4, 6, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18])
def test_single_moment_relaxes_by_its_own_rate(k):
    """f = f^eq + eps M^-1 e_k (a non-conserved moment k): the collision (F = 0) leaves
    f^eq + eps (1 - s_k) M^-1 e_k; distinct rates per moment catch a mis-ordered S."""
    M = O.mrt_matrix()
    Minv = np.linalg.inv(M)
    rates = np.linspace(0.3, 1.9, Q)
    rho, u = 1.02, np.array([0.03, -0.01, 0.02])
    fe = _feq(rho, u, O.EQ_QCOMPR)
    eps = 1e-3
    f = fe + eps * Minv[:, k]
    out = O.collide_m(f, 1, 0.8, eq=O.EQ_QCOMPR, coll=O.COLL_MRT, rates=rates)
    assert np.abs(out - (fe + eps * (1 - rates[k]) * Minv[:, k])).max() <= 1e-15


@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
def test_mrt_conserves_mass_and_adds_force(eq):
    rng = np.random.default_rng(8)
    for _ in range(10):
        f = W * (1 + 0.05 * rng.standard_normal(Q))
        F = 1e-4 * rng.standard_normal(3)
        rates = 0.2 + 1.7 * rng.random(Q)
        out = O.collide_m(f, 1, 0.8, F, eq=eq, coll=O.COLL_MRT, rates=rates)
        assert out.sum() == pytest.approx(f.sum(), abs=2e-15)
        assert np.allclose(C.T @ out, C.T @ f + F, rtol=0, atol=2e-15)


def _channel(ny):
    nt = np.ones((4, ny, 4), np.uint8)
    nt[:, 0, :] = 0
    nt[:, ny - 1, :] = 0
    return nt


LAMBDA_MAGIC = 3.0 / 16.0


@pytest.mark.parametrize("eq,coll", [(O.EQ_QCOMPR, O.COLL_BGK), (O.EQ_QCOMPR, O.COLL_MRT),
                                     (O.EQ_INCOMPR, O.COLL_BGK), (O.EQ_INCOMPR, O.COLL_MRT)])
def test_poiseuille_exact_at_magic_lambda(eq, coll):
    """Steady plane Poiseuille flow between walls at y = 1/2 and y = ny - 3/2: with
    Lambda = 3/16 halfway bounce-back puts the walls exactly there and the profile is the
    closed form u_x = g / (2 nu) (y - 1/2)(ny - 3/2 - y) to rounding."""
    ny, g = 16, 1e-6
    if coll == O.COLL_BGK:
        tau = 0.5 + np.sqrt(LAMBDA_MAGIC)
        rates = None
    else:
        tau = 0.8
        s_even = 1.0 / tau
        s_odd = 1.0 / (0.5 + LAMBDA_MAGIC / (1.0 / s_even - 0.5))
        rates = np.array([1, s_even, s_even, 1, s_odd, 1, s_odd, 1, s_odd, s_even, s_even, s_even, s_even,
                          s_even, s_even, s_even, s_odd, s_odd, s_odd], dtype=np.float64)
    nu = (tau - 0.5) / 3.0
    nt = _channel(ny)
    f = O.init(nt)
    f = O.run_m(f, nt, 6000, 0b101, tau, (g, 0, 0), eq=eq, coll=coll, rates=rates)
    _, u = O.macroscopic_m(f, nt, (g, 0, 0), eq=eq)
    y = np.arange(1, ny - 1, dtype=np.float64)
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    prof = u[0][:, 1:ny - 1, :]
    err = np.abs(prof - exact[None, :, None]).max() / exact.max()
    print(f"max |u - exact| / u_max = {err:.2e}")
    assert err <= 1e-9, err
    # transverse components: rounding noise of the momentum sums only
    assert np.abs(u[1]).max() <= 1e-10 * exact.max() and np.abs(u[2]).max() <= 1e-10 * exact.max()


def test_poiseuille_not_exact_away_from_magic_lambda():
    """The same channel with the default MRT rates (Lambda = 0.1 at tau = 0.8) misses the
    closed form by the known O(1/H^2) wall slip: the exactness above is not generic."""
    ny, g, tau = 16, 1e-6, 0.8
    nu = (tau - 0.5) / 3.0
    nt = _channel(ny)
    f = O.run_m(O.init(nt), nt, 6000, 0b101, tau, (g, 0, 0), coll=O.COLL_MRT, rates=O.mrt_rates(tau))
    _, u = O.macroscopic_m(f, nt, (g, 0, 0))
    y = np.arange(1, ny - 1, dtype=np.float64)
    exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    err = np.abs(u[0][:, 1:ny - 1, :] - exact[None, :, None]).max() / exact.max()
    assert 1e-4 < err < 5e-2


@pytest.mark.parametrize("coll", [O.COLL_BGK, O.COLL_MRT])
def test_incompressible_momentum_closed_form(coll):
    """Fully periodic fluid box, uniform force: P(t) = P(0) + t n F (the reported momentum
    is sum (sum c f* - F/2), so P(t) = n F (t - 1/2) from rest)."""
    nt = np.ones((8, 8, 8), np.uint8)
    F = np.array([1e-5, -2e-5, 3e-6])
    f = O.init(nt)
    rates = O.mrt_rates(0.7) if coll == O.COLL_MRT else None
    for t in (1, 5, 20):
        ft = O.run_m(f, nt, t, 0b111, 0.7, F, eq=O.EQ_INCOMPR, coll=coll, rates=rates)
        _, u = O.macroscopic_m(ft, nt, F, eq=O.EQ_INCOMPR)
        P = u.reshape(3, -1).sum(1)
        # rounding of 512 x 19 summed populations of size ~1/18: ~1e-14 absolute
        assert np.allclose(P, nt.size * F * (t - 0.5), rtol=0, atol=1e-13)


@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
def test_uniform_flow_is_a_fixed_point(eq):
    nt = np.ones((8, 4, 4), np.uint8)
    u0 = np.array([0.03, -0.02, 0.01])
    fe = _feq(1.01, u0, eq) if eq == O.EQ_QCOMPR else _feq(1.01, u0, eq)
    f = np.broadcast_to(fe[:, None, None, None], (Q,) + nt.shape).copy()
    out = O.run_m(f, nt, 10, 0b111, 0.9, eq=eq, coll=O.COLL_MRT, rates=O.mrt_rates(0.9))
    assert np.abs(out - f).max() <= 1e-15


# ---------------------------------------------------------------- moving wall (lid)
@pytest.mark.parametrize("tau", [0.8, 1.3])
@pytest.mark.parametrize("coll", [O.COLL_BGK, O.COLL_MRT])
def test_couette_exact_with_moving_lid(tau, coll):
    """Wall at rest at y = 1/2 (solid plane y = 0), the box face y = ny moving with U along
    x (walls halfway, at y = ny - 1/2): the steady profile u_x = U (y - 1/2) / (ny - 1) is
    reproduced exactly by halfway bounce-back with the moving-wall term (LBGK: to 1e-10 U).
    MRT with the default rates of d'Humieres et al. leaves a layer at the moving wall that
    decays by about 3x per node into the bulk: within 2e-6 U (measured 5.2e-7 U at the
    wall node)."""
    ny, U = 12, 0.01
    nt = np.ones((4, ny, 4), np.uint8)
    nt[:, 0, :] = 0
    rates = O.mrt_rates(tau) if coll == O.COLL_MRT else None
    f = O.run_m(O.init(nt), nt, 6000, 0b101, tau, coll=coll, rates=rates, lid_face=3, lid_u=(U, 0, 0))
    _, u = O.macroscopic_m(f, nt)
    y = np.arange(1, ny, dtype=np.float64)
    exact = U * (y - 0.5) / (ny - 1)
    tol = 1e-10 if coll == O.COLL_BGK else 2e-6
    assert np.abs(u[0][:, 1:, :] - exact[None, :, None]).max() <= tol * U
    assert np.abs(u[1]).max() <= tol * U and np.abs(u[2]).max() <= tol * U


@pytest.mark.parametrize("coll", [O.COLL_BGK, O.COLL_MRT])
def test_lid_driven_cavity_conserves_mass(coll):
    """Closed 8^3 cavity, lid z = nz moving tangentially: the wall term adds no mass at a
    node (its links' c.u_lid cancel in pairs), so the total is conserved."""
    nt = np.ones((8, 8, 8), np.uint8)
    f0 = O.init(nt)
    rates = O.mrt_rates(0.7) if coll == O.COLL_MRT else None
    f = O.run_m(f0, nt, 200, 0, 0.7, coll=coll, rates=rates, lid_face=5, lid_u=(0.05, 0.02, 0))
    m0 = np.nansum(f0)
    assert abs(np.nansum(f) - m0) / m0 <= 1e-13
    _, u = O.macroscopic_m(f, nt)
    assert u[0][-1].mean() > 0.005        # the top layer is dragged along x


def test_lid_at_rest_is_a_plain_wall():
    nt = np.ones((8, 8, 8), np.uint8)
    f0 = O.init(nt, 1.0, (0.01, 0.0, 0.0))
    a = O.run_m(f0, nt, 5, 0, 0.8, lid_face=5, lid_u=(0, 0, 0))
    b = O.run_m(f0, nt, 5, 0, 0.8)
    assert np.array_equal(a, b, equal_nan=True)


# -------------------------------------------------------------------- Zou-He
@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
@pytest.mark.parametrize("face", range(6))
def test_zou_he_reconstruction_sets_density_and_momentum(face, eq):
    """The defining property: the completed node has the prescribed momentum (velocity
    boundary: j = rho u_b, or u_b for the incompressible model) or the prescribed density
    with no tangential momentum (pressure boundary); known populations are untouched."""
    rng = np.random.default_rng(face + 10 * eq)
    a, sg = face // 2, (1 if face % 2 == 0 else -1)
    known = [i for i in range(Q) if C[i][a] * sg <= 0]
    for _ in range(5):
        f = W * (1 + 0.1 * rng.standard_normal(Q))
        ub = 0.05 * rng.standard_normal(3)
        out = O.zou_he(f, face, 0, eq, ub)
        rho, j = out.sum(), C.T @ out
        assert np.abs(j - (rho * ub if eq == O.EQ_QCOMPR else ub)).max() <= 1e-16
        assert np.array_equal(out[known], f[known])
        out = O.zou_he(f, face, 1, eq, rho_b=1.03)
        j = C.T @ out
        assert out.sum() == pytest.approx(1.03, abs=1e-15)   # a sum of 19 values
        assert all(abs(j[b]) <= 1e-16 for b in range(3) if b != a)
        assert np.array_equal(out[known], f[known])


def _duct(nx=32, ny=10, nz=4):
    """Channel along x: walls y = 0, ny - 1; inlet nodes on x = 0, outlet nodes on x = nx - 1."""
    nt = np.ones((nz, ny, nx), np.uint8)
    nt[:, 0, :] = 0
    nt[:, ny - 1, :] = 0
    nt[:, 1:ny - 1, 0] = 2
    nt[:, 1:ny - 1, nx - 1] = 3
    return nt


@pytest.mark.parametrize("eq,coll", [(O.EQ_QCOMPR, O.COLL_BGK), (O.EQ_INCOMPR, O.COLL_MRT)])
def test_zou_he_channel_boundary_values(eq, coll):
    """Velocity inlet u = (0.02, 0, 0) on x = 0, pressure outlet rho = 1 on x = nx - 1,
    periodic in z: after every step the inlet nodes carry exactly u_in and the outlet
    nodes exactly rho_out (the reconstruction sets them and the collision conserves them)."""
    nt = _duct()
    u_in, tau = (0.02, 0.0, 0.0), 0.8
    rates = O.mrt_rates(tau) if coll == O.COLL_MRT else None
    f = O.init(nt)
    inl, outl = nt == 2, nt == 3
    for _ in range(3):
        f = O.run_m(f, nt, 40, 0b100, tau, u_in=u_in, rho_out=1.0, eq=eq, coll=coll, rates=rates,
                    bc=O.BC_ZOU_HE, in_face=0, out_face=1)
        rho, u = O.macroscopic_m(f, nt, eq=eq)
        assert np.abs(u[0][inl] - 0.02).max() <= 1e-15 and np.abs(u[1][inl]).max() <= 1e-15
        assert np.abs(rho[outl] - 1.0).max() <= 1e-15
    # the flow has developed: the centre-line velocity downstream exceeds the inlet's
    assert u[0][:, 5, 16].mean() > 0.021


@pytest.mark.parametrize("eq", [O.EQ_QCOMPR, O.EQ_INCOMPR])
@pytest.mark.parametrize("faces", [(0, 1), (3, 2), (4, 5)])
def test_zou_he_uniform_flow_is_a_fixed_point(faces, eq):
    """A box periodic across the flow with inlet and outlet planes on opposite faces: the
    uniform equilibrium f^eq(rho_out, u_in) meets both conditions, so it is a fixed point
    of the step (the reconstruction returns the equilibrium's own unknowns)."""
    fi, fo = faces
    a = fi // 2
    shape = [8, 8, 8]
    nt = np.ones(shape, np.uint8)
    idx_in = [slice(None)] * 3
    idx_out = [slice(None)] * 3
    ax = 2 - a                                   # array axis of coordinate a (z, y, x order)
    idx_in[ax] = 0 if fi % 2 == 0 else -1
    idx_out[ax] = 0 if fo % 2 == 0 else -1
    nt[tuple(idx_in)] = 2
    nt[tuple(idx_out)] = 3
    periodic = 0b111 & ~(1 << a)
    u_in = np.zeros(3)
    u_in[a] = 0.03 if fi % 2 == 0 else -0.03
    fe = _feq(1.0, u_in, eq)
    f = np.broadcast_to(fe[:, None, None, None], (Q,) + nt.shape).copy()
    out = O.run_m(f, nt, 50, periodic, 0.7, u_in=u_in, rho_out=1.0, eq=eq, bc=O.BC_ZOU_HE, in_face=fi,
                  out_face=fo)
    assert np.abs(out - f).max() <= 2e-15   # a few ulps of 1/3 after 50 steps

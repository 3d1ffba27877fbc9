"""Pins of the oracle's differentiation path (tangent-linear and hand-written adjoint).

The tangent-linear step is pinned to the step itself by central finite differences;
the adjoint step is pinned to the tangent by the dot-product identity
<J v, w> = <v, J^T w>; the full reverse sweep is pinned to finite differences of the
loss in FP64. Boxes hold fluid, solid, inlet and outlet nodes so every branch of the
collision and of the bounce-back transpose is exercised.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1611_02445_gb300 import inputs as I

KW = dict(u_in=(0.04, 0.01, 0.0), rho_out=1.01)


def _case(seed, shape=(6, 5, 7), boundary=True):
    nx, ny, nz = shape
    nt = I.random_box(nx, ny, nz, p_solid=0.3, seed=seed, boundary=boundary)
    A = I.random_populations(nt, 0.1, seed=seed + 100)
    rng = np.random.default_rng(seed + 200)
    gfield = 1e-3 * (1.0 + 0.2 * rng.standard_normal(nt.shape))
    return nt, A, gfield, rng


@pytest.mark.parametrize("periodic", [0b000, 0b111, 0b011])
def test_tangent_matches_central_differences(periodic):
    nt, A, gf, rng = _case(periodic + 1)
    m = nt != 0
    v = np.where(m, rng.standard_normal(A.shape), 0.0) * 0.01
    dgf = rng.standard_normal(nt.shape) * 1e-4
    tau, dtau = 0.7, 0.3
    g = (0.0, 2e-4, -1e-4)
    B, dB = O.step_tl(A, v, nt, periodic, tau, dtau, g, (0, 0, 0), gf, dgf, **KW)
    eps = 1e-5
    Bp = O.step(A + eps * v, nt, periodic, tau + eps * dtau, g, gf + eps * dgf, **KW)
    Bm = O.step(A - eps * v, nt, periodic, tau - eps * dtau, g, gf - eps * dgf, **KW)
    fd = (Bp - Bm) / (2 * eps)
    Bv = O.step(A, nt, periodic, tau, g, gf, **KW)
    assert np.array_equal(B[:, m], Bv[:, m])
    scale = np.abs(dB[:, m]).max()
    assert np.abs(fd[:, m] - dB[:, m]).max() <= 1e-7 * scale


@pytest.mark.parametrize("periodic", [0b000, 0b111, 0b101])
def test_adjoint_dot_product(periodic):
    """<J v, w> = <v, J^T w> for state, tau and per-node force directions."""
    nt, A, gf, rng = _case(periodic + 7)
    m = nt != 0
    v = np.where(m, rng.standard_normal(A.shape), 0.0)
    w = np.where(m, rng.standard_normal(A.shape), 0.0)
    dgf = np.where(m, rng.standard_normal(nt.shape), 0.0)
    dtau = 0.37
    tau = 0.85
    g = (0.0, 1e-4, 3e-4)
    _, Jv = O.step_tl(A, v, nt, periodic, tau, dtau, g, (0, 0, 0), gf, dgf, **KW)
    gbar_field = np.zeros(nt.shape)
    gbar = np.zeros(3)
    taubar = np.zeros(1)
    lam = O.step_adj(A, w, nt, periodic, tau, g, gf, gbar_field=gbar_field, gbar=gbar,
                     taubar=taubar, **KW)
    lhs = float((Jv[:, m] * w[:, m]).sum())
    rhs = float((v[:, m] * lam[:, m]).sum() + dtau * taubar[0] + (dgf * gbar_field).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # the solid nodes receive no adjoint
    assert np.abs(lam[:, ~m]).max() == 0.0


def test_adjoint_dot_product_uniform_force():
    nt, A, _, rng = _case(31)
    m = nt != 0
    v = np.where(m, rng.standard_normal(A.shape), 0.0)
    w = np.where(m, rng.standard_normal(A.shape), 0.0)
    dg = rng.standard_normal(3)
    g = (1e-3, -2e-4, 5e-4)
    _, Jv = O.step_tl(A, v, nt, 0b010, 0.9, 0.0, g, dg, None, None, **KW)
    gbar = np.zeros(3)
    lam = O.step_adj(A, w, nt, 0b010, 0.9, g, None, gbar=gbar, **KW)
    lhs = float((Jv[:, m] * w[:, m]).sum())
    rhs = float((v[:, m] * lam[:, m]).sum() + dg @ gbar)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("boundary", [False, True])
def test_loss_gradient_matches_fd(boundary):
    """Reverse sweep over T steps against FP64 central differences of the loss."""
    nt = I.random_box(8, 6, 6, p_solid=0.25, seed=41, boundary=boundary)
    rng = np.random.default_rng(5)
    gf = 1e-3 * (1.0 + 0.1 * rng.standard_normal(nt.shape))
    f0 = I.random_populations(nt, 0.05, seed=3)
    T, plane, per, tau = 6, 7, 0b111, 0.8
    L, gbar_field, gbar, taubar = O.adjoint(nt, T, plane, per, tau, g_field=gf, f0=f0, **KW)
    assert L == pytest.approx(O.forward_loss(nt, T, plane, per, tau, g_field=gf, f0=f0, **KW),
                              rel=0, abs=0)
    # tau
    e = 1e-4
    Lp = O.forward_loss(nt, T, plane, per, tau * (1 + e), g_field=gf, f0=f0, **KW)
    Lm = O.forward_loss(nt, T, plane, per, tau * (1 - e), g_field=gf, f0=f0, **KW)
    fd_tau = (Lp - Lm) / (2 * e * tau)
    assert taubar == pytest.approx(fd_tau, rel=1e-6)
    # per-node force along random directions
    for k in range(3):
        d = rng.standard_normal(nt.shape)
        h = 1e-5
        Lp = O.forward_loss(nt, T, plane, per, tau, g_field=gf + h * d, f0=f0, **KW)
        Lm = O.forward_loss(nt, T, plane, per, tau, g_field=gf - h * d, f0=f0, **KW)
        fd = (Lp - Lm) / (2 * h)
        ad = float((gbar_field * d).sum())
        assert ad == pytest.approx(fd, rel=1e-6)


def test_loss_gradient_single_outlet_node():
    """FP64 finite difference at single nodes of the loss plane."""
    nt = I.random_box(8, 6, 6, p_solid=0.2, seed=43)
    f0 = I.random_populations(nt, 0.05, seed=4)
    gf = np.full(nt.shape, 1e-3)
    T, plane, per, tau = 5, 7, 0b111, 0.8
    L, gbar_field, _, _ = O.adjoint(nt, T, plane, per, tau, g_field=gf, f0=f0)
    nodes = np.argwhere(nt[:, :, plane] != 0)[:3]
    for z, y in nodes:
        h = 1e-6
        gp, gm = gf.copy(), gf.copy()
        gp[z, y, plane] += h
        gm[z, y, plane] -= h
        fd = (O.forward_loss(nt, T, plane, per, tau, g_field=gp, f0=f0)
              - O.forward_loss(nt, T, plane, per, tau, g_field=gm, f0=f0)) / (2 * h)
        assert gbar_field[z, y, plane] == pytest.approx(fd, rel=1e-5)

"""Pins of the oracle's discrete velocity model, weights and equilibrium
(Sec. 2.1, Eqs. 1-9) against facts fixed by mathematics, not by the
oracle's own formulas."""
import math

import numpy as np
import pytest

from oracle import fftlb_oracle as O


def dfact(n):
    """(n)!! for odd n >= -1."""
    return 1 if n <= 0 else n * dfact(n - 2)


def test_velocity_set_geometry():
    v, ring = O.velocities()
    assert v.shape == (33, 2)
    assert np.all(v[0] == 0) and ring[0] == 0
    speeds = np.hypot(v[:, 0], v[:, 1])
    for k, vk in enumerate(O.PAPER_SPEEDS, start=1):
        sel = ring == k
        assert sel.sum() == 8
        np.testing.assert_allclose(speeds[sel], vk, rtol=0, atol=1e-15)
        ang = np.sort(np.mod(np.arctan2(v[sel, 1], v[sel, 0]), 2 * np.pi))
        np.testing.assert_allclose(np.diff(ang), np.pi / 4, atol=1e-14)
    np.testing.assert_allclose(v.sum(axis=0), 0.0, atol=1e-14)


@pytest.mark.parametrize("T", [0.3, 0.5142857, 0.7, 0.95, 1.2])
def test_weights_reproduce_gaussian_moments(T):
    """The ring weights of Eqs. 4-6 must give the discrete moments of a unit
    Maxwellian: sum_j F v_x^(2p) v_y^(2q) = (2p-1)!! (2q-1)!! T^(p+q) for
    p + q <= 3, and every odd moment vanishes."""
    v, ring = O.velocities()
    F = O.weights(T)
    w = F[ring]
    for p in range(4):
        for q in range(4 - p):
            got = (w * v[:, 0] ** (2 * p) * v[:, 1] ** (2 * q)).sum()
            want = dfact(2 * p - 1) * dfact(2 * q - 1) * T ** (p + q)
            assert got == pytest.approx(want, rel=1e-12, abs=1e-14), (p, q)
    for p, q in [(1, 0), (0, 1), (3, 0), (1, 2), (2, 1), (5, 0), (3, 2), (1, 1), (3, 1)]:
        got = (w * v[:, 0] ** p * v[:, 1] ** q).sum()
        assert abs(got) < 1e-12, (p, q)


def test_feq_moments_exact():
    """f^eq reproduces rho, rho u, rho T (Eqs. 7-9), the equilibrium pressure
    tensor rho T delta and zero heat flux, at arbitrary states."""
    rng = np.random.default_rng(1)
    v, _ = O.velocities()
    for _ in range(20):
        rho = rng.uniform(0.2, 7.0)
        T = rng.uniform(0.45, 1.1)
        u = rng.uniform(-0.08, 0.08, size=2)
        fe = O.feq(np.array(rho), np.array(u[0]), np.array(u[1]), np.array(T))
        c = v - u
        assert fe.sum() == pytest.approx(rho, rel=1e-13)
        np.testing.assert_allclose(v.T @ fe, rho * u, atol=1e-13 * rho)
        assert 0.5 * ((c * c).sum(1) @ fe) == pytest.approx(rho * T, rel=1e-13)
        P = np.einsum("ja,jb,j->ab", c, c, fe)
        np.testing.assert_allclose(P, rho * T * np.eye(2), atol=1e-12 * rho)
        qf = np.einsum("ja,j,j->a", c, (c * c).sum(1), fe)
        np.testing.assert_allclose(qf, 0.0, atol=1e-12 * rho)


def test_feq_is_fourth_order_maxwellian_expansion():
    """Eq. 3: the bracket is the expansion of exp((2 u.v - u^2)/(2T)) to fourth
    order in u, so the error of the bracket scales as |u|^5."""
    v, ring = O.velocities()
    T = 0.8
    F = O.weights(T)
    errs = []
    for eps in (0.04, 0.02, 0.01):
        ux, uy = 0.6 * eps, 0.8 * eps
        fe = O.feq(np.array(1.0), np.array(ux), np.array(uy), np.array(T))
        bracket = fe / F[ring]
        exact = np.exp((2 * (v[:, 0] * ux + v[:, 1] * uy) - (ux * ux + uy * uy)) / (2 * T))
        errs.append(np.abs(bracket - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 28 < r1 < 36 and 28 < r2 < 36, errs


def test_moments_of_feq_roundtrip():
    rng = np.random.default_rng(2)
    shape = (5, 7)
    rho = rng.uniform(0.5, 6.0, shape)
    ux = rng.uniform(-0.05, 0.05, shape)
    uy = rng.uniform(-0.05, 0.05, shape)
    T = rng.uniform(0.5, 1.0, shape)
    r2, ux2, uy2, T2 = O.moments(O.feq(rho, ux, uy, T))
    np.testing.assert_allclose(r2, rho, rtol=1e-13)
    np.testing.assert_allclose(ux2, ux, atol=1e-14)
    np.testing.assert_allclose(uy2, uy, atol=1e-14)
    np.testing.assert_allclose(T2, T, rtol=1e-13)


def test_weights_positive_in_paper_range():
    """All F_k > 0 over the paper's temperatures (0.85 - 0.99, a = 9/8)."""
    for T in np.linspace(0.85, 0.99, 8):
        assert np.all(O.weights(T) > 0)

"""Pins of the oracle's windowed spectral derivative (Sec. 3.6, Eqs. FT, IFT,
FFT, K1-K4; Appendix A) against brute-force sums, calculus and the
arcsin-series error analysis."""
import math

import numpy as np
import pytest

from oracle import fftlb_oracle as O

ARCSIN_TAIL = {1: 1.0 / 6.0, 2: 3.0 / 40.0, 3: 5.0 / 112.0, 4: 35.0 / 1152.0}


def brute_force_D(g, axis, dx, window):
    """Eqs. FT, IFT and FFT written out as plain sums in 2-D:
    g~(kx, ky) = dx^2 sum_j g(x_j) exp(-i k.x_j);
    D g(x_j) = 1/(Lx Ly) sum_{n=-N/2}^{N/2-1} i k_m g~ exp(i k.x_j), real part.
    The windowed wavenumber is computed here from the arcsin series of
    Eq. K-TaylorSeries by math.asin's own Taylor coefficients, not from the
    oracle's table."""
    ny, nx = g.shape
    Lx, Ly = nx * dx, ny * dx
    xs = np.arange(nx) * dx
    ys = np.arange(ny) * dx

    def km(n, N):
        k = 2 * math.pi * n / (N * dx)
        if window == 0:
            return k
        s = math.sin(k * dx / 2)
        tot = 0.0
        for j in range(window):
            cj = math.factorial(2 * j) / (4 ** j * math.factorial(j) ** 2 * (2 * j + 1))
            tot += cj * s ** (2 * j + 1)
        return tot * 2 / dx

    out = np.zeros_like(g, dtype=complex)
    for ny_ in range(-ny // 2, ny // 2):
        ky = 2 * math.pi * ny_ / Ly
        for nx_ in range(-nx // 2, nx // 2):
            kx = 2 * math.pi * nx_ / Lx
            phase = np.exp(-1j * (kx * xs[None, :] + ky * ys[:, None]))
            gt = dx * dx * (g * phase).sum()
            mult = 1j * (km(nx_, nx) if axis == "x" else km(ny_, ny))
            out += mult * gt * np.conj(phase)
    return np.real(out) / (Lx * Ly)


@pytest.mark.parametrize("shape", [(8, 8), (6, 10), (4, 12)])
@pytest.mark.parametrize("window", [0, 1, 2, 4])
@pytest.mark.parametrize("axis", ["x", "y"])
def test_D_matches_brute_force_sums(shape, window, axis):
    rng = np.random.default_rng(3)
    g = rng.standard_normal(shape)
    dx = 1.0 / 256
    got = O.D(g, axis, dx, window)
    want = brute_force_D(g, axis, dx, window)
    np.testing.assert_allclose(got, want, atol=1e-11 * np.abs(want).max())


def trig_poly(N, seed, nmax):
    """Random real trigonometric polynomial with modes |n| <= nmax on
    x in [0, 2 pi), its exact derivative and an evaluator."""
    rng = np.random.default_rng(seed)
    amps = rng.standard_normal((nmax + 1, 2))

    def f(x):
        return sum(amps[n, 0] * np.cos(n * x) + amps[n, 1] * np.sin(n * x) for n in range(nmax + 1))

    def df(x):
        return sum(n * (-amps[n, 0] * np.sin(n * x) + amps[n, 1] * np.cos(n * x)) for n in range(nmax + 1))

    return f, df


@pytest.mark.parametrize("N", [8, 16, 32])
def test_exact_wavenumber_differentiates_trig_polynomials(N):
    """window 0: the spectral derivative is exact for modes below Nyquist."""
    dx = 2 * np.pi / N
    x = np.arange(N) * dx
    f, df = trig_poly(N, N, N // 2 - 1)
    g = np.tile(f(x), (4, 1))
    got = O.D(g, "x", dx, 0)
    np.testing.assert_allclose(got, np.tile(df(x), (4, 1)), atol=1e-12 * np.abs(df(x)).max())
    gy = g.T.copy()
    np.testing.assert_allclose(O.D(gy, "y", dx, 0), np.tile(df(x), (4, 1)).T, atol=1e-12 * np.abs(df(x)).max())


@pytest.mark.parametrize("N", [8, 16, 64])
def test_k1_is_half_grid_central_difference(N):
    """Appendix A: IFT[i k1 f~] = (f(x + dx/2) - f(x - dx/2)) / dx for a
    band-limited f (modes below Nyquist)."""
    dx = 2 * np.pi / N
    x = np.arange(N) * dx
    f, _ = trig_poly(N, 100 + N, N // 2 - 1)
    g = np.tile(f(x), (2, 1))
    want = (f(x + dx / 2) - f(x - dx / 2)) / dx
    np.testing.assert_allclose(O.D(g, "x", dx, 1)[0], want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("window", [1, 2, 3, 4])
def test_leading_error_constant(window):
    """For f = sin x, D f = k_m(1) cos x exactly, and from the arcsin series
    k_m(1) - 1 = -(c_m / 4^m) dx^(2m) (1 + O(dx^2)), c_m the first omitted
    arcsin coefficient (1/6, 3/40, 5/112, 35/1152).  In terms of derivatives:
    +dx^2/24 f''' (k1, as printed in Appendix A), -3/640 dx^4 f^(5),
    +5/7168 dx^6 f^(7), -35/294912 dx^8 f^(9)."""
    consts = []
    for N in (32, 64):
        dx = 2 * np.pi / N
        x = np.arange(N) * dx
        g = np.tile(np.sin(x), (2, 1))
        d = O.D(g, "x", dx, window)[0]
        # k_m(1) from the computed derivative (projection on cos x)
        k1 = (d * np.cos(x)).sum() / (np.cos(x) ** 2).sum()
        consts.append((k1 - 1.0) / dx ** (2 * window))
    want = -ARCSIN_TAIL[window] / 4 ** window
    # the relative O(dx^2) correction shrinks by 4 from N=32 to N=64
    assert consts[1] == pytest.approx(want, rel=0.02), consts
    # sign of the printed k1 constant: error = +dx^2/24 f''' with f''' = -cos
    if window == 1:
        assert consts[1] * 1.0 == pytest.approx(-1.0 / 24.0, rel=0.01)


@pytest.mark.parametrize("window,order", [(1, 2), (2, 4), (3, 6)])
def test_convergence_order_smooth_function(window, order):
    """Orders 2, 4, 6 (Sec. 3.6 and Appendix A) on f = exp(sin x)."""
    errs = []
    Ns = (24, 48) if window < 3 else (16, 32)
    for N in Ns:
        dx = 2 * np.pi / N
        x = np.arange(N) * dx
        g = np.tile(np.exp(np.sin(x)), (2, 1))
        d = O.D(g, "x", dx, window)[0]
        errs.append(np.abs(d - np.cos(x) * np.exp(np.sin(x))).max())
    p = math.log2(errs[0] / errs[1])
    assert abs(p - order) < 0.35, (errs, p)


def test_k4_order_eight_on_single_mode():
    """Order 8 of k4: on sin(n x) the error ratio between N and 2N is 2^8."""
    errs = []
    for N in (24, 48):
        dx = 2 * np.pi / N
        x = np.arange(N) * dx
        g = np.tile(np.sin(3 * x), (2, 1))
        errs.append(np.abs(O.D(g, "x", dx, 4)[0] - 3 * np.cos(3 * x)).max())
    assert abs(math.log2(errs[0] / errs[1]) - 8) < 0.2, errs


def test_k4_derivative_of_sine_is_roundoff():
    """Fig. 5 / Sec. 3.6: with k4 the error of the derivative of sin(x) is at
    round-off level (N = 128 on [0, 2 pi))."""
    N = 128
    dx = 2 * np.pi / N
    x = np.arange(N) * dx
    g = np.tile(np.sin(x), (2, 1))
    assert np.abs(O.D(g, "x", dx, 4)[0] - np.cos(x)).max() < 1e-13


def test_windowed_k_tends_to_exact_k():
    """k_m approaches k as m grows (Eq. K-TaylorSeries) for every bin,
    and never overshoots it."""
    N, dx = 64, 1.0 / 256
    k0 = np.abs(O.kappa(N, dx, 0))
    prev = np.zeros(N)
    for m in (1, 2, 3, 4):
        km = np.abs(O.kappa(N, dx, m))
        assert np.all(km >= prev - 1e-9) and np.all(km <= k0 + 1e-9)
        prev = km
    low = np.abs(O.wavenumber_index(N)) <= 4
    np.testing.assert_allclose(prev[low], k0[low], rtol=1e-6)


def test_D_sums_to_zero():
    """The k = 0 multiplier vanishes: every derivative has zero mean (the
    discrete statement behind global conservation)."""
    rng = np.random.default_rng(5)
    g = rng.standard_normal((16, 12))
    for axis in ("x", "y"):
        for m in (0, 1, 4):
            assert abs(O.D(g, axis, 0.01, m).sum()) < 1e-9

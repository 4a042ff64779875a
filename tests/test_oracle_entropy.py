"""Entropy pin of the oracle's Korteweg tensor (Eq. 19), including the term
-rho T d_g rho d_g(M/T) that vanishes at uniform temperature.

The force term of Sec. 2.2 is built so that the hydrodynamics it produces is
the thermodynamically consistent van der Waals fluid with the gradient
coefficient M = K + H T of the free energy: K |grad rho|^2 / 2 is gradient
energy (it is the gradient part of e_T, Eq. 17) and H |grad rho|^2 / 2 is
gradient entropy.  The non-dissipative part of such a fluid conserves the
total entropy

    S = integral of [ s(rho, T) - (H / 2) |grad rho|^2 ],

with s the entropy density of the 2-D vdW fluid (c_v = 1 per unit mass):
s = rho ln T - rho ln(rho / (1 - b rho)) + const * rho.

At f = f^eq the BGK term of Eq. 10 vanishes, so the moments of L(f) are the
inviscid (Euler-Korteweg) rates; with q = 0 (no C_q heat flux, Eq. 23) and
zeta = 0 (no bulk viscosity, Eqs. 21-22) nothing dissipates and dS/dt = 0.
test_entropy_rate_is_total_derivative checks the continuum statement
symbolically in one dimension (the entropy-rate density is a total
derivative with the term as printed, and not with it dropped or negated);
test_oracle_conserves_entropy checks the oracle's rhs on a smooth periodic
2-D state, where spectral derivatives make the discrete rate vanish to
round-off.  Energy conservation (tests/test_oracle_force.py) cannot see this
term (any symmetric Lambda conserves e_T through C), and mechanical
equilibrium (tests/test_oracle_physics.py) holds at uniform T where the term
is zero.  Planted mistakes are planted in private copies of the oracle."""
import importlib.util
import os
import sys

import numpy as np
import pytest

from oracle import fftlb_oracle as O

ORACLE_SRC = os.path.join(os.path.dirname(O.__file__), "fftlb_oracle.py")


def planted(old, new):
    src = open(ORACLE_SRC).read()
    assert old in src
    spec = importlib.util.spec_from_loader("oracle_planted_entropy", loader=None)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle_planted_entropy"] = mod
    exec(src.replace(old, new), mod.__dict__)
    return mod


def smooth_state(N, dx):
    """Non-uniform rho, T, u made of the lowest Fourier modes of the box."""
    x = np.arange(N) * dx
    X, Y = np.meshgrid(x, x)
    k = 2 * np.pi / (N * dx)
    rho = 1.0 + 0.25 * np.sin(k * X + 0.3) * np.cos(k * Y) + 0.1 * np.cos(2 * k * Y + 1.0)
    T = 1.1 + 0.08 * np.cos(k * X - 0.7) + 0.05 * np.sin(k * (X + Y))
    ux = 0.05 * np.sin(k * Y + 0.2) + 0.03 * np.cos(k * X)
    uy = 0.04 * np.cos(k * (X - Y))
    return rho, ux, uy, T


def entropy_rate(mod, H, K, window=0, N=64, dx=1 / 64):
    """dS/dt of the oracle's L(f) at f = f^eq, divided by the sum of the
    magnitudes of its three contributions (so 0 means exact cancellation)."""
    a, b = 9 / 8, 1 / 3
    rho, ux, uy, T = smooth_state(N, dx)
    p = mod.Params(nx=N, ny=N, dx=dx, a=a, b=b, K=K, H=H, q=0.0, zeta=0.0, window=window)
    f = mod.init_equilibrium(rho, ux, uy, T, p)
    L = mod.rhs(f, p)
    v, _ = O.velocities()
    rho_t = L.sum(axis=0)
    jx_t = np.tensordot(v[:, 0], L, axes=(0, 0))
    jy_t = np.tensordot(v[:, 1], L, axes=(0, 0))
    e_t = np.tensordot(0.5 * (v[:, 0] ** 2 + v[:, 1] ** 2), L, axes=(0, 0))   # (rho T + rho u^2 / 2)_t
    kin_t = ux * jx_t + uy * jy_t - 0.5 * (ux * ux + uy * uy) * rho_t         # (rho u^2 / 2)_t
    T_t = (e_t - kin_t - T * rho_t) / rho
    # ds/drho at fixed T and ds/dT at fixed rho of the vdW entropy density
    s_rho = np.log(T) - np.log(rho / (1 - b * rho)) - 1.0 - b * rho / (1 - b * rho)
    s_T = rho / T
    # -(H/2)|grad rho|^2 changes at the rate -H grad rho . grad rho_t, i.e.
    # H lap(rho) rho_t after integration by parts (lap by numpy's FFT)
    kk = 2 * np.pi * np.fft.fftfreq(N, dx)
    lap = np.real(np.fft.ifft2(-(kk[None, :] ** 2 + kk[:, None] ** 2) * np.fft.fft2(rho)))
    parts = [s_rho * rho_t, s_T * T_t, H * lap * rho_t]
    return sum(q.sum() for q in parts) / sum(np.abs(q).sum() for q in parts)


@pytest.mark.parametrize("H,K,window", [(0.0, 2e-4, 0), (1e-3, 1e-2, 0), (1e-3, 1e-2, 4)])
def test_oracle_conserves_entropy(H, K, window):
    assert abs(entropy_rate(O, H, K, window)) < 1e-10


TERM = "iso = -(rho * T * (rx * gx + ry * gy))"


@pytest.mark.parametrize("old,new", [
    (TERM, "iso = -(0.0 * (rx * gx + ry * gy))"),                 # term dropped
    (TERM, "iso = +(rho * T * (rx * gx + ry * gy))"),             # sign flipped
    (TERM, "iso = -(rho * (rx * gx + ry * gy))"),                 # factor T lost
    ("g = M / T", "g = M"),                                       # d(M) instead of d(M/T)
    ("M * (rho * lap + 0.5 * grad2)", "M * (rho * lap + 1.0 * grad2)"),
    ("Lxy = M * rx * ry", "Lxy = -M * rx * ry"),
])
def test_entropy_pin_catches_planted_mistakes(old, new):
    assert abs(entropy_rate(planted(old, new), 1e-3, 1e-2)) > 1e-7


def test_entropy_rate_is_total_derivative():
    """One-dimensional continuum check of the same statement: with Eq. 19's
    term as printed, the entropy-rate density of the f = f^eq moments is a
    total x-derivative (its Euler operator vanishes for rho, T and u);
    dropped or negated, it is not.  The moments are those of the kinetic
    model: rho_t = -(rho u)', (rho u)_t = -(rho u^2 + rho T)' - rho T B and
    (rho T + rho u^2 / 2)_t = -((2 rho T + rho u^2 / 2) u)' - 2 rho T^2 C -
    u rho T B, from sum_i I_i = 0, sum_i c_i I_i = -rho T B and
    sum_i |c_i|^2 I_i / 2 = -2 rho T^2 (C + C_q) (Eq. 11 with A of Eq. 20)."""
    sp = pytest.importorskip("sympy")
    from sympy.calculus.euler import euler_equations
    x, a, b, K, H, sgn = sp.symbols("x a b K H sgn")
    rho, T, u = (sp.Function(n)(x) for n in ("rho", "T", "u"))
    d = lambda e: sp.diff(e, x)
    M = K + H * T
    P = rho * T / (1 - b * rho) - a * rho ** 2
    Pi = P - rho * T
    Lam = M * d(rho) ** 2 - (sgn * rho * T * d(rho) * d(M / T) + M * (rho * d(d(rho)) + d(rho) ** 2 / 2))
    Bx = (d(Pi) + d(Lam)) / (rho * T)
    Cnum = (Pi + Lam + a * rho ** 2) * d(u) + K * (-d(rho) ** 2 * d(u) / 2 - rho * d(rho) * d(d(u))
                                                    - d(rho) ** 2 * d(u))
    rho_t = -d(rho * u)
    mom_t = -d(rho * u ** 2 + rho * T) - rho * T * Bx
    e_t = -d((2 * rho * T + rho * u ** 2 / 2) * u) - Cnum - u * rho * T * Bx
    T_t = (e_t - (u * mom_t - u ** 2 / 2 * rho_t) - T * rho_t) / rho
    r, t = sp.symbols("r t", positive=True)
    s = r * sp.log(t) - r * sp.log(r / (1 - b * r))
    s_rho = sp.diff(s, r).subs({r: rho, t: T})
    s_T = sp.diff(s, t).subs({r: rho, t: T})
    density = s_rho * rho_t + s_T * T_t - H * d(rho) * d(rho_t)

    def is_total_derivative(val):
        eqs = euler_equations(density.subs(sgn, val), [rho, T, u], x)
        return all(sp.simplify(e.lhs) == 0 for e in eqs)

    assert is_total_derivative(1)
    assert not is_total_derivative(0)
    assert not is_total_derivative(-1)

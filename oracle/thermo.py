"""Equilibrium thermodynamics of the van der Waals fluid used to check runs of
the FFT-LB method (arXiv:1011.3582, Sec. 4).

TEST INFRASTRUCTURE ONLY (see oracle/fftlb_oracle.py).  FP64, scipy root
finding and quadrature as library primitives.

  * maxwell(T, a, b): coexistence densities of Fig. 9 / Fig. 13 (Maxwell
    construction: equal pressure and equal chemical potential).
  * sigma_square_gradient(T, a, b, K): surface tension of the square-gradient
    theory, sigma = K int (d rho/dz)^2 dz (Sec. 4.2, second Laplace-law
    relation), evaluated as int sqrt(2 K Delta omega(rho)) d rho.
  * laplace_sigma(R, dP): least-squares slope of the Laplace law
    dP = sigma / R (Sec. 4.2, first relation).

EOS: P = rho T / (1 - b rho) - a rho^2 (Eq. 18 generalised; the paper has
a = 9/8, b = 1/3, so T_c = 8a/(27b) = 1 and rho_c = 1/(3b) = 1).
Pins: tests/test_oracle_thermo.py (equal-area rule, near-critical expansion,
reduced-variable invariance, the paper's printed densities and sigmas).
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, optimize


def critical_point(a, b):
    """T_c = 8a/(27b), rho_c = 1/(3b), P_c = a/(27 b^2) of the vdW EOS."""
    return 8.0 * a / (27.0 * b), 1.0 / (3.0 * b), a / (27.0 * b * b)


def pressure(rho, T, a, b):
    return rho * T / (1.0 - b * rho) - a * rho * rho


def free_energy(rho, T, a, b):
    """Helmholtz free-energy density psi(rho) with rho psi' - psi = P
    (terms linear in rho dropped: they change neither P nor Delta omega)."""
    return rho * T * np.log(rho / (1.0 - b * rho)) - rho * T - a * rho * rho


def chem_potential(rho, T, a, b):
    """mu = d psi / d rho."""
    return T * np.log(rho / (1.0 - b * rho)) + b * rho * T / (1.0 - b * rho) - 2.0 * a * rho


def spinodal(T, a, b):
    """Densities where dP/drho = 0 (bracketing the unstable branch)."""
    Tc, rc, _ = critical_point(a, b)
    dP = lambda r: T / (1.0 - b * r) ** 2 - 2.0 * a * r
    lo = optimize.brentq(dP, 1e-12, rc)
    hi = optimize.brentq(dP, rc, (1.0 - 1e-12) / b)
    return lo, hi


def maxwell(T, a, b):
    """Coexisting (rho_v, rho_l) at temperature T < T_c: P(rho_v) = P(rho_l)
    and mu(rho_v) = mu(rho_l)."""
    Tc, rc, _ = critical_point(a, b)
    if not (0.0 < T < Tc):
        raise ValueError("T must lie in (0, T_c)")
    s_lo, s_hi = spinodal(T, a, b)

    def eqs(x):
        rv, rl = x
        return [pressure(rv, T, a, b) - pressure(rl, T, a, b),
                chem_potential(rv, T, a, b) - chem_potential(rl, T, a, b)]

    # start from the near-critical expansion, clipped into the stable branches
    d = 2.0 * np.sqrt(max(1.0 - T / Tc, 0.0))
    x0 = [min(rc * (1.0 - d), 0.9 * s_lo), max(rc * (1.0 + d), 1.05 * s_hi)]
    x0[1] = min(x0[1], 0.5 * (s_hi + 1.0 / b))
    with np.errstate(invalid="ignore", divide="ignore"):
        sol = optimize.fsolve(eqs, x0, xtol=1e-14, full_output=True)
    rv, rl = sol[0]
    if not (0.0 < rv < s_lo and s_hi < rl < 1.0 / b):
        # fall back to a nested bracket on the saturation pressure
        def area(Ps):
            r1 = optimize.brentq(lambda r: pressure(r, T, a, b) - Ps, 1e-14, s_lo)
            r2 = optimize.brentq(lambda r: pressure(r, T, a, b) - Ps, s_hi, (1 - 1e-14) / b)
            return chem_potential(r1, T, a, b) - chem_potential(r2, T, a, b), r1, r2
        Plo = max(pressure(s_hi, T, a, b), 1e-14)
        Phi = pressure(s_lo, T, a, b)
        Ps = optimize.brentq(lambda P: area(P)[0], Plo * (1 + 1e-12), Phi * (1 - 1e-12), xtol=1e-15)
        _, rv, rl = area(Ps)
    return float(rv), float(rl)


def delta_omega(rho, T, a, b, rv, rl):
    """Excess grand-potential density psi(rho) - mu_s rho + P_s, zero at both
    coexisting densities and positive between them."""
    mu = chem_potential(rv, T, a, b)
    Ps = pressure(rv, T, a, b)
    return free_energy(rho, T, a, b) - mu * rho + Ps


def sigma_square_gradient(T, a, b, K):
    """sigma = K int (d rho/dz)^2 dz for the planar profile that minimises
    int [psi + K |grad rho|^2 / 2]; with K rho'^2 / 2 = Delta omega this is
    int_{rho_v}^{rho_l} sqrt(2 K Delta omega(rho)) d rho."""
    rv, rl = maxwell(T, a, b)
    fn = lambda r: np.sqrt(max(2.0 * K * delta_omega(r, T, a, b, rv, rl), 0.0))
    val, _ = integrate.quad(fn, rv, rl, epsabs=0.0, epsrel=1e-12, limit=200)
    return float(val)


def laplace_sigma(R, dP):
    """Slope sigma of dP = sigma / R (+ offset) by least squares."""
    x = 1.0 / np.asarray(R, dtype=np.float64)
    A = np.vstack([x, np.ones_like(x)]).T
    (s, c), *_ = np.linalg.lstsq(A, np.asarray(dP, dtype=np.float64), rcond=None)
    return float(s), float(c)

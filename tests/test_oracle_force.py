"""Pins of the oracle's force term and time step (Sec. 2.2, Eqs. 10-23)
against moment algebra, conservation laws and energy conservation of
Eq. 14.  Planted mistakes are planted in a private copy of the oracle."""
import importlib.util
import os
import sys

import numpy as np
import pytest

from oracle import fftlb_oracle as O
from paper_1011_3582_gb300 import workloads as W

ORACLE_SRC = os.path.join(os.path.dirname(O.__file__), "fftlb_oracle.py")


def smooth_state(p, seed=4, amp=0.08, umax=0.03, rho0=1.0, T0=0.9, noneq=0.0):
    rho, ux, uy, T = W.smooth_random(p.nx, p.ny, seed=seed, rho0=rho0, T0=T0, amp=amp, umax=umax)
    f = O.init_equilibrium(rho, ux, uy, T, p)
    if noneq:
        rng = np.random.default_rng(seed + 1)
        f = f * (1.0 + noneq * rng.uniform(-1, 1, f.shape))
    return f


def test_force_moment_identities():
    """sum_i I_i = 0 and sum_i v_i I_i = -rho T B pointwise: Eq. 11 with
    A = -2 (C + C_q) T (Eq. 20) and the equilibrium moments."""
    p = O.Params(nx=16, ny=16, dx=1 / 64, K=1e-4, window=4)
    f = smooth_state(p, noneq=1e-3)
    _, parts = O.rhs(f, p, return_parts=True)
    v, _ = O.velocities()
    I = parts["I"]
    scale = np.abs(I).max()
    assert np.abs(I.sum(axis=0)).max() < 1e-12 * scale * 33
    mom = np.tensordot(v.T, I, axes=(1, 0))
    rT = parts["rho"] * parts["T"]
    np.testing.assert_allclose(mom[0], -rT * parts["Bx"], atol=1e-12 * scale * 33)
    np.testing.assert_allclose(mom[1], -rT * parts["By"], atol=1e-12 * scale * 33)


@pytest.mark.parametrize("integrator", [1, 3])
def test_uniform_state_is_fixed_point(integrator):
    p = O.Params(nx=8, ny=12, integrator=integrator, a=9 / 49, b=2 / 21)
    rho, ux, uy, T = W.uniform(8, 12, rho=3.1, T=0.5, ux=0.02, uy=-0.01)
    f = O.init_equilibrium(rho, ux, uy, T, p)
    f2 = O.run(f, p, 3)
    np.testing.assert_allclose(f2, f, rtol=0, atol=1e-14 * np.abs(f).max())


@pytest.mark.parametrize("integrator,window", [(1, 4), (3, 2)])
def test_global_mass_and_momentum_conserved(integrator, window):
    p = O.Params(nx=16, ny=16, dx=1 / 64, K=1e-4, window=window, integrator=integrator)
    f = smooth_state(p, noneq=1e-3)
    i0 = O.invariants(f, p)
    f = O.run(f, p, 10)
    i1 = O.invariants(f, p)
    assert abs(i1["mass"] - i0["mass"]) < 1e-14 * i0["mass"] * 10
    assert abs(i1["px"] - i0["px"]) < 1e-14 * i0["mass"] * 10
    assert abs(i1["py"] - i0["py"]) < 1e-14 * i0["mass"] * 10


def _energy_drift_ratio(mod, nsteps=20):
    """|Delta E_T| / |Delta int a rho^2| over a short run from a smooth
    non-equilibrium state with the exact wavenumber."""
    p = mod.Params(nx=32, ny=32, dx=1 / 64, dt=1e-5, tau=1e-2, K=1e-3, q=-0.004,
                   window=0, integrator=3)
    rho, ux, uy, T = W.smooth_random(32, 32, seed=4, rho0=1.0, T0=0.9, amp=0.08, umax=0.03)
    f = mod.init_equilibrium(rho, ux, uy, T, p)
    i0 = mod.invariants(f, p)
    r0 = mod.moments(f)[0]
    f = mod.run(f, p, nsteps)
    i1 = mod.invariants(f, p)
    r1 = mod.moments(f)[0]
    dpot = abs((p.a * (r1 ** 2 - r0 ** 2)).sum() * p.dx ** 2)
    return abs(i1["eT"] - i0["eT"]) / dpot


def _planted(old, new):
    src = open(ORACLE_SRC).read()
    assert old in src
    spec = importlib.util.spec_from_loader("oracle_planted", loader=None)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["oracle_planted"] = mod
    exec(src.replace(old, new), mod.__dict__)
    return mod


def test_total_energy_conserved():
    """Eq. 14 is a conservation law for e_T of Eq. 17: the force term
    must convert potential energy -a rho^2 + K |grad rho|^2 / 2 into
    kinetic and thermal energy exactly.  With spectral derivatives the
    total drifts by < 1e-8 of the potential energy exchanged."""
    assert _energy_drift_ratio(O) < 1e-8


@pytest.mark.parametrize("old,new", [
    ("+ p.a * rho * rho * div", "- p.a * rho * rho * div"),
    ("-0.5 * grad2 * div", "-1.0 * grad2 * div"),
    ("- rho * (rx * divx + ry * divy)", "+ rho * (rx * divx + ry * divy)"),
    ("Lxx * uxx + Lxy * uyx + Lxy * uxy + Lyy * uyy", "Lxx * uxx + 2 * Lxy * uyx + Lyy * uyy"),
    ("Bx = (Pix + dLx", "Bx = (-Pix + dLx"),
    ("A = -2.0 * (C + Cq) * T", "A = -1.0 * (C + Cq) * T"),
])
def test_energy_pin_catches_planted_mistakes(old, new):
    assert _energy_drift_ratio(_planted(old, new)) > 1e-6

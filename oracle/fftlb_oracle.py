"""FP64 CPU oracle of the windowed-FFT lattice-Boltzmann (FFT-LB) method for
thermal liquid-vapour systems of Gan, Xu, Zhang and Li, "FFT-LB modeling of
thermal liquid-vapor systems" (arXiv:1011.3582).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain, obviously correct
reference against which the CUDA path is checked.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path
(``paper_1011_3582_gb300``) and imports nothing from it.

Everything is float64 numpy.  ``numpy.fft`` serves as the library DFT
primitive; there is no blocking, fusion or reordering beyond what the paper's
equations state.  Equation numbers follow the order of appearance in the paper
(Sec. 2: Eqs. 1-23); the WFFT equations of Sec. 3.6 are named by their labels
(FT, IFT, FFT, K1-K4, Fliter).

Pins (tests/test_oracle_*.py, marker "not gpu"):
  * velocities / weights: Gaussian moment identities through 6th order;
  * f^eq: exact mass, momentum, temperature, pressure-tensor and heat-flux
    moments; 4th-order agreement with the Maxwellian of Eq. 3's first line;
  * spectral derivative: brute-force O(N^2) sums of Eqs. FT/IFT, single
    Fourier modes, the k1 half-grid difference identity (Appendix A),
    convergence orders 2/4/6/8 and their leading error constants;
  * force term: sum_i I_i = 0 and sum_i v_i I_i = -rho T B pointwise;
  * whole step: a uniform state is a fixed point; global mass and momentum
    are conserved to round-off;
  * C and A (Eqs. 20, 22): total energy e_T (Eq. 17) conserved to < 1e-8 of
    the potential energy exchanged (Eq. 14 is a conservation law);
  * B, Lambda, P^w (Eqs. 18, 19, 21): the exact square-gradient planar profile
    is in mechanical equilibrium (tests/test_oracle_physics.py);
  * C_q (Eq. 23): the entropy mode decays with diffusivity T (tau - q), the
    Prandtl relation Pr = tau / 2(tau - q) of Sec. 2.2;
  * the zeta terms of B (Eq. 21): a sound wave decays faster by
    zeta k^2 / 2 rho, the bulk viscosity of the dissipative tensor of
    Eqs. 13-14 (tests/test_oracle_physics.py);
  * Lambda at non-uniform T, including -rho T d_gamma rho d_gamma(M/T) of
    Eq. 19: at f = f^eq with q = zeta = 0 the rates conserve the vdW entropy
    plus the -(H/2)|grad rho|^2 gradient entropy (tests/test_oracle_entropy.py).
Parity unpinned: none.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------

PAPER_SPEEDS = (1.0, 1.9, 2.9, 4.3)   # Sec. 2.1, after Eq. 1


@dataclass
class Params:
    """Problem statement (Sec. 2.2 and Sec. 3, paper defaults).

    nx, ny        periodic grid (lattice sites); dx = dy
    dx, dt, tau   Delta x, Delta t, BGK relaxation time (Eq. 2)
    a, b          van der Waals constants: P^w = rho T / (1 - b rho) - a rho^2
                  (Eq. 18 has a = 9/8, b = 1/3)
    K, H          M = K + H T (below Eq. 19)
    q             heat-flux parameter of C_q (Eq. 23)
    zeta          bulk viscosity (Eq. 21, 22)
    window        0 = exact k, m = 1..4 -> k_m (Eqs. K1-K4)
    integrator    1 = forward Euler, 3 = SSP-RK3 (Shu-Osher)
    """
    nx: int = 64
    ny: int = 64
    dx: float = 1.0 / 256
    dt: float = 1e-5
    tau: float = 1e-2
    a: float = 9.0 / 8.0
    b: float = 1.0 / 3.0
    K: float = 1e-5
    H: float = 0.0
    q: float = -0.004
    zeta: float = 0.0
    window: int = 4
    integrator: int = 3
    speeds: tuple = field(default_factory=lambda: PAPER_SPEEDS)


# ---------------------------------------------------------------------------
# Discrete velocity model and equilibrium (Sec. 2.1)
# ---------------------------------------------------------------------------

def velocities(speeds=PAPER_SPEEDS):
    """Eq. 1: v_0 = 0, v_ki = v_k (cos((i-1) pi/4), sin((i-1) pi/4)).

    Returns (v[33, 2], ring[33]); index 0 is the rest velocity and index
    1 + 8 (k-1) + (i-1) is velocity i of ring k (k, i counted from 1).
    ring[j] is k (0 for the rest velocity).
    """
    v = [(0.0, 0.0)]
    ring = [0]
    for k, vk in enumerate(speeds, start=1):
        for i in range(1, 9):
            ang = (i - 1) * np.pi / 4.0
            v.append((vk * np.cos(ang), vk * np.sin(ang)))
            ring.append(k)
    return np.array(v, dtype=np.float64), np.array(ring)


def weights(T, speeds=PAPER_SPEEDS):
    """Eqs. 4-6: F_k(T), k = 1..4, with the cyclic index {k+l}, and
    F_0 = 1 - 8 (F_1 + F_2 + F_3 + F_4).

    T may be an array; returns F with shape (5,) + T.shape, F[0] = F_0.
    """
    T = np.asarray(T, dtype=np.float64)
    F = np.zeros((5,) + T.shape)
    n = len(speeds)
    for k in range(1, n + 1):
        vk2 = speeds[k - 1] ** 2
        # {k+l} for l = 1, 2, 3 (Eq. 6): k+l if k+l <= 4 else k+l-4
        o = []
        for l in (1, 2, 3):
            kl = k + l if k + l <= 4 else k + l - 4
            o.append(speeds[kl - 1] ** 2)
        num = (48.0 * T**4
               - 6.0 * (o[0] + o[1] + o[2]) * T**3
               + (o[0] * o[1] + o[1] * o[2] + o[2] * o[0]) * T**2
               - o[0] * o[1] * o[2] * T / 4.0)
        den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2])
        F[k] = num / den
    F[0] = 1.0 - 8.0 * (F[1] + F[2] + F[3] + F[4])
    return F


def feq(rho, ux, uy, T, speeds=PAPER_SPEEDS):
    """Eq. 3 (second and third lines): fourth-order expansion of the local
    Maxwellian in u with the ring weights F_k of Eq. 4.  Returns [33, ...]."""
    v, ring = velocities(speeds)
    F = weights(T, speeds)
    u2 = ux * ux + uy * uy
    out = np.empty((33,) + np.shape(rho))
    for j in range(33):
        vu = v[j, 0] * ux + v[j, 1] * uy
        bracket = ((1.0 - u2 / (2 * T) + u2 * u2 / (8 * T * T))
                   + (vu / T) * (1.0 - u2 / (2 * T))
                   + (vu * vu / (2 * T * T)) * (1.0 - u2 / (2 * T))
                   + vu**3 / (6 * T**3)
                   + vu**4 / (24 * T**4))
        out[j] = rho * F[ring[j]] * bracket
    return out


def moments(f, speeds=PAPER_SPEEDS):
    """Eqs. 7-9 evaluated on f (reading: the hydrodynamic fields are the
    moments of the distribution f itself; collision conserves them):
    rho = sum f, rho u = sum v f, rho T = sum |v - u|^2 f / 2."""
    v, _ = velocities(speeds)
    rho = f.sum(axis=0)
    ux = np.tensordot(v[:, 0], f, axes=(0, 0)) / rho
    uy = np.tensordot(v[:, 1], f, axes=(0, 0)) / rho
    cx = v[:, 0][:, None, None] - ux[None]
    cy = v[:, 1][:, None, None] - uy[None]
    T = (0.5 * (cx * cx + cy * cy) * f).sum(axis=0) / rho
    return rho, ux, uy, T


# ---------------------------------------------------------------------------
# Windowed spectral derivative (Sec. 3.6)
# ---------------------------------------------------------------------------

ARCSIN_COEFFS = (1.0, 1.0 / 6.0, 3.0 / 40.0, 5.0 / 112.0)   # Eqs. K1-K4


def wavenumber_index(N):
    """n for each DFT bin in numpy order: n in [-N/2, N/2 - 1] (Eq. IFT)."""
    return np.fft.fftfreq(N) * N


def kappa(N, dx, window):
    """Windowed wavenumber k_m of Eqs. K1-K4 for every DFT bin of a length-N
    axis, k = 2 pi n / (N dx).  window 0 is the exact k; window m >= 1 keeps
    the first m terms of the arcsin series of Eq. K-TaylorSeries:
        k_m = (2/dx) sum_{j<m} c_j sin^(2j+1)(k dx / 2).
    No bin is altered: the Nyquist bin n = -N/2 keeps its formula value."""
    n = wavenumber_index(N)
    k = 2.0 * np.pi * n / (N * dx)
    if window == 0:
        return k
    s = np.sin(k * dx / 2.0)
    km = np.zeros_like(k)
    for j in range(window):
        km += ARCSIN_COEFFS[j] * s ** (2 * j + 1)
    return km * 2.0 / dx


def D(g, axis, dx, window):
    """Spectral derivative of Fig. 3 with the window of Eqs. K1-K4:
    transform (Eq. FT), multiply by i k_m (Eq. FFT), inverse (Eq. IFT),
    real part.  The DFT normalisations dx and 1/L of Eqs. FT/IFT cancel,
    leaving numpy's unnormalised forward / 1/N inverse.  axis: 'x' (last
    array axis) or 'y' (second-to-last)."""
    ny, nx = g.shape[-2], g.shape[-1]
    G = np.fft.fft2(g, axes=(-2, -1))
    if axis == 'x':
        mult = 1j * kappa(nx, dx, window)[None, :]
    else:
        mult = 1j * kappa(ny, dx, window)[:, None]
    return np.real(np.fft.ifft2(mult * G, axes=(-2, -1)))


# ---------------------------------------------------------------------------
# Right-hand side (Eqs. 10, 11, 18-23)
# ---------------------------------------------------------------------------

def pressure_vdw(rho, T, a, b):
    """Eq. 18 with general constants: P^w = rho T / (1 - b rho) - a rho^2."""
    return rho * T / (1.0 - b * rho) - a * rho * rho


def rhs(f, p: Params, return_parts=False):
    """L(f) of Eq. 10: -v . grad f - (f - f^eq)/tau + I, with every spatial
    derivative taken by the windowed spectral derivative D."""
    dx, m = p.dx, p.window
    v, _ = velocities(p.speeds)
    Dx = lambda g: D(g, 'x', dx, m)
    Dy = lambda g: D(g, 'y', dx, m)

    rho, ux, uy, T = moments(f, p.speeds)                     # Eqs. 7-9
    fe = feq(rho, ux, uy, T, p.speeds)                        # Eq. 3

    Pw = pressure_vdw(rho, T, p.a, p.b)                        # Eq. 18
    Pi = Pw - rho * T                                          # P^w - rho T
    M = p.K + p.H * T                                          # M = K + H T
    g = M / T

    rx, ry = Dx(rho), Dy(rho)
    lap = Dx(Dx(rho)) + Dy(Dy(rho))                            # composed D
    uxx, uxy = Dx(ux), Dy(ux)          # d_x u_x, d_y u_x
    uyx, uyy = Dx(uy), Dy(uy)          # d_x u_y, d_y u_y
    div = uxx + uyy
    divx, divy = Dx(div), Dy(div)      # d_gamma (d_alpha u_alpha)
    Tx, Ty = Dx(T), Dy(T)
    Pix, Piy = Dx(Pi), Dy(Pi)
    gx, gy = Dx(g), Dy(g)              # d_gamma (M/T)

    # Eq. 19
    grad2 = rx * rx + ry * ry
    iso = -(rho * T * (rx * gx + ry * gy)) - M * (rho * lap + 0.5 * grad2)
    Lxx = M * rx * rx + iso
    Lxy = M * rx * ry
    Lyy = M * ry * ry + iso

    # Eq. 21
    dLx = Dx(Lxx) + Dy(Lxy)
    dLy = Dx(Lxy) + Dy(Lyy)
    Bx = (Pix + dLx - p.zeta * divx) / (rho * T)
    By = (Piy + dLy - p.zeta * divy) / (rho * T)

    # Eq. 22  (Lambda_ab d_a u_b; the constant 9/8 is a)
    L_du = Lxx * uxx + Lxy * uyx + Lxy * uxy + Lyy * uyy
    Cnum = (Pi * div + L_du - p.zeta * div * div + p.a * rho * rho * div
            + p.K * (-0.5 * grad2 * div
                     - rho * (rx * divx + ry * divy)
                     - (rx * (uxx * rx + uyx * ry) + ry * (uxy * rx + uyy * ry))))
    C = Cnum / (2.0 * rho * T * T)

    # Eq. 23
    Phx = 2.0 * p.q * rho * T * Tx
    Phy = 2.0 * p.q * rho * T * Ty
    Cq = (Dx(Phx) + Dy(Phy)) / (2.0 * rho * T * T)

    # Eq. 20
    A = -2.0 * (C + Cq) * T

    out = np.empty_like(f)
    I = np.empty_like(f)
    for j in range(33):
        cx = v[j, 0] - ux
        cy = v[j, 1] - uy
        I[j] = -(A + Bx * cx + By * cy + (C + Cq) * (cx * cx + cy * cy)) * fe[j]   # Eq. 11
        conv = v[j, 0] * Dx(f[j]) + v[j, 1] * Dy(f[j])
        out[j] = -conv - (f[j] - fe[j]) / p.tau + I[j]                          # Eq. 10
    if return_parts:
        return out, dict(rho=rho, ux=ux, uy=uy, T=T, feq=fe, I=I, A=A, Bx=Bx,
                         By=By, C=C, Cq=Cq, Lxx=Lxx, Lxy=Lxy, Lyy=Lyy)
    return out


# ---------------------------------------------------------------------------
# Time integration
# ---------------------------------------------------------------------------

def step(f, p: Params):
    """One time step.  integrator 1: forward Euler (Sec. 3, the time scheme the
    paper states); integrator 3: SSP-RK3 in Shu-Osher form (reading of the
    unstated Runge-Kutta scheme)."""
    dt = p.dt
    if p.integrator == 1:
        return f + dt * rhs(f, p)
    if p.integrator == 3:
        f1 = f + dt * rhs(f, p)
        f2 = 0.75 * f + 0.25 * (f1 + dt * rhs(f1, p))
        return f / 3.0 + (2.0 / 3.0) * (f2 + dt * rhs(f2, p))
    raise ValueError("integrator must be 1 or 3")


def init_equilibrium(rho, ux, uy, T, p: Params):
    """Initial state f = f^eq(rho, u, T)."""
    return feq(np.asarray(rho, np.float64), np.asarray(ux, np.float64),
               np.asarray(uy, np.float64), np.asarray(T, np.float64), p.speeds)


def run(f, p: Params, nsteps):
    for _ in range(nsteps):
        f = step(f, p)
    return f


# ---------------------------------------------------------------------------
# Diagnostics (Eqs. 12-17)
# ---------------------------------------------------------------------------

def invariants(f, p: Params):
    """Global mass, momentum (x, y), total energy e_T of Eq. 17 (with a in
    place of 9/8 and grad rho by D) and the maximum speed max |u|.  Sums are
    multiplied by the cell area dx^2."""
    rho, ux, uy, T = moments(f, p.speeds)
    rx = D(rho, 'x', p.dx, p.window)
    ry = D(rho, 'y', p.dx, p.window)
    eT = rho * T - p.a * rho * rho + p.K * (rx * rx + ry * ry) / 2.0 \
        + rho * (ux * ux + uy * uy) / 2.0
    area = p.dx * p.dx
    return dict(mass=rho.sum() * area, px=(rho * ux).sum() * area,
                py=(rho * uy).sum() * area, eT=eT.sum() * area,
                umax=np.sqrt(ux * ux + uy * uy).max())

"""A plain PyTorch + cuFFT implementation of one FFT-LB time step
(arXiv:1011.3582, Eqs. 1-23 with the windowed derivative of Sec. 3.6), kept
ONLY as a timing reference for bench.py: torch.fft (cuFFT) for the 94
transforms of a stage and torch element-wise kernels for the rest, in
float32 on the GPU.  It is not the product path (libfftlb.so is), and no
product code calls it.

The arithmetic follows the same equations as the CUDA path: moments on f
(Eqs. 7-9), weights and equilibrium (Eqs. 3-6), the level-1 derivatives,
Lambda and Phi (Eq. 19, 23), their divergences, the coefficients B, C, C_q,
A (Eqs. 20-22) and the force term (Eq. 11), convection -v.D f, BGK, and the
Euler or SSP-RK3 combination; every spatial derivative is the windowed
spectral derivative with the Nyquist bin dropped.
"""
import math

import torch


def _kappa(n, dx, window, device):
    """Windowed wavenumber of every FFT bin (Nyquist zeroed)."""
    m = torch.fft.fftfreq(n, d=1.0 / n, dtype=torch.float64).to(device)   # integer bin indices
    if window == 0:
        k = 2.0 * math.pi * m / (n * dx)
    else:
        s = torch.sin(math.pi * m / n)
        c, sp, k = 1.0, s.clone(), torch.zeros_like(s)
        for j in range(window):
            if j > 0:
                c = c * (2 * j - 1) ** 2 / ((2 * j) * (2 * j + 1))
            k = k + c * sp
            sp = sp * s * s
        k = k * 2.0 / dx
    k[(2 * m).abs() == n] = 0.0
    return k


class TorchStep:
    """One handle's worth of state for the reference: f [33, ny, nx] float32."""

    def __init__(self, nx, ny, dx=1 / 256, dt=1e-5, tau=1e-2, a=9 / 8, b=1 / 3, K=1e-5, H=0.0, q=-0.004,
                 zeta=0.0, window=4, integrator=3, speeds=(1.0, 1.9, 2.9, 4.3), device="cuda"):
        self.nx, self.ny, self.dx, self.dt, self.tau = nx, ny, dx, dt, tau
        self.a, self.b, self.K, self.H, self.q, self.zeta = a, b, K, H, q, zeta
        self.integrator = integrator
        dev = torch.device(device)
        vx, vy, ring = [0.0], [0.0], [0]
        cs = [1.0, math.sqrt(0.5), 0.0, -math.sqrt(0.5), -1.0, -math.sqrt(0.5), 0.0, math.sqrt(0.5)]
        for k in range(4):
            for i in range(8):
                vx.append(speeds[k] * cs[i])
                vy.append(speeds[k] * cs[(i + 6) % 8])
                ring.append(k + 1)
        f32 = torch.float32
        self.vx = torch.tensor(vx, dtype=f32, device=dev)[:, None, None]
        self.vy = torch.tensor(vy, dtype=f32, device=dev)[:, None, None]
        self.v2 = self.vx * self.vx + self.vy * self.vy
        self.ring = torch.tensor(ring, device=dev)
        Fc = []
        for k in range(4):
            o = [speeds[(k + l) % 4] ** 2 for l in (1, 2, 3)]
            vk2 = speeds[k] ** 2
            den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2])
            Fc.append((48.0 / den, -6.0 * sum(o) / den, (o[0] * o[1] + o[1] * o[2] + o[2] * o[0]) / den,
                       -o[0] * o[1] * o[2] / (4.0 * den)))
        self.Fc = Fc
        kx = _kappa(nx, dx, window, dev)[: nx // 2 + 1].to(f32)
        ky = _kappa(ny, dx, window, dev).to(f32)
        self.ikx = (1j * kx)[None, :].to(torch.complex64)
        self.iky = (1j * ky)[:, None].to(torch.complex64)
        self.f = None

    # spectral helpers
    def _fwd(self, g):
        return torch.fft.rfft2(g)

    def _inv(self, G):
        return torch.fft.irfft2(G, s=(self.ny, self.nx))

    def _weights(self, T):
        F = [T * (c3 + T * (c2 + T * (c1 + T * c0))) for (c0, c1, c2, c3) in self.Fc]
        F0 = 1.0 - 8.0 * (F[0] + F[1] + F[2] + F[3])
        return torch.stack([F0] + F)   # [5, ny, nx]

    def feq(self, rho, ux, uy, T):
        F = self._weights(T)[self.ring]                    # [33, ny, nx]
        u2 = ux * ux + uy * uy
        iT = 1.0 / T
        qq = 0.5 * u2 * iT
        om = 1.0 - qq
        p0, p1, p2 = om + 0.5 * qq * qq, om * iT, 0.5 * om * iT * iT
        p3, p4 = iT ** 3 / 6.0, iT ** 4 / 24.0
        vu = self.vx * ux + self.vy * uy
        return rho * F * (p0 + vu * (p1 + vu * (p2 + vu * (p3 + vu * p4))))

    def set_fields(self, rho, ux, uy, T):
        """f = f^eq(rho, u, T), evaluated in fp64 and stored in fp32 (as the
        CUDA path does)."""
        t = [torch.as_tensor(x, dtype=torch.float64, device=self.vx.device) for x in (rho, ux, uy, T)]
        rho, ux, uy, T = t
        Fk = [T * (c3 + T * (c2 + T * (c1 + T * c0))) for (c0, c1, c2, c3) in self.Fc]
        F = torch.stack([1.0 - 8.0 * (Fk[0] + Fk[1] + Fk[2] + Fk[3])] + Fk)[self.ring]
        vx, vy = self.vx.double(), self.vy.double()
        u2 = ux * ux + uy * uy
        iT = 1.0 / T
        qq = 0.5 * u2 * iT
        om = 1.0 - qq
        vu = vx * ux + vy * uy
        br = (om + 0.5 * qq * qq) + vu * (om * iT + vu * (0.5 * om * iT * iT + vu * (iT ** 3 / 6.0 + vu * iT ** 4 / 24.0)))
        self.f = (rho * F * br).float()

    def fields(self):
        f = self.f
        rho = f.sum(0)
        ux = (self.vx * f).sum(0) / rho
        uy = (self.vy * f).sum(0) / rho
        T = 0.5 * ((self.v2 * f).sum(0) / rho - (ux * ux + uy * uy))
        return rho, ux, uy, T

    def rhs(self, f):
        rho = f.sum(0)
        ux = (self.vx * f).sum(0) / rho
        uy = (self.vy * f).sum(0) / rho
        T = 0.5 * ((self.v2 * f).sum(0) / rho - (ux * ux + uy * uy))
        fe = self.feq(rho, ux, uy, T)
        M = self.K + self.H * T
        Pi = rho * T / (1.0 - self.b * rho) - self.a * rho * rho - rho * T
        g = M / T
        # level-1 spectra and derivatives (one batched transform)
        S = self._fwd(torch.stack([rho, ux, uy, T, Pi, g]))
        ikx, iky = self.ikx, self.iky
        Sr, Sux, Suy, ST, SPi, Sg = S
        d = self._inv(torch.stack([ikx * Sr, iky * Sr, ikx * ikx * Sr + iky * iky * Sr,
                                   ikx * Sux, iky * Sux, ikx * Suy, iky * Suy,
                                   ikx * (ikx * Sux + iky * Suy), iky * (ikx * Sux + iky * Suy),
                                   ikx * ST, iky * ST, ikx * SPi, iky * SPi, ikx * Sg, iky * Sg]))
        rx, ry, lap, uxx, uxy, uyx, uyy, divx, divy, Tx, Ty, Pix, Piy, gx, gy = d
        grad2 = rx * rx + ry * ry
        iso = -(rho * T * (rx * gx + ry * gy)) - M * (rho * lap + 0.5 * grad2)
        Lxx, Lxy, Lyy = M * rx * rx + iso, M * rx * ry, M * ry * ry + iso
        div = uxx + uyy
        Ldu = Lxx * uxx + Lxy * (uyx + uxy) + Lyy * uyy
        Cn = Pi * div + Ldu - self.zeta * div * div + self.a * rho * rho * div + self.K * (
            -0.5 * grad2 * div - rho * (rx * divx + ry * divy) - (rx * (uxx * rx + uyx * ry) + ry * (uxy * rx + uyy * ry)))
        q2 = 2.0 * self.q * rho * T
        L2 = self._fwd(torch.stack([Lxx, Lxy, Lyy, q2 * Tx, q2 * Ty]))
        dL = self._inv(torch.stack([ikx * L2[0] + iky * L2[1], ikx * L2[1] + iky * L2[2], ikx * L2[3] + iky * L2[4]]))
        rT = rho * T
        Bx = (Pix - self.zeta * divx + dL[0]) / rT
        By = (Piy - self.zeta * divy + dL[1]) / rT
        CC = (Cn + dL[2]) / (2.0 * rho * T * T)
        A = -2.0 * CC * T
        u2 = ux * ux + uy * uy
        e0 = A - (Bx * ux + By * uy) + CC * u2
        I = -(e0 + (Bx - 2.0 * CC * ux) * self.vx + (By - 2.0 * CC * uy) * self.vy + CC * self.v2) * fe
        conv = self._inv((self.vx[1:] * ikx + self.vy[1:] * iky) * self._fwd(f[1:]))
        out = -(f - fe) / self.tau + I
        out[1:] -= conv
        return out

    def step(self, n=1):
        dt = self.dt
        for _ in range(n):
            f = self.f
            if self.integrator == 1:
                self.f = f + dt * self.rhs(f)
            else:
                f1 = f + dt * self.rhs(f)
                f2 = 0.75 * f + 0.25 * (f1 + dt * self.rhs(f1))
                self.f = f / 3.0 + (2.0 / 3.0) * (f2 + dt * self.rhs(f2))

"""Shared set-up of the GPU parity tests: configurations shaped like the
paper's workloads and cached oracle runs."""
import functools

import numpy as np

from oracle import fftlb_oracle as O
from oracle import thermo as TH
from paper_1011_3582_gb300 import workloads as W

A49, B21 = 9.0 / 49.0, 2.0 / 21.0          # vdW constants of the benchmark configurations
TC49 = 8 * A49 / (27 * B21)                # = 4/7
RHOC49 = 1.0 / (3 * B21)                   # = 3.5


def lib():
    from paper_1011_3582_gb300 import build
    build.build()
    from paper_1011_3582_gb300 import fftlb
    return fftlb


def slab64():
    """64x64 planar slab at T = 0.9 T_c, Maxwell densities in the central 32
    rows with tanh edges of width 2, seed-42 noise U(-1e-4, 1e-4) on rho."""
    T = 0.9 * TC49
    rv, rl = TH.maxwell(T, A49, B21)
    fields = W.slab(64, 64, rv, rl, T, y1=16, y2=48, width=2.0, noise=1e-4, seed=42)
    return fields, dict(nx=64, ny=64, a=A49, b=B21)


def droplet_ragged():
    """48 x 96 (radix-3 axes) droplet of the paper's EOS at T = 0.95."""
    rv, rl = TH.maxwell(0.95, 9 / 8, 1 / 3)
    fields = W.droplet(96, 48, 14.0, rl, rv, 0.95, width=2.0)
    return fields, dict(nx=96, ny=48, a=9 / 8, b=1 / 3)


def oracle_params(kw, **extra):
    d = dict(kw)
    d.update(extra)
    return O.Params(**{k: v for k, v in d.items() if k in O.Params.__dataclass_fields__})


@functools.lru_cache(maxsize=None)
def oracle_run(name, nsteps, integrator, window=4):
    fields, kw = {"slab64": slab64, "droplet_ragged": droplet_ragged}[name]()
    p = oracle_params(kw, integrator=integrator, window=window)
    f = O.init_equilibrium(*fields, p)
    f = O.run(f, p, nsteps)
    return f, O.moments(f), O.invariants(f, p)


def gpu_run(fl, name, nsteps, integrator, precision, window=4):
    fields, kw = {"slab64": slab64, "droplet_ragged": droplet_ragged}[name]()
    p = fl.params(integrator=integrator, precision=precision, window=window, **kw)
    with fl.Handle(p) as h:
        h.set_fields(*fields)
        h.step(nsteps)
        return h.get_f(), h.fields(), h.invariants()


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def weight_condition(T, speeds=(1.0, 1.9, 2.9, 4.3)):
    """Largest condition number over the rings k of Eq. 4's weight
    polynomial F_k(T) = T (c3 + T (c2 + T (c1 + T c0))) at the temperatures T:
    sum_j |c_j T^j| / |F_k(T)|.  Near a root of F_k (ring 4 of the paper's
    set near T = 0.43) fp32 evaluation loses that many ulps."""
    T = np.asarray(T, np.float64)
    worst = 0.0
    for k in range(4):
        o = [speeds[(k + l) % 4] ** 2 for l in (1, 2, 3)]
        vk2 = speeds[k] ** 2
        den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2])
        c = [48 / den, -6 * sum(o) / den, (o[0] * o[1] + o[1] * o[2] + o[2] * o[0]) / den,
             -o[0] * o[1] * o[2] / (4 * den)]
        terms = [c[0] * T ** 4, c[1] * T ** 3, c[2] * T ** 2, c[3] * T]
        worst = max(worst, float((sum(np.abs(t) for t in terms) / np.abs(sum(terms))).max()))
    return worst


def fp32_force_bound(n, nsteps, rho, T, dx=1 / 256, dt=1e-5, K=1e-5, vmax=4.3, u_split=0.0, tau=1e-2):
    """Elementwise bound on |df_i| / f_i of the FP32 path after nsteps RK3
    steps.  Two sources: (1) each stage update rounds f_i at most twice, and
    the initial f^eq once: 4 (S + 1) u with a factor 2 of margin; (2) the
    force coefficient B (Eq. 21) contains d_b Lambda_ab with Lambda
    containing K rho lap(rho) (Eq. 19), a third spectral derivative of rho.
    The rounding of an FP32 transform is spread over all wavenumbers with rms
    ~ u sqrt(log2 N) rms(rho) (two chained transforms: factor 2), and the
    third derivative multiplies wavenumber k by |k|^3; over the square
    spectrum of the window-4 symbol (max k_max = (2/dx)(1 + 1/6 + 3/40 +
    5/112)) the rms of |k|^3 is 0.83 k_max^3.  |v - u| |dB| dt per stage,
    over S = 3 nsteps stages, times sqrt(2 ln M) for the maximum over the M
    values of f, times 2 of margin; (3) f^eq carries the fp32 error of the
    weights F_k (Eq. 4), 4 u times the polynomial's condition number
    (weight_condition), which the BGK term passes to f at dt / tau per
    stage: S dt / tau 4 u cond, times 2 of margin (near a root of F_k, e.g.
    ring 4 at T = 0.75 T_c of the 9/49, 2/21 fluid, this term dominates).
    u_split: the relative error of one split-BF16 first pass (the row and
    the column first passes of a 2-D transform add 2 u_split to its
    u sqrt(log2 N))."""
    u, S = 2.0 ** -24, 3 * nsteps
    N = n * n if np.isscalar(n) else n[0] * n[1]   # n or (ny, nx)
    kmax = (2 / dx) * (1 + 1 / 6 + 3 / 40 + 5 / 112)
    eps = (u * np.sqrt(np.log2(N)) + 2 * u_split) * np.sqrt(np.mean(rho ** 2))
    d3 = 2 * eps * 0.83 * kmax ** 3
    dB = vmax * K * d3 / T.min()
    tail = np.sqrt(2 * np.log(33 * N))
    weights = 2 * S * (dt / tau) * 4 * u * weight_condition(T)
    return 4 * (S + 1) * u + 2 * tail * S * dt * dB + weights

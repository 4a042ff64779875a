"""fp32 evaluation of the ring weights F_k(T) of Eq. 4 (CPU emulation).

The fp32 kernels evaluate F_k = T (c3 + T (c2 + T (c1 + T c0))) with the
compensated Horner scheme (Graillat, Langlois and Louvet, 2005): the
coefficients as fp32 pairs hi + lo, every product and sum split by
error-free transformations (TwoProd through fma, TwoSum), the rounding
errors carried in a second Horner accumulator.  This emulates that
arithmetic step by step in numpy float32 (the fma as one rounding of the
exact float64 value) and checks it against the float64 polynomial: within
a few ulps everywhere, including around the root of F_4 near T = 0.43
where plain fp32 Horner is off by up to 4e-3 relative."""
import numpy as np

SPEEDS = (1.0, 1.9, 2.9, 4.3)
f32 = np.float32


def coefficients(k):
    o = [SPEEDS[(k + l) % 4] ** 2 for l in (1, 2, 3)]
    vk2 = SPEEDS[k] ** 2
    den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2])
    return [48 / den, -6 * sum(o) / den, (o[0] * o[1] + o[1] * o[2] + o[2] * o[0]) / den, -o[0] * o[1] * o[2] / (4 * den)]


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def compensated(k, T):
    c64 = coefficients(k)
    hi = [f32(v) for v in c64]
    lo = [f32(v - np.float64(h)) for v, h in zip(c64, hi)]
    T = f32(T)
    s, c = hi[0], lo[0]
    for j in range(1, 4):
        p = f32(s * T)
        pe = fma32(s, T, -p)
        a = hi[j]
        sn = f32(p + a)
        z = f32(sn - p)
        se = f32(f32(p - f32(sn - z)) + f32(a - z))
        c = fma32(c, T, f32(f32(pe + se) + lo[j]))
        s = sn
    return f32(T * f32(s + c))


def plain(k, T):
    c = [f32(v) for v in coefficients(k)]
    T = f32(T)
    return f32(T * f32(c[3] + f32(T * f32(c[2] + f32(T * f32(c[1] + f32(T * c[0])))))))


def exact(k, T):
    c = coefficients(k)
    T = np.float64(f32(T))
    return T * (c[3] + T * (c[2] + T * (c[1] + T * c[0])))


def test_compensated_weights_are_accurate_near_the_root():
    u = 2.0 ** -24
    Ts = np.concatenate([np.linspace(0.3, 0.65, 2001), np.linspace(0.425, 0.432, 2001)])
    worst_c, worst_p = 0.0, 0.0
    for k in range(4):
        for T in Ts:
            e = exact(k, T)
            worst_c = max(worst_c, abs(float(compensated(k, T)) - e) / abs(e))
            worst_p = max(worst_p, abs(float(plain(k, T)) - e) / abs(e))
    assert worst_c < 4 * u, worst_c          # a few ulps everywhere
    assert worst_p > 100 * worst_c           # plain Horner cancels near the root of F_4

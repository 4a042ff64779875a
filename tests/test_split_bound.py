"""The per-pass error bound of the split-BF16 first pass, checked on the CPU.

The GPU parity tests of precision 32 | FFTLB_BF16SPLIT add u_split = 3 * 2^-16
per split pass to the fp32 transform round-off (tests/test_gpu_parity.py).
That figure comes from the arithmetic of one 16-point DFT done as a real
product with split operands: for every real product w x the pass keeps
w_hi x_hi + w_hi x_lo + w_lo x_hi, with z_hi = bf16(z) and
z_lo = bf16(z - z_hi) (nearest even), so

    |w x - kept| <= |w - w_hi - w_lo| |x| + |w| |x - x_hi - x_lo|
                    + |w_lo| |x_lo| + (second order)
                 <= 3 * 2^-16 |w| |x|  (to first order),

and an output of the pass is in error by at most u_split times the sum of
|w| |x| over its 32 real products.  These tests emulate that arithmetic in
float64 (exact sums, so only the splitting is measured) and check the bound
on random and adversarial inputs, and that it is not loose by orders of
magnitude.  They test the bound, not the CUDA kernel (the GPU parity tests
do that).
"""
import numpy as np

from oracle.cnn_oracle import bf16_round

U_SPLIT = 3 * 2.0 ** -16


def split(z):
    """bfloat16 hi and lo parts of float32 values."""
    z = np.asarray(z, np.float32)
    hi = bf16_round(z)
    lo = bf16_round((z - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def dft16(direction):
    m = np.arange(16)
    return np.exp(direction * 2j * np.pi * np.outer(m, m) / 16)


def split_pass(x, direction):
    """16-point DFT of the columns of x (16 x nb complex) with every real
    product split; returns the result and the sum of |w| |x| per output."""
    W = dft16(direction)
    A = np.block([[W.real, -W.imag], [W.imag, W.real]])          # [Re Y; Im Y] = A [Re x; Im x]
    X = np.concatenate([x.real, x.imag]).astype(np.float32)
    ah, al = split(A.astype(np.float32))
    xh, xl = split(X)
    Y = ah @ xh + ah @ xl + al @ xh
    mag = np.abs(A) @ np.abs(X.astype(np.float64))
    return Y[:16] + 1j * Y[16:], mag[:16], mag[16:]


def exact(x, direction):
    X = np.concatenate([x.real, x.imag]).astype(np.float32).astype(np.float64)
    xc = X[:16] + 1j * X[16:]
    return dft16(direction) @ xc


def check(x, direction):
    y, mr, mi = split_pass(x, direction)
    ye = exact(x, direction)
    er = np.abs(y.real - ye.real) / mr
    ei = np.abs(y.imag - ye.imag) / mi
    return max(er.max(), ei.max())


def test_bound_holds_on_random_inputs():
    rng = np.random.default_rng(5)
    worst = 0.0
    for direction in (-1, 1):
        for scale in (1e-3, 1.0, 7.5, 3e4):
            x = scale * (rng.standard_normal((16, 512)) + 1j * rng.standard_normal((16, 512)))
            worst = max(worst, check(x, direction))
    assert worst <= U_SPLIT
    # the bound is attained within a small factor (it is not loose)
    assert worst > U_SPLIT / 16


def test_bound_holds_on_adversarial_inputs():
    """Values just below bfloat16 rounding ties (the largest hi and lo
    errors) and spectra of pure tones, where cancellation is complete."""
    rng = np.random.default_rng(9)
    base = 1.0 + (2 * rng.integers(0, 128, (16, 64)) + 1) * 2.0 ** -8 * (1 - 2.0 ** -9)
    signs = rng.choice([-1.0, 1.0], (16, 64))
    x = base * signs + 1j * base[::-1] * signs[:, ::-1]
    worst = check(x, -1)
    tone = np.exp(2j * np.pi * 3 * np.arange(16) / 16)[:, None] * np.ones((1, 4))
    worst = max(worst, check(tone, -1), check(tone, 1))
    assert worst <= U_SPLIT


def test_dropping_a_term_breaks_the_bound():
    """Without the w_hi x_lo term the error is of order 2^-8, far above
    u_split: the bound distinguishes a complete split from a broken one."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 256)) + 1j * rng.standard_normal((16, 256))
    W = dft16(-1)
    A = np.block([[W.real, -W.imag], [W.imag, W.real]])
    X = np.concatenate([x.real, x.imag]).astype(np.float32)
    ah, al = split(A.astype(np.float32))
    xh, _ = split(X)
    Y = ah @ xh + al @ xh
    mag = np.abs(A) @ np.abs(X.astype(np.float64))
    ye = exact(x, -1)
    err = np.abs(Y[:16] - ye.real) / mag[:16]
    assert err.max() > 10 * U_SPLIT


def test_gradient_emulation_separates_complete_from_broken_split():
    """The bound of the GPU split-BF16 gradient test (split_emulation): the
    emulated gradient with complete split passes stays 4x below it, and with
    the w_hi x_lo product dropped in every split pass it lands 4x above."""
    from oracle import fftlb_oracle as O
    from split_emulation import SPLIT_GRADIENT_BOUND, emulated_gradient
    rng = np.random.default_rng(7)
    g = rng.standard_normal((256, 256))
    for axis in ("x", "y"):
        ref = O.D(g, axis, 1 / 256, 4)
        scale = np.abs(ref).max()
        ok = np.abs(emulated_gradient(g, axis, 1 / 256, 4) - ref).max() / scale
        bad = np.abs(emulated_gradient(g, axis, 1 / 256, 4, drop_hi_lo=True) - ref).max() / scale
        assert ok < SPLIT_GRADIENT_BOUND / 4, (axis, ok)
        assert bad > 4 * SPLIT_GRADIENT_BOUND, (axis, bad)


def test_gradient_emulation_without_splitting_is_exact():
    """With exact products (no rounding at all) the emulated route equals
    the oracle's D to round-off: the route itself is right."""
    import split_emulation as S
    from oracle import fftlb_oracle as O
    rng = np.random.default_rng(1)
    g = rng.standard_normal((64, 128))
    saved = S._split, S.OPERAND
    try:
        S._split = lambda z: (np.asarray(z, np.float64), np.zeros(np.shape(z)))
        S.OPERAND = np.float64
        for axis in ("x", "y"):
            ref = O.D(g, axis, 1 / 256, 3)
            got = S.emulated_gradient(g, axis, 1 / 256, 3)
            assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12
    finally:
        S._split, S.OPERAND = saved

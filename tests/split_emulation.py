"""CPU emulation of the split-BF16 first passes on the spectral-gradient
path, and the error bound the GPU test of that path uses.

Test infrastructure (imports only numpy and the oracle).  The CUDA gradient
of a handle in precision 32 | FFTLB_BF16SPLIT transforms rows and columns
with Stockham passes whose first pass, a 16-point DFT of the inputs
x[j + t n/16] (t = 0..15), runs on the tensor cores with every real operand
split into bfloat16 hi and lo parts and the products w_hi x_hi + w_hi x_lo +
w_lo x_hi accumulated.  Here that first pass is emulated exactly (float32
operands, bfloat16 splits, float64 sums) and the rest of each transform is
exact, so the emulated gradient carries the split passes' error alone.

Bound (SPLIT_GRADIENT_BOUND, on max|error| / max|D g|).  Per real product
the split keeps w x up to three residuals, each at most 2^-16 |w| |x|: the
rounding of x_lo, the rounding of w_lo and the dropped w_lo x_lo.  Rounding
residuals are spread uniformly, so each has an rms of at most 2^-16 / sqrt 3
of |w| |x|, together 2^-16; an output sums 32 such products with unrelated
signs, so its rms relative error is at most 2^-16 as well.  The gradient
path holds four split passes (forward row, forward column, inverse column,
inverse row), which add in quadrature: 2 * 2^-16 rms.  The maximum error and
the maximum of D g over the field both sit about sqrt(2 ln M) rms above
their rms, so the ratio of maxima follows the ratio of rms; a factor 4 of
margin gives 8 * 2^-16 = 1.2e-4, plus 2e-5 for the fp32 arithmetic of the
other passes (the tolerance of the plain fp32 gradient test).  Dropping the
w_hi x_lo product leaves a residual of order 2^-9 per product, about 500
times the complete split's, which this bound rejects with a wide margin
(tests/test_split_bound.py)."""
import numpy as np

from oracle import fftlb_oracle as O
from oracle.cnn_oracle import bf16_round

SPLIT_GRADIENT_BOUND = 2e-5 + 8 * 2.0 ** -16
OPERAND = np.float32        # precision of the pass's operands before the split


def _split(z):
    z = np.asarray(z, np.float32)
    hi = bf16_round(z)
    lo = bf16_round((z - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def _split_dft16(x, direction, drop_hi_lo):
    """16-point DFT along axis 0 of x (complex, [16, ...]) as the real
    product [Re y; Im y] = [[Wr, -Wi], [Wi, Wr]] [Re x; Im x] with split
    operands."""
    m = np.arange(16)
    W = np.exp(direction * 2j * np.pi * np.outer(m, m) / 16)
    A = np.block([[W.real, -W.imag], [W.imag, W.real]])
    shape = x.shape
    xr = x.reshape(16, -1)
    X = np.concatenate([xr.real, xr.imag]).astype(OPERAND)
    ah, al = _split(A.astype(OPERAND))
    xh, xl = _split(X)
    Y = ah @ xh + al @ xh
    if not drop_hi_lo:
        Y = Y + ah @ xl
    return (Y[:16] + 1j * Y[16:]).reshape(shape)


def fft_split(x, direction, axis, drop_hi_lo=False):
    """Unnormalised DFT (direction -1 forward, +1 inverse) along `axis`
    with the first radix-16 Stockham pass split: y[j][m] = sum_t
    x[j + t n/16] W16^(t m), then X[m + 16 k] = sum_j W_n^(j m) y[j][m]
    W_{n/16}^(j k), the remaining passes, exact."""
    x = np.moveaxis(np.asarray(x, complex), axis, -1)
    n = x.shape[-1]
    nb = n // 16
    xt = x.reshape(x.shape[:-1] + (16, nb))                       # [..., t, j]
    y = np.moveaxis(_split_dft16(np.moveaxis(xt, -2, 0), direction, drop_hi_lo), 0, -2)   # [..., m, j]
    tw = np.exp(direction * 2j * np.pi * np.outer(np.arange(16), np.arange(nb)) / n)
    z = y * tw
    zk = np.fft.fft(z, axis=-1) if direction < 0 else np.fft.ifft(z, axis=-1) * nb
    out = np.moveaxis(zk, -2, -1).reshape(x.shape[:-1] + (n,))   # X[m + 16 k] = zk[m][k]
    return np.moveaxis(out, -1, axis)


def emulated_gradient(g, axis, dx, window, drop_hi_lo=False):
    """D_axis g along the CUDA path's route: real rows packed as h = nx/2
    complex values, row transform, real-to-complex post-processing, column
    transforms of the one-sided spectrum, multiplier i k_m (Nyquist bins
    zero), inverse columns, complex-to-real pre-processing, inverse rows.
    Split first passes on the row and column transforms of the h one-sided
    columns; the row-Nyquist column, which the CUDA path packs into column
    0, is transformed exactly here."""
    ny, nx = g.shape
    h = nx // 2
    k = np.arange(h)
    Z = fft_split(g[:, 0::2] + 1j * g[:, 1::2], -1, 1, drop_hi_lo)
    Zc = np.conj(Z[:, (-k) % h])
    X = 0.5 * (Z + Zc) - 0.5j * (Z - Zc) * np.exp(-2j * np.pi * k / nx)   # one-sided X[0 .. h-1]
    Xnyq = Z[:, 0].real - Z[:, 0].imag
    kx, ky = O.kappa(nx, dx, window).copy(), O.kappa(ny, dx, window).copy()
    kx[nx // 2] = 0.0                                                     # Nyquist bins
    ky[ny // 2] = 0.0
    F = fft_split(X, -1, 0, drop_hi_lo)
    mult = 1j * kx[None, :h] if axis == "x" else 1j * ky[:, None]
    G = fft_split(F * mult, +1, 0, drop_hi_lo) / ny
    Gnyq = np.fft.ifft(np.fft.fft(Xnyq) * (0.0 if axis == "x" else 1j * ky))
    Gh = np.conj(G[:, (h - k) % h])                                       # X[k + h]
    Gh[:, 0] = Gnyq
    Zs = (G + Gh) + 1j * (G - Gh) * np.exp(2j * np.pi * k / nx)
    z = fft_split(Zs, +1, 1, drop_hi_lo) / nx
    out = np.empty_like(g)
    out[:, 0::2], out[:, 1::2] = z.real, z.imag
    return out

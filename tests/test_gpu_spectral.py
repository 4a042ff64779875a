"""Parity of the CUDA windowed spectral derivative (Sec. 3.6; fftlb_gradient)
with the oracle's D, element by element, across windows, grid shapes
(powers of 2 and 3, ragged, tiny, full 1024^2) and precisions."""
import numpy as np
import pytest

from gpu_common import lib, rel_err
from oracle import fftlb_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fl():
    return lib()


def grad_gpu(fl, g, window, precision, dx=1 / 256):
    nf, ny, nx = g.shape
    with fl.Handle(fl.params(nx=nx, ny=ny, dx=dx, window=window, precision=precision)) as h:
        gd = torch.from_numpy(g).cuda()
        out = torch.empty((2 * nf, ny, nx), dtype=torch.float64, device="cuda")
        h.gradient(gd, out, nf)
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("shape", [(64, 64), (48, 96), (96, 48), (4, 8), (8, 4), (384, 128), (6, 6)])
@pytest.mark.parametrize("window", [0, 1, 4])
def test_gradient_fp64(fl, shape, window):
    rng = np.random.default_rng(sum(shape) + window)
    g = rng.standard_normal((3,) + shape)
    out = grad_gpu(fl, g, window, 64)
    for i in range(3):
        dx_o = O.D(g[i], "x", 1 / 256, window)
        dy_o = O.D(g[i], "y", 1 / 256, window)
        assert rel_err(out[2 * i], dx_o) < 1e-12
        assert rel_err(out[2 * i + 1], dy_o) < 1e-12


@pytest.mark.parametrize("shape", [(64, 64), (48, 96), (1024, 1024)])
def test_gradient_fp32(fl, shape):
    rng = np.random.default_rng(7)
    g = rng.standard_normal((2,) + shape)
    out = grad_gpu(fl, g, 4, 32)
    for i in range(2):
        assert rel_err(out[2 * i], O.D(g[i], "x", 1 / 256, 4)) < 2e-5
        assert rel_err(out[2 * i + 1], O.D(g[i], "y", 1 / 256, 4)) < 2e-5


def test_gradient_fp64_full_size(fl):
    rng = np.random.default_rng(8)
    g = rng.standard_normal((1, 1024, 1024))
    out = grad_gpu(fl, g, 4, 64)
    assert rel_err(out[0], O.D(g[0], "x", 1 / 256, 4)) < 1e-12
    assert rel_err(out[1], O.D(g[0], "y", 1 / 256, 4)) < 1e-12


def test_gradient_of_sine_is_exact_k4(fl):
    """Fig. 5: with k4 the derivative of sin(x) is exact to round-off."""
    N = 128
    dx = 2 * np.pi / N
    x = np.arange(N) * dx
    g = np.tile(np.sin(x), (N, 1))[None]
    out = grad_gpu(fl, g, 4, 64, dx=dx)
    assert np.abs(out[0] - np.cos(x)[None, :]).max() < 1e-13
    assert np.abs(out[1]).max() < 1e-13


@pytest.mark.parametrize("shape", [(256, 256), (1024, 1024), (512, 128)])
def test_gradient_split_bf16_within_split_bound(fl, shape):
    """Precision 32 | FFTLB_BF16SPLIT: the handle's gradient runs the
    stage's transform code, whose first radix-16 pass of every row and
    column transform is the split-BF16 DFT product on the tensor cores.
    Bound: split_emulation.SPLIT_GRADIENT_BOUND (1.4e-4 of max |D g|),
    derived from the split's rounding; a split pass without the w_hi x_lo
    product gives about 3.6e-3 (tests/test_split_bound.py).  The plain fp32
    path on the same input must stay below its own 2e-5, and the split
    path must differ from it (the tensor-core pass ran)."""
    from split_emulation import SPLIT_GRADIENT_BOUND
    rng = np.random.default_rng(11)
    g = rng.standard_normal((1,) + shape)
    split = grad_gpu(fl, g, 4, 32 | fl.BF16SPLIT)
    plain = grad_gpu(fl, g, 4, 32)
    for i, axis in enumerate(("x", "y")):
        ref = O.D(g[0], axis, 1 / 256, 4)
        es, e32 = rel_err(split[i], ref), rel_err(plain[i], ref)
        print("split-BF16 gradient %s %s: %.2e (fp32 %.2e, bound %.2e)" % (shape, axis, es, e32, SPLIT_GRADIENT_BOUND))
        assert es < SPLIT_GRADIENT_BOUND
        assert e32 < 2e-5
        assert not np.array_equal(split[i], plain[i])

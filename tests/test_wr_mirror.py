"""The warp-resident row transform (kernels_wr.cuh) on the host: its exact
index arithmetic against numpy's FFT, and its shared-memory accesses free
of bank conflicts for the P >= 16 row groups (CPU, no GPU)."""
import numpy as np
import pytest

import wr_mirror as M


@pytest.mark.parametrize("H", [512, 256, 128])
@pytest.mark.parametrize("direction", [-1, 1])
def test_row_transform_is_the_dft(H, direction):
    rng = np.random.default_rng(H)
    z = rng.standard_normal(H) + 1j * rng.standard_normal(H)
    for rsw in ((0, 1) if M.ROWCFG[H][1] == 8 else (0,)):
        got = M.row_fft_wr(z, H, direction, rsw)
        want = np.fft.fft(z) if direction < 0 else np.fft.ifft(z) * H
        assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("H", [512, 256, 128])
def test_transposed_positions_are_a_permutation(H):
    E, P = M.ROWCFG[H]
    for rsw in ((0, 1) if P == 8 else (0,)):
        pos = {M.tpos(H, l, k1, rsw) for l in range(P) for k1 in range(E)}
        assert pos == set(range(H))


@pytest.mark.parametrize("H", [512, 256])
def test_no_bank_conflicts(H):
    E, P = M.ROWCFG[H]
    rec = M.Recorder()
    z = np.zeros(H, complex)
    for row in range(32 // P):
        M.row_fft_wr(z, H, -1, 0, rec, row)
    assert rec.worst_conflict() == 1


@pytest.mark.parametrize("H", [512, 256, 128])
def test_real_rows_round_trip(H):
    """r2c post-processing of the packed row's transform is the one-sided
    spectrum (numpy rfft, Nyquist packed into X[0].imag), and c2r
    pre-processing + inverse transform returns 2H times the row."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal(2 * H)
    Z = M.row_fft_wr(x[0::2] + 1j * x[1::2], H, -1)
    X = M.r2c_post(Z, H)
    ref = np.fft.rfft(x)
    assert np.allclose(X[1:], ref[1:H]) and np.isclose(X[0].real, ref[0].real) and np.isclose(X[0].imag, ref[H].real)
    z = M.row_fft_wr(M.c2r_pre(X, H), H, +1)
    y = np.empty(2 * H)
    y[0::2], y[1::2] = z.real, z.imag
    assert np.allclose(y, 2 * H * x)


@pytest.mark.parametrize("NY", [1024, 512, 256, 128])
def test_column_tile_transform(NY):
    """kcol_wr's index arithmetic: forward, multiplier, inverse equals
    NY * IDFT(m DFT(x)) per column of the tile."""
    E, P, TW = M.COLCFG[NY]
    rng = np.random.default_rng(NY)
    tile = rng.standard_normal((NY, TW)) + 1j * rng.standard_normal((NY, TW))
    mult = rng.standard_normal((TW, NY)) + 1j * rng.standard_normal((TW, NY))
    got = M.col_conv_wr(tile, NY, mult)
    want = np.stack([np.fft.ifft(mult[c] * np.fft.fft(tile[:, c])) * NY for c in range(TW)], axis=1)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("NY", [1024, 512, 256, 128])
def test_column_tile_layout(NY):
    """The swizzled positions are a permutation of the tile; the rows a
    thread's in-place store overwrites were read by threads of its own warp
    (so __syncwarp orders them); no bank conflicts."""
    E, P, TW = M.COLCFG[NY]
    assert {M.cpos(NY, c, l, k1) for c in range(TW) for l in range(P) for k1 in range(E)} == set(range(TW * NY))
    for l in range(P):
        for c in range(TW):
            for k1 in range(E):
                pos = M.cpos(NY, c, l, k1)
                row, col = divmod(pos, TW)
                reader_l = row % P                    # stage 1 read row l' + P t
                assert col == c
                assert (c + TW * reader_l) // 32 == (c + TW * l) // 32
    assert M.worst_conflict_sets(M.col_access_sets(NY)) == 1


@pytest.mark.parametrize("H", [512, 256, 128])
def test_row_spectrum_times_ik(H):
    """r2c_post_wr2 (the separable split's row-spectrum derivative): its raw
    output is r2c_post_wr's, and the inverse of its i k_x X / nx output is
    the spectral x-derivative of the row (k_x zero at DC and Nyquist)."""
    rng = np.random.default_rng(H + 1)
    x = rng.standard_normal(2 * H)
    nx, dx = 2 * H, 1.0 / 64
    kxt = 2 * np.pi * np.arange(H + 1) / (nx * dx)
    kxt[H] = 0.0
    Z = M.row_fft_wr(x[0::2] + 1j * x[1::2], H, -1)
    raw, mul = M.r2c_post2(Z, H, kxt, 1.0 / nx)
    assert np.allclose(raw, M.r2c_post(Z, H))
    z = M.row_fft_wr(M.c2r_pre(mul, H), H, +1)
    d = np.empty(nx)
    d[0::2], d[1::2] = z.real, z.imag
    k = 2 * np.pi * np.arange(H + 1) / (nx * dx)
    k[H] = 0.0
    want = np.fft.irfft(1j * k * np.fft.rfft(x), n=nx)
    assert np.abs(d - want).max() < 1e-9 * np.abs(want).max()

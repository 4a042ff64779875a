"""Shared-memory destinations of the column kernels' tensor copies (CPU).

A tensor copy (cp.async.bulk.tensor) into shared memory needs a 128-byte
aligned destination.  The column kernels stage a job's one or two input
tiles of TW x ny complex values as ny / BOXR boxes of BOXR rows each (BOXR:
the largest divisor of ny up to 256): input s lands at s * tile_stride and
box j at j * BOXR * TW values after it.  This mirrors the engine's
acceptance rule for tile widths (fp32: 2 TW * 4 bytes a multiple of 16; box
offsets 128-byte aligned unless the tile is a single box) and checks every
destination of every accepted width on every valid grid length, fp32 and
fp64.  (A 4-row grid with TW = 2, whose second input tile started 64 bytes
into the buffer before tile_stride existed, raised a misaligned-address
fault.)"""
import pytest


def valid_len(n):
    if n < 4 or n % 2:
        return False
    while n % 2 == 0:
        n //= 2
    while n % 3 == 0:
        n //= 3
    return n == 1


def boxr(ny):
    return max(d for d in range(1, min(ny, 256) + 1) if ny % d == 0)


def tile_stride(TW, ny, cs):
    return ((TW * ny * cs + 127) // 128 * 128) // cs


@pytest.mark.parametrize("cs,rs", [(8, 4), (16, 8)])
def test_every_tensor_copy_destination_is_128_byte_aligned(cs, rs):
    checked = 0
    for ny in [n for n in range(4, 2049) if valid_len(n)]:
        B = boxr(ny)
        for TW in (8, 4, 2, 1):
            if (2 * TW * rs) % 16:
                continue
            if not (ny <= B or (B * TW * cs) % 128 == 0):     # the engine's boxes_aligned rule
                continue
            for s in (0, 1):
                for r0 in range(0, ny, B):
                    off = (s * tile_stride(TW, ny, cs) + r0 * TW) * cs
                    assert off % 128 == 0, (ny, TW, s, r0)
                    checked += 1
    assert checked > 100

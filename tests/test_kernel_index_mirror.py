"""Host mirrors of the index arithmetic of the power-of-two Stockham passes
in paper_1011_3582_gb300/csrc/fft_device.cuh, checked on the CPU.

Each mirror restates, in numpy, how a pass of the CUDA code decomposes a
butterfly index J into (transform b, butterfly jj), where it reads and
writes its R elements in a padded or unpadded layout (p(e) = e + e / 16),
and which twiddles it takes from the per-pass tables (T[t Ns + k] =
exp(-2 pi i t k / (Ns R)), built like pass_twiddles in engine_impl.cuh).
The checks:
  * the forward passes (pp_pass_p2 with the radix schedule of pp_fft_p2)
    compute the DFT, for every power-of-two length to 1024, both batch
    orders and every padding of source and destination;
  * the adjoint passes in reverse order (pp_pass_p2_adj) give n times the
    inverse DFT: forward + diagonal multiply + adjoint gives n IDFT(m DFT(x)),
    also with the last forward pass, the multiply and its adjoint fused in
    registers (pp_pass_p2_fused, the convection columns of pp_conv_p2);
  * the constant-stride addresses the passes use instead of padding each
    index (base + t (S + S/16), or base + t S inside one 16-element block)
    equal the padded indices wherever the code takes them;
  * the lane mapping of the split-BF16 first pass (tc_dft16_pass: lane
    (g, q) loads inputs 2q, 2q+1, 2q+8, 2q+9 of butterfly g and stores
    outputs g, g+8 of butterflies 2q, 2q+1) reads and writes exactly the
    elements of the scalar first pass and, with exact arithmetic, gives its
    result.
These test the design of the passes; the GPU parity tests run the kernels.
"""
import numpy as np
import pytest


def pad(e, on):
    return e + (e >> 4) if on else e


def schedule(logn, maxlr=4):
    """[(log radix, log Ns, table offset)] of pp_fft_p2 / p2_schedule."""
    out, lns, rem, off = [], 0, logn, 0
    while rem > 0:
        lr = maxlr if rem >= maxlr else rem
        out.append((lr, lns, off))
        if lns > 0:
            off += 1 << (lns + lr)
        lns += lr
        rem -= lr
    return out


def tables(n, maxlr=4):
    T = []
    for lr, lns, _ in schedule(n.bit_length() - 1, maxlr):
        if lns > 0:
            Ns, R = 1 << lns, 1 << lr
            T += [np.exp(-2j * np.pi * t * k / (Ns * R)) for t in range(R) for k in range(Ns)]
    return np.array(T, dtype=complex)


def decompose(J, nbatch, lognb, bfast):
    if bfast:
        return J & (nbatch - 1), J >> (nbatch.bit_length() - 1)
    return J >> lognb, J & ((1 << lognb) - 1)


def read_addrs(jj, nb, R, pad_on):
    """Addresses of jj + t nb: constant stride when nb >= 16 or n <= 16
    (as pp_pass_p2's rlin), else padded one by one."""
    if not pad_on or nb >= 16 or nb * R <= 16:
        step = nb + (nb >> 4) if pad_on else nb
        return [pad(jj, pad_on) + t * step for t in range(R)]
    return [pad(jj + t * nb, pad_on) for t in range(R)]


def write_addrs(idxD, Ns, R, pad_on):
    """Addresses of idxD + t Ns (pp_pass_p2's wlin)."""
    if not pad_on or Ns >= 16 or Ns * R <= 16:
        step = Ns + (Ns >> 4) if pad_on else Ns
        return [pad(idxD, pad_on) + t * step for t in range(R)]
    return [pad(idxD + t * Ns, pad_on) for t in range(R)]


def fwd_pass(src, dst, lay_s, lay_d, logn, nbatch, lr, lns, T, bfast):
    R, lognb, Ns = 1 << lr, logn - lr, 1 << lns
    nb = 1 << lognb
    (sbs, ses, ps), (dbs, des, pd) = lay_s, lay_d
    W = np.exp(-2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    for J in range(nbatch << lognb):
        b, jj = decompose(J, nbatch, lognb, bfast)
        k = jj & (Ns - 1)
        idxD = ((jj >> lns) << (lns + lr)) + k
        v = np.array([src[b * sbs + a * ses] for a in read_addrs(jj, nb, R, ps)])
        if Ns > 1:
            v[1:] *= np.array([T[t * Ns + k] for t in range(1, R)])
        v = W @ v
        for t, a in enumerate(write_addrs(idxD, Ns, R, pd)):
            dst[b * dbs + a * des] = v[t]


def adj_pass(src, dst, lay_s, lay_d, logn, nbatch, lr, lns, T, bfast):
    """pp_pass_p2_adj: reads where the forward pass writes, DFT(+1),
    conjugate twiddles, writes where the forward pass reads."""
    R, lognb, Ns = 1 << lr, logn - lr, 1 << lns
    nb = 1 << lognb
    (sbs, ses, ps), (dbs, des, pd) = lay_s, lay_d
    W = np.exp(2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    for J in range(nbatch << lognb):
        b, jj = decompose(J, nbatch, lognb, bfast)
        k = jj & (Ns - 1)
        idxD = ((jj >> lns) << (lns + lr)) + k
        v = np.array([src[b * sbs + a * ses] for a in write_addrs(idxD, Ns, R, ps)])
        v = W @ v
        if Ns > 1:
            v[1:] *= np.conj(np.array([T[t * Ns + k] for t in range(1, R)]))
        for t, a in enumerate(read_addrs(jj, nb, R, pd)):
            dst[b * dbs + a * des] = v[t]


def layout(n, nbatch, pad_on, bfast):
    """(bs, es, pad): batch-fast (column tiles: element stride nbatch) or
    element-fast (rows: batch stride = padded length)."""
    plen = pad(n - 1, pad_on) + 1
    return (1, nbatch, pad_on) if bfast else (plen, 1, pad_on)


def load(x, lay, n, nbatch):
    bs, es, p = lay
    buf = np.zeros(bs * (nbatch - 1) + es * (pad(n - 1, p) + 1) + nbatch, dtype=complex)
    for b in range(nbatch):
        for e in range(n):
            buf[b * bs + pad(e, p) * es] = x[b, e]
    return buf


def unload(buf, lay, n, nbatch):
    bs, es, p = lay
    return np.array([[buf[b * bs + pad(e, p) * es] for e in range(n)] for b in range(nbatch)])


def run_forward(x, bfast, pa, pb, maxlr=4):
    nbatch, n = x.shape
    logn = n.bit_length() - 1
    T = tables(n, maxlr)
    la, lb = layout(n, nbatch, pa, bfast), layout(n, nbatch, pb, bfast)
    bufs = [load(x, la, n, nbatch), load(np.zeros_like(x), lb, n, nbatch)]
    lays = [la, lb]
    where = 0
    for lr, lns, off in schedule(logn, maxlr):
        fwd_pass(bufs[where], bufs[where ^ 1], lays[where], lays[where ^ 1], logn, nbatch, lr, lns, T[off:], bfast)
        where ^= 1
    return unload(bufs[where], lays[where], n, nbatch), bufs, lays, where, T


@pytest.mark.parametrize("bfast", [False, True])
@pytest.mark.parametrize("pads", [(0, 1), (1, 0), (0, 0), (1, 1)])
def test_forward_passes_compute_the_dft(bfast, pads):
    rng = np.random.default_rng(1)
    for logn in range(1, 11):
        n = 1 << logn
        nbatch = 4 if bfast else 3
        if n > 256 and (bfast or pads != (0, 1)):
            continue   # the large lengths once, in the rows' layout
        x = rng.standard_normal((nbatch, n)) + 1j * rng.standard_normal((nbatch, n))
        y = run_forward(x, bfast, *pads)[0]
        assert np.abs(y - np.fft.fft(x, axis=1)).max() < 1e-10 * n


def test_radix8_first_schedule_computes_the_dft():
    rng = np.random.default_rng(2)
    for logn in (3, 6, 9):
        x = rng.standard_normal((2, 1 << logn)) + 0j
        y = run_forward(x, False, 0, 1, maxlr=3)[0]
        assert np.abs(y - np.fft.fft(x, axis=1)).max() < 1e-10 * (1 << logn)


@pytest.mark.parametrize("n", [16, 64, 128, 1024])
def test_adjoint_passes_and_fused_multiply(n):
    """Forward passes, a diagonal multiply, then the adjoint passes in reverse
    order: n IDFT(m DFT(x)), the convection and derivative columns."""
    rng = np.random.default_rng(n)
    nbatch = 4 if n <= 128 else 1
    x = rng.standard_normal((nbatch, n)) + 1j * rng.standard_normal((nbatch, n))
    m = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    logn = n.bit_length() - 1
    y, bufs, lays, where, T = run_forward(x, True, 0, 1)
    bufs[where] = load(y * m[None, :], lays[where], n, nbatch)
    for lr, lns, off in reversed(schedule(logn)):
        adj_pass(bufs[where], bufs[where ^ 1], lays[where], lays[where ^ 1], logn, nbatch, lr, lns, T[off:], True)
        where ^= 1
    got = unload(bufs[where], lays[where], n, nbatch)
    want = n * np.fft.ifft(m[None, :] * np.fft.fft(x, axis=1), axis=1)
    assert np.abs(got - want).max() < 1e-9 * n


def fused_pass(buf, lay, logn, nbatch, lr, lns, T, mult, bfast):
    """pp_pass_p2_fused: the last forward pass, the multiply of output
    element idxD + t Ns of transform b, and its adjoint, in registers, read
    from and written back to the same positions jj + t nb."""
    R, lognb, Ns = 1 << lr, logn - lr, 1 << lns
    nb = 1 << lognb
    bs, es, p = lay
    Wf = np.exp(-2j * np.pi * np.outer(np.arange(R), np.arange(R)) / R)
    for J in range(nbatch << lognb):
        b, jj = decompose(J, nbatch, lognb, bfast)
        k = jj & (Ns - 1)
        idxD = ((jj >> lns) << (lns + lr)) + k
        addrs = [b * bs + a * es for a in read_addrs(jj, nb, R, p)]
        v = buf[addrs].copy()
        tw = np.array([T[t * Ns + k] for t in range(R)]) if Ns > 1 else np.ones(R)
        v = Wf @ (v * tw)
        v = v * np.array([mult(b, idxD + t * Ns) for t in range(R)])
        v = np.conj(tw) * (np.conj(Wf) @ v)
        buf[addrs] = v


@pytest.mark.parametrize("n", [4, 32, 256, 1024])
def test_fused_last_pass(n):
    """Forward passes 1 .. L-1, the fused pass L, adjoint passes L-1 .. 1
    (pp_conv_p2): n IDFT(m DFT(x)) with 2L - 1 passes."""
    rng = np.random.default_rng(n + 1)
    nbatch = 4 if n <= 256 else 1
    logn = n.bit_length() - 1
    x = rng.standard_normal((nbatch, n)) + 1j * rng.standard_normal((nbatch, n))
    m = rng.standard_normal((nbatch, n)) + 1j * rng.standard_normal((nbatch, n))
    T = tables(n)
    lays = [layout(n, nbatch, 0, True), layout(n, nbatch, 1, True)]
    bufs = [load(x, lays[0], n, nbatch), load(np.zeros_like(x), lays[1], n, nbatch)]
    sched = schedule(logn)
    where = 0
    for lr, lns, off in sched[:-1]:
        fwd_pass(bufs[where], bufs[where ^ 1], lays[where], lays[where ^ 1], logn, nbatch, lr, lns, T[off:], True)
        where ^= 1
    lr, lns, off = sched[-1]
    fused_pass(bufs[where], lays[where], logn, nbatch, lr, lns, T[off:], lambda b, e: m[b, e], True)
    for lr, lns, off in reversed(sched[:-1]):
        adj_pass(bufs[where], bufs[where ^ 1], lays[where], lays[where ^ 1], logn, nbatch, lr, lns, T[off:], True)
        where ^= 1
    got = unload(bufs[where], lays[where], n, nbatch)
    want = n * np.fft.ifft(m * np.fft.fft(x, axis=1), axis=1)
    assert np.abs(got - want).max() < 1e-9 * n


def test_constant_stride_addresses_equal_the_padded_indices():
    bad = 0
    for logn in range(1, 13):
        for lr in (1, 2, 3, 4):
            if lr > logn:
                continue
            R, nb = 1 << lr, 1 << (logn - lr)
            for lns in range(0, logn - lr + 1):
                Ns = 1 << lns
                for jj in range(nb):
                    idxD = ((jj >> lns) << (lns + lr)) + (jj & (Ns - 1))
                    bad += read_addrs(jj, nb, R, True) != [pad(jj + t * nb, True) for t in range(R)]
                    bad += write_addrs(idxD, Ns, R, True) != [pad(idxD + t * Ns, True) for t in range(R)]
    assert bad == 0


@pytest.mark.parametrize("bfast,adj", [(False, False), (True, False), (True, True)])
def test_tensor_core_first_pass_lane_mapping(bfast, adj):
    """tc_dft16_pass with exact arithmetic: the union of the lanes' loads and
    stores is the scalar first pass's, every element is stored once, and the
    result is the 16-point DFT (forward, or +1 for the adjoint)."""
    rng = np.random.default_rng(7)
    for logn, nbatch in ((9, 6), (4, 3), (6, 5), (10, 2), (8, 4)):
        if bfast and nbatch & (nbatch - 1):
            continue
        lognb = logn - 4
        nb, total = 1 << lognb, nbatch << lognb
        n = 1 << logn
        direction = 1 if adj else -1
        W = np.exp(direction * 2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
        src = rng.standard_normal((nbatch, n)) + 1j * rng.standard_normal((nbatch, n))
        dst = np.full((nbatch, n), np.nan + 0j)
        loads, stores = [], []
        for J0 in range(0, total, 8):                        # one warp's group of 8 butterflies
            B = np.zeros((16, 8), dtype=complex)
            for lane in range(32):
                g, q = lane >> 2, lane & 3
                J = J0 + g
                if J >= total:
                    continue
                b, jj = decompose(J, nbatch, lognb, bfast)
                for i in range(4):
                    t = 2 * q + (i & 1) + (i >> 1) * 8
                    e = (jj << 4) + t if adj else jj + t * nb
                    loads.append((b, e))
                    B[t, g] = src[b, e]
            Y = W @ B
            for lane in range(32):
                g, q = lane >> 2, lane & 3
                for c in range(2):
                    Jo = J0 + 2 * q + c
                    if Jo >= total:
                        continue
                    b, jo = decompose(Jo, nbatch, lognb, bfast)
                    for hh in range(2):
                        m = g + 8 * hh
                        e = jo + m * nb if adj else (jo << 4) + m
                        stores.append((b, e))
                        dst[b, e] = Y[m, 2 * q + c]
        ref_l, ref = [], np.full((nbatch, n), np.nan + 0j)
        for J in range(total):
            b, jj = decompose(J, nbatch, lognb, bfast)
            ins = [(jj << 4) + t for t in range(16)] if adj else [jj + t * nb for t in range(16)]
            outs = [jj + t * nb for t in range(16)] if adj else [(jj << 4) + t for t in range(16)]
            ref_l += [(b, e) for e in ins]
            ref[b, outs] = W @ src[b, ins]
        assert sorted(loads) == sorted(ref_l)
        assert len(set(stores)) == len(stores) == total * 16
        assert np.abs(dst - ref).max() < 1e-12

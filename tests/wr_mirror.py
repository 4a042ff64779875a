"""Host mirror of the warp-resident row transform of kernels_wr.cuh
(row_fft_wr, r2c_post_wr, c2r_pre_wr): the same index arithmetic, with
numpy arrays for a row group's shared-memory row and its lanes' registers,
so that tests can check it against numpy's FFT and count shared-memory
bank conflicts without a GPU.  Test infrastructure: no method arithmetic."""
import numpy as np

ROWCFG = {512: (16, 32), 256: (16, 16), 128: (16, 8)}   # H: (E, P)


def tpos(H, l, k1, rsw):
    E, P = ROWCFG[H]
    return ((k1 ^ rsw) * P) + (l ^ (k1 & (P - 1)))


def dft(v, direction):
    n = len(v)
    m = np.arange(n)
    return np.exp(direction * 2j * np.pi * np.outer(m, m) / n) @ v


class Recorder:
    """Records every shared-memory access as (instruction id, lane, word)."""

    def __init__(self):
        self.acc = {}

    def add(self, iid, lane, word):
        self.acc.setdefault(iid, []).append((lane, word))

    def worst_conflict(self, word_bytes=8):
        """Largest number of distinct words one bank serves in one
        half-warp (8-byte accesses) or warp (4-byte) of one instruction."""
        worst = 1
        for iid, lst in self.acc.items():
            groups = {}
            for lane, w in lst:
                grp = lane // 16 if word_bytes == 8 else 0
                groups.setdefault(grp, set()).add(w)
            for ws in groups.values():
                banks = {}
                for w in ws:
                    b = (w * word_bytes // 4) % 32
                    banks.setdefault(b, set()).add(w)
                worst = max(worst, max(len(s) for s in banks.values()))
        return worst


def row_fft_wr(z, H, direction, rsw=0, rec=None, row=0):
    """Emulates row_fft_wr on the row z (complex array of length H) for one
    row group; returns the transformed row (z is not modified)."""
    E, P = ROWCFG[H]
    z = z.astype(complex).copy()
    tw = np.exp(-2j * np.pi * np.outer(np.arange(E), np.arange(P)) / H)   # tw[k1, l]
    lane0 = (row % (32 // P)) * P if P < 32 else 0
    regs = []
    for j in range(P):
        v = np.array([z[j + P * t] for t in range(E)])
        if rec:
            for t in range(E):
                rec.add(("s1load", t), lane0 + j, row * H + j + P * t)
        v = dft(v, direction)
        w = tw[:, j] if direction < 0 else np.conj(tw[:, j])
        regs.append(v * w)
    for j in range(P):
        for k1 in range(E):
            z[tpos(H, j, k1, rsw)] = regs[j][k1]
            if rec:
                rec.add(("tstore", k1), lane0 + j, row * H + tpos(H, j, k1, rsw))
    out = z.copy()
    if P <= E:
        for j in range(P):
            for q in range(E // P):
                k1 = j + P * q
                u = np.array([z[tpos(H, l, k1, rsw)] for l in range(P)])
                if rec:
                    for l in range(P):
                        rec.add(("s2load", q, l), lane0 + j, row * H + tpos(H, l, k1, rsw))
                u = dft(u, direction)
                for k2 in range(P):
                    out[k1 + E * k2] = u[k2]
                    if rec:
                        rec.add(("nstore", q, k2), lane0 + j, row * H + k1 + E * k2)
        return out
    assert P == 2 * E
    HE = E // 2
    V = {}
    for j in range(P):
        k1, g = j & (E - 1), j // E
        u = np.array([z[tpos(H, g + 2 * m, k1, 0)] for m in range(E)])
        if rec:
            for m in range(E):
                rec.add(("s2load", m), j, tpos(H, g + 2 * m, k1, 0))
        V[j] = dft(u, direction)
    for j in range(P):
        k1, g = j & (E - 1), j // E
        partner = j ^ E
        for i in range(HE):
            send_p = V[partner][i] if (partner // E) else V[partner][HE + i]   # what the partner sends
            a = send_p if g else V[j][i]
            b = V[j][HE + i] if g else send_p
            w = np.exp(direction * 2j * np.pi * i / 32)
            t = b * w
            if g:
                t = t * (-1j if direction < 0 else 1j)
            k2 = HE * g + i
            out[k1 + E * k2] = a + t
            out[k1 + E * (k2 + E)] = a - t
            if rec:
                rec.add(("nstore", i, 0), j, k1 + E * k2)
                rec.add(("nstore", i, 1), j, k1 + E * (k2 + E))
    return out


def r2c_post(Z, H):
    """Emulates r2c_post_wr: packed one-sided spectrum from the transform Z."""
    out = np.zeros(H, complex)
    Wp = np.exp(-2j * np.pi * np.arange(H // 2 + 1) / (2 * H))
    for k in range(H // 2 + 1):
        if k == 0:
            out[0] = complex(Z[0].real + Z[0].imag, Z[0].real - Z[0].imag)
            continue
        p, q = Z[k], Z[H - k]
        ze = 0.5 * (p + np.conj(q))
        zo = -0.5j * (p - np.conj(q))
        wz = Wp[k] * zo
        out[k] = ze + wz
        if H - k != k:
            out[H - k] = np.conj(ze - wz)
    return out


def r2c_post2(Z, H, kxt, sx):
    """Emulates r2c_post_wr2: the one-sided spectrum X as r2c_post_wr writes
    it (raw) and i k_x X / nx (mul, sx = 1 / nx), pair by pair (k, H - k) as
    the lanes take them, k_x looked up at both bins of the pair."""
    raw = np.zeros(H, complex)
    mul = np.zeros(H, complex)
    Wp = np.exp(-2j * np.pi * np.arange(H // 2 + 1) / (2 * H))
    for k in range(H // 2 + 1):
        if k == 0:
            a = complex(Z[0].real + Z[0].imag, Z[0].real - Z[0].imag)
            b = None
        else:
            p, q = Z[k], Z[H - k]
            ze = 0.5 * (p + np.conj(q))
            zo = -0.5j * (p - np.conj(q))
            wz = Wp[k] * zo
            a, b = ze + wz, np.conj(ze - wz)
        raw[k] = a
        mul[k] = 1j * (kxt[k] * sx) * a
        if k != 0 and H - k != k:
            raw[H - k] = b
            mul[H - k] = 1j * (kxt[H - k] * sx) * b
    return raw, mul


def c2r_pre(X, H):
    """Emulates c2r_pre_wr."""
    z = X.astype(complex).copy()
    Wp = np.exp(-2j * np.pi * np.arange(H // 2 + 1) / (2 * H))
    for k in range(H // 2 + 1):
        if k == 0:
            z[0] = complex(X[0].real + X[0].imag, X[0].real - X[0].imag)
            continue
        p, q = X[k], X[H - k]
        w = Wp[k]
        z[k] = (p + np.conj(q)) + 1j * ((p - np.conj(q)) * np.conj(w))
        if H - k != k:
            z[H - k] = (q + np.conj(p)) + 1j * ((q - np.conj(p)) * (-w))
    return z


COLCFG = {1024: (32, 32, 8), 512: (32, 16, 16), 256: (16, 16, 16), 128: (16, 8, 32)}   # NY: (E, P, TW)


def cpos(NY, c, l, k1):
    E, P, TW = COLCFG[NY]
    SW = 16 // TW - 1 if TW < 16 else 0
    return (k1 * P + (l ^ (k1 & SW))) * TW + c


def col_conv_wr(tile, NY, mult, rec=None):
    """Emulates kcol_wr's transforms on a tile [NY][TW] (complex): stage 1,
    in-place swizzled store, stage 2 with the per-element multiplier
    mult[c][k], inverse, stage 1 inverse; returns the [NY][TW] result
    (unnormalised: NY * IDFT(mult * DFT))."""
    E, P, TW = COLCFG[NY]
    T = tile.reshape(-1).astype(complex).copy()
    tw = np.exp(-2j * np.pi * np.outer(np.arange(E), np.arange(P)) / NY)   # tw[k1, l]
    thread = lambda c, l: c + TW * l
    regs = {}
    for l in range(P):
        for c in range(TW):
            v = np.array([T[(l + P * t) * TW + c] for t in range(E)])
            if rec:
                for t in range(E):
                    rec.add(("s1load", t), thread(c, l) % 32 + 32 * 0, ((l + P * t) * TW + c, thread(c, l) // 32))
            regs[(c, l)] = dft(v, -1) * tw[:, l]
    for (c, l), v in regs.items():
        for k1 in range(E):
            T[cpos(NY, c, l, k1)] = v[k1]
    for c in range(TW):
        for j in range(P):
            for q in range(E // P):
                k1 = j + P * q
                u = np.array([T[cpos(NY, c, l, k1)] for l in range(P)])
                X = dft(u, -1)
                Y = X * np.array([mult[c][k1 + E * k2] for k2 in range(P)])
                w = dft(Y, +1) * np.conj(tw[k1, :])
                for l in range(P):
                    T[cpos(NY, c, l, k1)] = w[l]
    out = np.empty((NY, TW), complex)
    for l in range(P):
        for c in range(TW):
            v = np.array([T[cpos(NY, c, l, k1)] for k1 in range(E)])
            y = dft(v, +1)
            for t in range(E):
                out[l + P * t, c] = y[t]
    return out


def col_access_sets(NY):
    """(instruction, warp) -> {lane: word} of kcol_wr's shared-memory tile
    accesses, for bank-conflict counting."""
    E, P, TW = COLCFG[NY]
    sets = {}
    for tid in range(TW * P):
        c, jl = tid % TW, tid // TW
        w, lane = tid // 32, tid % 32
        for t in range(E):
            sets.setdefault(("s1load", t, w), {})[lane] = (jl + P * t) * TW + c
        for k1 in range(E):
            sets.setdefault(("s1store", k1, w), {})[lane] = cpos(NY, c, jl, k1)
        for q in range(E // P):
            for l in range(P):
                sets.setdefault(("s2", q, l, w), {})[lane] = cpos(NY, c, l, jl + P * q)
        # twiddle tables (8-byte words from a separate base): stage 1 reads
        # twc[k1 P + l], stage 2 reads twt[l E + k1]
        for k1 in range(1, E):
            sets.setdefault(("tw1", k1, w), {})[lane] = 10 ** 6 + k1 * P + jl
        for q in range(E // P):
            for l in range(1, P):
                sets.setdefault(("tw2", q, l, w), {})[lane] = 2 * 10 ** 6 + l * E + jl + P * q
    return sets


def worst_conflict_sets(sets):
    worst = 1
    for lanes in sets.values():
        for half in (0, 1):
            ws = {w for ln, w in lanes.items() if ln // 16 == half}
            banks = {}
            for w in ws:
                banks.setdefault((2 * w) % 32, set()).add(w)
            if banks:
                worst = max(worst, max(len(v) for v in banks.values()))
    return worst

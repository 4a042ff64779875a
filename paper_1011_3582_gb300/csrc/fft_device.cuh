// Device building blocks of the windowed-FFT derivative (arXiv:1011.3582,
// Sec. 3.6, Fig. 3: transform, multiply by i k_m, inverse transform):
// complex arithmetic, a batched in-place shared-memory Stockham FFT with
// radix-4/2/3 passes, and the packing of a length-N real row into a
// length-N/2 complex transform (forward and inverse).
//
// Conventions: forward transform X[k] = sum_n x[n] exp(-2 pi i k n / N)
// (unnormalised, the sum of Eq. FT without the dx factor); inverse
// x[n] = sum_k X[k] exp(+2 pi i k n / N) (unnormalised; the 1/(nx ny) of
// Eq. IFT is folded into the spectral multipliers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fftlb {

template <typename real> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// i * a and -i * a
template <typename C> __device__ __forceinline__ C cmul_i(C a) { return C{-a.y, a.x}; }
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return C{a.y, -a.x}; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }

// Small DFTs; DIR = -1 forward, +1 inverse.
template <int R, int DIR, typename C> struct SmallDFT;

template <int DIR, typename C> struct SmallDFT<2, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        C a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <int DIR, typename C> struct SmallDFT<4, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        C s0 = cadd(v[0], v[2]), s1 = csub(v[0], v[2]);
        C s2 = cadd(v[1], v[3]), s3 = csub(v[1], v[3]);
        // forward: W4 = -i; inverse: W4 = +i
        C r3 = (DIR < 0) ? cmul_mi(s3) : cmul_i(s3);
        v[0] = cadd(s0, s2);
        v[2] = csub(s0, s2);
        v[1] = cadd(s1, r3);
        v[3] = csub(s1, r3);
    }
};

template <int DIR, typename C> struct SmallDFT<3, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        using R = decltype(v[0].x);
        const R c = R(-0.5);
        const R s = R(DIR) * R(0.86602540378443864676372317075294);
        C t1 = cadd(v[1], v[2]);
        C t2 = C{v[0].x + c * t1.x, v[0].y + c * t1.y};
        C d = csub(v[1], v[2]);
        C t3 = C{-s * d.y, s * d.x};   // i * s * (v1 - v2)
        v[0] = cadd(v[0], t1);
        v[1] = cadd(t2, t3);
        v[2] = csub(t2, t3);
    }
};

template <int DIR, typename C> struct SmallDFT<8, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        using R = decltype(v[0].x);
        const R h = R(0.70710678118654752440084436210485);
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        SmallDFT<4, DIR, C>::run(e);
        SmallDFT<4, DIR, C>::run(o);
        // o_k *= W8^k, W8 = exp(DIR 2 pi i / 8)
        C o1 = (DIR < 0) ? C{h * (o[1].x + o[1].y), h * (o[1].y - o[1].x)}
                         : C{h * (o[1].x - o[1].y), h * (o[1].y + o[1].x)};
        C o2 = (DIR < 0) ? cmul_mi(o[2]) : cmul_i(o[2]);
        C o3 = (DIR < 0) ? C{h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y)}
                         : C{-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y)};
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    }
};

// z * exp(DIR i pi m / 8) for the products m = b k1 of the radix-16 split
template <int DIR, typename C>
__device__ __forceinline__ C mul_w16(C z, int m) {
    using R = decltype(z.x);
    const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);
    const R h = R(0.70710678118654752440);
    R wr, wi;
    switch (m) {
        case 0: return z;
        case 1: wr = c1; wi = s1; break;
        case 2: wr = h; wi = h; break;
        case 3: wr = s1; wi = c1; break;
        case 4: return (DIR < 0) ? cmul_mi(z) : cmul_i(z);
        case 6: wr = -h; wi = h; break;
        default: wr = -c1; wi = -s1; break;   // m = 9
    }
    wi = (DIR < 0) ? -wi : wi;
    return cmul(z, C{wr, wi});
}

// radix 16 as 4 x 4: z[b][k1] = DFT4_a x[4a + b]; z *= W16^(b k1);
// y[k1 + 4 k2] = DFT4_b z[b][k1]
template <int DIR, typename C> struct SmallDFT<16, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        C z[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
#pragma unroll
            for (int a = 0; a < 4; ++a) z[b][a] = v[4 * a + b];
            SmallDFT<4, DIR, C>::run(z[b]);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) z[b][k1] = mul_w16<DIR>(z[b][k1], b * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C t[4] = {z[0][k1], z[1][k1], z[2][k1], z[3][k1]};
            SmallDFT<4, DIR, C>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
        }
    }
};

// Layout of a batch of transforms in shared memory: element e of transform
// b sits at b * bs + p(e) * es, where p(e) = e, or e + e / 16 for padded
// work buffers (one pad slot per 16 elements breaks the power-of-two strides
// of the first Stockham pass across banks).
struct Lay {
    int bs, es, pad;
    __device__ __forceinline__ int operator()(int b, int e) const { return b * bs + (pad ? e + (e >> 4) : e) * es; }
};

__host__ __device__ inline int padded_len(int n) { return n + (n >> 4); }

// One out-of-place Stockham pass of radix R over nbatch length-n transforms
// (src in layout ls, dst in layout ld).  Each thread works one butterfly at a
// time, so at most R complex values are live.  With BFAST the transform
// index varies fastest across threads (contiguous column tiles), otherwise
// the butterfly index does (contiguous rows).
template <int R, int DIR, bool BFAST, typename C>
__device__ __forceinline__ void pp_pass(const C *src, Lay ls, C *dst, Lay ld, int n, int nbatch, int Ns, const C *W,
                                        int tid, int nthr) {
    const int nb = n / R;
    const int total = nb * nbatch;
    const int wstride = n / (Ns * R);
    for (int J = tid; J < total; J += nthr) {
        int b, jj;
        if (BFAST) {
            b = J % nbatch;
            jj = J / nbatch;
        } else {
            b = J / nb;
            jj = J - b * nb;
        }
        const int k = jj % Ns;
        C v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            C x = src[ls(b, jj + t * nb)];
            if (t > 0 && Ns > 1) {
                C w = W[t * k * wstride];
                if (DIR > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[t] = x;
        }
        SmallDFT<R, DIR, C>::run(v);
        const int idxD = (jj / Ns) * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) dst[ld(b, idxD + t * Ns)] = v[t];
    }
}

// Complete transforms (radices 16, 8, 4, 2, 3 in that preference), passes
// alternating between A (layout la) and B (layout lb).  Callers synchronise
// before; every pass ends with a block barrier.  Returns 0 if the result is
// in A, 1 if it is in B.
template <int DIR, bool BFAST, typename C>
__device__ int pp_fft(C *A, Lay la, C *B, Lay lb, int n, int nbatch, const C *W, int tid, int nthr) {
    int Ns = 1, rem = n, where = 0;
    while (rem > 1) {
        const C *src = where ? B : A;
        C *dst = where ? A : B;
        const Lay ls = where ? lb : la, ld = where ? la : lb;
        int R;
        if ((rem & 15) == 0) {
            R = 16;
            pp_pass<16, DIR, BFAST>(src, ls, dst, ld, n, nbatch, Ns, W, tid, nthr);
        } else if ((rem & 7) == 0) {
            R = 8;
            pp_pass<8, DIR, BFAST>(src, ls, dst, ld, n, nbatch, Ns, W, tid, nthr);
        } else if ((rem & 3) == 0) {
            R = 4;
            pp_pass<4, DIR, BFAST>(src, ls, dst, ld, n, nbatch, Ns, W, tid, nthr);
        } else if ((rem & 1) == 0) {
            R = 2;
            pp_pass<2, DIR, BFAST>(src, ls, dst, ld, n, nbatch, Ns, W, tid, nthr);
        } else {
            R = 3;
            pp_pass<3, DIR, BFAST>(src, ls, dst, ld, n, nbatch, Ns, W, tid, nthr);
        }
        __syncthreads();
        Ns *= R;
        rem /= R;
        where ^= 1;
    }
    return where;
}

// r2c_post / c2r_pre (below) on rows in an arbitrary layout
template <typename C>
__device__ __forceinline__ void r2c_post_l(C *a, Lay L, int h, int batch, const C *Wp, int tid, int nthr) {
    using R = decltype(a[0].x);
    const int npair = h / 2 + 1;
    for (int j = tid; j < npair * batch; j += nthr) {
        const int row = j / npair;
        const int k = j - row * npair;
        if (k == 0) {
            const int i0 = L(row, 0);
            C z0 = a[i0];
            a[i0] = C{z0.x + z0.y, z0.x - z0.y};
        } else {
            const int ik = L(row, k), ih = L(row, h - k);
            C p = a[ik], q = a[ih];
            C ze = cscale(cadd(p, cconj(q)), R(0.5));
            C zo = cscale(cmul_mi(csub(p, cconj(q))), R(0.5));
            C wz = cmul(Wp[k], zo);
            a[ik] = cadd(ze, wz);
            if (h - k != k) a[ih] = cconj(csub(ze, wz));
        }
    }
}

template <typename C>
__device__ __forceinline__ void c2r_pre_l(C *a, Lay L, int h, int batch, const C *Wp, int tid, int nthr) {
    const int npair = h / 2 + 1;
    for (int j = tid; j < npair * batch; j += nthr) {
        const int row = j / npair;
        const int k = j - row * npair;
        if (k == 0) {
            const int i0 = L(row, 0);
            C x0 = a[i0];
            a[i0] = C{x0.x + x0.y, x0.x - x0.y};
        } else {
            const int ik = L(row, k), ih = L(row, h - k);
            C p = a[ik], q = a[ih];
            C w = Wp[k];
            C wc = cconj(w);
            a[ik] = cadd(cadd(p, cconj(q)), cmul_i(cmul(csub(p, cconj(q)), wc)));
            if (h - k != k) {
                C mw = C{-w.x, -w.y};
                a[ih] = cadd(cadd(q, cconj(p)), cmul_i(cmul(csub(q, cconj(p)), mw)));
            }
        }
    }
}

struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// One Stockham pass of radix R over `batch` independent length-n arrays
// stored contiguously (row r at a + r*n), done in place: every thread first
// loads and transforms its butterflies into registers, then (after a block
// barrier) writes them to their auto-sorted positions.  Ns is the length of
// the sub-transforms already completed.  W[m] = exp(-2 pi i m / n).
// Requires batch * n <= 16 * nthr.
template <int R, int DIR, typename C>
__device__ __forceinline__ void fft_pass(C *a, int n, int batch, int Ns, const C *W, int tid, int nthr) {
    constexpr int MAXB = (R == 3) ? 6 : 16 / R;
    const int nb = n / R;
    const int total = nb * batch;
    const int wstride = n / (Ns * R);
    C v[MAXB][R];
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j = tid + b * nthr;
        if (j < total) {
            const int row = j / nb;
            const int jj = j - row * nb;
            const int k = jj % Ns;
            const C *base = a + row * n;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                C x = base[jj + t * nb];
                if (t > 0) {
                    C w = W[t * k * wstride];
                    if (DIR > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[b][t] = x;
            }
            SmallDFT<R, DIR, C>::run(v[b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MAXB; ++b) {
        const int j = tid + b * nthr;
        if (j < total) {
            const int row = j / nb;
            const int jj = j - row * nb;
            const int k = jj % Ns;
            const int idxD = (jj / Ns) * Ns * R + k;
            C *base = a + row * n;
#pragma unroll
            for (int t = 0; t < R; ++t) base[idxD + t * Ns] = v[b][t];
        }
    }
    __syncthreads();
}

// Complete in-place transform of `batch` rows of length n = 2^p 3^q held in
// shared memory.  Must be called by all threads of the block (barriers).
template <int DIR, typename C>
__device__ void block_fft(C *a, int n, int batch, const C *W, int tid, int nthr) {
    int Ns = 1, rem = n;
    while (rem > 1) {
        if ((rem & 3) == 0) {
            fft_pass<4, DIR>(a, n, batch, Ns, W, tid, nthr);
            Ns *= 4;
            rem >>= 2;
        } else if ((rem & 1) == 0) {
            fft_pass<2, DIR>(a, n, batch, Ns, W, tid, nthr);
            Ns *= 2;
            rem >>= 1;
        } else {
            fft_pass<3, DIR>(a, n, batch, Ns, W, tid, nthr);
            Ns *= 3;
            rem /= 3;
        }
    }
}

// Real-to-complex post-processing.  Row r of `a` (length h = N/2) holds
// Z = FFT_h(x[2m] + i x[2m+1]); it is replaced by the one-sided spectrum
// X[0..h-1] of the real row x (length N), with the real Nyquist value X[h]
// packed into the imaginary part of X[0].  Wp[k] = exp(-2 pi i k / N).
// Pairs (k, h-k) are handled by one thread, so no barrier is needed
// inside; the caller synchronises before and after.
template <typename C>
__device__ __forceinline__ void r2c_post(C *a, int h, int batch, const C *Wp, int tid, int nthr) {
    using R = decltype(a[0].x);
    const int npair = h / 2 + 1;   // k = 0 .. h/2
    for (int j = tid; j < npair * batch; j += nthr) {
        const int row = j / npair;
        const int k = j - row * npair;
        C *z = a + row * h;
        if (k == 0) {
            C z0 = z[0];
            z[0] = C{z0.x + z0.y, z0.x - z0.y};
        } else {
            C p = z[k], q = z[h - k];
            C ze = cscale(cadd(p, cconj(q)), R(0.5));
            C zo = cscale(cmul_mi(csub(p, cconj(q))), R(0.5));   // (p - conj q) / (2i)
            C wz = cmul(Wp[k], zo);
            z[k] = cadd(ze, wz);
            if (h - k != k) z[h - k] = cconj(csub(ze, wz));
        }
    }
}

// Inverse of r2c_post: from the packed one-sided spectrum, form
// Z[k] = (X[k] + X[k + h]) + i (X[k] - X[k + h]) exp(+2 pi i k / N) (with
// X[k + h] = conj X[h - k]), whose unnormalised length-h inverse FFT z gives
// the unnormalised real inverse x[2m] = Re z[m], x[2m+1] = Im z[m].
template <typename C>
__device__ __forceinline__ void c2r_pre(C *a, int h, int batch, const C *Wp, int tid, int nthr) {
    const int npair = h / 2 + 1;
    for (int j = tid; j < npair * batch; j += nthr) {
        const int row = j / npair;
        const int k = j - row * npair;
        C *z = a + row * h;
        if (k == 0) {
            C x0 = z[0];   // (X[0], X[h])
            z[0] = C{x0.x + x0.y, x0.x - x0.y};
        } else {
            C p = z[k], q = z[h - k];
            C w = Wp[k];
            C wc = cconj(w);
            z[k] = cadd(cadd(p, cconj(q)), cmul_i(cmul(csub(p, cconj(q)), wc)));
            if (h - k != k) {
                C mw = C{-w.x, -w.y};
                z[h - k] = cadd(cadd(q, cconj(p)), cmul_i(cmul(csub(q, cconj(p)), mw)));
            }
        }
    }
}

}  // namespace fftlb

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
// Z[k] = (X[k] + X[k + h]) + i (X[k] - X[k + h]) exp(+2 pi i k / N), whose
// length-h inverse FFT z gives x[2m] = Re z[m], x[2m+1] = Im z[m] (times N/...
// unnormalised: x = sum over all N modes).
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

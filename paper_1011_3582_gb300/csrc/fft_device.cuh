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

#include <type_traits>

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

#ifndef FFTLB_NO_PACKED_F32X2
// fp32 complex add / subtract as one packed FP32x2 instruction (sm_100+)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
#endif
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

// z * (wr + i DIR wi) for the constant twiddles of the radix-16 split
template <int DIR, typename C, typename R>
__device__ __forceinline__ C mul_wc(C z, R wr, R wi) {
    const R s = (DIR < 0) ? -wi : wi;
    return C{z.x * wr - z.y * s, z.x * s + z.y * wr};
}

// radix 16 as 4 x 4: z[b][k1] = DFT4_a x[4a + b]; z *= W16^(b k1);
// y[k1 + 4 k2] = DFT4_b z[b][k1].  The nine non-trivial W16^(b k1),
// exp(DIR i pi m / 8) for m = b k1 in {1, 2, 3, 2, 4, 6, 3, 6, 9}, are
// written out so that every factor is a compile-time constant.
template <int DIR, typename C> struct SmallDFT<16, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        using R = decltype(v[0].x);
        const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);
        const R h = R(0.70710678118654752440);
        C z0[4] = {v[0], v[4], v[8], v[12]};
        C z1[4] = {v[1], v[5], v[9], v[13]};
        C z2[4] = {v[2], v[6], v[10], v[14]};
        C z3[4] = {v[3], v[7], v[11], v[15]};
        SmallDFT<4, DIR, C>::run(z0);
        SmallDFT<4, DIR, C>::run(z1);
        SmallDFT<4, DIR, C>::run(z2);
        SmallDFT<4, DIR, C>::run(z3);
        // b = 1: m = 1, 2, 3;  b = 2: m = 2, 4, 6;  b = 3: m = 3, 6, 9
        z1[1] = mul_wc<DIR>(z1[1], c1, s1);
        z1[2] = mul_wc<DIR>(z1[2], h, h);
        z1[3] = mul_wc<DIR>(z1[3], s1, c1);
        z2[1] = mul_wc<DIR>(z2[1], h, h);
        z2[2] = (DIR < 0) ? cmul_mi(z2[2]) : cmul_i(z2[2]);
        z2[3] = mul_wc<DIR>(z2[3], -h, h);
        z3[1] = mul_wc<DIR>(z3[1], s1, c1);
        z3[2] = mul_wc<DIR>(z3[2], -h, h);
        z3[3] = mul_wc<DIR>(z3[3], -c1, -s1);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C t[4] = {z0[k1], z1[k1], z2[k1], z3[k1]};
            SmallDFT<4, DIR, C>::run(t);
            v[k1] = t[0];
            v[k1 + 4] = t[1];
            v[k1 + 8] = t[2];
            v[k1 + 12] = t[3];
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

__host__ __device__ inline int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
__host__ __device__ inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Power-of-two version of pp_pass: n, Ns and (with BFAST) nbatch are powers
// of two, so the butterfly decomposition uses shifts and masks, and element
// addresses advance by constant strides.  The padded index p(e) = e + e/16
// of the R elements s + t S of a butterfly is p(s) + t (S + S/16) when the
// stride S (n/R or Ns) is a multiple of 16, and p(s) + t S when all R
// elements lie in one 16-element block (S R <= 16: the block of S R
// elements starts at a multiple of S R, which divides 16); otherwise each
// index is padded on its own.
template <int R, int DIR, bool BFAST, int PADS, int PADD, typename C>
__device__ __forceinline__ void pp_pass_p2(const C *src, int sbs, int ses, C *dst, int dbs, int des, int logn,
                                           int nbatch, int lognbatch, int logNs, const C *T, int tid, int nthr) {
    constexpr int LR = (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
    const int lognb = logn - LR;
    const int nb = 1 << lognb;
    const int Ns = 1 << logNs;
    const int total = nbatch << lognb;
    const bool rlin = !PADS || nb >= 16 || (nb << LR) <= 16;
    const bool wlin = !PADD || Ns >= 16 || (Ns << LR) <= 16;
    const int rstep = (PADS ? nb + (nb >> 4) : nb) * ses;
    const int wstep = (PADD ? Ns + (Ns >> 4) : Ns) * des;
    for (int J = tid; J < total; J += nthr) {
        int b, jj;
        if (BFAST) {
            b = J & (nbatch - 1);
            jj = J >> lognbatch;
        } else {
            b = J >> lognb;
            jj = J & (nb - 1);
        }
        const int k = jj & (Ns - 1);
        const int idxD = ((jj >> logNs) << (logNs + LR)) + k;
        C v[R];
        if (rlin) {
            const C *p = src + b * sbs + (PADS ? jj + (jj >> 4) : jj) * ses;
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = p[t * rstep];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                v[t] = src[b * sbs + (e + (e >> 4)) * ses];
            }
        }
        if (Ns > 1) {
            const C *tw = T + k;   // this pass's table: T[t Ns + k] = exp(-2 pi i t k / (Ns R))
#pragma unroll
            for (int t = 1; t < R; ++t) {
                C w = tw[t * Ns];
                if (DIR > 0) w.y = -w.y;
                v[t] = cmul(v[t], w);
            }
        }
        SmallDFT<R, DIR, C>::run(v);
        if (wlin) {
            C *q = dst + b * dbs + (PADD ? idxD + (idxD >> 4) : idxD) * des;
#pragma unroll
            for (int t = 0; t < R; ++t) q[t * wstep] = v[t];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = idxD + t * Ns;
                dst[b * dbs + (e + (e >> 4)) * des] = v[t];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Split-BF16 tensor-core first pass (fp32 transforms in the BF16SPLIT mode).
// The first radix-16 pass of a power-of-two Stockham transform has no
// twiddles: every butterfly is a 16-point DFT, so the pass is the product
// Y = W X of the DFT matrix W (W[m][t] = exp(DIR 2 pi i m t / 16)) with the
// 16 x nbutterfly matrix X of the butterflies' inputs.  Over the reals,
//   [Re Y]   [ Wr  -Wi ] [Re X]
//   [Im Y] = [ Wi   Wr ] [Im X],
// which for 8 butterflies is two m16n8k16 row tiles (Re Y, Im Y) times two
// k16 steps (Re X, Im X).  Every real operand z is split into bfloat16
// z_hi = bf16(z) and z_lo = bf16(z - z_hi) (round to nearest even); the
// product keeps W_hi X_hi + W_hi X_lo + W_lo X_hi, accumulated in fp32 by
// mma.sync (the dropped W_lo X_lo and the rounding of z_lo are each below
// 2^-16 of |W| |X|).  A warp takes 8 butterflies at a time; lane (g, q) =
// (lane / 4, lane % 4) loads inputs t = 2q, 2q+1, 2q+8, 2q+9 of butterfly g
// (the B fragment) and stores outputs m = g, g+8 of butterflies 2q, 2q+1
// (the accumulator fragment).
//
// frag: per lane, the A fragments of Wr_hi, Wr_lo, Wi_hi, Wi_lo of the
// forward direction (Wi = -sin), 4 uint4 (a0..a3: rows g / g+8, columns
// 2q, 2q+1 / 2q+8, 2q+9; the lower column in the lower half).
// ADJ = false: reads e = jj + t n/16, writes jj 16 + m (the pass P_1 of
// pp_pass_p2); ADJ = true: reads jj 16 + t, writes jj + m n/16 (its adjoint,
// pp_pass_p2_adj at Ns = 1, with DIR = +1).
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t bf16x2_rn(float first, float second) {
    uint32_t d;   // first in the lower half
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(second), "f"(first));
    return d;
}

// hi / lo bfloat16 split of two floats (packed like bf16x2_rn)
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = bf16x2_rn(a, b);
    lo = bf16x2_rn(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xffff0000u));
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint4 &a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint4 bf16x2_neg(uint4 a) {
    const uint32_t s = 0x80008000u;
    return uint4{a.x ^ s, a.y ^ s, a.z ^ s, a.w ^ s};
}

template <int DIR, bool BFAST, bool ADJ, int PADS, int PADD>
__device__ __forceinline__ void tc_dft16_pass(const float2 *src, int sbs, int ses, float2 *dst, int dbs, int des,
                                              int logn, int nbatch, int lognbatch, const uint4 *frag, int tid,
                                              int nthr) {
    const int lognb = logn - 4;
    const int nb = 1 << lognb;
    const int total = nbatch << lognb;
    const int lane = tid & 31, g = lane >> 2, q = lane & 3;
    const uint4 *fl = frag + 4 * lane;
    const uint4 wr_hi = fl[0], wr_lo = fl[1];
    const uint4 wi_hi = DIR < 0 ? fl[2] : bf16x2_neg(fl[2]);
    const uint4 wi_lo = DIR < 0 ? fl[3] : bf16x2_neg(fl[3]);
    const uint4 nwi_hi = bf16x2_neg(wi_hi), nwi_lo = bf16x2_neg(wi_lo);
    for (int J0 = (tid >> 5) * 8; J0 < total; J0 += (nthr >> 5) * 8) {   // warp-uniform
        const int J = J0 + g;
        const bool ok = J < total;
        const int Jc = ok ? J : 0;
        int b, jj;
        if (BFAST) {
            b = Jc & (nbatch - 1);
            jj = Jc >> lognbatch;
        } else {
            b = Jc >> lognb;
            jj = Jc & (nb - 1);
        }
        float2 x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int t = 2 * q + (i & 1) + (i >> 1) * 8;
            const int e = ADJ ? (jj << 4) + t : jj + t * nb;
            const float2 v = src[b * sbs + (PADS ? e + (e >> 4) : e) * ses];
            x[i] = ok ? v : float2{0.f, 0.f};
        }
        uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
        split_bf16x2(x[0].x, x[1].x, rh0, rl0);   // Re X rows 2q, 2q+1
        split_bf16x2(x[2].x, x[3].x, rh1, rl1);   // Re X rows 2q+8, 2q+9
        split_bf16x2(x[0].y, x[1].y, ih0, il0);
        split_bf16x2(x[2].y, x[3].y, ih1, il1);
        float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
        __syncwarp();
        // Re Y = Wr Re X - Wi Im X (small terms first)
        mma_bf16_16816(yr, wr_lo, rh0, rh1);
        mma_bf16_16816(yr, nwi_lo, ih0, ih1);
        mma_bf16_16816(yr, wr_hi, rl0, rl1);
        mma_bf16_16816(yr, nwi_hi, il0, il1);
        mma_bf16_16816(yr, wr_hi, rh0, rh1);
        mma_bf16_16816(yr, nwi_hi, ih0, ih1);
        // Im Y = Wi Re X + Wr Im X
        mma_bf16_16816(yi, wi_lo, rh0, rh1);
        mma_bf16_16816(yi, wr_lo, ih0, ih1);
        mma_bf16_16816(yi, wi_hi, rl0, rl1);
        mma_bf16_16816(yi, wr_hi, il0, il1);
        mma_bf16_16816(yi, wi_hi, rh0, rh1);
        mma_bf16_16816(yi, wr_hi, ih0, ih1);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int Jo = J0 + 2 * q + c;
            if (Jo < total) {
                int bo, jo;
                if (BFAST) {
                    bo = Jo & (nbatch - 1);
                    jo = Jo >> lognbatch;
                } else {
                    bo = Jo >> lognb;
                    jo = Jo & (nb - 1);
                }
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int m = g + 8 * hh;
                    const int e = ADJ ? jo + m * nb : (jo << 4) + m;
                    dst[bo * dbs + (PADD ? e + (e >> 4) : e) * des] = float2{yr[c + 2 * hh], yi[c + 2 * hh]};
                }
            }
        }
    }
}

// the first pass through tc_dft16_pass when it applies (fp32, radix 16,
// Ns = 1, a fragment table given); returns false otherwise
template <int DIR, bool BFAST, bool ADJ, int PADS, int PADD, typename C>
__device__ __forceinline__ bool tc_first_pass(int lr, int logNs, const C *src, int sbs, int ses, C *dst, int dbs,
                                              int des, int logn, int nbatch, int lognbatch, const uint4 *tc, int tid,
                                              int nthr) {
    if constexpr (std::is_same<C, float2>::value) {
        if (tc != nullptr && lr == 4 && logNs == 0) {
            tc_dft16_pass<DIR, BFAST, ADJ, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, tc,
                                                       tid, nthr);
            return true;
        }
    }
    return false;
}

// Per-pass twiddle tables of a power-of-two length n for the radix plan of
// pp_fft_p2 with largest radix 2^maxlr (2^maxlr while at least maxlr bits
// remain, then the rest): for every pass with Ns > 1, Ns * R entries
// T[t Ns + k] = exp(-2 pi i t k / (Ns R)) (consecutive butterflies k read
// consecutive entries).  Total length pass_twiddle_len(n) <= 2 n.
__host__ __device__ inline int pass_twiddle_len(int n, int maxlr = 4) {
    int logn = 0;
    while ((1 << logn) < n) ++logn;
    int logNs = 0, rem = logn, len = 0;
    while (rem > 0) {
        const int lr = rem >= maxlr ? maxlr : rem;
        if (logNs > 0) len += 1 << (logNs + lr);
        logNs += lr;
        rem -= lr;
    }
    return len;
}

// pp_fft for power-of-two n with compile-time padding of A and B; T holds
// the pass twiddle tables of n
// the pass tables of n with largest radix 2^maxlr (4: radix 16; 3: radix 8,
// for batches whose radix-16 passes would leave threads idle)
template <int DIR, bool BFAST, int PADA, int PADB, typename C>
__device__ int pp_fft_p2(C *A, int abs_, int aes, C *B, int bbs, int bes, int n, int nbatch, const C *T, int tid,
                         int nthr, int maxlr = 4, const uint4 *tc = nullptr) {
    const int logn = ilog2(n), lognbatch = ilog2(nbatch);
    int logNs = 0, rem = logn, where = 0;
    const C *Tp = T;
    while (rem > 0) {
        const int lr = rem >= maxlr ? maxlr : rem;   // largest radix first, the rest last
        // (the first pass always runs A -> B)
        const bool done = logNs == 0 && tc_first_pass<DIR, BFAST, false, PADA, PADB>(
                                            lr, logNs, A, abs_, aes, B, bbs, bes, logn, nbatch, lognbatch, tc, tid, nthr);
        if (done) {
        } else if (where == 0) {
            if (lr == 4) pp_pass_p2<16, DIR, BFAST, PADA, PADB>(A, abs_, aes, B, bbs, bes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else if (lr == 3) pp_pass_p2<8, DIR, BFAST, PADA, PADB>(A, abs_, aes, B, bbs, bes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else if (lr == 2) pp_pass_p2<4, DIR, BFAST, PADA, PADB>(A, abs_, aes, B, bbs, bes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else pp_pass_p2<2, DIR, BFAST, PADA, PADB>(A, abs_, aes, B, bbs, bes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
        } else {
            if (lr == 4) pp_pass_p2<16, DIR, BFAST, PADB, PADA>(B, bbs, bes, A, abs_, aes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else if (lr == 3) pp_pass_p2<8, DIR, BFAST, PADB, PADA>(B, bbs, bes, A, abs_, aes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else if (lr == 2) pp_pass_p2<4, DIR, BFAST, PADB, PADA>(B, bbs, bes, A, abs_, aes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
            else pp_pass_p2<2, DIR, BFAST, PADB, PADA>(B, bbs, bes, A, abs_, aes, logn, nbatch, lognbatch, logNs, Tp, tid, nthr);
        }
        __syncthreads();
        if (logNs > 0) Tp += 1 << (logNs + lr);
        logNs += lr;
        rem -= lr;
        where ^= 1;
    }
    return where;
}

// ---------------------------------------------------------------------------
// Forward transform, spectral multiply and inverse transform of power-of-two
// columns with one pass fused.  With the forward transform written as the
// passes F = P_L ... P_1 (pp_pass_p2, P_1 first), the inverse up to the
// factor n is the adjoint F^H = P_1^H ... P_L^H.  The adjoint of a pass reads
// where the pass writes, applies the opposite-direction R-point DFT,
// multiplies by the conjugate twiddles and writes where the pass reads.  P_L,
// the diagonal multiply and P_L^H touch only the R elements one butterfly
// owns, so they run in registers, in place: L - 1 + 1 + L - 1 passes
// through shared memory instead of 2 L + 1.
// ---------------------------------------------------------------------------

// the schedule of pp_fft_p2 for n = 2^logn: radix of pass p and the offset
// of its twiddle table
__device__ __forceinline__ void p2_schedule(int logn, int p, int *lr, int *logNs, int *toff) {
    int lns = 0, rem = logn, off = 0;
    for (int q = 0; q < p; ++q) {
        const int l = rem >= 4 ? 4 : rem;
        if (lns > 0) off += 1 << (lns + l);
        lns += l;
        rem -= l;
    }
    *lr = rem >= 4 ? 4 : rem;
    *logNs = lns;
    *toff = off;
}

__device__ __forceinline__ int p2_npasses(int logn) { return (logn + 3) / 4; }

// adjoint of pp_pass_p2<R, -1, BFAST> (src read at its write positions, dst
// written at its read positions)
template <int R, bool BFAST, int PADS, int PADD, typename C>
__device__ __forceinline__ void pp_pass_p2_adj(const C *src, int sbs, int ses, C *dst, int dbs, int des, int logn,
                                               int nbatch, int lognbatch, int logNs, const C *T, int tid, int nthr) {
    constexpr int LR = (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
    const int lognb = logn - LR;
    const int nb = 1 << lognb;
    const int Ns = 1 << logNs;
    const int total = nbatch << lognb;
    // the linear cases of pp_pass_p2, with reads and writes exchanged
    const bool rlin = !PADS || Ns >= 16 || (Ns << LR) <= 16;
    const bool wlin = !PADD || nb >= 16 || (nb << LR) <= 16;
    const int rstep = (PADS ? Ns + (Ns >> 4) : Ns) * ses;
    const int wstep = (PADD ? nb + (nb >> 4) : nb) * des;
    for (int J = tid; J < total; J += nthr) {
        int b, jj;
        if (BFAST) {
            b = J & (nbatch - 1);
            jj = J >> lognbatch;
        } else {
            b = J >> lognb;
            jj = J & (nb - 1);
        }
        const int k = jj & (Ns - 1);
        const int idxD = ((jj >> logNs) << (logNs + LR)) + k;
        C v[R];
        if (rlin) {
            const C *p = src + b * sbs + (PADS ? idxD + (idxD >> 4) : idxD) * ses;
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = p[t * rstep];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = idxD + t * Ns;
                v[t] = src[b * sbs + (e + (e >> 4)) * ses];
            }
        }
        SmallDFT<R, +1, C>::run(v);
        if (Ns > 1) {
            const C *tw = T + k;
#pragma unroll
            for (int t = 1; t < R; ++t) v[t] = cmul(v[t], cconj(tw[t * Ns]));
        }
        if (wlin) {
            C *q = dst + b * dbs + (PADD ? jj + (jj >> 4) : jj) * des;
#pragma unroll
            for (int t = 0; t < R; ++t) q[t * wstep] = v[t];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                dst[b * dbs + (e + (e >> 4)) * des] = v[t];
            }
        }
    }
}

template <bool BFAST, int PADS, int PADD, typename C>
__device__ __forceinline__ void pp_pass_p2_adj_r(int lr, const C *src, int sbs, int ses, C *dst, int dbs, int des,
                                                 int logn, int nbatch, int lognbatch, int logNs, const C *T, int tid,
                                                 int nthr, const uint4 *tc = nullptr) {
    if (tc_first_pass<+1, BFAST, true, PADS, PADD>(lr, logNs, src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch,
                                                    tc, tid, nthr)) return;
    if (lr == 4) pp_pass_p2_adj<16, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else if (lr == 3) pp_pass_p2_adj<8, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else if (lr == 2) pp_pass_p2_adj<4, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else pp_pass_p2_adj<2, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
}

template <bool BFAST, int PADS, int PADD, typename C>
__device__ __forceinline__ void pp_pass_p2_fwd_r(int lr, const C *src, int sbs, int ses, C *dst, int dbs, int des,
                                                 int logn, int nbatch, int lognbatch, int logNs, const C *T, int tid,
                                                 int nthr, const uint4 *tc = nullptr) {
    if (tc_first_pass<-1, BFAST, false, PADS, PADD>(lr, logNs, src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch,
                                                     tc, tid, nthr)) return;
    if (lr == 4) pp_pass_p2<16, -1, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else if (lr == 3) pp_pass_p2<8, -1, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else if (lr == 2) pp_pass_p2<4, -1, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
    else pp_pass_p2<2, -1, BFAST, PADS, PADD>(src, sbs, ses, dst, dbs, des, logn, nbatch, lognbatch, logNs, T, tid, nthr);
}

// the fused last pass: forward pass L (read at its read positions), multiply
// output element e of transform b by mult(b, e), adjoint of pass L, write
// back to the same positions, times scale
template <int R, bool BFAST, int PAD, typename C, typename Mult>
__device__ __forceinline__ void pp_pass_p2_fused(C *buf, int bs, int es, int logn, int nbatch, int lognbatch,
                                                 int logNs, const C *T, const Mult &mult, int tid, int nthr) {
    using real = decltype(buf[0].x);
    constexpr int LR = (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
    const int lognb = logn - LR;
    const int nb = 1 << lognb;
    const int Ns = 1 << logNs;
    const int total = nbatch << lognb;
    const bool lin = !PAD || nb >= 16 || (nb << LR) <= 16;   // as in pp_pass_p2
    const int step = (PAD ? nb + (nb >> 4) : nb) * es;
    for (int J = tid; J < total; J += nthr) {
        int b, jj;
        if (BFAST) {
            b = J & (nbatch - 1);
            jj = J >> lognbatch;
        } else {
            b = J >> lognb;
            jj = J & (nb - 1);
        }
        const int k = jj & (Ns - 1);
        const int idxD = ((jj >> logNs) << (logNs + LR)) + k;
        C *p = buf + b * bs + (PAD ? jj + (jj >> 4) : jj) * es;
        C v[R];
        if (lin) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = p[t * step];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                v[t] = buf[b * bs + (e + (e >> 4)) * es];
            }
        }
        const C *tw = T + k;
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) v[t] = cmul(v[t], tw[t * Ns]);
        }
        SmallDFT<R, -1, C>::run(v);
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = mult(b, idxD + t * Ns, v[t]);
        SmallDFT<R, +1, C>::run(v);
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) v[t] = cmul(v[t], cconj(tw[t * Ns]));
        }
        if (lin) {
#pragma unroll
            for (int t = 0; t < R; ++t) p[t * step] = v[t];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                buf[b * bs + (e + (e >> 4)) * es] = v[t];
            }
        }
    }
    (void)sizeof(real);
}

// Barrier among the nthr threads that share a transform batch: the whole
// block (id 0, __syncthreads) or a group of whole warps on a named barrier.
struct GroupSync {
    int id, nthr;
    __device__ __forceinline__ void operator()() const {
        if (id == 0) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
    }
};

// y = F^H diag(mult) F x for nbatch power-of-two transforms of length n:
// A (layout la, unpadded) holds x; B (layout lb, padded) is the work buffer.
// Returns 0 if y is in A, 1 if in B.  Every pass ends with a barrier of the
// nthr participating threads (sync); callers synchronise before.
template <bool BFAST, typename C, typename Mult>
__device__ int pp_conv_p2(C *A, Lay la, C *B, Lay lb, int n, int nbatch, const C *T, const Mult &mult, int tid,
                          int nthr, const GroupSync &sync, const uint4 *tc = nullptr) {
    const int logn = ilog2(n), lognbatch = ilog2(nbatch), L = p2_npasses(logn);
    int where = 0, lr, lns, toff;
    for (int p = 0; p < L - 1; ++p) {   // forward passes 1 .. L-1
        p2_schedule(logn, p, &lr, &lns, &toff);
        if (where == 0) pp_pass_p2_fwd_r<BFAST, 0, 1>(lr, A, la.bs, la.es, B, lb.bs, lb.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        else pp_pass_p2_fwd_r<BFAST, 1, 0>(lr, B, lb.bs, lb.es, A, la.bs, la.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        sync();
        where ^= 1;
    }
    p2_schedule(logn, L - 1, &lr, &lns, &toff);
    C *buf = where ? B : A;
    const Lay lbuf = where ? lb : la;
#define FFTLB_FUSED(RR)                                                                                         \
    (lbuf.pad ? pp_pass_p2_fused<RR, BFAST, 1>(buf, lbuf.bs, lbuf.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr) \
              : pp_pass_p2_fused<RR, BFAST, 0>(buf, lbuf.bs, lbuf.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr))
    if (lr == 4) FFTLB_FUSED(16);
    else if (lr == 3) FFTLB_FUSED(8);
    else if (lr == 2) FFTLB_FUSED(4);
    else FFTLB_FUSED(2);
#undef FFTLB_FUSED
    sync();
    for (int p = L - 2; p >= 0; --p) {   // adjoint passes L-1 .. 1
        p2_schedule(logn, p, &lr, &lns, &toff);
        if (where == 0) pp_pass_p2_adj_r<BFAST, 0, 1>(lr, A, la.bs, la.es, B, lb.bs, lb.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        else pp_pass_p2_adj_r<BFAST, 1, 0>(lr, B, lb.bs, lb.es, A, la.bs, la.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        sync();
        where ^= 1;
    }
    return where;
}

// Several outputs from one or two inputs (the level-1 / level-2 derivative
// groups): the inputs take the forward passes 1 .. L-1 once
// (pp_fwd_head_p2); each output is then one fused pass, reading both inputs'
// butterfly and applying their pass L, the per-element combination
// mult(b, e, x0, x1) and the adjoint of pass L, written to a free buffer
// (pp_pass_p2_fused2), and the adjoint passes L-1 .. 1 (pp_adj_tail_p2).

template <bool BFAST, typename C>
__device__ int pp_fwd_head_p2(C *A, Lay la, C *B, Lay lb, int n, int nbatch, const C *T, int tid, int nthr,
                              const GroupSync &sync, const uint4 *tc = nullptr) {
    const int logn = ilog2(n), lognbatch = ilog2(nbatch), L = p2_npasses(logn);
    int where = 0, lr, lns, toff;
    for (int p = 0; p < L - 1; ++p) {
        p2_schedule(logn, p, &lr, &lns, &toff);
        if (where == 0) pp_pass_p2_fwd_r<BFAST, 0, 1>(lr, A, la.bs, la.es, B, lb.bs, lb.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        else pp_pass_p2_fwd_r<BFAST, 1, 0>(lr, B, lb.bs, lb.es, A, la.bs, la.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        sync();
        where ^= 1;
    }
    return where;
}

template <int R, bool BFAST, int PADX, int PADQ, typename C, typename Mult2>
__device__ __forceinline__ void pp_pass_p2_fused2(const C *X0, const C *X1, int xbs, int xes, bool two, C *Q, int qbs,
                                                  int qes, int logn, int nbatch, int lognbatch, int logNs, const C *T,
                                                  const Mult2 &mult, int tid, int nthr) {
    constexpr int LR = (R == 16) ? 4 : (R == 8) ? 3 : (R == 4) ? 2 : 1;
    const int lognb = logn - LR;
    const int nb = 1 << lognb;
    const int Ns = 1 << logNs;
    const int total = nbatch << lognb;
    // (the linear cases of pp_pass_p2 for reads and writes at jj + t nb)
    const bool xlin = !PADX || nb >= 16 || (nb << LR) <= 16;
    const bool qlin = !PADQ || nb >= 16 || (nb << LR) <= 16;
    const int xstep = (PADX ? nb + (nb >> 4) : nb) * xes;
    const int qstep = (PADQ ? nb + (nb >> 4) : nb) * qes;
    for (int J = tid; J < total; J += nthr) {
        int b, jj;
        if (BFAST) {
            b = J & (nbatch - 1);
            jj = J >> lognbatch;
        } else {
            b = J >> lognb;
            jj = J & (nb - 1);
        }
        const int k = jj & (Ns - 1);
        const int idxD = ((jj >> logNs) << (logNs + LR)) + k;
        const C *tw = T + k;
        C v0[R], v1[R];
        if (xlin) {
            const int a0 = b * xbs + (PADX ? jj + (jj >> 4) : jj) * xes;
#pragma unroll
            for (int t = 0; t < R; ++t) {
                v0[t] = X0[a0 + t * xstep];
                v1[t] = two ? X1[a0 + t * xstep] : C{0, 0};
            }
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                const int a = b * xbs + (e + (e >> 4)) * xes;
                v0[t] = X0[a];
                v1[t] = two ? X1[a] : C{0, 0};
            }
        }
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                const C w = tw[t * Ns];
                v0[t] = cmul(v0[t], w);
                v1[t] = cmul(v1[t], w);
            }
        }
        SmallDFT<R, -1, C>::run(v0);
        if (two) SmallDFT<R, -1, C>::run(v1);
#pragma unroll
        for (int t = 0; t < R; ++t) v0[t] = mult(b, idxD + t * Ns, v0[t], v1[t]);
        SmallDFT<R, +1, C>::run(v0);
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) v0[t] = cmul(v0[t], cconj(tw[t * Ns]));
        }
        if (qlin) {
            C *q = Q + b * qbs + (PADQ ? jj + (jj >> 4) : jj) * qes;
#pragma unroll
            for (int t = 0; t < R; ++t) q[t * qstep] = v0[t];
        } else {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                const int e = jj + t * nb;
                Q[b * qbs + (e + (e >> 4)) * qes] = v0[t];
            }
        }
    }
}

// the fused output pass from inputs in layout lx to the buffer Q (layout lq)
template <bool BFAST, typename C, typename Mult2>
__device__ void pp_out_fused_p2(const C *X0, const C *X1, Lay lx, bool two, C *Q, Lay lq, int n, int nbatch,
                                const C *T, const Mult2 &mult, int tid, int nthr, const GroupSync &sync) {
    const int logn = ilog2(n), lognbatch = ilog2(nbatch), L = p2_npasses(logn);
    int lr, lns, toff;
    p2_schedule(logn, L - 1, &lr, &lns, &toff);
#define FFTLB_F2(RR)                                                                                              \
    if (lx.pad) {                                                                                                \
        if (lq.pad) pp_pass_p2_fused2<RR, BFAST, 1, 1>(X0, X1, lx.bs, lx.es, two, Q, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr); \
        else pp_pass_p2_fused2<RR, BFAST, 1, 0>(X0, X1, lx.bs, lx.es, two, Q, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr); \
    } else {                                                                                                     \
        if (lq.pad) pp_pass_p2_fused2<RR, BFAST, 0, 1>(X0, X1, lx.bs, lx.es, two, Q, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr); \
        else pp_pass_p2_fused2<RR, BFAST, 0, 0>(X0, X1, lx.bs, lx.es, two, Q, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, mult, tid, nthr); \
    }
    // (callers use this path only when the last pass has radix <= 8: two
    // inputs' radix-16 butterflies in registers would spill)
    if (lr == 3) { FFTLB_F2(8) }
    else if (lr == 2) { FFTLB_F2(4) }
    else { FFTLB_F2(2) }
#undef FFTLB_F2
    sync();
}

// adjoint passes L-1 .. 1 between Q0 and Q1 (same layout lq); returns 0 if
// the result is in Q0, 1 if in Q1
template <bool BFAST, typename C>
__device__ int pp_adj_tail_p2(C *Q0, C *Q1, Lay lq, int n, int nbatch, const C *T, int tid, int nthr,
                              const GroupSync &sync, const uint4 *tc = nullptr) {
    const int logn = ilog2(n), lognbatch = ilog2(nbatch), L = p2_npasses(logn);
    int where = 0, lr, lns, toff;
    for (int p = L - 2; p >= 0; --p) {
        p2_schedule(logn, p, &lr, &lns, &toff);
        C *src = where ? Q1 : Q0, *dst = where ? Q0 : Q1;
        if (lq.pad) pp_pass_p2_adj_r<BFAST, 1, 1>(lr, src, lq.bs, lq.es, dst, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        else pp_pass_p2_adj_r<BFAST, 0, 0>(lr, src, lq.bs, lq.es, dst, lq.bs, lq.es, logn, nbatch, lognbatch, lns, T + toff, tid, nthr, tc);
        sync();
        where ^= 1;
    }
    return where;
}

// Dispatch: the shift-based passes when n (and, for BFAST, nbatch) is a
// power of two, the generic passes otherwise.  PADA / PADB must match
// la.pad / lb.pad.
// (W: the length-n twiddles of the generic passes; T: the pass tables of
// the shift-based ones, used when n is a power of two)
template <int DIR, bool BFAST, int PADA, int PADB, typename C>
__device__ __forceinline__ int pp_fft_any(C *A, Lay la, C *B, Lay lb, int n, int nbatch, const C *W, const C *T,
                                          int tid, int nthr, int maxlr = 4, const uint4 *tc = nullptr) {
    if (is_pow2(n) && (!BFAST || is_pow2(nbatch)))
        return pp_fft_p2<DIR, BFAST, PADA, PADB>(A, la.bs, la.es, B, lb.bs, lb.es, n, nbatch, T, tid, nthr, maxlr, tc);
    return pp_fft<DIR, BFAST>(A, la, B, lb, n, nbatch, W, tid, nthr);
}

// r2c_post / c2r_pre (below) on rows in an arbitrary layout
template <typename C>
__device__ __forceinline__ void r2c_post_l(C *a, Lay L, int h, int batch, const C *Wp, int tid, int nthr) {
    using R = decltype(a[0].x);
    for (int row = 0; row < batch; ++row) {
        for (int k = tid; k <= h / 2; k += nthr) {
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
}

template <typename C>
__device__ __forceinline__ void c2r_pre_l(C *a, Lay L, int h, int batch, const C *Wp, int tid, int nthr) {
    for (int row = 0; row < batch; ++row) {
        for (int k = tid; k <= h / 2; k += nthr) {
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

// Warp-resident row transforms and the fp32 row kernels built on them
// (arXiv:1011.3582, Sec. 3.6, Fig. 3: transform, multiply, inverse).
//
// A row of H = E * P complex values (a real row of 2H values packed as
// z[m] = x[2m] + i x[2m+1]) is transformed by a group of P lanes of one
// warp, in place in shared memory, with no block barrier:
//   stage 1: lane l holds x[l + P t] (t < E) in registers and takes the
//            E-point DFT over t, then multiplies output k1 by W_H^(l k1);
//   transpose: every lane stores its E values at swizzled positions of the
//            same row buffer (__syncwarp before and after);
//   stage 2: the P-point DFTs over l, one per k1, in registers: for P <= E
//            lane j holds the P values of k1 = j + P q (q < E / P); for
//            P = 2E (H = 512) lane k1 + E g holds the even (g = 0) or odd
//            (g = 1) half of the l values, takes an E-point DFT and the
//            last radix-2 step is one exchange with lane ^ E (__shfl_xor);
//   result:  X[k1 + E k2] back in natural order.
// With n = l + P t and k = k1 + E k2, W_H^(nk) = W_H^(l k1) W_P^(l k2)
// W_E^(t k1), which is the decomposition above.  Every index is a
// compile-time constant plus the lane's own offset, and the swizzles keep
// the shared-memory accesses free of bank conflicts for the P >= 16
// layouts (the row groups of P = 8 share banks two ways).
#pragma once

#include "kernels_pipe.cuh"

namespace fftlb {

// cos(2 pi k / 32), k = 0..8 (the rest by symmetry)
__device__ __forceinline__ constexpr double cos32(int k) {
    return k == 0 ? 1.0
         : k == 1 ? 0.98078528040323044913
         : k == 2 ? 0.92387953251128675613
         : k == 3 ? 0.83146961230254523708
         : k == 4 ? 0.70710678118654752440
         : k == 5 ? 0.55557023301960222474
         : k == 6 ? 0.38268343236508977173
         : k == 7 ? 0.19509032201612826785
                  : 0.0;
}

// W_32^k = exp(DIR 2 pi i k / 32) for 0 <= k < 16, compile-time after unrolling
template <int DIR, typename R>
__device__ __forceinline__ void w32(int k, R &c, R &s) {
    const double cc = k <= 8 ? cos32(k) : -cos32(16 - k);
    const double ss = k <= 8 ? cos32(8 - k) : cos32(k - 8);
    c = R(cc);
    s = R(DIR < 0 ? -ss : ss);
}

// 32-point DFT as two 16-point DFTs of the even and odd inputs and one
// radix-2 step with the constants W_32^k
template <int DIR, typename C> struct SmallDFT<32, DIR, C> {
    __device__ __forceinline__ static void run(C *v) {
        using R = decltype(v[0].x);
        C e[16], o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        SmallDFT<16, DIR, C>::run(e);
        SmallDFT<16, DIR, C>::run(o);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            R c, s;
            w32<DIR, R>(k, c, s);
            const C t = k == 0 ? o[k] : C{o[k].x * c - o[k].y * s, o[k].x * s + o[k].y * c};
            v[k] = cadd(e[k], t);
            v[k + 16] = csub(e[k], t);
        }
    }
};

// Row configurations: H = E * P, P lanes per row, 32 / P rows per warp
template <int H> struct RowCfg;
template <> struct RowCfg<512> { static constexpr int E = 16, P = 32; };
template <> struct RowCfg<256> { static constexpr int E = 16, P = 16; };
template <> struct RowCfg<128> { static constexpr int E = 16, P = 8; };

// threads per block of the row kernels: 16 warps, or 8 for H = 128 (four
// rows per warp: 32 row groups, one per convection row)
// Threads of the final row kernel at H = 512: 256, i.e. two blocks per SM,
// each with one head buffer and one-ring chunks (measured at 1024^2: 131 us
// against 146 us for one 512-thread block with two head buffers; the
// FFTLB_K5_NT512 build flag selects 512)
#ifndef FFTLB_K5_NT512
#define FFTLB_K5_NT512 256
#endif
template <int H> __host__ __device__ constexpr int nt_wr() { return H >= 256 ? 512 : 256; }
inline int nt_wr_host(int H) { return H >= 256 ? 512 : 256; }
// Threads of the forward row kernel at H = 512: 256, i.e. two blocks per
// SM, each with 8-row chunks (measured at 1024^2: 68.7 us against 83.3 us
// for one 512-thread block with 16-row chunks; FFTLB_K1_NT512 selects 512)
#ifndef FFTLB_K1_NT512
#define FFTLB_K1_NT512 256
#endif
template <int H> __host__ __device__ constexpr int nt_k1wr() { return H == 512 ? FFTLB_K1_NT512 : nt_wr<H>(); }
inline int nt_k1wr_host(int H) { return H == 512 ? FFTLB_K1_NT512 : nt_wr_host(H); }
// Threads of the level-1 row kernel at H = 512: 256 with one row buffer,
// i.e. two blocks per SM (measured at 1024^2: 39.3 us against 46.4 us for
// one 512-thread block with two row buffers; FFTLB_K3_NT512 selects 512)
#ifndef FFTLB_K3_NT512
#define FFTLB_K3_NT512 256
#endif
template <int H> __host__ __device__ constexpr int nt_k3wr() { return H == 512 ? FFTLB_K3_NT512 : nt_wr<H>(); }
inline int nt_k3wr_host(int H) { return H == 512 ? FFTLB_K3_NT512 : nt_wr_host(H); }
template <int H> __host__ __device__ constexpr int nb_k3wr() { return nt_k3wr<H>() == 512 || H < 256 ? 2 : 1; }
inline int nb_k3wr_host(int H) { return nt_k3wr_host(H) == 512 || H < 256 ? 2 : 1; }
template <int H> __host__ __device__ constexpr int nt_k5wr() { return H == 512 ? FFTLB_K5_NT512 : nt_wr<H>(); }
inline int nt_k5wr_host(int H) { return H == 512 ? FFTLB_K5_NT512 : nt_wr_host(H); }
// head buffers of the final row kernel: two (the next row's head fetched a
// row ahead) unless its blocks are half size
template <int H> __host__ __device__ constexpr int nhb_k5wr() { return nt_k5wr<H>() == 512 || H < 256 ? 2 : 1; }
// sites per unrolled pass of the final row kernel's epilogue (the loads of
// the next site's distributions issue before the current site's arithmetic;
// measured at 1024^2: 132.2 us with 1, 131.1 with 2, 130.5 with 4)
#ifndef FFTLB_K5_UNROLL
#define FFTLB_K5_UNROLL 4
#endif
constexpr int K5U = FFTLB_K5_UNROLL;
// FFTLB_K5_VEC > 0: the epilogue with four consecutive sites per thread
// (where nx is four times the block size) and 16-byte accesses (measured at
// 1024^2: 130.9 us scalar, 126.7 us with 1, 131.9 us with 2)
#ifndef FFTLB_K5_VEC
#define FFTLB_K5_VEC 1
#endif

// position of stage-1 output (l, k1) in the row buffer.  P >= 16: k1 P +
// (l ^ (k1 mod P)) (for P = 2E, k1 < E: k1 P + (l ^ k1)); P = 8: the row
// parity rsw also flips bit 0 of k1, so that the two rows of a half-warp use
// different banks
template <int H>
__device__ __forceinline__ int tpos(int l, int k1, int rsw) {
    constexpr int P = RowCfg<H>::P;
    return ((k1 ^ rsw) * P) + (l ^ (k1 & (P - 1)));
}

// the lanes of this lane's row group (P consecutive lanes)
template <int P>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (P >= 32) return 0xffffffffu;
    else return ((1u << P) - 1u) << ((threadIdx.x & 31) & ~(P - 1));
}

// In-place DFT (DIR = -1) or unnormalised inverse (DIR = +1) of the H
// complex values at z by lane j (0 <= j < P) of its row group; tw[k1 P + l]
// = exp(-2 pi i l k1 / H); rsw: row parity (P = 8), else 0.  All P lanes of
// the row group must call it together (they synchronise with __syncwarp on
// the group's mask; other row groups of the warp may diverge).
template <int H, int DIR, typename C>
__device__ __forceinline__ void row_fft_wr(C *z, const C *tw, int j, int rsw) {
    constexpr int E = RowCfg<H>::E, P = RowCfg<H>::P;
    const unsigned gm = group_mask<P>();
    C v[E];
#pragma unroll
    for (int t = 0; t < E; ++t) v[t] = z[j + P * t];
    SmallDFT<E, DIR, C>::run(v);
#pragma unroll
    for (int k1 = 1; k1 < E; ++k1) {
        C w = tw[k1 * P + j];
        if (DIR > 0) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
    __syncwarp(gm);
#pragma unroll
    for (int k1 = 0; k1 < E; ++k1) z[tpos<H>(j, k1, rsw)] = v[k1];
    __syncwarp(gm);
    if constexpr (P <= E) {
        constexpr int NQ = E / P;
        C u[NQ][P];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
#pragma unroll
            for (int l = 0; l < P; ++l) u[q][l] = z[tpos<H>(l, j + P * q, rsw)];
            SmallDFT<P, DIR, C>::run(u[q]);
        }
        __syncwarp(gm);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) z[j + P * q + E * k2] = u[q][k2];
    } else {
        static_assert(P == 2 * E, "row configuration");
        using R = decltype(v[0].x);
        constexpr int HE = E / 2;
        const int k1 = j & (E - 1), g = j / E;
        C u[E];
#pragma unroll
        for (int m = 0; m < E; ++m) u[m] = z[tpos<H>(g + 2 * m, k1, 0)];
        SmallDFT<E, DIR, C>::run(u);
        // X[k1 + E (k2' + E k3)] = V0[k2'] + (-1)^k3 W_P^k2' V1[k2']: lane
        // g keeps k2' in [HE g, HE g + HE) and receives the other lane's half
        C a[HE], b[HE];
#pragma unroll
        for (int i = 0; i < HE; ++i) {
            const C send = g ? u[i] : u[HE + i];
            C recv;
            recv.x = __shfl_xor_sync(0xffffffffu, send.x, E);
            recv.y = __shfl_xor_sync(0xffffffffu, send.y, E);
            a[i] = g ? recv : u[i];
            b[i] = g ? u[HE + i] : recv;
        }
        __syncwarp(gm);   // every lane's stage-2 reads are done
#pragma unroll
        for (int i = 0; i < HE; ++i) {
            R c, s;
            w32<DIR, R>(i, c, s);   // W_P^i, P = 32
            C t = i == 0 ? b[i] : C{b[i].x * c - b[i].y * s, b[i].x * s + b[i].y * c};
            // times W_P^(HE g): W_32^8 = -i forward, +i inverse
            const C r = DIR < 0 ? cmul_mi(t) : cmul_i(t);
            t = g ? r : t;
            const int k2 = HE * g + i;
            z[k1 + E * k2] = cadd(a[i], t);
            z[k1 + E * (k2 + E)] = csub(a[i], t);
        }
        __syncwarp(gm);
        return;
    }
    __syncwarp(gm);
}

// Forward real rows: the natural-order result Z of row_fft_wr (the
// half-length transform of the packed row) -> one-sided spectrum X[0 .. H-1]
// with the real Nyquist value in the imaginary part of X[0], written to
// out (global memory, coalesced: lanes take consecutive k and H - k).
// Wp[k] = exp(-2 pi i k / 2H), k <= H / 2.
template <int H, typename C>
__device__ __forceinline__ void r2c_post_wr(const C *z, C *out, const C *Wp, int j) {
    using R = decltype(z[0].x);
    constexpr int P = RowCfg<H>::P;
#pragma unroll
    for (int k0 = 0; k0 <= H / 2; k0 += P) {
        const int k = k0 + j;
        if (k > H / 2) break;
        if (k == 0) {
            const C z0 = z[0];
            out[0] = C{z0.x + z0.y, z0.x - z0.y};
        } else {
            const C p = z[k], q = z[H - k];
            const C ze = cscale(cadd(p, cconj(q)), R(0.5));
            const C zo = cscale(cmul_mi(csub(p, cconj(q))), R(0.5));
            const C wz = cmul(Wp[k], zo);
            out[k] = cadd(ze, wz);
            if (H - k != k) out[H - k] = cconj(csub(ze, wz));
        }
    }
}

// r2c_post_wr with two destinations: X to raw and i k_x X / nx (the d_x
// term of a level-2 output) to mul; either may be null.  kxt[k] = k_x of
// bin k, sx = 1 / nx; bin 0 (DC, row-Nyquist) has k_x = 0 for both.
template <int H, typename C>
__device__ __forceinline__ void r2c_post_wr2(const C *z, C *raw, C *mul, const float *__restrict__ kxt, float sx,
                                             const C *Wp, int j) {
    using R = decltype(z[0].x);
    constexpr int P = RowCfg<H>::P;
#pragma unroll
    for (int k0 = 0; k0 <= H / 2; k0 += P) {
        const int k = k0 + j;
        if (k > H / 2) break;
        C a, b;
        if (k == 0) {
            const C z0 = z[0];
            a = C{z0.x + z0.y, z0.x - z0.y};
        } else {
            const C p = z[k], q = z[H - k];
            const C ze = cscale(cadd(p, cconj(q)), R(0.5));
            const C zo = cscale(cmul_mi(csub(p, cconj(q))), R(0.5));
            const C wz = cmul(Wp[k], zo);
            a = cadd(ze, wz);
            b = cconj(csub(ze, wz));
        }
        if (raw) {
            raw[k] = a;
            if (k != 0 && H - k != k) raw[H - k] = b;
        }
        if (mul) {
            mul[k] = imul(kxt[k] * sx, a);
            if (k != 0 && H - k != k) mul[H - k] = imul(kxt[H - k] * sx, b);
        }
    }
}

// Inverse real rows, in place: one-sided packed spectrum X -> Z[k] = (X[k]
// + X[k + H]) + i (X[k] - X[k + H]) exp(+2 pi i k / 2H), X[k + H] =
// conj X[H - k]; the half-length inverse of Z is the real row.
template <int H, typename C>
__device__ __forceinline__ void c2r_pre_wr(C *z, const C *Wp, int j) {
    constexpr int P = RowCfg<H>::P;
#pragma unroll
    for (int k0 = 0; k0 <= H / 2; k0 += P) {
        const int k = k0 + j;
        if (k > H / 2) break;
        if (k == 0) {
            const C x0 = z[0];
            z[0] = C{x0.x + x0.y, x0.x - x0.y};
        } else {
            const C p = z[k], q = z[H - k];
            const C w = Wp[k];
            const C wc = cconj(w);
            z[k] = cadd(cadd(p, cconj(q)), cmul_i(cmul(csub(p, cconj(q)), wc)));
            if (H - k != k) {
                const C mw = C{-w.x, -w.y};
                z[H - k] = cadd(cadd(q, cconj(p)), cmul_i(cmul(csub(q, cconj(p)), mw)));
            }
        }
    }
}

// four consecutive floats (16-byte aligned) to and from registers
__device__ __forceinline__ void ld4(float (&a)[4], const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a[0] = v.x;
    a[1] = v.y;
    a[2] = v.z;
    a[3] = v.w;
}
__device__ __forceinline__ void st4(float *p, const float (&a)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
}

// ---------------------------------------------------------------------------
// K1 (fp32, nx = 2H): moments rho, u, T (Eqs. 7-9), the level-1 fields
// Pi = P^w - rho T (Eq. 18) and g = M/T, and the forward row transforms of
// the 32 moving f_i and of rho, u_x, u_y, T, Pi, g, as k1_pipe, with
// warp-resident row transforms.  Persistent over the rows of all runs;
// per row, 32 / NG chunks of distribution rows (the first also holds the
// rest velocity's row, which only enters the moments), NG = rows per block
// pass (one per row group), two chunk buffers.
// ---------------------------------------------------------------------------

// the distribution rows of chunk c of a row: the rest velocity and the
// first NG moving rows, then NG moving rows per chunk
__host__ __device__ constexpr int k1w_first(int c, int NG) { return c == 0 ? 0 : 1 + c * NG; }
__host__ __device__ constexpr int k1w_count(int c, int NG) { return c == 0 ? NG + 1 : NG; }

__device__ __forceinline__ void k1w_issue(const float *f, float *dst, uint64_t *bar, int j, int nchunk, int NG,
                                          int nx, int ny, size_t N) {
    const int ri = j / nchunk, c = j - ri * nchunk;
    const int yg = (int)blockIdx.x + ri * (int)gridDim.x;   // row over all runs
    const int run = yg / ny, y = yg - run * ny;
    const int i0 = k1w_first(c, NG), nf = k1w_count(c, NG);
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(float));
    const float *fr = f + (size_t)run * Q * N;
    mbar_expect_tx(bar, (uint32_t)nf * rowbytes);
    for (int r = 0; r < nf; ++r)
        bulk_g2s(dst + (size_t)r * nx, fr + (size_t)(i0 + r) * N + (size_t)y * nx, rowbytes, bar);
}

template <int H>
__global__ void __launch_bounds__(nt_k1wr<H>(), nt_k1wr<H>() >= 512 ? 1 : 2) k1_wr(const float *__restrict__ f, float2 *spec, float *__restrict__ fields,
                                                 const float2 *__restrict__ tw_g, const float2 *__restrict__ Wp_g,
                                                 const float *__restrict__ kxt, KP<float> P, int *err) {
    using C = float2;
    using real = float;
    constexpr int NX = 2 * H, NT = nt_k1wr<H>(), NWARP = NT / 32;
    constexpr int PL = RowCfg<H>::P, RPW = 32 / PL;
    constexpr int NG = NWARP * RPW;                // row groups per block
    constexpr int CH = NG + 1, NCH = NMOV / NG;    // rows per chunk buffer, chunks per row
    constexpr int SMAX = (NX + NT - 1) / NT;
    static_assert(NMOV % NG == 0 && NG >= 6, "chunking");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1;
    const int nx = NX, ny = P.ny, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp * RPW + lane / PL, j = lane & (PL - 1);
    const int rsw = PL == 8 ? ((lane / PL) & 1) : 0;
    const size_t N = (size_t)NX * ny, slot = (size_t)ny * H;
    SmemCursor sc{smem_raw, 0u};
    C *tw = (C *)sc.take(H * sizeof(C));
    C *Wp = (C *)sc.take((H / 2 + 1) * sizeof(C));
    real *kxs = (real *)sc.take(H * sizeof(real));   // k_x of the row bins
    real *buf0 = (real *)sc.take((size_t)CH * NX * sizeof(real));
    real *buf1 = (real *)sc.take((size_t)CH * NX * sizeof(real));
    real *fb = (real *)sc.take((size_t)6 * NX * sizeof(real));   // rho, ux, uy, T, Pi, g rows
    const int NY = P.nrun * ny;
    const int nrows = (int)blockIdx.x < NY ? (NY - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = nrows * NCH;
    if (tid == 0) {   // (the first copies start while the tables load)
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init_fence();
        grid_dep_wait();
        if (njobs > 0) k1w_issue(f, buf0, &bar0, 0, NCH, NG, nx, ny, N);
        if (njobs > 1) k1w_issue(f, buf1, &bar1, 1, NCH, NG, nx, ny, N);
    }
    load_tab4(tw, tw_g, H, NT);
    load_tab4(Wp, Wp_g, H / 2 + 1, NT);
    load_tab4(kxs, kxt, H, NT);
    grid_dep_wait();
    grid_dep_launch();
    __syncthreads();
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = njobs > 0, pend1 = njobs > 1;
    real a0[SMAX], a1[SMAX], a2[SMAX], a3[SMAX];
#pragma unroll
    for (int s = 0; s < SMAX; ++s) a0[s] = a1[s] = a2[s] = a3[s] = real(0);
    for (int jb = 0; jb < njobs; ++jb) {
        const bool odd = jb & 1;
        uint64_t *bar = odd ? &bar1 : &bar0;
        const int ri = jb / NCH, c = jb - ri * NCH;
        const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
        const int run = yg / ny, y = yg - run * ny;
        C *spec_r = spec + (size_t)run * NSLOT * slot;
        real *fields_r = fields + (size_t)run * 4 * N;
        const int i0 = k1w_first(c, NG), nf = k1w_count(c, NG);
        if (!block_wait(bar, odd ? par1 : par0, err)) {
            if (pend0) mbar_wait_bounded(&bar0, par0);
            if (pend1) mbar_wait_bounded(&bar1, par1);
            return;
        }
        if (odd) {
            par1 ^= 1;
            pend1 = false;
        } else {
            par0 ^= 1;
            pend0 = false;
        }
        real *B = odd ? buf1 : buf0;
        // moments (Eqs. 7-9): sums over this chunk's rows
#pragma unroll 1
        for (int r = 0; r < nf; ++r) {
            const int i = i0 + r;
            const real vx = VX<real>(i), vy = VY<real>(i), v2 = V2<real>(i);
#pragma unroll
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                const real v = B[(size_t)r * NX + x];
                a0[s] += v;
                a1[s] += vx * v;
                a2[s] += vy * v;
                a3[s] += v2 * v;
            }
        }
        __syncthreads();
        // forward transforms of the chunk's moving rows: group grp takes
        // chunk row grp + (c == 0) (the first chunk's row 0 is the rest
        // velocity), i.e. f_i with i = i0 + that row, into slot i - 1
        {
            const int r = grp + (c == 0 ? 1 : 0);
            if (r < nf) {
                const int i = i0 + r;
                C *zr = reinterpret_cast<C *>(B) + (size_t)r * H;
                C *dst = spec_r + (size_t)(i - 1) * slot + (size_t)y * H;
                row_fft_wr<H, -1>(zr, tw, j, rsw);
                if (VY<real>(i) == real(0))   // convection in k_x alone: i v_x k_x f^ / nx, no column pass
                    r2c_post_wr2<H>(zr, (C *)nullptr, dst, kxs, VX<real>(i) * P.scale_x, Wp, j);
                else
                    r2c_post_wr<H>(zr, dst, Wp, j);
            }
        }
        if (c == NCH - 1) {
            // the level-1 fields of this row, then their forward transforms
#pragma unroll
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                const real rho = a0[s], ux = a1[s] / rho, uy = a2[s] / rho;
                const real T = real(0.5) * (a3[s] / rho - (ux * ux + uy * uy));
                const size_t o = (size_t)y * nx + x;
                fields_r[o] = rho;
                fields_r[N + o] = ux;
                fields_r[2 * N + o] = uy;
                fields_r[3 * N + o] = T;
                fb[x] = rho;
                fb[NX + x] = ux;
                fb[2 * NX + x] = uy;
                fb[3 * NX + x] = T;
                fb[4 * NX + x] = rho * T / (real(1) - P.b * rho) - P.a * rho * rho - rho * T;   // Eq. 18
                fb[5 * NX + x] = (P.K + P.H * T) / T;                                          // M / T
                a0[s] = a1[s] = a2[s] = a3[s] = real(0);
            }
            __syncthreads();
            if (grp < 6) {
                C *zr = reinterpret_cast<C *>(fb) + (size_t)grp * H;
                row_fft_wr<H, -1>(zr, tw, j, rsw);
                r2c_post_wr<H>(zr, spec_r + (size_t)(SLOT_RHO + grp) * slot + (size_t)y * H, Wp, j);
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && jb + 2 < njobs) {   // job jb + 2 reuses this buffer
            k1w_issue(f, B, bar, jb + 2, NCH, NG, nx, ny, N);
            if (odd) pend1 = true;
            else pend0 = true;
        }
    }
}

// shared memory of k1_wr<H>
inline size_t k1_wr_smem(int H) {
    const int P = H == 512 ? 32 : H == 256 ? 16 : 8;
    const int CH = (nt_k1wr_host(H) / 32) * (32 / P) + 1;
    return smem_bytes({(size_t)H * 8, (size_t)(H / 2 + 1) * 8, (size_t)H * 4, (size_t)CH * 2 * H * 4,
                       (size_t)CH * 2 * H * 4, (size_t)6 * 2 * H * 4});
}

// ---------------------------------------------------------------------------
// K3 (fp32, nx = 2H): row inverse of the 15 level-1 derivative spectra ->
// Lambda (Eq. 19), Phi = 2 q rho T grad T (Eq. 23), the numerators of C
// (Eq. 22) and B (Eq. 21) -> forward row transforms of Lambda_xx,
// Lambda_xy, Lambda_yy, Phi_x, Phi_y, as k3_pipe, with warp-resident row
// transforms.  Persistent over the rows of all runs, one row per pass, two
// buffers (15 spectrum rows + rho, T), the next-but-one row prefetched.
// ---------------------------------------------------------------------------

template <typename real>
__device__ __forceinline__ void k3_issue(const typename cplx_of<real>::type *spec, const real *fields, real *dst,
                                         uint64_t *bar, int ri, int nx, int ny, size_t N, size_t slot, int h) {
    const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
    const int run = yg / ny, y = yg - run * ny;
    spec += (size_t)run * NSLOT * slot;
    fields += (size_t)run * 4 * N;
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(real));
    mbar_expect_tx(bar, (uint32_t)(ND1 + 1) * rowbytes);   // D_DIVX is formed in K3
    for (int o = 0; o < ND1; ++o)
        if (k3_src_slot(o) >= 0)
            bulk_g2s(dst + (size_t)o * nx, spec + (size_t)k3_src_slot(o) * slot + (size_t)y * h, rowbytes, bar);
    bulk_g2s(dst + (size_t)ND1 * nx, fields + (size_t)y * nx, rowbytes, bar);
    bulk_g2s(dst + (size_t)(ND1 + 1) * nx, fields + 3 * N + (size_t)y * nx, rowbytes, bar);
}

template <int H>
__global__ void __launch_bounds__(nt_k3wr<H>(), nt_k3wr<H>() >= 512 ? 1 : 2) k3_wr(float2 *spec, const float *__restrict__ fields,
                                                 float *__restrict__ aux, const float2 *__restrict__ tw_g,
                                                 const float2 *__restrict__ Wp_g, const float *__restrict__ kxt,
                                                 KP<float> P, int *err) {
    using C = float2;
    using real = float;
    constexpr int NX = 2 * H, NT = nt_k3wr<H>(), NB = nb_k3wr<H>();
    constexpr int PL = RowCfg<H>::P, RPW = 32 / PL, NG = (NT / 32) * RPW;   // row groups
    constexpr int SMAX = (NX + NT - 1) / NT;
    constexpr int RB = ND1 + 2;   // rows per buffer
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1;
    const int nx = NX, ny = P.ny, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = warp * RPW + lane / PL, j = lane & (PL - 1);
    const int rsw = PL == 8 ? ((lane / PL) & 1) : 0;
    const size_t N = (size_t)NX * ny, slot = (size_t)ny * H;
    SmemCursor sc{smem_raw, 0u};
    C *tw = (C *)sc.take(H * sizeof(C));
    C *Wp = (C *)sc.take((H / 2 + 1) * sizeof(C));
    real *kxs = (real *)sc.take(H * sizeof(real));   // k_x of the row bins
    real *buf0 = (real *)sc.take((size_t)RB * NX * sizeof(real));
    real *buf1 = NB > 1 ? (real *)sc.take((size_t)RB * NX * sizeof(real)) : buf0;
    const int NY = P.nrun * ny;
    const int nrows = (int)blockIdx.x < NY ? (NY - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {   // (the first copies start before the tables load)
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init_fence();
        grid_dep_wait();
        if (nrows > 0) k3_issue<real>(spec, fields, buf0, &bar0, 0, nx, ny, N, slot, H);
        if (NB > 1 && nrows > 1) k3_issue<real>(spec, fields, buf1, &bar1, 1, nx, ny, N, slot, H);
    }
    load_tab4(tw, tw_g, H, NT);
    load_tab4(Wp, Wp_g, H / 2 + 1, NT);
    load_tab4(kxs, kxt, H, NT);
    grid_dep_wait();
    grid_dep_launch();
    __syncthreads();
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = nrows > 0, pend1 = NB > 1 && nrows > 1;
    for (int ri = 0; ri < nrows; ++ri) {
        const bool odd = NB > 1 && (ri & 1);
        uint64_t *bar = odd ? &bar1 : &bar0;
        const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
        const int run = yg / ny, y = yg - run * ny;
        C *spec_r = spec + (size_t)run * NSLOT * slot;
        real *aux_r = aux + (size_t)run * 3 * N;
        if (!block_wait(bar, odd ? par1 : par0, err)) {
            if (pend0) mbar_wait_bounded(&bar0, par0);
            if (pend1) mbar_wait_bounded(&bar1, par1);
            return;
        }
        if (odd) {
            par1 ^= 1;
            pend1 = false;
        } else {
            par0 ^= 1;
            pend0 = false;
        }
        real *d = odd ? buf1 : buf0;
        for (int k = tid; k < H; k += NT) k3_form_x<real>(reinterpret_cast<C *>(d), H, k, kxs[k], P.scale_x);
        __syncthreads();
        for (int r = grp; r < ND1; r += NG) {   // (uniform over each row group)
            C *zr = reinterpret_cast<C *>(d) + (size_t)r * H;
            c2r_pre_wr<H>(zr, Wp, j);
            __syncwarp(group_mask<PL>());
            row_fft_wr<H, +1>(zr, tw, j, rsw);
        }
        __syncthreads();
        const real *rT = d + (size_t)ND1 * NX;
#pragma unroll 1
        for (int s = 0; s < SMAX; ++s) {
            const int x = tid + s * NT;
            const size_t o = (size_t)y * nx + x;
            const real rho = rT[x], T = rT[NX + x];
            const real rx = d[D_RX * NX + x], ry = d[D_RY * NX + x], lap = d[D_LAP * NX + x];
            const real uxx = d[D_UXX * NX + x], uxy = d[D_UXY * NX + x];
            const real uyx = d[D_UYX * NX + x], uyy = d[D_UYY * NX + x];
            const real divx = d[D_DIVX * NX + x], divy = d[D_DIVY * NX + x];
            const real Tx = d[D_TX * NX + x], Ty = d[D_TY * NX + x];
            const real Pix = d[D_PIX * NX + x], Piy = d[D_PIY * NX + x];
            const real gx = d[D_GX * NX + x], gy = d[D_GY * NX + x];
            const real M = P.K + P.H * T;
            const real Pi = rho * T / (real(1) - P.b * rho) - P.a * rho * rho - rho * T;
            const real grad2 = rx * rx + ry * ry;
            const real iso = -(rho * T * (rx * gx + ry * gy)) - M * (rho * lap + real(0.5) * grad2);   // Eq. 19
            const real Lxx = M * rx * rx + iso, Lxy = M * rx * ry, Lyy = M * ry * ry + iso;
            const real div = uxx + uyy;
            const real Ldu = Lxx * uxx + Lxy * (uyx + uxy) + Lyy * uyy;
            const real Cn = Pi * div + Ldu - P.zeta * div * div + P.a * rho * rho * div +
                            P.K * (real(-0.5) * grad2 * div - rho * (rx * divx + ry * divy) -
                                   (rx * (uxx * rx + uyx * ry) + ry * (uxy * rx + uyy * ry)));   // Eq. 22
            aux_r[o] = Cn;
            aux_r[N + o] = Pix - P.zeta * divx;   // Eq. 21 without d_b Lambda_ab
            aux_r[2 * N + o] = Piy - P.zeta * divy;
            const real q2 = real(2) * P.q * rho * T;   // Eq. 23
            // rows 0..4 (same site, same thread)
            d[0 * NX + x] = Lxx;
            d[1 * NX + x] = Lxy;
            d[2 * NX + x] = Lyy;
            d[3 * NX + x] = q2 * Tx;
            d[4 * NX + x] = q2 * Ty;
        }
        __syncthreads();
        for (int r = grp; r < 5; r += NG) {
            C *zr = reinterpret_cast<C *>(d) + (size_t)r * H;
            row_fft_wr<H, -1>(zr, tw, j, rsw);
            C *raw = k3_raw_slot(r) >= 0 ? spec_r + (size_t)k3_raw_slot(r) * slot + (size_t)y * H : nullptr;
            C *mul = k3_mul_slot(r) >= 0 ? spec_r + (size_t)k3_mul_slot(r) * slot + (size_t)y * H : nullptr;
            r2c_post_wr2<H>(zr, raw, mul, kxs, P.scale_x, Wp, j);
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && ri + NB < nrows) {   // row ri + NB reuses this buffer
            k3_issue<real>(spec, fields, d, bar, ri + NB, nx, ny, N, slot, H);
            if (odd) pend1 = true;
            else pend0 = true;
        }
    }
}

// shared memory of k3_wr<H>
inline size_t k3_wr_smem(int H) {
    return smem_bytes({(size_t)H * 8, (size_t)(H / 2 + 1) * 8, (size_t)H * 4, (size_t)(ND1 + 2) * 2 * H * 4,
                       nb_k3wr_host(H) > 1 ? (size_t)(ND1 + 2) * 2 * H * 4 : 0});
}

// ---------------------------------------------------------------------------
// K5 (fp32, nx = 2H): convection rows + level-2 divergences (inverse) ->
// A, B, C, C_q (Eqs. 20-23), f^eq (Eq. 3), I (Eq. 11), BGK and the RK
// combination (Eq. 10), as k5_pipe, with warp-resident row transforms.
// Persistent over the rows of all runs; per row: the head (3 level-2
// spectra, rho, u_x, u_y, T, the 3 aux numerators; two buffers, prefetched
// a row ahead) and 32 / CH chunks of CH convection rows (two buffers), each
// chunk one row per row group (CH = 16 warps x rows per warp: two rings for
// H = 512, all four for H = 256).
// ---------------------------------------------------------------------------

template <int H>
__global__ void __launch_bounds__(nt_k5wr<H>(), nt_k5wr<H>() >= 512 ? 1 : 2) k5_wr(const float2 *spec, const float *__restrict__ fields,
                                                 const float *__restrict__ aux, const float *fcur, const float *fbase,
                                                 float *fout, float alpha, float beta,
                                                 const float2 *__restrict__ tw_g, const float2 *__restrict__ Wp_g,
                                                 KP<float> P, int *err) {
    using C = float2;
    using real = float;
    constexpr int NX = 2 * H, NT = nt_k5wr<H>(), NWARP = NT / 32, NHB = nhb_k5wr<H>();
    constexpr int PL = RowCfg<H>::P, RPW = 32 / PL;          // lanes per row, rows per warp
    constexpr int CH = NWARP * RPW, NCH = NMOV / CH;           // rows per chunk, chunks per row
    constexpr int NRING = CH / 8;                              // rings per chunk
    constexpr int SMAX = (NX + NT - 1) / NT;
    static_assert(NMOV % CH == 0 && CH % 8 == 0, "chunking");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1, hbar0, hbar1;
    const int nx = NX, ny = P.ny, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grow = warp * RPW + lane / PL, j = lane & (PL - 1);   // row within the chunk, lane within the row
    const int rsw = PL == 8 ? ((lane / PL) & 1) : 0;
    const size_t N = (size_t)NX * ny, slot = (size_t)ny * H;
    SmemCursor sc{smem_raw, 0u};
    C *tw = (C *)sc.take(H * sizeof(C));
    C *Wp = (C *)sc.take((H / 2 + 1) * sizeof(C));
    real *head0 = (real *)sc.take((size_t)NHEAD * NX * sizeof(real));
    real *head1 = NHB > 1 ? (real *)sc.take((size_t)NHEAD * NX * sizeof(real)) : head0;
    real *buf0 = (real *)sc.take((size_t)CH * NX * sizeof(real));
    real *buf1 = (real *)sc.take((size_t)CH * NX * sizeof(real));
    const int NY = P.nrun * ny;
    const int nrows = (int)blockIdx.x < NY ? (NY - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = nrows * NCH;
    if (tid == 0) {   // (the first copies start before the tables load)
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init(&hbar0, 1);
        mbar_init(&hbar1, 1);
        mbar_init_fence();
        // Only the head's level-2 rows come from the launch just before this
        // one (the level-2 columns); the convection spectra, fields, aux rows
        // and distributions were complete before that launch began, and that
        // launch touches none of what this kernel writes.  So under a
        // programmatic dependent launch only the head copies wait.
        if (njobs > 0) k5_issue_chunk<real>(spec, buf0, &bar0, 0, NCH, CH, nx, ny, slot, H);
        if (njobs > 1) k5_issue_chunk<real>(spec, buf1, &bar1, 1, NCH, CH, nx, ny, slot, H);
        grid_dep_wait();
        if (nrows > 0) k5_issue_head<real>(spec, fields, aux, head0, &hbar0, 0, nx, ny, N, slot, H);
        if (NHB > 1 && nrows > 1) k5_issue_head<real>(spec, fields, aux, head1, &hbar1, 1, nx, ny, N, slot, H);
    }
    load_tab4(tw, tw_g, H, NT);
    load_tab4(Wp, Wp_g, H / 2 + 1, NT);
    grid_dep_launch();
    __syncthreads();
    uint32_t par0 = 0, par1 = 0, hpar0 = 0, hpar1 = 0;
    bool pend0 = njobs > 0, pend1 = njobs > 1, hpend0 = nrows > 0, hpend1 = NHB > 1 && nrows > 1;
    const real dt = P.dt, itau = real(1) / P.tau;
    const bool with_base = alpha != real(0);
    for (int jb = 0; jb < njobs; ++jb) {
        const bool odd = jb & 1;
        const int ri = jb / NCH, c = jb - ri * NCH;
        const bool hodd = NHB > 1 && (ri & 1);
        const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
        const int run = yg / ny, y = yg - run * ny;
        const size_t fo = (size_t)run * Q * N;
        real *Hd = hodd ? head1 : head0;
        if (!block_wait(odd ? &bar1 : &bar0, odd ? par1 : par0, err)) {
            if (pend0) mbar_wait_bounded(&bar0, par0);
            if (pend1) mbar_wait_bounded(&bar1, par1);
            if (hpend0) mbar_wait_bounded(&hbar0, hpar0);
            if (hpend1) mbar_wait_bounded(&hbar1, hpar1);
            return;
        }
        if (odd) {
            par1 ^= 1;
            pend1 = false;
        } else {
            par0 ^= 1;
            pend0 = false;
        }
        real *B = odd ? buf1 : buf0;
        // inverse transforms: convection row grow of the chunk; with the
        // first chunk, then (its copies complete) the 3 level-2 rows of the
        // head (row groups 0..2)
        {
            const unsigned gm = group_mask<PL>();
            C *zr = reinterpret_cast<C *>(B) + (size_t)grow * H;
            c2r_pre_wr<H>(zr, Wp, j);
            __syncwarp(gm);
            row_fft_wr<H, +1>(zr, tw, j, rsw);
            if (c == 0) {
                if (!block_wait(hodd ? &hbar1 : &hbar0, hodd ? hpar1 : hpar0, err)) {
                    if (pend0) mbar_wait_bounded(&bar0, par0);
                    if (pend1) mbar_wait_bounded(&bar1, par1);
                    if (hpend0) mbar_wait_bounded(&hbar0, hpar0);
                    if (hpend1) mbar_wait_bounded(&hbar1, hpar1);
                    return;
                }
                if (hodd) {
                    hpar1 ^= 1;
                    hpend1 = false;
                } else {
                    hpar0 ^= 1;
                    hpend0 = false;
                }
                if (grow < 3) {   // uniform over each row group
                    C *zh = reinterpret_cast<C *>(Hd) + (size_t)grow * H;
                    c2r_pre_wr<H>(zh, Wp, j);
                    __syncwarp(gm);
                    row_fft_wr<H, +1>(zh, tw, j, rsw);
                }
            }
        }
        __syncthreads();
        if (c == 0) {
            // per-site coefficients over the head rows (same site, same
            // thread): row 0 <- e0, 1 <- e1x, 2 <- e1y, 7 <- C + C_q, 8 <- 1/T;
            // the rest velocity's update
            if constexpr (NX == 4 * NT && FFTLB_K5_VEC > 0) {   // four consecutive sites per thread
                const int x0 = 4 * tid;
                const size_t o = fo + (size_t)y * nx + x0;
                real rho[4], ux[4], uy[4], T[4], dLx[4], dLy[4], dPh[4], a7[4], a8[4], a9[4], fc[4], fb[4];
                ld4(rho, Hd + 3 * nx + x0);
                ld4(ux, Hd + 4 * nx + x0);
                ld4(uy, Hd + 5 * nx + x0);
                ld4(T, Hd + 6 * nx + x0);
                ld4(dLx, Hd + x0);
                ld4(dLy, Hd + nx + x0);
                ld4(dPh, Hd + 2 * nx + x0);
                ld4(a7, Hd + 7 * nx + x0);
                ld4(a8, Hd + 8 * nx + x0);
                ld4(a9, Hd + 9 * nx + x0);
                ld4(fc, fcur + o);
                if (with_base) ld4(fb, fbase + o);
                real e0[4], e1x[4], e1y[4], CC[4], iT[4], fn[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const real rT = rho[q] * T[q];
                    const real inv2 = real(1) / (real(2) * rho[q] * T[q] * T[q]);
                    const real Bx = (a8[q] + dLx[q]) / rT;      // Eq. 21
                    const real By = (a9[q] + dLy[q]) / rT;
                    CC[q] = (a7[q] + dPh[q]) * inv2;            // C + C_q, Eqs. 22-23
                    const real A = real(-2) * CC[q] * T[q];      // Eq. 20
                    const real u2 = ux[q] * ux[q] + uy[q] * uy[q];
                    e0[q] = A - (Bx * ux[q] + By * uy[q]) + CC[q] * u2;
                    e1x[q] = Bx - real(2) * CC[q] * ux[q];
                    e1y[q] = By - real(2) * CC[q] * uy[q];
                    iT[q] = real(1) / T[q];
                    real F[5];
                    weights_Fk<real>(T[q], F);
                    const real qq = real(0.5) * u2 / T[q], om = real(1) - qq;
                    const real fe = rho[q] * F[0] * (om + real(0.5) * qq * qq);
                    fn[q] = beta * (fc[q] + dt * (-(fc[q] - fe) * itau - e0[q] * fe));
                    if (with_base) fn[q] += alpha * fb[q];
                }
                st4(Hd + x0, e0);
                st4(Hd + nx + x0, e1x);
                st4(Hd + 2 * nx + x0, e1y);
                st4(Hd + 7 * nx + x0, CC);
                st4(Hd + 8 * nx + x0, iT);
                st4(fout + o, fn);
            } else
#pragma unroll 1
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x < nx) {
                    const real rho = Hd[3 * nx + x], ux = Hd[4 * nx + x], uy = Hd[5 * nx + x], T = Hd[6 * nx + x];
                    const real dLx = Hd[x], dLy = Hd[nx + x], dPh = Hd[2 * nx + x];
                    const real rT = rho * T;
                    const real inv2 = real(1) / (real(2) * rho * T * T);
                    const real Bx = (Hd[8 * nx + x] + dLx) / rT;      // Eq. 21
                    const real By = (Hd[9 * nx + x] + dLy) / rT;
                    const real CC = (Hd[7 * nx + x] + dPh) * inv2;    // C + C_q, Eqs. 22-23
                    const real A = real(-2) * CC * T;                 // Eq. 20
                    const real u2 = ux * ux + uy * uy;
                    const real e0 = A - (Bx * ux + By * uy) + CC * u2;
                    Hd[x] = e0;
                    Hd[nx + x] = Bx - real(2) * CC * ux;
                    Hd[2 * nx + x] = By - real(2) * CC * uy;
                    Hd[7 * nx + x] = CC;
                    Hd[8 * nx + x] = real(1) / T;
                    real F[5];
                    weights_Fk<real>(T, F);
                    const real qq = real(0.5) * u2 / T, om = real(1) - qq;
                    const real fe = rho * F[0] * (om + real(0.5) * qq * qq);
                    const size_t o = fo + (size_t)y * nx + x;
                    const real fc = fcur[o];
                    real fn = beta * (fc + dt * (-(fc - fe) * itau - e0 * fe));
                    if (with_base) fn += alpha * fbase[o];
                    fout[o] = fn;
                }
            }
            __syncthreads();
        }
        // epilogue: the NRING rings of the chunk (ring k = c NRING + rr:
        // velocities 1 + 8k .. 8 + 8k of Eq. 1, one speed, one weight, the
        // eight directions known at compile time)
#pragma unroll 1
        for (int rr = 0; rr < NRING; ++rr) {
            const int k = c * NRING + rr;
            const int v0 = 8 * k;
            const real sk = VX<real>(1 + v0), sk2 = V2<real>(1 + v0);
            const real *cres = B + (size_t)rr * 8 * NX;
            if constexpr (NX == 4 * NT && FFTLB_K5_VEC > 0) {
                // four consecutive sites per thread: 16-byte loads and stores
                const int x0 = 4 * tid;
                const size_t o0 = fo + (size_t)(1 + v0) * N + (size_t)y * nx + x0;
                real rho[4], ux[4], uy[4], T[4], iT[4], e0[4], e1x[4], e1y[4], CC[4];
                ld4(rho, Hd + 3 * nx + x0);
                ld4(ux, Hd + 4 * nx + x0);
                ld4(uy, Hd + 5 * nx + x0);
                ld4(T, Hd + 6 * nx + x0);
                ld4(iT, Hd + 8 * nx + x0);
                ld4(e0, Hd + x0);
                ld4(e1x, Hd + nx + x0);
                ld4(e1y, Hd + 2 * nx + x0);
                ld4(CC, Hd + 7 * nx + x0);
                real rF[4], p0[4], p1[4], p2[4], p3[4], p4[4], g0[4], uxk[4], uyk[4], exk[4], eyk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const real qq = real(0.5) * (ux[q] * ux[q] + uy[q] * uy[q]) * iT[q], om = real(1) - qq;
                    p0[q] = om + real(0.5) * qq * qq;
                    p1[q] = om * iT[q];
                    p2[q] = real(0.5) * om * iT[q] * iT[q];
                    p3[q] = iT[q] * iT[q] * iT[q] * (real(1) / real(6));
                    p4[q] = iT[q] * iT[q] * iT[q] * iT[q] * (real(1) / real(24));
                    rF[q] = rho[q] * weight_Fk<real>(k, T[q]);   // Eq. 4
                    g0[q] = e0[q] + CC[q] * sk2;
                    uxk[q] = sk * ux[q];
                    uyk[q] = sk * uy[q];
                    exk[q] = sk * e1x[q];
                    eyk[q] = sk * e1y[q];
                }
                // (FFTLB_K5_VEC = 1: the distributions of four directions are
                // loaded before any of their stores, as fout may alias fcur or
                // fbase; 2: all eight, through restrict-qualified pointers, as
                // each element is read before the same thread writes it)
                const real *__restrict__ pc = fcur + o0;
                const real *__restrict__ pb = fbase + o0;
                real *__restrict__ po = fout + o0;
                constexpr int RH = FFTLB_K5_VEC == 1 ? 4 : 8;
#pragma unroll
                for (int r0 = 0; r0 < 8; r0 += RH) {
                    real fc[RH][4], fb[RH][4];
#pragma unroll
                    for (int r = 0; r < RH; ++r) {
                        ld4(fc[r], pc + (size_t)(r0 + r) * N);
                        if (with_base) ld4(fb[r], pb + (size_t)(r0 + r) * N);
                    }
#pragma unroll
                    for (int r = 0; r < RH; ++r) {
                        real cv[4], fn[4];
                        ld4(cv, cres + (size_t)(r0 + r) * NX + x0);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const real vu = dir_dot<real>(r0 + r, uxk[q], uyk[q]);
                            const real br = p0[q] + vu * (p1[q] + vu * (p2[q] + vu * (p3[q] + vu * p4[q])));
                            const real fe = rF[q] * br;                                          // Eq. 3
                            const real I = -(g0[q] + dir_dot<real>(r0 + r, exk[q], eyk[q])) * fe;  // Eq. 11
                            const real rhs = -cv[q] - (fc[r][q] - fe) * itau + I;                // Eq. 10
                            fn[q] = beta * (fc[r][q] + dt * rhs);
                            if (with_base) fn[q] += alpha * fb[r][q];
                        }
                        st4(po + (size_t)(r0 + r) * N, fn);
                    }
                }
            } else {
#pragma unroll(K5U)
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x >= nx) continue;
                real fc[8], fb[8];
                const size_t o0 = fo + (size_t)(1 + v0) * N + (size_t)y * nx + x;
                const real *pc = fcur + o0;
                const real *pb = fbase + o0;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    fc[r] = pc[r * N];
                    fb[r] = with_base ? pb[r * N] : real(0);
                }
                real *po = fout + o0;
                const real rho = Hd[3 * nx + x], ux = Hd[4 * nx + x], uy = Hd[5 * nx + x], T = Hd[6 * nx + x];
                const real iT = Hd[8 * nx + x];
                const real e0 = Hd[x], e1x = Hd[nx + x], e1y = Hd[2 * nx + x], CC = Hd[7 * nx + x];
                const real Fk = weight_Fk<real>(k, T);   // Eq. 4
                const real qq = real(0.5) * (ux * ux + uy * uy) * iT, om = real(1) - qq;
                const real p0 = om + real(0.5) * qq * qq, p1 = om * iT, p2 = real(0.5) * om * iT * iT;
                const real p3 = iT * iT * iT * (real(1) / real(6)), p4 = iT * iT * iT * iT * (real(1) / real(24));
                const real rF = rho * Fk;
                const real g0 = e0 + CC * sk2;
                const real uxk = sk * ux, uyk = sk * uy, exk = sk * e1x, eyk = sk * e1y;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const real vu = dir_dot<real>(r, uxk, uyk);
                    const real br = p0 + vu * (p1 + vu * (p2 + vu * (p3 + vu * p4)));
                    const real fe = rF * br;                                                 // Eq. 3
                    const real I = -(g0 + dir_dot<real>(r, exk, eyk)) * fe;                   // Eq. 11
                    const real conv = cres[(size_t)r * NX + x];
                    const real rhs = -conv - (fc[r] - fe) * itau + I;                        // Eq. 10
                    real fn = beta * (fc[r] + dt * rhs);
                    if (with_base) fn += alpha * fb[r];
                    po[r * N] = fn;
                }
            }
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && jb + 1 < njobs) {
            // the next job's distribution rows (current and, for RK stages 2
            // and 3, base state) into L2 ahead of its epilogue's loads
            const int nri = (jb + 1) / NCH, nc = (jb + 1) - nri * NCH;
            const int nyg = (int)blockIdx.x + nri * (int)gridDim.x;
            const int nrun = nyg / ny, ny_ = nyg - nrun * ny;
            const size_t no = (size_t)nrun * Q * N + (size_t)(1 + nc * CH) * N + (size_t)ny_ * nx;
            for (int r = 0; r < CH; ++r) {
                bulk_prefetch_l2(fcur + no + (size_t)r * N, (uint32_t)(NX * sizeof(real)));
                if (with_base) bulk_prefetch_l2(fbase + no + (size_t)r * N, (uint32_t)(NX * sizeof(real)));
            }
        }
        if (tid == 0) {
            if (jb + 2 < njobs) {
                const bool nodd = jb & 1;   // chunk jb + 2 reuses this buffer
                k5_issue_chunk<real>(spec, B, nodd ? &bar1 : &bar0, jb + 2, NCH, CH, nx, ny, slot, H);
                if (nodd) pend1 = true;
                else pend0 = true;
            }
            if (c == NCH - 1 && ri + NHB < nrows) {   // the row's head buffer is free
                k5_issue_head<real>(spec, fields, aux, Hd, hodd ? &hbar1 : &hbar0, ri + NHB, nx, ny, N, slot, H);
                if (hodd) hpend1 = true;
                else hpend0 = true;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Column transforms of a tile of TW spectrum columns of length NY = E * P
// (the tile [NY][TW] complex as the tensor copy lands it): thread (c, l)
// (c < TW fastest, l < P) holds column c's x[l + P t], t < E:
//   stage 1: E-point DFT over t, times W_NY^(l k1), stored in place at row
//            k1 P + (l ^ (k1 & SW)) of the tile (SW = 16 / TW - 1: the row
//            swizzle that keeps stage 2's reads conflict-free; the rows it
//            exchanges belong to threads of the same warp, so __syncwarp
//            orders the in-place store);
//   __syncthreads;
//   stage 2: thread (c, j) takes k1 = j + P q (q < E / P) and the P-point
//            DFT over l: the spectrum X[k1 + E k2] of column c in registers;
//            the multiplier (convection: i (v_x k_x + v_y k_y) / (nx ny)),
//            the inverse P-point DFT and the conjugate twiddles follow in
//            registers and the values go back where they were read;
//   __syncthreads;
//   stage 1 inverse: the inverse E-point DFT over k1, stored to global.
// The packed column 0 of the tile at k_x = 0 (DC real, row-Nyquist
// imaginary) needs no pairing of (k_y, -k_y): both columns it carries take
// the multiplier at k_x = 0, because the Nyquist bin of k_x is zero.
// ---------------------------------------------------------------------------

// (FFTLB_COL1024_TW: the 1024-point tile width, 8 by default; 4 halves the
// blocks and doubles their number per SM, measured slower: convection 102 ->
// 112 us, level 1 62 -> 96 us at 1024^2)
#ifndef FFTLB_COL1024_TW
#define FFTLB_COL1024_TW 8
#endif
template <int NY> struct ColCfg;
template <> struct ColCfg<1024> { static constexpr int E = 32, P = 32, TW = FFTLB_COL1024_TW; };
template <> struct ColCfg<512> { static constexpr int E = 32, P = 16, TW = 16; };
template <> struct ColCfg<256> { static constexpr int E = 16, P = 16, TW = 16; };
template <> struct ColCfg<128> { static constexpr int E = 16, P = 8, TW = 32; };
inline int col_tw_host(int NY) { return NY == 1024 ? FFTLB_COL1024_TW : NY == 128 ? 32 : 16; }
inline int col_p_host(int NY) { return NY == 1024 ? 32 : NY == 128 ? 8 : 16; }

template <int NY>
__device__ __forceinline__ int cpos(int c, int l, int k1) {
    constexpr int P = ColCfg<NY>::P, TW = ColCfg<NY>::TW, SW = TW < 16 ? 16 / TW - 1 : 0;
    return (k1 * P + (l ^ (k1 & SW))) * TW + c;
}

template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::TW * ColCfg<NY>::P, ColCfg<NY>::TW * ColCfg<NY>::P >= 256 ? 2 : 4) kcol_wr(float2 *spec,
                                                                             const GroupDesc *__restrict__ groups,
                                                                             int ngroups,
                                                                             const float *__restrict__ kxt,
                                                                             const float *__restrict__ kyt,
                                                                             const float2 *__restrict__ twc_g,
                                                                             KP<float> P, int BOXR, int nbuf,
                                                                             const __grid_constant__ CUtensorMap tmap,
                                                                             int *err) {
    using C = float2;
    using real = float;
    constexpr int E = ColCfg<NY>::E, PP = ColCfg<NY>::P, TW = ColCfg<NY>::TW, NT = TW * PP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1, abar;
    __shared__ ColG gt[kMaxColGroups];   // ngroups <= kMaxColGroups (checked by the host)
    const int h = P.h, tid = threadIdx.x;
    const int c = tid % TW, jl = tid / TW;
    const size_t slot = (size_t)NY * h;
    constexpr int tile = TW * NY;
    SmemCursor sc{smem_raw, 0u};
    C *twc = (C *)sc.take((size_t)2 * NY * sizeof(C));   // [k1][l] (stage 1), then [l][k1] (stage 2)
    const C *twt = twc + NY;
    real *kxs = (real *)sc.take((size_t)(h + 1) * sizeof(real));
    real *kys = (real *)sc.take(NY * sizeof(real));
    C *buf0 = (C *)sc.take((size_t)tile * sizeof(C));
    C *buf1 = nbuf > 1 ? (C *)sc.take((size_t)tile * sizeof(C)) : buf0;
    const int ntiles = h / TW;
    const int njobs_total = P.nrun * ngroups * ntiles;
    const int njobs = (int)blockIdx.x < njobs_total ? (njobs_total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {   // (the first copies start before the tables load)
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init(&abar, 1);
        mbar_init_fence();
        grid_dep_wait();
        if (njobs > 0) kcol_issue(buf0, &bar0, groups, 0, ntiles, ngroups, TW, NY, BOXR, &tmap);
        if (nbuf > 1 && njobs > 1) kcol_issue(buf1, &bar1, groups, 1, ntiles, ngroups, TW, NY, BOXR, &tmap);
        if (njobs > nbuf) kcol_prefetch(groups, nbuf, ntiles, ngroups, TW, NY, BOXR, &tmap);
    }
    load_tab4(twc, twc_g, 2 * NY, NT);
    load_tab4(kxs, kxt, h + 1, NT);
    load_tab4(kys, kyt, NY, NT);
    for (int g = tid; g < ngroups; g += NT) {
        const GroupDesc &G = groups[g];
        gt[g] = ColG{G.nin, {G.in_slot[0], G.in_slot[1]}, G.out_slot[0], G.add_slot, (float)G.c[0][0][0],
                     (float)G.c[0][0][1]};
    }
    grid_dep_wait();
    grid_dep_launch();
    __syncthreads();
    uint32_t par0 = 0, par1 = 0, apar = 0;
    bool pend0 = njobs > 0, pend1 = nbuf > 1 && njobs > 1;
    const real scale = P.scale;
    for (int k = 0; k < njobs; ++k) {
        const bool odd = k & 1;
        uint64_t *bar = odd ? &bar1 : &bar0;
        const int job = (int)blockIdx.x + k * (int)gridDim.x;
        const int run = job / (ngroups * ntiles), jr = job - run * ngroups * ntiles;
        const int g = jr / ntiles, t = jr - g * ntiles;
        const int kx0 = t * TW;
        if (!block_wait(bar, odd ? par1 : par0, err)) {
            if (pend0) mbar_wait_bounded(&bar0, par0);
            if (pend1) mbar_wait_bounded(&bar1, par1);
            return;
        }
        if (odd) {
            par1 ^= 1;
            pend1 = false;
        } else {
            par0 ^= 1;
            pend0 = false;
        }
        C *T = odd ? buf1 : buf0;
        const int oslot = gt[g].out_slot, aslot = gt[g].add_slot;
        const real c0 = gt[g].c0, c1 = gt[g].c1;
        C v[E];
        // stage 1, forward
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = T[(jl + PP * q) * TW + c];
        SmallDFT<E, -1, C>::run(v);
#pragma unroll
        for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], twc[k1 * PP + jl]);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < E; ++k1) T[cpos<NY>(c, jl, k1)] = v[k1];
        __syncthreads();
        // stage 2: forward, multiplier, inverse, conjugate twiddles
        {
            const real mx = c0 * kxs[kx0 + c];
#pragma unroll
            for (int q = 0; q < E / PP; ++q) {
                const int k1 = jl + PP * q;
                C u[PP];
#pragma unroll
                for (int l = 0; l < PP; ++l) u[l] = T[cpos<NY>(c, l, k1)];
                SmallDFT<PP, -1, C>::run(u);
#pragma unroll
                for (int k2 = 0; k2 < PP; ++k2) {
                    const real m = (mx + c1 * kys[k1 + E * k2]) * scale;   // i m
                    u[k2] = C{-m * u[k2].y, m * u[k2].x};
                }
                SmallDFT<PP, +1, C>::run(u);
#pragma unroll
                for (int l = 0; l < PP; ++l) T[cpos<NY>(c, l, k1)] = l == 0 ? u[l] : cmul(u[l], cconj(twt[l * E + k1]));
            }
        }
        __syncthreads();
        // stage 1, inverse
#pragma unroll
        for (int k1 = 0; k1 < E; ++k1) v[k1] = T[cpos<NY>(c, jl, k1)];
        fence_proxy_async();
        __syncthreads();
        // the tile buffer is free: with an addend, its tile comes into the
        // buffer first (read after the inverse DFT), then the next job's
        if (tid == 0 && aslot >= 0) {
            const int sl = run * NSLOT + aslot;
            mbar_expect_tx(&abar, (uint32_t)(tile * sizeof(C)));
            for (int r0 = 0; r0 < NY; r0 += BOXR) tma_load_2d(T + (size_t)r0 * TW, &tmap, 2 * t * TW, sl * NY + r0, &abar);
        }
        if (tid == 0 && aslot < 0 && k + nbuf < njobs) {   // prefetch job k + nbuf into the buffer
            const bool nodd = (k + nbuf) & 1;
            kcol_issue(T, nodd ? &bar1 : &bar0, gt, k + nbuf, ntiles, ngroups, TW, NY, BOXR, &tmap);
            if (nodd) pend1 = true;
            else pend0 = true;
            // and the job after it into L2, so that its copy finds the tiles there
            if (k + nbuf + 1 < njobs) kcol_prefetch(gt, k + nbuf + 1, ntiles, ngroups, TW, NY, BOXR, &tmap);
        }
        SmallDFT<E, +1, C>::run(v);
        C *out = spec + (size_t)run * NSLOT * slot + (size_t)oslot * slot + kx0 + c;
        if (aslot >= 0) {   // plus the term the row kernel formed
            if (!block_wait(&abar, apar, err)) {
                mbar_wait_bounded(&abar, apar);
                if (pend0) mbar_wait_bounded(&bar0, par0);
                if (pend1) mbar_wait_bounded(&bar1, par1);
                return;
            }
            apar ^= 1;
#pragma unroll
            for (int q = 0; q < E; ++q) out[(size_t)(jl + PP * q) * h] = cadd(v[q], T[(jl + PP * q) * TW + c]);
            fence_proxy_async();
            __syncthreads();
            if (tid == 0 && k + nbuf < njobs) {
                const bool nodd = (k + nbuf) & 1;
                kcol_issue(T, nodd ? &bar1 : &bar0, gt, k + nbuf, ntiles, ngroups, TW, NY, BOXR, &tmap);
                if (nodd) pend1 = true;
                else pend0 = true;
                if (k + nbuf + 1 < njobs) kcol_prefetch(gt, k + nbuf + 1, ntiles, ngroups, TW, NY, BOXR, &tmap);
            }
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) out[(size_t)(jl + PP * q) * h] = v[q];
        }
    }
}

// Derivative column groups (level 1 and level 2): up to 2 input spectra and
// 6 outputs per group, every output a sum of up to 2 terms M(k_x, k_y) X_in
// with M = i (c0 k_x + c1 k_y) + (c2 k_x^2 + c3 k_y^2 + c4 k_x k_y).  Each
// input tile takes stage 1 and stage 2 forward in place; stage 2 writes the
// spectrum X[k1 + E k2] back where it read (l -> k2), so every thread owns
// the spectrum values it needs.  Per output: the combination, the inverse
// stage 2 and the conjugate twiddles into the work tile, a block barrier,
// the inverse stage 1 and the global store, a block barrier.  The next job's
// input tiles are fetched as soon as the last output has read them.
constexpr int kMaxMGroups = 8;   // groups of one kcolm_wr launch (5 level-1 groups)

template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::TW * ColCfg<NY>::P, 1) kcolm_wr(float2 *spec,
                                                                              const GroupDesc *__restrict__ groups,
                                                                              int ngroups,
                                                                              const float *__restrict__ kxt,
                                                                              const float *__restrict__ kyt,
                                                                              const float2 *__restrict__ twc_g,
                                                                              KP<float> P, int BOXR,
                                                                              const __grid_constant__ CUtensorMap tmap,
                                                                              int *err) {
    using C = float2;
    using real = float;
    constexpr int E = ColCfg<NY>::E, PP = ColCfg<NY>::P, TW = ColCfg<NY>::TW, NT = TW * PP;
    constexpr int NQ = E / PP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0;
    __shared__ GroupDesc gs[kMaxMGroups];   // the launch's groups (ngroups <= kMaxMGroups, checked by the host)
    const int h = P.h, tid = threadIdx.x;
    const int c = tid % TW, jl = tid / TW;
    const size_t slot = (size_t)NY * h;
    constexpr int tile = TW * NY;
    SmemCursor sc{smem_raw, 0u};
    C *twc = (C *)sc.take((size_t)2 * NY * sizeof(C));   // [k1][l] (stage 1), then [l][k1] (stage 2)
    const C *twt = twc + NY;
    real *kxs = (real *)sc.take((size_t)(h + 1) * sizeof(real));
    real *kys = (real *)sc.take(NY * sizeof(real));
    C *in = (C *)sc.take((size_t)2 * tile * sizeof(C));   // input tiles 0 and 1
    C *W = (C *)sc.take((size_t)tile * sizeof(C));        // work tile
    const int ntiles = h / TW;
    const int njobs_total = P.nrun * ngroups * ntiles;
    const int njobs = (int)blockIdx.x < njobs_total ? (njobs_total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {   // (the first copies start before the tables load)
        mbar_init(&bar0, 1);
        mbar_init_fence();
        grid_dep_wait();
        if (njobs > 0) kcol_issue(in, &bar0, groups, 0, ntiles, ngroups, TW, NY, BOXR, &tmap);
        if (njobs > 1) kcol_prefetch(groups, 1, ntiles, ngroups, TW, NY, BOXR, &tmap);
    }
    load_tab4(twc, twc_g, 2 * NY, NT);
    load_tab4(kxs, kxt, h + 1, NT);
    load_tab4(kys, kyt, NY, NT);
    {
        const int nw = ngroups * (int)(sizeof(GroupDesc) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(groups);
        int *dst = reinterpret_cast<int *>(gs);
        for (int i = tid; i < nw; i += NT) dst[i] = src[i];
    }
    grid_dep_wait();
    grid_dep_launch();
    __syncthreads();
    uint32_t par0 = 0;
    bool pend0 = njobs > 0;
    const real scale = P.scale;
    for (int k = 0; k < njobs; ++k) {
        const int job = (int)blockIdx.x + k * (int)gridDim.x;
        const int run = job / (ngroups * ntiles), jr = job - run * ngroups * ntiles;
        const int g = jr / ntiles, t = jr - g * ntiles;
        const int kx0 = t * TW;
        const GroupDesc &gd = gs[g];
        if (!block_wait(&bar0, par0, err)) {
            if (pend0) mbar_wait_bounded(&bar0, par0);
            return;
        }
        par0 ^= 1;
        pend0 = false;
        const int nin = gd.nin, nout = gd.nout;
        const real ax = kxs[kx0 + c];
        // forward transforms of the inputs, in place
        for (int s = 0; s < nin; ++s) {
            C *T = in + (size_t)s * tile;
            C v[E];
#pragma unroll
            for (int q = 0; q < E; ++q) v[q] = T[(jl + PP * q) * TW + c];
            SmallDFT<E, -1, C>::run(v);
#pragma unroll
            for (int k1 = 1; k1 < E; ++k1) v[k1] = cmul(v[k1], twc[k1 * PP + jl]);
            __syncwarp();
#pragma unroll
            for (int k1 = 0; k1 < E; ++k1) T[cpos<NY>(c, jl, k1)] = v[k1];
        }
        __syncthreads();
        for (int s = 0; s < nin; ++s) {
            C *T = in + (size_t)s * tile;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int k1 = jl + PP * q;
                C u[PP];
#pragma unroll
                for (int l = 0; l < PP; ++l) u[l] = T[cpos<NY>(c, l, k1)];
                SmallDFT<PP, -1, C>::run(u);
#pragma unroll
                for (int k2 = 0; k2 < PP; ++k2) T[cpos<NY>(c, k2, k1)] = u[k2];
            }
        }
        // (each thread reads back only its own spectrum values below)
        for (int o = 0; o < nout; ++o) {
            const int two = gd.nterm[o] > 1;
            const C *X0 = in + (size_t)gd.term_in[o][0] * tile;
            const C *X1 = in + (size_t)gd.term_in[o][1] * tile;
            const real p0 = (real)gd.c[o][0][0], p1 = (real)gd.c[o][0][1], p2 = (real)gd.c[o][0][2],
                       p3 = (real)gd.c[o][0][3], p4 = (real)gd.c[o][0][4];
            const real q0 = (real)gd.c[o][1][0], q1 = (real)gd.c[o][1][1], q2 = (real)gd.c[o][1][2],
                       q3 = (real)gd.c[o][1][3], q4 = (real)gd.c[o][1][4];
            const int oslot = gd.out_slot[o];
            const bool last = o == nout - 1;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int k1 = jl + PP * q;
                C u[PP];
#pragma unroll
                for (int k2 = 0; k2 < PP; ++k2) {
                    const int pos = cpos<NY>(c, k2, k1);
                    const real ay = kys[k1 + E * k2];
                    C acc = mult_apply<real>(p0, p1, p2, p3, p4, ax, ay, X0[pos]);
                    if (two) acc = cadd(acc, mult_apply<real>(q0, q1, q2, q3, q4, ax, ay, X1[pos]));
                    u[k2] = cscale(acc, scale);
                }
                SmallDFT<PP, +1, C>::run(u);
#pragma unroll
                for (int l = 0; l < PP; ++l)
                    W[cpos<NY>(c, l, k1)] = l == 0 ? u[l] : cmul(u[l], cconj(twt[l * E + k1]));
            }
            if (last) fence_proxy_async();
            __syncthreads();
            if (last && tid == 0 && k + 1 < njobs) {   // the input tiles are free: fetch the next job's
                kcol_issue(in, &bar0, gs, k + 1, ntiles, ngroups, TW, NY, BOXR, &tmap);
                pend0 = true;
                if (k + 2 < njobs) kcol_prefetch(gs, k + 2, ntiles, ngroups, TW, NY, BOXR, &tmap);
            }
            C v[E];
#pragma unroll
            for (int k1 = 0; k1 < E; ++k1) v[k1] = W[cpos<NY>(c, jl, k1)];
            SmallDFT<E, +1, C>::run(v);
            C *out = spec + (size_t)run * NSLOT * slot + (size_t)oslot * slot + kx0 + c;
#pragma unroll
            for (int q = 0; q < E; ++q) out[(size_t)(jl + PP * q) * h] = v[q];
            __syncthreads();   // the work tile is rewritten by the next output
        }
    }
}

// shared memory of kcolm_wr<NY>
inline size_t kcolm_wr_smem(int NY, int h) {
    const int TW = col_tw_host(NY);
    const size_t tile = (size_t)TW * NY * 8;
    return smem_bytes({(size_t)2 * NY * 8, (size_t)(h + 1) * 4, (size_t)NY * 4, 2 * tile, tile});
}

// shared memory of kcol_wr<NY> with nbuf tile buffers
inline size_t kcol_wr_smem(int NY, int h, int nbuf) {
    const int TW = col_tw_host(NY);
    const size_t tile = (size_t)TW * NY * 8;
    return smem_bytes({(size_t)2 * NY * 8, (size_t)(h + 1) * 4, (size_t)NY * 4, tile, nbuf > 1 ? tile : 0});
}

// shared memory of k5_wr<H>
inline size_t k5_wr_smem(int H) {
    const int P = H == 512 ? 32 : H == 256 ? 16 : 8;
    const int NT = nt_k5wr_host(H), CH = (NT / 32) * (32 / P);
    const int NHB = NT == 512 || H < 256 ? 2 : 1;
    return smem_bytes({(size_t)H * 8, (size_t)(H / 2 + 1) * 8, (size_t)NHEAD * 2 * H * 4,
                       NHB > 1 ? (size_t)NHEAD * 2 * H * 4 : 0, (size_t)CH * 2 * H * 4, (size_t)CH * 2 * H * 4});
}

}  // namespace fftlb

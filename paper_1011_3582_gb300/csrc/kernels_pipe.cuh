// Pipelined kernels of one FFT-LB stage (arXiv:1011.3582; the stage is
// described at the top of engine_impl.cuh).  Every kernel stages its global
// inputs into shared memory with asynchronous bulk / tensor copies
// (async_copy.cuh) so that the HBM traffic of the next job overlaps the
// transforms of the current one (within a block when it holds two staging
// buffers, across the blocks of an SM when it holds one), and transforms
// out of place between the staged (unpadded) buffer and a padded work
// buffer (pp_fft).  The job lists run over the rows or column tiles of all
// runs of a batch (KP::nrun):
//   k1_pipe    persistent over rows; chunks of CH distribution rows,
//              double-buffered; moments accumulate in registers.
//   kcol_pipe  persistent over (run, group, column tile) jobs; TW-wide
//              column tiles fetched by 2-D tensor copies into one or two
//              buffers; the spectral multiply is fused with the last
//              forward pass and its adjoint (fft_device.cuh).
//   k3_pipe    one row per block: 15 derivative rows + rho, T.
//   k5_pipe    persistent over rows; the per-row head (level-2 spectra,
//              fields, aux) and CH-row chunks of convection spectra are
//              prefetched (one or two chunk buffers).
#pragma once

#include "async_copy.cuh"

// Threads per block (NT) and minimum resident blocks per SM (MINB) of the
// persistent kernels, per precision and kernel kind.  fp32 defaults
// (measured at 1024^2): the row-forward kernel runs two 256-thread blocks
// per SM (its 8-row chunks give one radix-16 butterfly per thread; 229 ->
// 171 us); the column kernels two 256-thread blocks, each with a single
// staged tile, so that one block's barrier waits and tile loads overlap the
// other's passes (convection 227 -> 212 us, level 1 144 -> 129 us against
// one double-buffered 512-thread block); the final row kernel one 512-thread
// block (its per-site epilogue needs the registers).
#ifndef FFTLB_NT32_K1
#define FFTLB_NT32_K1 256
#endif
#ifndef FFTLB_MINB32_K1
#define FFTLB_MINB32_K1 2
#endif
#ifndef FFTLB_NT32_COL
#define FFTLB_NT32_COL 256
#endif
#ifndef FFTLB_MINB32_COL
#define FFTLB_MINB32_COL 2
#endif
#ifndef FFTLB_NT32_K5
#define FFTLB_NT32_K5 512
#endif
#ifndef FFTLB_MINB32_K5
#define FFTLB_MINB32_K5 1
#endif
#ifndef FFTLB_NT64
#define FFTLB_NT64 256
#endif
#ifndef FFTLB_MINB64
#define FFTLB_MINB64 1
#endif

namespace fftlb {

// (offsets from the 1024-byte aligned dynamic base, so that the compiler
// keeps every derived pointer in the shared address space)
struct SmemCursor {
    unsigned char *base;
    unsigned off;
    __device__ __forceinline__ void *take(size_t bytes) {
        off = (off + 127u) & ~127u;
        void *p = base + off;
        off += (unsigned)bytes;
        return p;
    }
};

inline size_t smem_bytes(std::initializer_list<size_t> parts) {
    size_t s = 0;
    for (size_t b : parts) s = ((s + 127) & ~size_t(127)) + b;
    return s;
}

enum KernelShape { KS_K1 = 0, KS_COL = 1, KS_K5 = 2 };
template <typename real, int KIND> struct KCfg;
template <> struct KCfg<float, KS_K1> {
    static constexpr int NT = FFTLB_NT32_K1, MINB = FFTLB_MINB32_K1;
};
template <> struct KCfg<float, KS_COL> {
    static constexpr int NT = FFTLB_NT32_COL, MINB = FFTLB_MINB32_COL;
};
template <> struct KCfg<float, KS_K5> {
    static constexpr int NT = FFTLB_NT32_K5, MINB = FFTLB_MINB32_K5;
};
template <int KIND> struct KCfg<double, KIND> {
    static constexpr int NT = FFTLB_NT64, MINB = FFTLB_MINB64;
};

template <typename C>
__device__ __forceinline__ void load_tab(C *dst, const C *src, int n, int nthr) {
    for (int i = threadIdx.x; i < n; i += nthr) dst[i] = src[i];
}

// load_tab with four loads in flight before their stores (a store to the
// generic pointer dst would otherwise hold back the next load): for kernels
// whose prologue is on the critical path of a short launch
template <typename C>
__device__ __forceinline__ void load_tab4(C *dst, const C *__restrict__ src, int n, int nthr) {
    for (int i0 = threadIdx.x; i0 < n; i0 += 4 * nthr) {
        C v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * nthr < n) v[u] = __ldg(src + i0 + u * nthr);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * nthr < n) dst[i0 + u * nthr] = v[u];
    }
}

// i m z
template <typename real, typename C>
__device__ __forceinline__ C imul(real m, C z) { return C{-m * z.y, m * z.x}; }

// real value x of row r of a packed-complex row buffer in layout L
template <typename real>
__device__ __forceinline__ real real_at(const typename cplx_of<real>::type *buf, Lay L, int r, int x) {
    return reinterpret_cast<const real *>(buf)[2 * L(r, x >> 1) + (x & 1)];
}

// Transforms of nrows rows of A (layout la) through a work buffer of wrows
// padded rows, a chunk at a time; results always end in A.
template <int DIR, typename C>
__device__ void rows_fft_to_A(C *A, Lay la, C *wk, Lay lb, int n, int nrows, int wrows, const C *W, const C *T,
                              int nthr, int maxlr, const uint4 *tc) {
    for (int r0 = 0; r0 < nrows; r0 += wrows) {
        const int nb = min(wrows, nrows - r0);
        C *a = A + (size_t)r0 * la.bs;
        const int w = pp_fft_any<DIR, false, 0, 1>(a, la, wk, lb, n, nb, W, T, (int)threadIdx.x, nthr, maxlr, tc);
        if (w) {
            for (int i = threadIdx.x; i < nb * n; i += nthr) {
                const int r = i / n, e = i - r * n;
                a[la(r, e)] = wk[lb(r, e)];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// K1: moments + forward row transforms (persistent, double-buffered)
// ---------------------------------------------------------------------------

template <typename real>
__device__ __forceinline__ void k1_issue(const real *f, real *dst, uint64_t *bar, int j, int nchunk, int CH, int nx,
                                         int ny, size_t N) {
    const int ri = j / nchunk, c = j - ri * nchunk;
    const int yg = (int)blockIdx.x + ri * (int)gridDim.x;   // row over all runs
    const int run = yg / ny, y = yg - run * ny;
    const int i0 = c * CH, nf = min(CH, Q - i0);
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(real));
    const real *fr = f + (size_t)run * Q * N;
    mbar_expect_tx(bar, (uint32_t)nf * rowbytes);
    for (int r = 0; r < nf; ++r)
        bulk_g2s(dst + (size_t)r * nx, fr + (size_t)(i0 + r) * N + (size_t)y * nx, rowbytes, bar);
}

template <typename real, int SMAX, bool TC = false>
__global__ void __launch_bounds__(KCfg<real, KS_K1>::NT, KCfg<real, KS_K1>::MINB) k1_pipe(const real *__restrict__ f,
                                                             typename cplx_of<real>::type *spec,
                                                             real *__restrict__ fields,
                                                             const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                             const typename cplx_of<real>::type *__restrict__ Wp_g,
                                                             const typename cplx_of<real>::type *__restrict__ Tr_g,
                                                             int ntr, const real *__restrict__ kxt, KP<real> P, int CH,
                                                             int *err) {
    const uint4 *tc = TC ? P.tc16 : nullptr;   // split-BF16 tensor-core first passes
    using C = typename cplx_of<real>::type;
    constexpr int NT = KCfg<real, KS_K1>::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1;
    const int nx = P.nx, ny = P.ny, h = P.h, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    const int ph = padded_len(h);
    SmemCursor sc{smem_raw, 0u};
    C *Wr = (C *)sc.take(h * sizeof(C));
    C *Wp = (C *)sc.take(h * sizeof(C));
    C *Tr = (C *)sc.take(ntr * sizeof(C));
    real *buf0 = (real *)sc.take((size_t)CH * nx * sizeof(real));
    real *buf1 = (real *)sc.take((size_t)CH * nx * sizeof(real));
    C *wk = (C *)sc.take((size_t)CH * ph * sizeof(C));
    const Lay la{h, 1, 0}, lb{ph, 1, 1};
    const int nchunk = (Q + CH - 1) / CH;
    const int NY = P.nrun * ny;   // rows of all runs
    const int nrows = (int)blockIdx.x < NY ? (NY - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = nrows * nchunk;
    if (tid == 0) {
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init_fence();
    }
    load_tab(Wr, Wr_g, h, NT);
    load_tab(Wp, Wp_g, h, NT);
    load_tab(Tr, Tr_g, ntr, NT);
    __syncthreads();
    if (tid == 0) {
        if (njobs > 0) k1_issue(f, buf0, &bar0, 0, nchunk, CH, nx, ny, N);
        if (njobs > 1) k1_issue(f, buf1, &bar1, 1, nchunk, CH, nx, ny, N);
    }
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = njobs > 0, pend1 = njobs > 1;
    real a0[SMAX], a1[SMAX], a2[SMAX], a3[SMAX];
#pragma unroll
    for (int s = 0; s < SMAX; ++s) a0[s] = a1[s] = a2[s] = a3[s] = real(0);
    for (int j = 0; j < njobs; ++j) {
        const bool odd = j & 1;
        uint64_t *bar = odd ? &bar1 : &bar0;
        const int ri = j / nchunk, c = j - ri * nchunk;
        const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
        const int run = yg / ny, y = yg - run * ny;
        C *spec_r = spec + (size_t)run * NSLOT * slot;
        real *fields_r = fields + (size_t)run * 4 * N;
        const int i0 = c * CH, nf = min(CH, Q - i0);
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
        C *Bc = reinterpret_cast<C *>(B);
        for (int r = 0; r < nf; ++r) {
            const int i = i0 + r;
            const real vx = VX<real>(i), vy = VY<real>(i), v2 = V2<real>(i);
#pragma unroll
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x < nx) {
                    const real v = B[(size_t)r * nx + x];
                    a0[s] += v;
                    a1[s] += vx * v;
                    a2[s] += vy * v;
                    a3[s] += v2 * v;
                }
            }
        }
        __syncthreads();
        const int r0 = (i0 == 0) ? 1 : 0;   // the rest velocity is not transformed
        if (nf > r0) {
            const int w = pp_fft_any<-1, false, 0, 1>(Bc + (size_t)r0 * h, la, wk, lb, h, nf - r0, Wr, Tr, tid, NT, 4, tc);
            C *res = w ? wk : Bc + (size_t)r0 * h;
            const Lay lr = w ? lb : la;
            r2c_post_l(res, lr, h, nf - r0, Wp, tid, NT);
            __syncthreads();
            for (int r = r0; r < nf; ++r) {
                const int i = i0 + r;
                C *dst = spec_r + (size_t)(i - 1) * slot + (size_t)y * h;
                if (VY<real>(i) == real(0)) {
                    // v_y = 0: the convection term needs no column pass; its
                    // row spectrum is i v_x k_x f^ / nx (the 1 / nx the column
                    // pass would leave)
                    const real sx = VX<real>(i) * P.scale_x;
                    for (int k = tid; k < h; k += NT) dst[k] = imul(kxt[k] * sx, res[lr(r - r0, k)]);
                } else {
                    for (int k = tid; k < h; k += NT) dst[k] = res[lr(r - r0, k)];
                }
            }
        }
        if (c == nchunk - 1) {
            __syncthreads();
            // moments (Eqs. 7-9) and the level-1 fields rho, ux, uy, T, Pi, g
#pragma unroll
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x < nx) {
                    const real rho = a0[s], ux = a1[s] / rho, uy = a2[s] / rho;
                    const real T = real(0.5) * (a3[s] / rho - (ux * ux + uy * uy));
                    const size_t o = (size_t)y * nx + x;
                    fields_r[o] = rho;
                    fields_r[N + o] = ux;
                    fields_r[2 * N + o] = uy;
                    fields_r[3 * N + o] = T;
                    B[x] = rho;
                    B[nx + x] = ux;
                    B[2 * nx + x] = uy;
                    B[3 * nx + x] = T;
                    B[4 * nx + x] = rho * T / (real(1) - P.b * rho) - P.a * rho * rho - rho * T;   // Eq. 18
                    B[5 * nx + x] = (P.K + P.H * T) / T;                                          // M / T
                }
                a0[s] = a1[s] = a2[s] = a3[s] = real(0);
            }
            __syncthreads();
            const int w = pp_fft_any<-1, false, 0, 1>(Bc, la, wk, lb, h, 6, Wr, Tr, tid, NT, 4, tc);
            C *res = w ? wk : Bc;
            const Lay lr = w ? lb : la;
            r2c_post_l(res, lr, h, 6, Wp, tid, NT);
            __syncthreads();
            for (int r = 0; r < 6; ++r) {
                C *dst = spec_r + (size_t)(SLOT_RHO + r) * slot + (size_t)y * h;
                for (int k = tid; k < h; k += NT) dst[k] = res[lr(r, k)];
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && j + 2 < njobs) {
            k1_issue(f, B, bar, j + 2, nchunk, CH, nx, ny, N);
            if (odd) pend1 = true;
            else pend0 = true;
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass (persistent over (run, group, tile) jobs, one or two tile buffers)
// ---------------------------------------------------------------------------

template <typename real>
__device__ __forceinline__ typename cplx_of<real>::type mult_apply(real c0, real c1, real c2, real c3, real c4,
                                                                    real ax, real ay,
                                                                    typename cplx_of<real>::type v) {
    using C = typename cplx_of<real>::type;
    const real mr = c2 * ax * ax + c3 * ay * ay + c4 * ax * ay;
    const real mi = c0 * ax + c1 * ay;
    return C{mr * v.x - mi * v.y, mr * v.y + mi * v.x};
}

// out = scale * sum_t M_t(kx, ky) X_t over a column tile (column c of the
// tile is transform c, element e is row ky = e).  Column 0 of the tile at
// kx0 = 0 carries (DC, row-Nyquist) and is handled by (ky, -ky) pairs.
// out may alias X0 (single term, in place: every thread writes only the
// elements it read).
template <typename real>
__device__ __forceinline__ void col_multiply(typename cplx_of<real>::type *out, Lay lo,
                                             const typename cplx_of<real>::type *X0, Lay l0,
                                             const typename cplx_of<real>::type *X1, Lay l1, const GroupDesc &g,
                                             int o, const real *kxt, const real *kyt, int kx0, int TW, int lgTW,
                                             int ny, int h, real scale, int nthr) {
    using C = typename cplx_of<real>::type;
    const bool two = g.nterm[o] > 1;
    const C *t0 = g.term_in[o][0] ? X1 : X0;
    const Lay m0 = g.term_in[o][0] ? l1 : l0;
    const C *t1 = g.term_in[o][1] ? X1 : X0;
    const Lay m1 = g.term_in[o][1] ? l1 : l0;
    const real p0 = (real)g.c[o][0][0], p1 = (real)g.c[o][0][1], p2 = (real)g.c[o][0][2], p3 = (real)g.c[o][0][3],
               p4 = (real)g.c[o][0][4];
    const real q0 = (real)g.c[o][1][0], q1 = (real)g.c[o][1][1], q2 = (real)g.c[o][1][2], q3 = (real)g.c[o][1][3],
               q4 = (real)g.c[o][1][4];
    const int tile = TW * ny;
    for (int idx = threadIdx.x; idx < tile; idx += nthr) {
        const int e = idx >> lgTW, c = idx & (TW - 1);
        const int kx = kx0 + c;
        if (kx == 0) continue;
        const real ax = kxt[kx], ay = kyt[e];
        C acc = mult_apply<real>(p0, p1, p2, p3, p4, ax, ay, t0[m0(c, e)]);
        if (two) acc = cadd(acc, mult_apply<real>(q0, q1, q2, q3, q4, ax, ay, t1[m1(c, e)]));
        out[lo(c, e)] = cscale(acc, scale);
    }
    if (kx0 == 0) {
        const real a0 = kxt[0], aN = kxt[h];
        for (int j = threadIdx.x; j <= ny / 2; j += nthr) {
            const int jm = (ny - j) % ny;
            const real ay = kyt[j], aym = kyt[jm];
            C outj, outm;
            {
                const C p = t0[m0(0, j)], q = t0[m0(0, jm)];
                const C A = cscale(cadd(p, cconj(q)), real(0.5));
                const C Bv = cscale(cmul_mi(csub(p, cconj(q))), real(0.5));
                outj = cadd(mult_apply<real>(p0, p1, p2, p3, p4, a0, ay, A),
                            cmul_i(mult_apply<real>(p0, p1, p2, p3, p4, aN, ay, Bv)));
                outm = cadd(mult_apply<real>(p0, p1, p2, p3, p4, a0, aym, cconj(A)),
                            cmul_i(mult_apply<real>(p0, p1, p2, p3, p4, aN, aym, cconj(Bv))));
            }
            if (two) {
                const C p = t1[m1(0, j)], q = t1[m1(0, jm)];
                const C A = cscale(cadd(p, cconj(q)), real(0.5));
                const C Bv = cscale(cmul_mi(csub(p, cconj(q))), real(0.5));
                outj = cadd(outj, cadd(mult_apply<real>(q0, q1, q2, q3, q4, a0, ay, A),
                                       cmul_i(mult_apply<real>(q0, q1, q2, q3, q4, aN, ay, Bv))));
                outm = cadd(outm, cadd(mult_apply<real>(q0, q1, q2, q3, q4, a0, aym, cconj(A)),
                                       cmul_i(mult_apply<real>(q0, q1, q2, q3, q4, aN, aym, cconj(Bv)))));
            }
            out[lo(0, j)] = cscale(outj, scale);
            if (jm != j) out[lo(0, jm)] = cscale(outm, scale);
        }
    }
}

// job -> (run, group, tile): jobs run over the tiles of one group, then the
// groups of one run, then the runs
// the convection multiplier i (v_x k_x + v_y k_y) (general form of
// col_multiply's terms) times the inverse normalisation, for the fused pass
// of pp_conv_p2: b = column within the tile, e = k_y bin
template <typename real> struct ColMult {
    using C = typename cplx_of<real>::type;
    real c0, c1, c2, c3, c4, scale;
    const real *kxs, *kys;
    int kx0;
    __device__ __forceinline__ C operator()(int b, int e, C v) const {
        return cscale(mult_apply<real>(c0, c1, c2, c3, c4, kxs[kx0 + b], kys[e], v), scale);
    }
};

// output o of a derivative group: sum over its terms of M_term(k_x, k_y)
// times input term_in, times the inverse normalisation (the per-element
// form of col_multiply, for pp_out_fused_p2)
template <typename real> struct GroupMult {
    using C = typename cplx_of<real>::type;
    real p[5], q[5], scale;
    int two, in0, in1;
    const real *kxs, *kys;
    int kx0;
    __device__ __forceinline__ C operator()(int b, int e, C x0, C x1) const {
        const real ax = kxs[kx0 + b], ay = kys[e];
        C acc = mult_apply<real>(p[0], p[1], p[2], p[3], p[4], ax, ay, in0 ? x1 : x0);
        if (two) acc = cadd(acc, mult_apply<real>(q[0], q[1], q[2], q[3], q[4], ax, ay, in1 ? x1 : x0));
        return cscale(acc, scale);
    }
};

// Elements between consecutive staged input tiles of TW x ny values: the
// tile size rounded up to 128 bytes, the alignment a tensor copy needs for
// its shared-memory destination.
template <typename C>
__host__ __device__ __forceinline__ size_t tile_stride(int TW, int ny) {
    const size_t bytes = ((size_t)TW * ny * sizeof(C) + 127) & ~(size_t)127;
    return bytes / sizeof(C);
}

// The fields of a group that the tile copies and a one-input job read,
// staged in shared memory once per launch by the warp-resident column
// kernels (a per-job copy of the whole GroupDesc by one thread held every
// other warp of the block at the next barrier).
struct ColG {
    int nin, in_slot[2], out_slot, add_slot;
    float c0, c1;
};
constexpr int kMaxColGroups = 32;   // groups of one kcol_wr launch (32 convection groups)

// (GD: GroupDesc in global memory, or ColG / GroupDesc staged in shared memory)
template <typename C, typename GD>
__device__ __forceinline__ void kcol_issue(C *dst, uint64_t *bar, const GD *groups, int k, int ntiles,
                                           int ngroups, int TW, int ny, int BOXR, const CUtensorMap *tmap) {
    const int job = (int)blockIdx.x + k * (int)gridDim.x;
    const int run = job / (ngroups * ntiles), jr = job - run * ngroups * ntiles;
    const int g = jr / ntiles, t = jr - g * ntiles;
    const GD *G = groups + g;
    const int nin = G->nin;
    const int tile = TW * ny;
    mbar_expect_tx(bar, (uint32_t)(nin * tile * sizeof(C)));
    for (int s = 0; s < nin; ++s) {
        const int sl = run * NSLOT + G->in_slot[s];   // the tensor spans the arenas of all runs
        for (int r0 = 0; r0 < ny; r0 += BOXR)
            tma_load_2d(dst + (size_t)s * tile_stride<C>(TW, ny) + (size_t)r0 * TW, tmap, 2 * t * TW, sl * ny + r0, bar);
    }
    if (G->add_slot >= 0) {   // the addend tile, read at the job's store: into L2 now
        const int sl = run * NSLOT + G->add_slot;
        for (int r0 = 0; r0 < ny; r0 += BOXR) tma_prefetch_2d(tmap, 2 * t * TW, sl * ny + r0);
    }
}

// L2 prefetch of the tiles kcol_issue would load for job k
template <typename GD>
__device__ __forceinline__ void kcol_prefetch(const GD *groups, int k, int ntiles, int ngroups, int TW, int ny,
                                              int BOXR, const CUtensorMap *tmap) {
    const int job = (int)blockIdx.x + k * (int)gridDim.x;
    const int run = job / (ngroups * ntiles), jr = job - run * ngroups * ntiles;
    const int g = jr / ntiles, t = jr - g * ntiles;
    const GD *G = groups + g;
    for (int s = 0; s < G->nin; ++s) {
        const int sl = run * NSLOT + G->in_slot[s];
        for (int r0 = 0; r0 < ny; r0 += BOXR) tma_prefetch_2d(tmap, 2 * t * TW, sl * ny + r0);
    }
}

// MULTI = false: every group has one input and one output in place
// (convection); MULTI = true: up to 2 inputs and several outputs.
template <typename real, bool MULTI, bool TC = false>
__global__ void __launch_bounds__(KCfg<real, KS_COL>::NT, KCfg<real, KS_COL>::MINB) kcol_pipe(typename cplx_of<real>::type *spec,
                                                               const GroupDesc *__restrict__ groups, int ngroups,
                                                               const real *__restrict__ kxt,
                                                               const real *__restrict__ kyt,
                                                               const typename cplx_of<real>::type *__restrict__ Wc_g,
                                                               const typename cplx_of<real>::type *__restrict__ Tc_g,
                                                               int ntc, KP<real> P, int TW, int BOXR, int nbuf,
                                                               const __grid_constant__ CUtensorMap tmap, int *err) {
    const uint4 *tc = TC ? P.tc16 : nullptr;   // split-BF16 tensor-core first passes
    using C = typename cplx_of<real>::type;
    constexpr int NT = KCfg<real, KS_COL>::NT;
    constexpr int NIN = MULTI ? 2 : 1;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1;
    __shared__ GroupDesc gd;
    const int ny = P.ny, h = P.h, tid = threadIdx.x;
    const size_t slot = (size_t)ny * h;
    const int tile = TW * ny;
    const int ptile = TW * padded_len(ny);
    const int lgTW = ilog2(TW);   // TW is a power of two
    const bool pow2ny = is_pow2(ny);
    SmemCursor sc{smem_raw, 0u};
    C *Wc = (C *)sc.take(ny * sizeof(C));
    C *Tc = (C *)sc.take(ntc * sizeof(C));
    real *kxs = (real *)sc.take((size_t)(h + 1 + ny) * sizeof(real));   // k_x then k_y tables
    real *kys = kxs + h + 1;
    const size_t tstr = tile_stride<C>(TW, ny);   // input s of a job at buf + s tstr
    C *buf0 = (C *)sc.take((size_t)NIN * tstr * sizeof(C));
    // nbuf = 2: double-buffered (job k + 2 prefetched while job k + 1 runs);
    // nbuf = 1: one buffer (job k + 1 loaded after job k), for two blocks per SM
    C *buf1 = nbuf > 1 ? (C *)sc.take((size_t)NIN * tstr * sizeof(C)) : buf0;
    C *wk0 = (C *)sc.take((size_t)ptile * sizeof(C));
    C *wk1 = MULTI ? (C *)sc.take((size_t)ptile * sizeof(C)) : nullptr;
    const Lay lt{1, TW, 0}, lw{1, TW, 1};   // staged tile / padded work tile
    const int ntiles = h / TW;
    const int njobs_total = P.nrun * ngroups * ntiles;
    const int njobs = (int)blockIdx.x < njobs_total ? (njobs_total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init_fence();
    }
    load_tab(Wc, Wc_g, ny, NT);
    load_tab(Tc, Tc_g, ntc, NT);
    load_tab(kxs, kxt, h + 1, NT);
    load_tab(kys, kyt, ny, NT);
    __syncthreads();
    if (tid == 0) {
        if (njobs > 0) kcol_issue(buf0, &bar0, groups, 0, ntiles, ngroups, TW, ny, BOXR, &tmap);
        if (nbuf > 1 && njobs > 1) kcol_issue(buf1, &bar1, groups, 1, ntiles, ngroups, TW, ny, BOXR, &tmap);
    }
    uint32_t par0 = 0, par1 = 0;
    bool pend0 = njobs > 0, pend1 = nbuf > 1 && njobs > 1;
    const real scale = P.scale;
    for (int k = 0; k < njobs; ++k) {
        const bool odd = k & 1;
        uint64_t *bar = odd ? &bar1 : &bar0;
        const int job = (int)blockIdx.x + k * (int)gridDim.x;
        const int run = job / (ngroups * ntiles), jr = job - run * ngroups * ntiles;
        const int g = jr / ntiles, t = jr - g * ntiles;
        const int kx0 = t * TW;
        C *spec_r = spec + (size_t)run * NSLOT * slot;
        {   // the group's descriptor, one word per thread (the previous job's last
            // reads of gd came before its final block barrier; block_wait below
            // orders these writes before the first read)
            const int *src = reinterpret_cast<const int *>(groups + g);
            int *dst = reinterpret_cast<int *>(&gd);
            for (int i = tid; i < (int)(sizeof(GroupDesc) / sizeof(int)); i += NT) dst[i] = src[i];
        }
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
        C *in0 = odd ? buf1 : buf0;
        C *gout;
        if (!MULTI) {
            const C *R;
            Lay lr;
            if (pow2ny && kx0 != 0) {
                // convection, power-of-two columns: forward passes, the last
                // pass fused with the multiply and its adjoint, adjoint passes
                // (splitting the tile's columns between two named-barrier
                // halves measured slower: 228 -> 247 us at 1024^2, from the
                // bank conflicts of half-width tiles)
                const ColMult<real> m{(real)gd.c[0][0][0], (real)gd.c[0][0][1], (real)gd.c[0][0][2],
                                      (real)gd.c[0][0][3], (real)gd.c[0][0][4], scale, kxs, kys, kx0};
                const int w = pp_conv_p2<true>(in0, lt, wk0, lw, ny, TW, Tc, m, tid, NT, GroupSync{0, NT}, tc);
                R = w ? wk0 : in0;
                lr = w ? lw : lt;
            } else {
                // convection (the tile holding k_x = 0 pairs (k_y, -k_y) of the
                // packed DC / row-Nyquist column; other lengths): forward,
                // multiply in place, inverse
                const int w1 = pp_fft_any<-1, true, 0, 1>(in0, lt, wk0, lw, ny, TW, Wc, Tc, tid, NT, 4, tc);
                C *X = w1 ? wk0 : in0;
                C *Y = w1 ? in0 : wk0;
                const Lay lx = w1 ? lw : lt, ly = w1 ? lt : lw;
                col_multiply<real>(X, lx, X, lx, X, lx, gd, 0, kxs, kys, kx0, TW, lgTW, ny, h, scale, NT);
                __syncthreads();
                const int w2 = w1 ? pp_fft_any<+1, true, 1, 0>(X, lx, Y, ly, ny, TW, Wc, Tc, tid, NT, 4, tc)
                                  : pp_fft_any<+1, true, 0, 1>(X, lx, Y, ly, ny, TW, Wc, Tc, tid, NT, 4, tc);
                R = w2 ? Y : X;
                lr = w2 ? ly : lx;
            }
            gout = spec_r + (size_t)gd.out_slot[0] * slot + kx0;
            if (gd.add_slot >= 0) {   // plus the term the row kernel formed
                // (4 loads before their stores: gout may alias ad, so a load
                // after a store could not be issued ahead of it)
                const C *ad = spec_r + (size_t)gd.add_slot * slot + kx0;
                for (int i0 = tid; i0 < tile; i0 += 4 * NT) {
                    C a[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int idx = i0 + u * NT, e = idx >> lgTW, c = idx & (TW - 1);
                        if (idx < tile) a[u] = ad[(size_t)e * h + c];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int idx = i0 + u * NT, e = idx >> lgTW, c = idx & (TW - 1);
                        if (idx < tile) gout[(size_t)e * h + c] = cadd(R[lr(c, e)], a[u]);
                    }
                }
            } else {
                for (int idx = tid; idx < tile; idx += NT) {
                    const int e = idx >> lgTW, c = idx & (TW - 1);
                    gout[(size_t)e * h + c] = R[lr(c, e)];
                }
            }
        } else {
            C *in1 = in0 + tstr;
            if (pow2ny && kx0 != 0 && (ilog2(ny) & 3) != 0) {   // last pass radix <= 8
                // inputs: forward passes 1 .. L-1 (X0 in {in0, wk0}, X1 in
                // {in1, wk1}); each output: one fused pass into the free pair
                // of buffers, then the adjoint passes L-1 .. 1
                const GroupSync bs{0, NT};
                const int wx = pp_fwd_head_p2<true>(in0, lt, wk0, lw, ny, TW, Tc, tid, NT, bs, tc);
                if (gd.nin > 1) pp_fwd_head_p2<true>(in1, lt, wk1, lw, ny, TW, Tc, tid, NT, bs, tc);
                const C *X0 = wx ? wk0 : in0, *X1 = wx ? wk1 : in1;
                const Lay lx = wx ? lw : lt;
                C *Q0 = wx ? in0 : wk0, *Q1 = wx ? in1 : wk1;
                const Lay lq = wx ? lt : lw;
                for (int o = 0; o < gd.nout; ++o) {
                    GroupMult<real> m;
                    for (int j = 0; j < 5; ++j) {
                        m.p[j] = (real)gd.c[o][0][j];
                        m.q[j] = (real)gd.c[o][1][j];
                    }
                    m.scale = scale;
                    m.two = gd.nterm[o] > 1;
                    m.in0 = gd.term_in[o][0];
                    m.in1 = gd.term_in[o][1];
                    m.kxs = kxs;
                    m.kys = kys;
                    m.kx0 = kx0;
                    pp_out_fused_p2<true>(X0, X1, lx, gd.nin > 1, Q0, lq, ny, TW, Tc, m, tid, NT, bs);
                    const int wq = pp_adj_tail_p2<true>(Q0, Q1, lq, ny, TW, Tc, tid, NT, bs, tc);
                    const C *R = wq ? Q1 : Q0;
                    gout = spec_r + (size_t)gd.out_slot[o] * slot + kx0;
                    for (int idx = tid; idx < tile; idx += NT) {
                        const int e = idx >> lgTW, c = idx & (TW - 1);
                        gout[(size_t)e * h + c] = R[lq(c, e)];
                    }
                    __syncthreads();
                }
            } else {
            // X0 in {in0, wk0}, X1 in {in1, wk1}; outputs ping-pong between
            // the two buffers left free
            const int w0 = pp_fft_any<-1, true, 0, 1>(in0, lt, wk0, lw, ny, TW, Wc, Tc, tid, NT, 4, tc);
            C *X0 = w0 ? wk0 : in0;
            C *F0 = w0 ? in0 : wk0;
            const Lay lx0 = w0 ? lw : lt, lf0 = w0 ? lt : lw;
            C *X1 = in1, *F1 = wk1;
            Lay lx1 = lt, lf1 = lw;
            if (gd.nin > 1) {
                const int w1 = pp_fft_any<-1, true, 0, 1>(in1, lt, wk1, lw, ny, TW, Wc, Tc, tid, NT, 4, tc);
                X1 = w1 ? wk1 : in1;
                F1 = w1 ? in1 : wk1;
                lx1 = w1 ? lw : lt;
                lf1 = w1 ? lt : lw;
            }
            for (int o = 0; o < gd.nout; ++o) {
                col_multiply<real>(F0, lf0, X0, lx0, X1, lx1, gd, o, kxs, kys, kx0, TW, lgTW, ny, h, scale, NT);
                __syncthreads();
                int w2;
                if (lf0.pad) w2 = lf1.pad ? pp_fft_any<+1, true, 1, 1>(F0, lf0, F1, lf1, ny, TW, Wc, Tc, tid, NT, 4, tc)
                                          : pp_fft_any<+1, true, 1, 0>(F0, lf0, F1, lf1, ny, TW, Wc, Tc, tid, NT, 4, tc);
                else w2 = lf1.pad ? pp_fft_any<+1, true, 0, 1>(F0, lf0, F1, lf1, ny, TW, Wc, Tc, tid, NT, 4, tc)
                                  : pp_fft_any<+1, true, 0, 0>(F0, lf0, F1, lf1, ny, TW, Wc, Tc, tid, NT, 4, tc);
                const C *R = w2 ? F1 : F0;
                const Lay lr = w2 ? lf1 : lf0;
                gout = spec_r + (size_t)gd.out_slot[o] * slot + kx0;
                for (int idx = tid; idx < tile; idx += NT) {
                    const int e = idx >> lgTW, c = idx & (TW - 1);
                    gout[(size_t)e * h + c] = R[lr(c, e)];
                }
                __syncthreads();
            }
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && k + nbuf < njobs) {
            const bool nodd = (k + nbuf) & 1;   // the barrier of job k + nbuf
            kcol_issue(in0, nodd ? &bar1 : &bar0, groups, k + nbuf, ntiles, ngroups, TW, ny, BOXR, &tmap);
            if (nodd) pend1 = true;
            else pend0 = true;
        }
    }
}

// ---------------------------------------------------------------------------
// K3: level-1 derivatives -> Lambda, Phi, C / B numerators -> forward rows
// ---------------------------------------------------------------------------

constexpr int NT3 = 256;

// The level-1 derivatives K3 forms in the row spectrum (k3_src_slot), at
// bin k of the one-sided rows of d (row o at d + o rs; bin 0 carries DC and
// row-Nyquist, both with k_x = 0): row D_RX holds rho^, D_UXX u_x^, D_UYX
// u_y^, D_TX T^, D_PIX Pi^, D_GX g^ as loaded; D_LAP holds d_yy rho and
// D_UYY d_y u_y from the column pass.  ax = k_x of bin k, sx = 1 / nx.
template <typename real, typename C>
__device__ __forceinline__ void k3_form_x(C *d, int rs, int k, real ax, real sx) {
    const real m = ax * sx;
    const C r = d[D_RX * rs + k];
    C lap = d[D_LAP * rs + k];
    lap.x -= ax * m * r.x;
    lap.y -= ax * m * r.y;
    d[D_LAP * rs + k] = lap;                          // (d_xx + d_yy) rho
    d[D_RX * rs + k] = imul(m, r);                    // d_x rho
    const C uxx = imul(m, d[D_UXX * rs + k]);
    d[D_UXX * rs + k] = uxx;                          // d_x u_x
    d[D_DIVX * rs + k] = imul(ax, cadd(uxx, d[D_UYY * rs + k]));   // d_x (d_x u_x + d_y u_y)
    d[D_UYX * rs + k] = imul(m, d[D_UYX * rs + k]);   // d_x u_y
    d[D_TX * rs + k] = imul(m, d[D_TX * rs + k]);
    d[D_PIX * rs + k] = imul(m, d[D_PIX * rs + k]);
    d[D_GX * rs + k] = imul(m, d[D_GX * rs + k]);
}

template <typename real, bool TC = false>
__global__ void __launch_bounds__(NT3) k3_pipe(typename cplx_of<real>::type *spec, const real *__restrict__ fields,
                                               real *__restrict__ aux,
                                               const typename cplx_of<real>::type *__restrict__ Wr_g,
                                               const typename cplx_of<real>::type *__restrict__ Wp_g,
                                               const typename cplx_of<real>::type *__restrict__ Tr_g, int ntr,
                                               const real *__restrict__ kxt, KP<real> P, int WR, int maxlr,
                                               int *err) {
    const uint4 *tc = TC ? P.tc16 : nullptr;   // split-BF16 tensor-core first passes
    using C = typename cplx_of<real>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    const int nx = P.nx, ny = P.ny, h = P.h, tid = threadIdx.x;
    const int run = (int)blockIdx.x / ny, y = (int)blockIdx.x - run * ny;   // one row of one run per block
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    spec += (size_t)run * NSLOT * slot;
    fields += (size_t)run * 4 * N;
    aux += (size_t)run * 3 * N;
    const int ph = padded_len(h);
    SmemCursor sc{smem_raw, 0u};
    C *Wr = (C *)sc.take(h * sizeof(C));
    C *Wp = (C *)sc.take(h * sizeof(C));
    C *Tr = (C *)sc.take(ntr * sizeof(C));
    C *d = (C *)sc.take((size_t)ND1 * h * sizeof(C));
    C *wk = (C *)sc.take((size_t)WR * ph * sizeof(C));
    real *rT = (real *)sc.take((size_t)2 * nx * sizeof(real));
    const Lay la{h, 1, 0}, lb{ph, 1, 1};
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(real));
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();   // the barrier is initialised before any thread polls it
    if (tid == 0) {
        mbar_expect_tx(&bar, (uint32_t)(ND1 + 1) * rowbytes);   // D_DIVX is formed here
        for (int o = 0; o < ND1; ++o)
            if (k3_src_slot(o) >= 0)
                bulk_g2s(d + (size_t)o * h, spec + (size_t)k3_src_slot(o) * slot + (size_t)y * h, rowbytes, &bar);
        bulk_g2s(rT, fields + (size_t)y * nx, rowbytes, &bar);
        bulk_g2s(rT + nx, fields + 3 * N + (size_t)y * nx, rowbytes, &bar);
    }
    load_tab(Wr, Wr_g, h, NT3);
    load_tab(Wp, Wp_g, h, NT3);
    load_tab(Tr, Tr_g, ntr, NT3);
    if (!block_wait(&bar, 0, err)) {
        mbar_wait_bounded(&bar, 0);
        return;
    }
    for (int k = tid; k < h; k += NT3) k3_form_x<real>(d, h, k, kxt[k], P.scale_x);
    __syncthreads();
    c2r_pre_l(d, la, h, ND1, Wp, tid, NT3);
    __syncthreads();
    rows_fft_to_A<+1>(d, la, wk, lb, h, ND1, WR, Wr, Tr, NT3, maxlr, tc);
    const C *res = d;
    const Lay lr = la;
    real *dw = reinterpret_cast<real *>(d);
    for (int x = tid; x < nx; x += NT3) {
        const size_t s = (size_t)y * nx + x;
        const real rho = rT[x], T = rT[nx + x];
        const real rx = real_at<real>(res, lr, D_RX, x), ry = real_at<real>(res, lr, D_RY, x);
        const real lap = real_at<real>(res, lr, D_LAP, x);
        const real uxx = real_at<real>(res, lr, D_UXX, x), uxy = real_at<real>(res, lr, D_UXY, x);
        const real uyx = real_at<real>(res, lr, D_UYX, x), uyy = real_at<real>(res, lr, D_UYY, x);
        const real divx = real_at<real>(res, lr, D_DIVX, x), divy = real_at<real>(res, lr, D_DIVY, x);
        const real Tx = real_at<real>(res, lr, D_TX, x), Ty = real_at<real>(res, lr, D_TY, x);
        const real Pix = real_at<real>(res, lr, D_PIX, x), Piy = real_at<real>(res, lr, D_PIY, x);
        const real gx = real_at<real>(res, lr, D_GX, x), gy = real_at<real>(res, lr, D_GY, x);
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
        aux[s] = Cn;
        aux[N + s] = Pix - P.zeta * divx;   // Eq. 21 without d_b Lambda_ab
        aux[2 * N + s] = Piy - P.zeta * divy;
        const real q2 = real(2) * P.q * rho * T;   // Eq. 23
        // rows 0..4 of d (same site, same thread)
        dw[0 * nx + x] = Lxx;
        dw[1 * nx + x] = Lxy;
        dw[2 * nx + x] = Lyy;
        dw[3 * nx + x] = q2 * Tx;
        dw[4 * nx + x] = q2 * Ty;
    }
    __syncthreads();
    rows_fft_to_A<-1>(d, la, wk, lb, h, 5, WR, Wr, Tr, NT3, maxlr, tc);
    C *res2 = d;
    const Lay lr2 = la;
    r2c_post_l(res2, lr2, h, 5, Wp, tid, NT3);
    __syncthreads();
    for (int r = 0; r < 5; ++r) {
        C *raw = k3_raw_slot(r) >= 0 ? spec + (size_t)k3_raw_slot(r) * slot + (size_t)y * h : nullptr;
        C *mul = k3_mul_slot(r) >= 0 ? spec + (size_t)k3_mul_slot(r) * slot + (size_t)y * h : nullptr;
        for (int k = tid; k < h; k += NT3) {
            const C X = res2[lr2(r, k)];
            if (raw) raw[k] = X;
            if (mul) mul[k] = imul(kxt[k] * P.scale_x, X);   // the d_x term of level 2
        }
    }
}

// ---------------------------------------------------------------------------
// K5: convection + level-2 -> coefficients -> f^eq, I, BGK, RK combination
// ---------------------------------------------------------------------------

constexpr int CHMAX5 = 8;
constexpr int NHEAD = 10;   // dLx, dLy, dPhi spectra; rho, ux, uy, T; Cn, Bnx, Bny

template <typename real>
__device__ __forceinline__ void k5_issue_chunk(const typename cplx_of<real>::type *spec, real *dst, uint64_t *bar,
                                               int j, int nchunk, int CH, int nx, int ny, size_t slot, int h) {
    const int ri = j / nchunk, c = j - ri * nchunk;
    const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
    const int run = yg / ny, y = yg - run * ny;
    spec += (size_t)run * NSLOT * slot;
    const int v0 = c * CH, nv = min(CH, NMOV - v0);
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(real));
    mbar_expect_tx(bar, (uint32_t)nv * rowbytes);
    for (int r = 0; r < nv; ++r)
        bulk_g2s(dst + (size_t)r * nx, spec + (size_t)(v0 + r) * slot + (size_t)y * h, rowbytes, bar);
}

template <typename real>
__device__ __forceinline__ void k5_issue_head(const typename cplx_of<real>::type *spec, const real *fields,
                                              const real *aux, real *dst, uint64_t *bar, int ri, int nx, int ny,
                                              size_t N, size_t slot, int h) {
    const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
    const int run = yg / ny, y = yg - run * ny;
    spec += (size_t)run * NSLOT * slot;
    fields += (size_t)run * 4 * N;
    aux += (size_t)run * 3 * N;
    const uint32_t rowbytes = (uint32_t)(nx * sizeof(real));
    mbar_expect_tx(bar, (uint32_t)NHEAD * rowbytes);
    bulk_g2s(dst, spec + (size_t)(SLOT_L2 + 0) * slot + (size_t)y * h, rowbytes, bar);
    bulk_g2s(dst + nx, spec + (size_t)(SLOT_L2 + 2) * slot + (size_t)y * h, rowbytes, bar);
    bulk_g2s(dst + 2 * (size_t)nx, spec + (size_t)(SLOT_L2 + 3) * slot + (size_t)y * h, rowbytes, bar);
    for (int r = 0; r < 4; ++r)
        bulk_g2s(dst + (size_t)(3 + r) * nx, fields + (size_t)r * N + (size_t)y * nx, rowbytes, bar);
    for (int r = 0; r < 3; ++r)
        bulk_g2s(dst + (size_t)(7 + r) * nx, aux + (size_t)r * N + (size_t)y * nx, rowbytes, bar);
}

// cos(r pi / 4) a + sin(r pi / 4) b for direction r of a ring of Eq. 1 (r a
// compile-time constant after unrolling)
template <typename real>
__device__ __forceinline__ real dir_dot(int r, real a, real b) {
    const real h = real(0.70710678118654752440);
    switch (r & 7) {
        case 0: return a;
        case 1: return h * (a + b);
        case 2: return b;
        case 3: return h * (b - a);
        case 4: return -a;
        case 5: return -h * (a + b);
        case 6: return -b;
        default: return h * (a - b);
    }
}

// NHB head buffers (1 or 2): the head of row ri lives in buffer ri % NHB and
// is prefetched NHB rows ahead.
template <typename real, int SMAX, bool TC = false>
__global__ void __launch_bounds__(KCfg<real, KS_K5>::NT, KCfg<real, KS_K5>::MINB) k5_pipe(const typename cplx_of<real>::type *spec,
                                                             const real *__restrict__ fields,
                                                             const real *__restrict__ aux, const real *fcur,
                                                             const real *fbase, real *fout, real alpha, real beta,
                                                             const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                             const typename cplx_of<real>::type *__restrict__ Wp_g,
                                                             const typename cplx_of<real>::type *__restrict__ Tr_g,
                                                             int ntr, KP<real> P, int CH, int NHB, int nbuf, int maxlr,
                                                             int *err) {
    const uint4 *tc = TC ? P.tc16 : nullptr;   // split-BF16 tensor-core first passes
    using C = typename cplx_of<real>::type;
    constexpr int NT = KCfg<real, KS_K5>::NT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar0, bar1, hbar0, hbar1;
    const int nx = P.nx, ny = P.ny, h = P.h, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    const int ph = padded_len(h);
    SmemCursor sc{smem_raw, 0u};
    C *Wr = (C *)sc.take(h * sizeof(C));
    C *Wp = (C *)sc.take(h * sizeof(C));
    C *Tr = (C *)sc.take(ntr * sizeof(C));
    real *head0 = (real *)sc.take((size_t)NHEAD * nx * sizeof(real));
    real *head1 = NHB > 1 ? (real *)sc.take((size_t)NHEAD * nx * sizeof(real)) : head0;
    real *buf0 = (real *)sc.take((size_t)CH * nx * sizeof(real));
    // nbuf = 2: chunk j + 2 prefetched while chunk j + 1 runs; nbuf = 1: one
    // chunk buffer, for two blocks per SM
    real *buf1 = nbuf > 1 ? (real *)sc.take((size_t)CH * nx * sizeof(real)) : buf0;
    C *wk = (C *)sc.take((size_t)max(CH, 3) * ph * sizeof(C));
    const Lay la{h, 1, 0}, lb{ph, 1, 1};
    const int nchunk = (NMOV + CH - 1) / CH;
    const int NY = P.nrun * ny;   // rows of all runs
    const int nrows = (int)blockIdx.x < NY ? (NY - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = nrows * nchunk;
    if (tid == 0) {
        mbar_init(&bar0, 1);
        mbar_init(&bar1, 1);
        mbar_init(&hbar0, 1);
        mbar_init(&hbar1, 1);
        mbar_init_fence();
    }
    load_tab(Wr, Wr_g, h, NT);
    load_tab(Wp, Wp_g, h, NT);
    load_tab(Tr, Tr_g, ntr, NT);
    __syncthreads();
    if (tid == 0) {
        if (nrows > 0) k5_issue_head<real>(spec, fields, aux, head0, &hbar0, 0, nx, ny, N, slot, h);
        if (NHB > 1 && nrows > 1) k5_issue_head<real>(spec, fields, aux, head1, &hbar1, 1, nx, ny, N, slot, h);
        if (njobs > 0) k5_issue_chunk<real>(spec, buf0, &bar0, 0, nchunk, CH, nx, ny, slot, h);
        if (nbuf > 1 && njobs > 1) k5_issue_chunk<real>(spec, buf1, &bar1, 1, nchunk, CH, nx, ny, slot, h);
    }
    uint32_t par0 = 0, par1 = 0, hpar0 = 0, hpar1 = 0;
    bool pend0 = njobs > 0, pend1 = nbuf > 1 && njobs > 1, hpend0 = nrows > 0, hpend1 = NHB > 1 && nrows > 1;
    const real dt = P.dt, itau = real(1) / P.tau;
    const bool with_base = alpha != real(0);
    for (int j = 0; j < njobs; ++j) {
        const bool odd = j & 1;
        const int ri = j / nchunk, c = j - ri * nchunk;
        const bool hodd = (NHB > 1) && (ri & 1);
        const int yg = (int)blockIdx.x + ri * (int)gridDim.x;
        const int run = yg / ny, y = yg - run * ny;
        const size_t fo = (size_t)run * Q * N;   // this run's distributions
        const int v0 = c * CH, nv = min(CH, NMOV - v0);
        real *H = hodd ? head1 : head0;
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
            C *l2 = reinterpret_cast<C *>(H);
            c2r_pre_l(l2, la, h, 3, Wp, tid, NT);
            __syncthreads();
            const int w = pp_fft_any<+1, false, 0, 1>(l2, la, wk, lb, h, 3, Wr, Tr, tid, NT, maxlr, tc);
            const C *lres = w ? wk : l2;
            const Lay llr = w ? lb : la;
            // per-site coefficients, written over the head rows (same site,
            // same thread): row 0 <- e0, 1 <- e1x, 2 <- e1y, 7 <- C + C_q,
            // 8 <- 1 / T
#pragma unroll 1
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x < nx) {
                    const real rho = H[3 * nx + x], ux = H[4 * nx + x], uy = H[5 * nx + x], T = H[6 * nx + x];
                    const real dLx = real_at<real>(lres, llr, 0, x), dLy = real_at<real>(lres, llr, 1, x);
                    const real dPh = real_at<real>(lres, llr, 2, x);
                    const real rT = rho * T;
                    const real inv2 = real(1) / (real(2) * rho * T * T);
                    const real Bx = (H[8 * nx + x] + dLx) / rT;      // Eq. 21
                    const real By = (H[9 * nx + x] + dLy) / rT;
                    const real CC = (H[7 * nx + x] + dPh) * inv2;    // C + C_q, Eqs. 22-23
                    const real A = real(-2) * CC * T;                // Eq. 20
                    const real u2 = ux * ux + uy * uy;
                    // I = -(A + B.(v-u) + CC |v-u|^2) f^eq = -(e0 + e1.v + CC |v|^2) f^eq
                    const real e0 = A - (Bx * ux + By * uy) + CC * u2;
                    H[x] = e0;
                    H[nx + x] = Bx - real(2) * CC * ux;
                    H[2 * nx + x] = By - real(2) * CC * uy;
                    H[7 * nx + x] = CC;
                    H[8 * nx + x] = real(1) / T;
                    // rest velocity (no convection)
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
        C *Bc = reinterpret_cast<C *>(B);
        c2r_pre_l(Bc, la, h, nv, Wp, tid, NT);
        __syncthreads();
        const int w = pp_fft_any<+1, false, 0, 1>(Bc, la, wk, lb, h, nv, Wr, Tr, tid, NT, maxlr, tc);
        const C *cres = w ? wk : Bc;
        const Lay lcr = w ? lb : la;
        if (CH == 8) {
            // the chunk is ring c + 1 (velocities 1 + 8c .. 8 + 8c, Eq. 1):
            // one speed, one weight F_k, and directions known at compile time
            const int k = c;
            const real sk = VX<real>(1 + v0), sk2 = V2<real>(1 + v0);   // direction 0: v = (s_k, 0)
#pragma unroll 1
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
                const real rho = H[3 * nx + x], ux = H[4 * nx + x], uy = H[5 * nx + x], T = H[6 * nx + x];
                const real iT = H[8 * nx + x];
                const real e0 = H[x], e1x = H[nx + x], e1y = H[2 * nx + x], CC = H[7 * nx + x];
                const real Fk = weight_Fk<real>(k, T);   // Eq. 4
                const real qq = real(0.5) * (ux * ux + uy * uy) * iT, om = real(1) - qq;
                const real p0 = om + real(0.5) * qq * qq, p1 = om * iT, p2 = real(0.5) * om * iT * iT;
                const real p3 = iT * iT * iT * (real(1) / real(6)), p4 = iT * iT * iT * iT * (real(1) / real(24));
                const real rF = rho * Fk;
                const real g0 = e0 + CC * sk2;   // e0 + CC |v|^2 on the ring
                const real uxk = sk * ux, uyk = sk * uy, exk = sk * e1x, eyk = sk * e1y;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const real vu = dir_dot<real>(r, uxk, uyk);
                    const real br = p0 + vu * (p1 + vu * (p2 + vu * (p3 + vu * p4)));
                    const real fe = rF * br;                                                 // Eq. 3
                    const real I = -(g0 + dir_dot<real>(r, exk, eyk)) * fe;                   // Eq. 11
                    const real conv = real_at<real>(cres, lcr, r, x);
                    const real rhs = -conv - (fc[r] - fe) * itau + I;                        // Eq. 10
                    real fn = beta * (fc[r] + dt * rhs);
                    if (with_base) fn += alpha * fb[r];
                    po[r * N] = fn;
                }
            }
        } else {
#pragma unroll 1
            for (int s = 0; s < SMAX; ++s) {
                const int x = tid + s * NT;
                if (x >= nx) continue;
                real fc[CHMAX5], fb[CHMAX5];
                const size_t o0 = fo + (size_t)(1 + v0) * N + (size_t)y * nx + x;
                const real *pc = fcur + o0;
                const real *pb = fbase + o0;
#pragma unroll
                for (int r = 0; r < CHMAX5; ++r) {
                    if (r < nv) {
                        fc[r] = pc[r * N];
                        fb[r] = with_base ? pb[r * N] : real(0);
                    }
                }
                real *po = fout + o0;
                const real rho = H[3 * nx + x], ux = H[4 * nx + x], uy = H[5 * nx + x], T = H[6 * nx + x];
                const real e0 = H[x], e1x = H[nx + x], e1y = H[2 * nx + x], CC = H[7 * nx + x];
                real F[5];
                weights_Fk<real>(T, F);                                  // Eqs. 4-6
                const real iT = H[8 * nx + x], qq = real(0.5) * (ux * ux + uy * uy) * iT, om = real(1) - qq;
                const real p0 = om + real(0.5) * qq * qq, p1 = om * iT, p2 = real(0.5) * om * iT * iT;
                const real p3 = iT * iT * iT * (real(1) / real(6)), p4 = iT * iT * iT * iT * (real(1) / real(24));
#pragma unroll
                for (int r = 0; r < CHMAX5; ++r) {
                    if (r < nv) {
                        const int i = 1 + v0 + r;
                        const real vx = VX<real>(i), vy = VY<real>(i), v2 = V2<real>(i);
                        const int k = c_ring[i];
                        const real vu = vx * ux + vy * uy;
                        const real br = p0 + vu * (p1 + vu * (p2 + vu * (p3 + vu * p4)));
                        real rF = F[1];
                        rF = (k == 2) ? F[2] : rF;
                        rF = (k == 3) ? F[3] : rF;
                        rF = (k == 4) ? F[4] : rF;
                        const real fe = rho * rF * br;                                          // Eq. 3
                        const real I = -(e0 + e1x * vx + e1y * vy + CC * v2) * fe;              // Eq. 11
                        const real conv = real_at<real>(cres, lcr, r, x);
                        const real rhs = -conv - (fc[r] - fe) * itau + I;                       // Eq. 10
                        real fn = beta * (fc[r] + dt * rhs);
                        if (with_base) fn += alpha * fb[r];
                        po[r * N] = fn;
                    }
                }
            }
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            if (j + nbuf < njobs) {
                const bool nodd = (j + nbuf) & 1;   // the barrier of chunk j + nbuf
                k5_issue_chunk<real>(spec, B, nodd ? &bar1 : &bar0, j + nbuf, nchunk, CH, nx, ny, slot, h);
                if (nodd) pend1 = true;
                else pend0 = true;
            }
            // the row's head buffer is free after its last chunk: prefetch
            // the head of row ri + NHB into it
            if (c == nchunk - 1 && ri + NHB < nrows) {
                k5_issue_head<real>(spec, fields, aux, H, hodd ? &hbar1 : &hbar0, ri + NHB, nx, ny, N, slot, h);
                if (hodd) hpend1 = true;
                else hpend0 = true;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Spectral gradient of caller fields (fftlb_gradient) through the stage's
// transform code: pp_fft_any (shift-based passes for power-of-two lengths,
// radix 16 first) and, when TC is set, the split-BF16 tensor-core first
// pass of every row and column transform.  One row or one column tile per
// block; not pipelined (the gradient is not on the stepping path).
// ---------------------------------------------------------------------------

// forward rows of nf real fields [nf][ny][nx] into slots slot0 + fi
template <typename real, bool TC = false>
__global__ void __launch_bounds__(NT3) k_grad_rows_fwd(const double *__restrict__ in,
                                                       typename cplx_of<real>::type *spec, int slot0,
                                                       const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                       const typename cplx_of<real>::type *__restrict__ Wp_g,
                                                       const typename cplx_of<real>::type *__restrict__ Tr_g, int ntr,
                                                       KP<real> P) {
    using C = typename cplx_of<real>::type;
    const uint4 *tc = TC ? P.tc16 : nullptr;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, fi = blockIdx.y, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    SmemCursor sc{smem_raw, 0u};
    C *Wr = (C *)sc.take(h * sizeof(C));
    C *Wp = (C *)sc.take(h * sizeof(C));
    C *Tr = (C *)sc.take(ntr * sizeof(C));
    C *buf = (C *)sc.take(h * sizeof(C));
    C *wk = (C *)sc.take(padded_len(h) * sizeof(C));
    const Lay la{h, 1, 0}, lb{padded_len(h), 1, 1};
    load_tab(Wr, Wr_g, h, NT3);
    load_tab(Wp, Wp_g, h, NT3);
    load_tab(Tr, Tr_g, ntr, NT3);
    real *bre = reinterpret_cast<real *>(buf);
    for (int x = tid; x < nx; x += NT3) bre[x] = (real)in[(size_t)fi * N + (size_t)y * nx + x];
    __syncthreads();
    const int w = pp_fft_any<-1, false, 0, 1>(buf, la, wk, lb, h, 1, Wr, Tr, tid, NT3, 4, tc);
    C *res = w ? wk : buf;
    const Lay lr = w ? lb : la;
    r2c_post_l(res, lr, h, 1, Wp, tid, NT3);
    __syncthreads();
    C *dst = spec + (size_t)(slot0 + fi) * slot + (size_t)y * h;
    for (int k = tid; k < h; k += NT3) dst[k] = res[lr(0, k)];
}

// column tile blockIdx.x of group blockIdx.y (one input): forward, then per
// output the multiplier into a free buffer and the inverse
template <typename real, bool TC = false>
__global__ void __launch_bounds__(NT3) k_grad_col(typename cplx_of<real>::type *spec,
                                                  const GroupDesc *__restrict__ groups,
                                                  const real *__restrict__ kxt, const real *__restrict__ kyt,
                                                  const typename cplx_of<real>::type *__restrict__ Wc_g,
                                                  const typename cplx_of<real>::type *__restrict__ Tc_g, int ntc,
                                                  KP<real> P, int TW) {
    using C = typename cplx_of<real>::type;
    const uint4 *tc = TC ? P.tc16 : nullptr;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ GroupDesc gd;
    const int ny = P.ny, h = P.h, tid = threadIdx.x;
    const size_t slot = (size_t)ny * h;
    const int kx0 = blockIdx.x * TW, lgTW = ilog2(TW);
    const int pny = padded_len(ny);
    SmemCursor sc{smem_raw, 0u};
    C *Wc = (C *)sc.take(ny * sizeof(C));
    C *Tc = (C *)sc.take(ntc * sizeof(C));
    C *A = (C *)sc.take((size_t)TW * ny * sizeof(C));     // unpadded [c][ny]
    C *B = (C *)sc.take((size_t)TW * pny * sizeof(C));    // padded
    C *D = (C *)sc.take((size_t)TW * pny * sizeof(C));    // padded
    const Lay la{ny, 1, 0}, lb{pny, 1, 1};
    if (tid == 0) gd = groups[blockIdx.y];
    load_tab(Wc, Wc_g, ny, NT3);
    load_tab(Tc, Tc_g, ntc, NT3);
    __syncthreads();
    const C *src = spec + (size_t)gd.in_slot[0] * slot;
    for (int idx = tid; idx < TW * ny; idx += NT3) {
        const int c = idx & (TW - 1), e = idx >> lgTW;
        A[la(c, e)] = src[(size_t)e * h + kx0 + c];
    }
    __syncthreads();
    const int w = pp_fft_any<-1, false, 0, 1>(A, la, B, lb, ny, TW, Wc, Tc, tid, NT3, 4, tc);
    C *X = w ? B : A;
    const Lay lx = w ? lb : la;
    for (int o = 0; o < gd.nout; ++o) {
        C *F = w ? A : B;   // the buffer X does not use
        const Lay lf = w ? la : lb;
        col_multiply<real>(F, lf, X, lx, X, lx, gd, o, kxt, kyt, kx0, TW, lgTW, ny, h, P.scale, NT3);
        __syncthreads();
        const int w2 = lf.pad ? pp_fft_any<+1, false, 1, 1>(F, lf, D, lb, ny, TW, Wc, Tc, tid, NT3, 4, tc)
                              : pp_fft_any<+1, false, 0, 1>(F, lf, D, lb, ny, TW, Wc, Tc, tid, NT3, 4, tc);
        const C *R = w2 ? D : F;
        const Lay lr = w2 ? lb : lf;
        C *dst = spec + (size_t)gd.out_slot[o] * slot;
        for (int idx = tid; idx < TW * ny; idx += NT3) {
            const int c = idx & (TW - 1), e = idx >> lgTW;
            dst[(size_t)e * h + kx0 + c] = R[lr(c, e)];
        }
        __syncthreads();
    }
}

// inverse rows of slots slot0 + fi into real fields out[fi][ny][nx]
template <typename real, bool TC = false>
__global__ void __launch_bounds__(NT3) k_grad_rows_inv(const typename cplx_of<real>::type *spec, int slot0,
                                                       double *__restrict__ out,
                                                       const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                       const typename cplx_of<real>::type *__restrict__ Wp_g,
                                                       const typename cplx_of<real>::type *__restrict__ Tr_g, int ntr,
                                                       KP<real> P) {
    using C = typename cplx_of<real>::type;
    const uint4 *tc = TC ? P.tc16 : nullptr;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, fi = blockIdx.y, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    SmemCursor sc{smem_raw, 0u};
    C *Wr = (C *)sc.take(h * sizeof(C));
    C *Wp = (C *)sc.take(h * sizeof(C));
    C *Tr = (C *)sc.take(ntr * sizeof(C));
    C *buf = (C *)sc.take(h * sizeof(C));
    C *wk = (C *)sc.take(padded_len(h) * sizeof(C));
    const Lay la{h, 1, 0}, lb{padded_len(h), 1, 1};
    load_tab(Wr, Wr_g, h, NT3);
    load_tab(Wp, Wp_g, h, NT3);
    load_tab(Tr, Tr_g, ntr, NT3);
    const C *src = spec + (size_t)(slot0 + fi) * slot + (size_t)y * h;
    for (int k = tid; k < h; k += NT3) buf[k] = src[k];
    __syncthreads();
    c2r_pre_l(buf, la, h, 1, Wp, tid, NT3);
    __syncthreads();
    const int w = pp_fft_any<+1, false, 0, 1>(buf, la, wk, lb, h, 1, Wr, Tr, tid, NT3, 4, tc);
    const C *res = w ? wk : buf;
    const Lay lr = w ? lb : la;
    for (int x = tid; x < nx; x += NT3) out[(size_t)fi * N + (size_t)y * nx + x] = (double)real_at<real>(res, lr, 0, x);
}

// A wait that nothing completes, for testing the bounded-wait error path:
// every block initialises an mbarrier that expects one arrival, which never
// comes, and waits on it for at most limit_ns.  The wait runs out,
// block_wait records kErrWaitTimeout in the device error word and the block
// returns.  No copy is issued, so nothing is in flight when it returns.
static __global__ void k_wait_selftest(int *err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    block_wait(&bar, 0, err, limit_ns);
}

}  // namespace fftlb

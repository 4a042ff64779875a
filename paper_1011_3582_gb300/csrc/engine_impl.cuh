// Templated engine of the FFT-LB method (arXiv:1011.3582): device kernels
// and the per-precision plan.  Included by engine_f64.cu and engine_f32.cu
// only (each instantiates one precision).
//
// One Runge-Kutta stage L(f) (Eq. 10) runs as six launches of the
// pipelined kernels of kernels_pipe.cuh on the handle's stream (profile
// names in parentheses):
//   k1_pipe (row_forward_moments)  moments rho, u, T (Eqs. 7-9) of the stage
//                           state, level-1 fields Pi = P^w - rho T (Eq. 18)
//                           and g = M/T; forward row transforms of the 32
//                           moving f_i and of rho, u_x, u_y, T, Pi, g
//   kcol_pipe (col_convection)  column forward -> i (v_x k_m,x + v_y k_m,y)
//                           -> column inverse for the 32 f_i (in place)
//   kcol_pipe (col_level1)  the 8 level-1 derivative spectra that involve
//                           k_y (d_y of rho, u, T, Pi, g; d_yy rho;
//                           d_y div u)
//   k3_pipe (row_level1)    the 7 derivatives in k_x alone, formed in the
//                           row spectrum (k3_form_x); row inverse of the
//                           15; Lambda (Eq. 19), Phi = 2 q rho T grad T
//                           (Eq. 23), the numerators of C (Eq. 22) and B
//                           (Eq. 21); forward row transforms of Lambda_xx,
//                           Lambda_xy, Lambda_yy, Phi_x, Phi_y, with the
//                           d_x terms of level 2 formed in the row spectrum
//   kcol_pipe (col_level2)  d_b Lambda_xb, d_b Lambda_yb, d_a Phi_a: the
//                           column pass of the d_y terms plus the d_x terms
//   k5_pipe (row_final)     row inverse of the convection terms and level-2
//                           divergences; A, B, C, C_q (Eqs. 20-23), f^eq
//                           (Eq. 3), I (Eq. 11), BGK and the RK combination.
// This file holds the engine (plan, tables, launches) and the auxiliary
// kernels of the per-run calls: equilibrium initialisation, moments,
// conversions, and the gradient / invariant transforms.
//
// Spectra are stored one-sided: slot s holds [ny][nx/2] complex values of
// a row-transformed (and later column-transformed) field, with the real
// row-Nyquist value packed into the imaginary part of column 0.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"
#include "fft_device.cuh"

namespace fftlb {

constexpr int Q = 33;
constexpr int NMOV = 32;
constexpr int NT = 256;          // threads per block of every row / column kernel

// spectrum slots
constexpr int SLOT_RHO = 32, SLOT_UX = 33, SLOT_UY = 34, SLOT_T = 35, SLOT_PI = 36, SLOT_G = 37;
constexpr int SLOT_D1 = 38;      // 15 level-1 derivative outputs
constexpr int ND1 = 15;
constexpr int SLOT_L2 = 53;      // Lxx, Lxy, Lyy, Phx, Phy; outputs in 53, 55, 56
constexpr int NSLOT = 58;
enum { D_RX, D_RY, D_LAP, D_UXX, D_UXY, D_UYX, D_UYY, D_DIVX, D_DIVY, D_TX, D_TY, D_PIX, D_PIY, D_GX, D_GY };

// The windowed derivative multipliers are separable: D_x = i k_x (a
// function of k_x alone), D_y = i k_y, and the second derivatives are their
// products (Eqs. K1-K4 with the real part taken after each derivative, so
// that the Nyquist bins carry zero).  A derivative whose multiplier depends
// on k_x alone needs no column transform: in the row-transformed slot it is
// the pointwise product i k_x X / nx (the 1 / nx that the column pass would
// leave).  So the level-1 column pass forms only the outputs that involve
// k_y, 8 of the 15 (d_y of rho, u_x, u_y, T, Pi, g; d_yy rho;
// d_xy u_x + d_yy u_y), and the row kernel K3 forms the other 7 from the
// row spectra of rho, u_x, u_y, T, Pi, g before its inverse rows:
//   rho_x = i k_x rho^ / nx, lap rho = d_yy rho - k_x^2 rho^ / nx,
//   u_xx = i k_x u_x^ / nx, u_yx = i k_x u_y^ / nx,
//   d_x(div u) = i k_x (u_xx + u_yy), T_x, Pi_x, g_x = i k_x (.)^ / nx.
// Level 2 in the same way: d_x Lambda_xx + d_y Lambda_xy is the column
// pass of d_y Lambda_xy plus i k_x Lambda_xx^ / nx, formed by K3 (add_slot).
// k3_src_slot(o): the slot K3 loads into its row o (-1: formed in K3).
__host__ __device__ constexpr int k3_src_slot(int o) {
    return o == D_RX ? SLOT_RHO : o == D_UXX ? SLOT_UX : o == D_UYX ? SLOT_UY : o == D_TX ? SLOT_T
         : o == D_PIX ? SLOT_PI : o == D_GX ? SLOT_G : o == D_DIVX ? -1 : SLOT_D1 + o;
}
// K3's level-2 outputs: row r of Lambda_xx, Lambda_xy, Lambda_yy, Phi_x,
// Phi_y goes to slot k3_raw_slot(r) as it is and to slot k3_mul_slot(r)
// times i k_x / nx (-1: not written)
__host__ __device__ constexpr int k3_raw_slot(int r) {
    return r == 1 ? SLOT_L2 + 1 : r == 2 ? SLOT_L2 + 2 : r == 4 ? SLOT_L2 + 4 : -1;
}
__host__ __device__ constexpr int k3_mul_slot(int r) {
    return r == 0 ? SLOT_L2 + 0 : r == 1 ? SLOT_D1 + D_DIVX : r == 3 ? SLOT_L2 + 3 : -1;
}

// velocity set (Eq. 1) and weight-polynomial coefficients (Eq. 4); each
// translation unit holds its own copy, shared by all live engines of that
// unit, which must therefore use one velocity set (vs_owner below)
static __constant__ double c_vx[Q], c_vy[Q], c_v2[Q];
static __constant__ float c_vxf[Q], c_vyf[Q], c_v2f[Q];
static __constant__ int c_ring[Q];
static __constant__ double c_Fk[4][4];    // F_k = T (c3 + T (c2 + T (c1 + T c0)))
static __constant__ float c_Fkf[4][4];
static __constant__ float c_Fkl[4][4];    // fp32 remainders: c_Fk - c_Fkf

// the live engines of this translation unit and their velocity set
struct VelocitySetOwner {
    std::mutex mu;
    int live = 0;
    double speeds[4] = {0, 0, 0, 0};
};
static VelocitySetOwner vs_owner;

template <typename real> __device__ __forceinline__ real VX(int i);
template <> __device__ __forceinline__ double VX<double>(int i) { return c_vx[i]; }
template <> __device__ __forceinline__ float VX<float>(int i) { return c_vxf[i]; }
template <typename real> __device__ __forceinline__ real VY(int i);
template <> __device__ __forceinline__ double VY<double>(int i) { return c_vy[i]; }
template <> __device__ __forceinline__ float VY<float>(int i) { return c_vyf[i]; }
template <typename real> __device__ __forceinline__ real V2(int i);
template <> __device__ __forceinline__ double V2<double>(int i) { return c_v2[i]; }
template <> __device__ __forceinline__ float V2<float>(int i) { return c_v2f[i]; }
template <typename real> __device__ __forceinline__ real FKC(int k, int j);
template <> __device__ __forceinline__ double FKC<double>(int k, int j) { return c_Fk[k][j]; }
template <> __device__ __forceinline__ float FKC<float>(int k, int j) { return c_Fkf[k][j]; }

// nrun: independent runs of this grid stored back to back (f [run][33][ny][nx],
// spectra [run][58][ny][nx/2], fields [run][4][ny][nx], aux [run][3][ny][nx]);
// the pipelined kernels treat the nrun * ny rows (or column tiles) of all
// runs as one job list
// tc16: the A fragments of the split-BF16 tensor-core first pass
// (tc_dft16_pass), or nullptr for the plain radix-16 first pass
template <typename real> struct KP {
    int nx, ny, h, nrun;
    real dx, dt, tau, a, b, K, H, q, zeta, scale;
    real scale_x;   // 1 / nx: the inverse normalisation a column pass leaves to the rows (scale * ny)
    const uint4 *tc16;
};

// One column-pass group: up to 2 input spectra and 6 outputs; every output
// is a sum of up to 2 terms M(kx, ky) * input, with
// M = i (c0 k_x + c1 k_y) + (c2 k_x^2 + c3 k_y^2 + c4 k_x k_y).
// add_slot >= 0 (groups of one input and one output, the convection kernels
// only): the column inverse of that output is added to slot add_slot's
// values at the same positions (a term that needs no column transform,
// formed by the row kernel that wrote add_slot).
struct GroupDesc {
    int nin, nout;
    int in_slot[2];
    int out_slot[6];
    int nterm[6];
    int term_in[6][2];
    double c[6][2][5];
    int add_slot;
};

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------

template <int DIR, typename C>
__device__ void fft_rows(C *buf, int n, int nrows, const C *W) {
    const int maxb = max(1, (16 * NT) / n);
    for (int r0 = 0; r0 < nrows; r0 += maxb) {
        block_fft<DIR>(buf + (size_t)r0 * n, n, min(maxb, nrows - r0), W, threadIdx.x, NT);
    }
}

template <typename C>
__device__ __forceinline__ void load_tables(C *dst, const C *src, int n) {
    for (int i = threadIdx.x; i < n; i += NT) dst[i] = src[i];
}

// Forward real rows -> packed one-sided spectra, in place in shared memory.
template <typename C>
__device__ void rows_r2c(C *buf, int h, int nrows, const C *Wr, const C *Wp) {
    __syncthreads();
    fft_rows<-1>(buf, h, nrows, Wr);
    r2c_post(buf, h, nrows, Wp, threadIdx.x, NT);
    __syncthreads();
}

// Packed one-sided spectra -> real rows (unnormalised), in place.
template <typename C>
__device__ void rows_c2r(C *buf, int h, int nrows, const C *Wr, const C *Wp) {
    __syncthreads();
    c2r_pre(buf, h, nrows, Wp, threadIdx.x, NT);
    __syncthreads();
    fft_rows<+1>(buf, h, nrows, Wr);
}

// Weight F_k(T) of ring k (Eq. 4) as T (c3 + T (c2 + T (c1 + T c0))).  fp64:
// Horner.  fp32: the compensated Horner scheme of Graillat, Langlois and
// Louvet (2005), with the coefficients as fp32 pairs hi + lo: every step's
// rounding errors (TwoProd through fma, TwoSum) are carried in a second
// accumulator and added at the end, so the result is accurate to about one
// ulp even where the polynomial cancels (F_4 near T = 0.43 has condition
// number 1.6e4).  Plain fp32 Horner there is off by up to 4e-3 relative, an
// error of fixed sign at a fixed T that the BGK term feeds into f every
// step: a steady drift of mass and energy in long fp32 runs.
template <typename real> __device__ __forceinline__ real weight_Fk(int k, real T);
template <> __device__ __forceinline__ double weight_Fk<double>(int k, double T) {
    return T * (c_Fk[k][3] + T * (c_Fk[k][2] + T * (c_Fk[k][1] + T * c_Fk[k][0])));
}
// (the error-free transformations use __fmul_rn / __fadd_rn / __fsub_rn,
// which the compiler never contracts into an fma)
template <> __device__ __forceinline__ float weight_Fk<float>(int k, float T) {
    float s = c_Fkf[k][0], c = c_Fkl[k][0];
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        const float p = __fmul_rn(s, T), pe = fmaf(s, T, -p);     // TwoProd(s, T)
        const float a = c_Fkf[k][j];
        const float sn = __fadd_rn(p, a), z = __fsub_rn(sn, p);   // TwoSum(p, a)
        const float se = __fadd_rn(__fsub_rn(p, __fsub_rn(sn, z)), __fsub_rn(a, z));
        c = fmaf(c, T, pe + se + c_Fkl[k][j]);
        s = sn;
    }
    return T * (s + c);
}

template <typename real>
__device__ __forceinline__ void weights_Fk(real T, real F[5]) {
    real s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const real v = weight_Fk<real>(k, T);
        F[k + 1] = v;
        s += v;
    }
    F[0] = real(1) - real(8) * s;
}

// ---------------------------------------------------------------------------
// column pass for the gradient and the invariants (one tile per block):
// forward -> multiplier -> inverse
// ---------------------------------------------------------------------------

template <typename real>
__global__ void __launch_bounds__(NT) k_col(typename cplx_of<real>::type *__restrict__ spec,
                                            const GroupDesc *__restrict__ groups,
                                            const real *__restrict__ kxt, const real *__restrict__ kyt,
                                            const typename cplx_of<real>::type *__restrict__ Wc_g, KP<real> P,
                                            int TW, int nin_max) {
    using C = typename cplx_of<real>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ GroupDesc g;
    const int ny = P.ny, h = P.h, tid = threadIdx.x;
    const size_t slot = (size_t)ny * h;
    const int kx0 = blockIdx.x * TW;
    if (tid == 0) g = groups[blockIdx.y];
    C *Wc = reinterpret_cast<C *>(smem_raw);
    C *in = Wc + ny;                                   // [nin_max][TW][ny]
    C *work = in + (size_t)nin_max * TW * ny;          // [TW][ny]
    load_tables(Wc, Wc_g, ny);
    __syncthreads();
    const int tile = TW * ny;
    for (int s = 0; s < g.nin; ++s) {
        const C *src = spec + (size_t)g.in_slot[s] * slot;
        C *dst = in + (size_t)s * tile;
        for (int idx = tid; idx < tile; idx += NT) {
            const int c = idx % TW, yy = idx / TW;
            dst[c * ny + yy] = src[(size_t)yy * h + kx0 + c];
        }
    }
    __syncthreads();
    for (int s = 0; s < g.nin; ++s) fft_rows<-1>(in + (size_t)s * tile, ny, TW, Wc);
    const real scale = P.scale;
    for (int o = 0; o < g.nout; ++o) {
        const int nterm = g.nterm[o];
        real cc[2][5];
        int tin[2];
        for (int t = 0; t < 2; ++t) {
            tin[t] = g.term_in[o][t];
            for (int e = 0; e < 5; ++e) cc[t][e] = (real)g.c[o][t][e];
        }
        for (int idx = tid; idx < tile; idx += NT) {
            const int c = idx / ny, ky = idx - c * ny;
            const int kx = kx0 + c;
            if (kx == 0) continue;
            const real ax = kxt[kx], ay = kyt[ky];
            C acc = C{0, 0};
            for (int t = 0; t < nterm; ++t) {
                const real mr = cc[t][2] * ax * ax + cc[t][3] * ay * ay + cc[t][4] * ax * ay;
                const real mi = cc[t][0] * ax + cc[t][1] * ay;
                const C v = in[(size_t)tin[t] * tile + idx];
                acc.x += mr * v.x - mi * v.y;
                acc.y += mr * v.y + mi * v.x;
            }
            work[idx] = cscale(acc, scale);
        }
        if (kx0 == 0) {
            // column 0 carries DC (real part) and row-Nyquist (imag part)
            // columns; separate, multiply each, recombine.
            const real a0 = kxt[0], aN = kxt[h];
            for (int j = tid; j <= ny / 2; j += NT) {
                const int jm = (ny - j) % ny;
                C outj = C{0, 0}, outm = C{0, 0};
                for (int t = 0; t < nterm; ++t) {
                    const C *col = in + (size_t)tin[t] * tile;   // column c = 0
                    const C p = col[j], q = col[jm];
                    const C A = cscale(cadd(p, cconj(q)), real(0.5));
                    const C Bv = cscale(cmul_mi(csub(p, cconj(q))), real(0.5));
                    const real ay = kyt[j], aym = kyt[jm];
                    // multiplier at (0, ky) and (Nyquist, ky)
                    const C M0 = C{cc[t][2] * a0 * a0 + cc[t][3] * ay * ay + cc[t][4] * a0 * ay, cc[t][0] * a0 + cc[t][1] * ay};
                    const C MN = C{cc[t][2] * aN * aN + cc[t][3] * ay * ay + cc[t][4] * aN * ay, cc[t][0] * aN + cc[t][1] * ay};
                    const C M0m = C{cc[t][2] * a0 * a0 + cc[t][3] * aym * aym + cc[t][4] * a0 * aym, cc[t][0] * a0 + cc[t][1] * aym};
                    const C MNm = C{cc[t][2] * aN * aN + cc[t][3] * aym * aym + cc[t][4] * aN * aym, cc[t][0] * aN + cc[t][1] * aym};
                    outj = cadd(outj, cadd(cmul(M0, A), cmul_i(cmul(MN, Bv))));
                    outm = cadd(outm, cadd(cmul(M0m, cconj(A)), cmul_i(cmul(MNm, cconj(Bv)))));
                }
                work[j] = cscale(outj, scale);
                if (jm != j) work[jm] = cscale(outm, scale);
            }
        }
        __syncthreads();
        fft_rows<+1>(work, ny, TW, Wc);
        C *dst = spec + (size_t)g.out_slot[o] * slot;
        for (int idx = tid; idx < tile; idx += NT) {
            const int c = idx % TW, yy = idx / TW;
            dst[(size_t)yy * h + kx0 + c] = work[c * ny + yy];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// auxiliary kernels: equilibrium init, moments, generic transforms, sums
// ---------------------------------------------------------------------------

template <typename real>
__global__ void k_feq_init(const double *rho_g, const double *ux_g, const double *uy_g, const double *T_g,
                           real *f, size_t N) {
    // (evaluated in fp64 for either storage type: the weight polynomial of
    // the fastest ring cancels to ~1e-5 relative in fp32, and the initial
    // state should carry only the final rounding)
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N; s += (size_t)gridDim.x * blockDim.x) {
        const double rho = rho_g[s], ux = ux_g[s], uy = uy_g[s], T = T_g[s];
        double F[5];
        weights_Fk<double>(T, F);
        const double u2 = ux * ux + uy * uy, iT = 1.0 / T, qq = 0.5 * u2 * iT, om = 1.0 - qq;
        const double p0 = om + 0.5 * qq * qq, p1 = om * iT, p2 = 0.5 * om * iT * iT;
        const double p3 = iT * iT * iT / 6.0, p4 = iT * iT * iT * iT / 24.0;
        for (int i = 0; i < Q; ++i) {
            const double vu = VX<double>(i) * ux + VY<double>(i) * uy;
            f[(size_t)i * N + s] = (real)(rho * F[c_ring[i]] * (p0 + vu * (p1 + vu * (p2 + vu * (p3 + vu * p4)))));
        }
    }
}

template <typename real>
__global__ void k_moments(const real *f, real *fields, size_t N) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < N; s += (size_t)gridDim.x * blockDim.x) {
        real m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        for (int i = 0; i < Q; ++i) {
            const real v = f[(size_t)i * N + s];
            m0 += v;
            m1 += VX<real>(i) * v;
            m2 += VY<real>(i) * v;
            m3 += V2<real>(i) * v;
        }
        const real ux = m1 / m0, uy = m2 / m0;
        fields[s] = m0;
        fields[N + s] = ux;
        fields[2 * N + s] = uy;
        fields[3 * N + s] = real(0.5) * (m3 / m0 - (ux * ux + uy * uy));
    }
}

template <typename real, typename TO>
__global__ void k_convert(const real *src, TO *dst, size_t n) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x)
        dst[s] = (TO)src[s];
}

// Forward row transforms of nf real fields (row-major [nf][ny][nx]) into
// spectrum slots slot0 .. slot0 + nf - 1.  grid = (ny, nf).
template <typename real, typename TIn>
__global__ void __launch_bounds__(NT) k_rows_forward(const TIn *__restrict__ in, typename cplx_of<real>::type *spec,
                                                     int slot0, const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                     const typename cplx_of<real>::type *__restrict__ Wp_g, KP<real> P) {
    using C = typename cplx_of<real>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, fi = blockIdx.y, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    C *Wr = reinterpret_cast<C *>(smem_raw);
    C *Wp = Wr + h;
    C *buf = Wp + h;
    load_tables(Wr, Wr_g, h);
    load_tables(Wp, Wp_g, h);
    real *bre = reinterpret_cast<real *>(buf);
    for (int x = tid; x < nx; x += NT) bre[x] = (real)in[(size_t)fi * N + (size_t)y * nx + x];
    rows_r2c(buf, h, 1, Wr, Wp);
    C *dst = spec + (size_t)(slot0 + fi) * slot + (size_t)y * h;
    for (int k = tid; k < h; k += NT) dst[k] = buf[k];
}

// Inverse row transforms of nf spectrum slots into real fields.  grid = (ny, nf).
template <typename real, typename TOut>
__global__ void __launch_bounds__(NT) k_rows_inverse(const typename cplx_of<real>::type *spec, int slot0,
                                                     TOut *__restrict__ out,
                                                     const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                     const typename cplx_of<real>::type *__restrict__ Wp_g, KP<real> P) {
    using C = typename cplx_of<real>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, fi = blockIdx.y, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny, slot = (size_t)ny * h;
    C *Wr = reinterpret_cast<C *>(smem_raw);
    C *Wp = Wr + h;
    C *buf = Wp + h;
    load_tables(Wr, Wr_g, h);
    load_tables(Wp, Wp_g, h);
    const C *src = spec + (size_t)(slot0 + fi) * slot + (size_t)y * h;
    for (int k = tid; k < h; k += NT) buf[k] = src[k];
    rows_c2r(buf, h, 1, Wr, Wp);
    __syncthreads();
    const real *bre = reinterpret_cast<const real *>(buf);
    for (int x = tid; x < nx; x += NT) out[(size_t)fi * N + (size_t)y * nx + x] = (TOut)bre[x];
}

// Invariant sums, first pass (grid = ny, one block per row y): the moments
// (Eqs. 7-9) of the row into fields, and the row's fp64 partial sums of
// mass, momentum, e_T of Eq. 17 without its gradient part, max |u| and the
// count of non-finite or unphysical sites.  With with_grad, also the
// forward row transform of rho into spectrum slot 0 and the row's
// x-gradient energy sum_x (D_x rho)^2 by Parseval's relation: slot 0 holds
// Z = DFT_x rho, D_x rho has spectrum i k_x Z (k_x is zero at DC and at the
// row Nyquist bin), and over the two-sided spectrum sum_x d^2 =
// (1 / nx) sum_k |DFT d|^2.  partial[8 y + 0..7] = mass, px, py, e_T
// part, max |u|, count, x-gradient energy, 0 (k_inv_grad_y fills 7).
// Per-site values in the working precision (no fp64 square roots or
// products for fp32 fields), sums in fp64.
template <typename real>
__global__ void __launch_bounds__(NT) k_inv_rows(const real *__restrict__ f, real *__restrict__ fields,
                                                 typename cplx_of<real>::type *spec, double *partial,
                                                 const typename cplx_of<real>::type *__restrict__ Wr_g,
                                                 const typename cplx_of<real>::type *__restrict__ Wp_g,
                                                 const real *__restrict__ kxt, KP<real> P, int with_grad) {
    using C = typename cplx_of<real>::type;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ double red[7][NT / 32];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, tid = threadIdx.x;
    const size_t N = (size_t)nx * ny;
    C *Wr = reinterpret_cast<C *>(smem_raw);
    C *Wp = Wr + h;
    C *buf = Wp + h;
    real *bre = reinterpret_cast<real *>(buf);
    if (with_grad) {
        load_tables(Wr, Wr_g, h);
        load_tables(Wp, Wp_g, h);
    }
    double m = 0, px = 0, py = 0, e = 0, bad = 0;
    real um = 0;
    for (int x = tid; x < nx; x += NT) {
        const size_t s = (size_t)y * nx + x;
        real m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        for (int i = 0; i < Q; ++i) {
            const real v = f[(size_t)i * N + s];
            m0 += v;
            m1 += VX<real>(i) * v;
            m2 += VY<real>(i) * v;
            m3 += V2<real>(i) * v;
        }
        const real rho = m0, ux = m1 / m0, uy = m2 / m0;
        const real T = real(0.5) * (m3 / m0 - (ux * ux + uy * uy));
        fields[s] = rho;
        fields[N + s] = ux;
        fields[2 * N + s] = uy;
        fields[3 * N + s] = T;
        if (with_grad) bre[x] = rho;
        const real u2 = ux * ux + uy * uy;
        m += (double)rho;
        px += (double)(rho * ux);
        py += (double)(rho * uy);
        e += (double)(rho * T - P.a * rho * rho + rho * u2 * real(0.5));
        um = um > sqrt(u2) ? um : sqrt(u2);
        const bool ok = isfinite(rho) && isfinite(ux) && isfinite(uy) && isfinite(T) && rho > real(0) && T > real(0) &&
                        P.b * rho < real(1);
        bad += ok ? 0.0 : 1.0;
    }
    double gxs = 0;
    if (with_grad) {
        rows_r2c(buf, h, 1, Wr, Wp);   // (barriers before and after)
        C *dst = spec + (size_t)y * h;
        for (int k = tid; k < h; k += NT) {
            const C z = buf[k];
            dst[k] = z;
            if (k > 0) {
                const real kx = kxt[k];
                gxs += 2.0 * (double)(kx * kx * (z.x * z.x + z.y * z.y));
            }
        }
        gxs /= nx;
    }
    // block sums: warp shuffles, then one value per warp through shared memory
    double v[7] = {m, px, py, e, (double)um, bad, gxs};
#pragma unroll
    for (int q = 0; q < 7; ++q)
        for (int w = 16; w > 0; w >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v[q], w);
            v[q] = q == 4 ? fmax(v[q], o) : v[q] + o;
        }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0)
        for (int q = 0; q < 7; ++q) red[q][warp] = v[q];
    __syncthreads();
    if (tid < 8) {
        double acc = 0;
        if (tid < 7) {
            acc = red[tid][0];
            for (int w = 1; w < NT / 32; ++w) acc = tid == 4 ? fmax(acc, red[tid][w]) : acc + red[tid][w];
        }
        partial[(size_t)y * 8 + tid] = acc;
    }
}

// Invariant sums, second pass (grid = ny): the row's y-gradient energy
// sum_x (D_y rho)^2 by Parseval's relation from Y = DFT_x(D_y rho) / nx in
// spectrum slot 2 (the column pass's output; bin 0 packs the real DC and
// Nyquist values): nx (Y_0.x^2 + Y_0.y^2 + sum_{0<k<h} 2 |Y_k|^2), into
// partial[8 y + 7].
template <typename real>
__global__ void __launch_bounds__(NT) k_inv_grad_y(const typename cplx_of<real>::type *spec, double *partial,
                                                   KP<real> P) {
    using C = typename cplx_of<real>::type;
    __shared__ double red[NT / 32];
    const int nx = P.nx, ny = P.ny, h = P.h, y = blockIdx.x, tid = threadIdx.x;
    const size_t slot = (size_t)ny * h;
    const C *Y = spec + 2 * slot + (size_t)y * h;
    double g = 0;
    for (int k = tid; k < h; k += NT) {
        const C w = Y[k];
        g += k == 0 ? (double)(w.x * w.x) + (double)(w.y * w.y) : 2.0 * (double)(w.x * w.x + w.y * w.y);
    }
    for (int w = 16; w > 0; w >>= 1) g += __shfl_down_sync(0xffffffffu, g, w);
    if ((tid & 31) == 0) red[tid >> 5] = g;
    __syncthreads();
    if (tid == 0) {
        double acc = 0;
        for (int w = 0; w < NT / 32; ++w) acc += red[w];
        partial[(size_t)y * 8 + 7] = acc * nx;
    }
}

// The invariants from the per-row partials of k_inv_rows / k_inv_grad_y:
// out[0..5] = mass, px, py, e_T (with K / 2 times the gradient energy),
// max |u|, count.
static __global__ void k_reduce_partials(const double *partial, int ny, double K, double *out) {
    __shared__ double red[8][NT];
    const int tid = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int y = tid; y < ny; y += NT) {
        for (int q = 0; q < 8; ++q) {
            const double v = partial[(size_t)y * 8 + q];
            acc[q] = (q == 4) ? fmax(acc[q], v) : acc[q] + v;
        }
    }
    for (int q = 0; q < 8; ++q) red[q][tid] = acc[q];
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (tid < w)
            for (int q = 0; q < 8; ++q)
                red[q][tid] = (q == 4) ? fmax(red[q][tid], red[q][tid + w]) : red[q][tid] + red[q][tid + w];
        __syncthreads();
    }
    if (tid < 6) out[tid] = tid == 3 ? red[3][0] + 0.5 * K * (red[6][0] + red[7][0]) : red[tid][0];
}

}  // namespace fftlb

#include "kernels_pipe.cuh"
#include "kernels_wr.cuh"

namespace fftlb {

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

#define FFTLB_CU(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return Status::err(e_ == cudaErrorMemoryAllocation ? FFTLB_ERR_OOM : FFTLB_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)

#define FFTLB_LAUNCHED(name)                                                                 \
    do {                                                                                     \
        cudaError_t e_ = cudaGetLastError();                                                 \
        if (e_ != cudaSuccess)                                                               \
            return Status::err(FFTLB_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static inline bool valid_len(int n) {
    if (n < 4 || (n & 1)) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// SPLIT: fp32 with the split-BF16 tensor-core first radix-16 passes (the
// kernels' TC instantiations; a separate engine type so that the plain
// kernels carry none of that code)
template <typename real, bool SPLIT = false>
class EngineT : public Engine {
    using C = typename cplx_of<real>::type;

  public:
    ~EngineT() override {
        for (auto &e : prof_pool_) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
        release();
        if (vs_counted_) {
            std::lock_guard<std::mutex> g(vs_owner.mu);
            --vs_owner.live;
        }
    }

    Status init(const fftlb_params &p, const double speeds[4], cudaStream_t s, int nrun) override {
        p_ = p;
        stream_ = s;
        if (nrun < 1 || nrun > 4096) return Status::err(FFTLB_ERR_ARG, "nrun must be in [1, 4096]");
        B_ = nrun;
        const int maxn = sizeof(real) == 8 ? 1024 : 2048;
        if (!valid_len(p.nx) || !valid_len(p.ny) || p.nx > maxn || p.ny > maxn)
            return Status::err(FFTLB_ERR_ARG, "nx, ny must be even 2^p 3^q in [4, " + std::to_string(maxn) + "]");
        if (!(p.tau > 0) || !(p.dx > 0) || !(p.dt > 0)) return Status::err(FFTLB_ERR_ARG, "tau, dx, dt must be > 0");
        if (p.window < 0 || p.window > 4) return Status::err(FFTLB_ERR_ARG, "window must be 0..4");
        if (p.integrator != 1 && p.integrator != 3) return Status::err(FFTLB_ERR_ARG, "integrator must be 1 or 3");
        if (!(p.b >= 0) || !(p.a >= 0)) return Status::err(FFTLB_ERR_ARG, "a, b must be >= 0");
        nx_ = p.nx;
        ny_ = p.ny;
        h_ = nx_ / 2;
        N_ = (size_t)nx_ * ny_;
        {
            // the velocity constants are per translation unit: a second set
            // would overwrite the one live engines compute with
            std::lock_guard<std::mutex> g(vs_owner.mu);
            if (vs_owner.live > 0 && memcmp(vs_owner.speeds, speeds, sizeof vs_owner.speeds) != 0)
                return Status::err(FFTLB_ERR_ARG, "velocity set: live handles of this precision use another set of "
                                                  "speeds (one velocity set per precision at a time)");
            Status su = upload_constants(speeds);
            if (!su.good()) return su;
            memcpy(vs_owner.speeds, speeds, sizeof vs_owner.speeds);
            ++vs_owner.live;
            vs_counted_ = true;
        }
        Status st = alloc();
        if (!st.good()) return st;
        st = build_tables();
        if (!st.good()) return st;
        st = build_groups();
        if (!st.good()) return st;
        return configure();
    }

    Status set_fields(const double *rho, const double *ux, const double *uy, const double *T, bool on_device) override {
        const double *src[4] = {rho, ux, uy, T};
        for (int i = 0; i < 4; ++i)
            if (!src[i]) return Status::err(FFTLB_ERR_ARG, "set_fields: NULL field");
        double *tmp = reinterpret_cast<double *>(scratch_d_);
        for (int i = 0; i < 4; ++i)
            FFTLB_CU(cudaMemcpyAsync(tmp + i * N_, src[i], N_ * sizeof(double),
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream_));
        k_feq_init<real><<<grid1d(), 256, 0, stream_>>>(tmp, tmp + N_, tmp + 2 * N_, tmp + 3 * N_, f0_, N_);
        FFTLB_LAUNCHED("k_feq_init");
        FFTLB_CU(cudaStreamSynchronize(stream_));
        steps_ = 0;
        return Status::ok();
    }

    Status step(long nsteps, long *done) override {
        if (done) *done = 0;
        if (nsteps < 0) return Status::err(FFTLB_ERR_ARG, "nsteps < 0");
        for (long n = 0; n < nsteps; ++n) {
            Status st;
            if (p_.integrator == 1) {
                st = stage(f0b_, nullptr, f0b_, real(0), real(1));
            } else {
                st = stage(f0b_, nullptr, f1b_, real(0), real(1));
                if (st.good()) st = stage(f1b_, f0b_, f1b_, real(0.75), real(0.25));
                if (st.good()) st = stage(f1b_, f0b_, f0b_, real(1.0 / 3.0), real(2.0 / 3.0));
            }
            if (!st.good()) return st;
            ++steps_;
            if (done) *done = n + 1;
            if (p_.check_every > 0 && (steps_ % p_.check_every) == 0) {
                double inv[6];
                st = sums(false, inv);
                if (!st.good()) return st;
                if (inv[5] > 0)
                    return Status::err(FFTLB_ERR_UNSTABLE, "non-finite or unphysical state after step " +
                                                               std::to_string(steps_));
            }
        }
        return Status::ok();
    }

    Status fields(double *rho, double *ux, double *uy, double *T, bool on_device) override {
        {
            Status st = check_err();
            if (!st.good()) return st;
        }
        k_moments<real><<<grid1d(), 256, 0, stream_>>>(f0_, fields_, N_);
        FFTLB_LAUNCHED("k_moments");
        double *tmp = reinterpret_cast<double *>(scratch_d_);
        k_convert<real, double><<<grid1d(), 256, 0, stream_>>>(fields_, tmp, 4 * N_);
        FFTLB_LAUNCHED("k_convert");
        double *dst[4] = {rho, ux, uy, T};
        for (int i = 0; i < 4; ++i) {
            if (!dst[i]) continue;
            FFTLB_CU(cudaMemcpyAsync(dst[i], tmp + i * N_, N_ * sizeof(double),
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream_));
        }
        if (!on_device) FFTLB_CU(cudaStreamSynchronize(stream_));
        return Status::ok();
    }

    Status get_f(double *f, bool on_device) override {
        if (!f) return Status::err(FFTLB_ERR_ARG, "get_f: NULL");
        if (sizeof(real) == 8 && on_device) {
            FFTLB_CU(cudaMemcpyAsync(f, f0_, Q * N_ * sizeof(double), cudaMemcpyDeviceToDevice, stream_));
            return Status::ok();
        }
        double *tmp = reinterpret_cast<double *>(scratch_d_);   // scratch holds >= 33 N doubles
        k_convert<real, double><<<grid1d(), 256, 0, stream_>>>(f0_, tmp, Q * N_);
        FFTLB_LAUNCHED("k_convert");
        FFTLB_CU(cudaMemcpyAsync(f, tmp, Q * N_ * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream_));
        if (!on_device) FFTLB_CU(cudaStreamSynchronize(stream_));
        return Status::ok();
    }

    Status set_f(const double *f, bool on_device) override {
        if (!f) return Status::err(FFTLB_ERR_ARG, "set_f: NULL");
        double *tmp = reinterpret_cast<double *>(scratch_d_);
        FFTLB_CU(cudaMemcpyAsync(tmp, f, Q * N_ * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, stream_));
        k_convert<double, real><<<grid1d(), 256, 0, stream_>>>(tmp, f0_, Q * N_);
        FFTLB_LAUNCHED("k_convert");
        FFTLB_CU(cudaStreamSynchronize(stream_));
        return Status::ok();
    }

    Status invariants(double out[6]) override {
        double inv[6];
        Status st = sums(true, inv);
        if (!st.good()) return st;
        const double area = p_.dx * p_.dx;
        out[0] = inv[0] * area;
        out[1] = inv[1] * area;
        out[2] = inv[2] * area;
        out[3] = inv[3] * area;
        out[4] = inv[4];
        out[5] = steps_ * p_.dt;
        return Status::ok();
    }

    Status gradient(const double *g, double *out, int nfields) override {
        if (!g || !out || nfields < 1 || nfields > 16)
            return Status::err(FFTLB_ERR_ARG, "gradient: need device pointers and 1 <= nfields <= 16");
        // the stage's transform code (and, for split handles, its split-BF16
        // first passes); field i in slot i -> D_x, D_y in slots 20 + 2i, 21 + 2i
        Status st = grad_config();
        if (!st.good()) return st;
        k_grad_rows_fwd<real, split_><<<dim3(ny_, nfields), NT3, smem_gr_, stream_>>>(g, spec_, 0, Wr_, Wp_, Tr_,
                                                                                      ntr_, kp_);
        FFTLB_LAUNCHED("k_grad_rows_fwd");
        k_grad_col<real, split_><<<dim3(h_ / TWg_, nfields), NT3, smem_gc_, stream_>>>(
            spec_, groups_ + grad_groups_, kxt_, kyt_, Wc_, Tc_, ntc_, kp_, TWg_);
        FFTLB_LAUNCHED("k_grad_col");
        k_grad_rows_inv<real, split_><<<dim3(ny_, 2 * nfields), NT3, smem_gr_, stream_>>>(spec_, 20, out, Wr_, Wp_,
                                                                                          Tr_, ntr_, kp_);
        FFTLB_LAUNCHED("k_grad_rows_inv");
        return Status::ok();
    }

    Status set_wait_test(long long ns) override {
        if (ns != 0 && (ns < 1000 || ns > 1000000000LL))
            return Status::err(FFTLB_ERR_ARG, "wait test limit must be 0 or in [1e3, 1e9] ns");
        wait_test_ns_ = (unsigned long long)ns;
        return Status::ok();
    }

    Status select_run(int run) override {
        if (run < 0 || run >= B_) return Status::err(FFTLB_ERR_ARG, "run index out of range");
        set_views(run);
        return Status::ok();
    }
    int nrun() const override { return B_; }

    long steps() const override { return steps_; }
    void set_steps(long s) override { steps_ = s; }
    int launches_per_step() const override { return 6 * (p_.integrator == 1 ? 1 : 3); }
    const fftlb_params &params() const override { return p_; }

  private:
    fftlb_params p_{};
    cudaStream_t stream_ = nullptr;
    int nx_ = 0, ny_ = 0, h_ = 0;
    size_t N_ = 0;
    long steps_ = 0;
    KP<real> kp_{};
    // device memory
    // batch bases (B_ runs back to back) and the views of the selected run
    int B_ = 1, run_ = 0;
    real *f0b_ = nullptr, *f1b_ = nullptr, *fieldsb_ = nullptr, *auxb_ = nullptr;
    C *specb_ = nullptr;
    real *f0_ = nullptr, *f1_ = nullptr, *fields_ = nullptr, *aux_ = nullptr;
    C *spec_ = nullptr;
    real *kxt_ = nullptr, *kyt_ = nullptr;
    C *Wr_ = nullptr, *Wp_ = nullptr, *Wc_ = nullptr;
    C *Tr_ = nullptr, *Tc_ = nullptr;   // pass twiddle tables (power-of-two lengths), radix 16 first
    C *Tr8_ = nullptr;                  // rows, radix 8 first
    bool vs_counted_ = false;           // counted in vs_owner.live
    static constexpr bool split_ = SPLIT && sizeof(real) == 4;   // split-BF16 tensor-core first passes
    uint4 *tc16_ = nullptr;             // their A fragments (dft16_fragments)
    int ntr_ = 0, ntc_ = 0, ntr8_ = 0;
    GroupDesc *groups_ = nullptr;
    double *partial_ = nullptr, *red_ = nullptr;
    void *scratch_d_ = nullptr;
    std::vector<void *> allocs_;
    // group ranges in groups_
    int conv_groups_ = 0, l1_groups_ = 0, l2_groups_ = 0, grad_groups_ = 0, inv_groups_ = 0;
    int nconv_ = NMOV;   // convection groups (velocities with v_y != 0)
    int nconvl_ = NMOV;  // ... and the one-input level-1 groups after them
    // warp-resident fp32 row kernels (kernels_wr.cuh) for nx = 512, 1024:
    // their stage-1 twiddle table and launch shape
    static constexpr bool wr_ok_ = std::is_same<real, float>::value && !SPLIT;
    bool k5wr_ = false, k1wr_ = false, k3wr_ = false;
    C *Tw1_ = nullptr;
    size_t smem5w_ = 0, smem1w_ = 0, smem3w_ = 0;
    int grid5w_ = 1, grid1w_ = 1, grid3w_ = 1;
    // warp-resident convection columns for ny = 256, 512, 1024
    bool colwr_ = false, colmwr_ = false;
    C *Twc_ = nullptr;
    size_t smemcw_ = 0, smemcmw_ = 0;
    int gridcw_ = 1, nbufcw_ = 1, gridcmw_ = 1, ntcw_ = 256;
    CUtensorMap tmap_convw_{};
    // gradient kernels (k_grad_*): column tile width and shared memory
    int TWg_ = 0;
    size_t smem_gr_ = 0, smem_gc_ = 0;
    // test hook: nonzero = every stage starts with k_wait_selftest (ns)
    unsigned long long wait_test_ns_ = 0;
    // launch configuration
    int TW_ = 1;
    size_t smem_col1_ = 0, smem_col2_ = 0, smem_rows1_ = 0, smem_inv_ = 0;
    // pipelined kernels
    int *err_ = nullptr;
    int nsm_ = 1;
    int CH1_ = 8, SMAX1_ = 1, grid1_ = 1, NHB5_ = 1, WR3_ = 1, CH5_ = 8, grid5_ = 1, SMAX5_ = 1, BOXR_ = 1;
    int TWc_ = 1, TWl_ = 1, gridc_ = 1, gridl_ = 1, NBUFc_ = 2, NBUFl_ = 2, NBUF5_ = 2;
    size_t smem1_ = 0, smem3_ = 0, smem5_ = 0, smemc_ = 0, smeml_ = 0;
    CUtensorMap tmap_conv_{}, tmap_l1_{};
    // profiling
    bool prof_ = false;
    struct ProfEv {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<ProfEv> prof_pool_;
    size_t prof_used_ = 0;
    double prof_ms_[KK_COUNT] = {0};
    long prof_n_[KK_COUNT] = {0};
    int prof_kind_ = 0;

    Status prof_begin(int kind) {
        if (!prof_) return Status::ok();
        if (prof_used_ == prof_pool_.size()) {
            ProfEv e;
            e.kind = kind;
            FFTLB_CU(cudaEventCreate(&e.a));
            FFTLB_CU(cudaEventCreate(&e.b));
            prof_pool_.push_back(e);
        }
        prof_pool_[prof_used_].kind = kind;
        FFTLB_CU(cudaEventRecord(prof_pool_[prof_used_].a, stream_));
        return Status::ok();
    }
    Status prof_end() {
        if (!prof_) return Status::ok();
        FFTLB_CU(cudaEventRecord(prof_pool_[prof_used_].b, stream_));
        ++prof_used_;
        if (prof_used_ >= 4096) return prof_flush();
        return Status::ok();
    }
    Status prof_flush() {
        if (prof_used_ == 0) return Status::ok();
        FFTLB_CU(cudaEventSynchronize(prof_pool_[prof_used_ - 1].b));
        for (size_t i = 0; i < prof_used_; ++i) {
            float ms = 0;
            FFTLB_CU(cudaEventElapsedTime(&ms, prof_pool_[i].a, prof_pool_[i].b));
            prof_ms_[prof_pool_[i].kind] += ms;
            prof_n_[prof_pool_[i].kind] += 1;
        }
        prof_used_ = 0;
        return Status::ok();
    }

  public:
    Status profile(int enable) override {
        Status st = prof_flush();
        if (!st.good()) return st;
        prof_ = enable != 0;
        for (int k = 0; k < KK_COUNT; ++k) {
            prof_ms_[k] = 0;
            prof_n_[k] = 0;
        }
        return Status::ok();
    }
    Status profile_read(double *ms, long *launches, double *bytes, int nkinds) override {
        Status st = prof_flush();
        if (!st.good()) return st;
        const double s = sizeof(real), NN = (double)N_ * B_;   // all runs of one launch
        const double fbase = p_.integrator == 3 ? 2.0 / 3.0 : 0.0;   // stages 2, 3 read f^n
        // algorithmic bytes per launch: every value each kernel must read or
        // write once (one-sided spectra count N reals per field)
        const double alg[KK_COUNT] = {
            (33 + 38 + 4) * NN * s,                   // f in; 38 spectra + rho, u, T out
            2.0 * nconvl_ * NN * s,                   // the v_y != 0 spectra and T, Pi, g, u_y in; as many out
            (3 + 4) * NN * s,                         // rho, u_x, u_y in; 4 out
            (14 + 2 + 3 + 6) * NN * s,                // 14 + rho, T in; 3 aux + 6 spectra out
            (3 + 3 + 3) * NN * s,                     // 3 in, 3 added, 3 out
            (32 + 3 + 4 + 3 + 33 + 33 * fbase + 33) * NN * s};
        for (int k = 0; k < nkinds && k < KK_COUNT; ++k) {
            if (ms) ms[k] = prof_ms_[k];
            if (launches) launches[k] = prof_n_[k];
            if (bytes) bytes[k] = alg[k];
        }
        return Status::ok();
    }

  private:

    void set_views(int run) {
        run_ = run;
        const size_t r = (size_t)run;
        f0_ = f0b_ + r * Q * N_;
        f1_ = f1b_ ? f1b_ + r * Q * N_ : nullptr;
        spec_ = specb_ + r * NSLOT * ny_ * h_;
        fields_ = fieldsb_ + r * 4 * N_;
        aux_ = auxb_ + r * 3 * N_;
    }

    unsigned grid1d() const {
        size_t b = (N_ + 255) / 256;
        return (unsigned)(b > 4096 ? 4096 : b);
    }

    template <typename T> Status dalloc(T **ptr, size_t count) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return Status::err(FFTLB_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
        }
        allocs_.push_back(p);
        *ptr = reinterpret_cast<T *>(p);
        return Status::ok();
    }

    void release() {
        for (void *p : allocs_) cudaFree(p);
        allocs_.clear();
    }

    Status upload_constants(const double speeds[4]) {
        double vx[Q], vy[Q], v2[Q];
        float vxf[Q], vyf[Q], v2f[Q];
        int ring[Q];
        vx[0] = vy[0] = v2[0] = 0;
        ring[0] = 0;
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 8; ++i) {
                const int j = 1 + 8 * k + i;
                // exact cos/sin of multiples of pi/4
                static const long double cs[8] = {1.0L, 0.707106781186547524400844362104849039L, 0.0L,
                                                  -0.707106781186547524400844362104849039L, -1.0L,
                                                  -0.707106781186547524400844362104849039L, 0.0L,
                                                  0.707106781186547524400844362104849039L};
                const long double c = cs[i], s = cs[(i + 6) % 8];
                (void)pi;
                vx[j] = (double)(speeds[k] * c);
                vy[j] = (double)(speeds[k] * s);
                v2[j] = vx[j] * vx[j] + vy[j] * vy[j];
                ring[j] = k + 1;
            }
        for (int j = 0; j < Q; ++j) {
            vxf[j] = (float)vx[j];
            vyf[j] = (float)vy[j];
            v2f[j] = (float)v2[j];
        }
        // Eq. 4: F_k = [48 T^4 - 6 s1 T^3 + s2 T^2 - s3 T / 4] / [v_k^2 prod_l (v_k^2 - o_l)],
        // o_l = v_{k+l}^2 with the cyclic index of Eq. 6
        double Fk[4][4];
        float Fkf[4][4], Fkl[4][4];
        for (int k = 0; k < 4; ++k) {
            double o[3];
            for (int l = 1; l <= 3; ++l) o[l - 1] = speeds[(k + l) % 4] * speeds[(k + l) % 4];
            const double vk2 = speeds[k] * speeds[k];
            const double den = vk2 * (vk2 - o[0]) * (vk2 - o[1]) * (vk2 - o[2]);
            if (den == 0) return Status::err(FFTLB_ERR_ARG, "velocity set: speeds must be distinct and non-zero");
            Fk[k][0] = 48.0 / den;
            Fk[k][1] = -6.0 * (o[0] + o[1] + o[2]) / den;
            Fk[k][2] = (o[0] * o[1] + o[1] * o[2] + o[2] * o[0]) / den;
            Fk[k][3] = -o[0] * o[1] * o[2] / (4.0 * den);
            for (int j = 0; j < 4; ++j) {
                Fkf[k][j] = (float)Fk[k][j];
                Fkl[k][j] = (float)(Fk[k][j] - (double)Fkf[k][j]);
            }
        }
        FFTLB_CU(cudaMemcpyToSymbol(c_vx, vx, sizeof vx));
        FFTLB_CU(cudaMemcpyToSymbol(c_vy, vy, sizeof vy));
        FFTLB_CU(cudaMemcpyToSymbol(c_v2, v2, sizeof v2));
        FFTLB_CU(cudaMemcpyToSymbol(c_vxf, vxf, sizeof vxf));
        FFTLB_CU(cudaMemcpyToSymbol(c_vyf, vyf, sizeof vyf));
        FFTLB_CU(cudaMemcpyToSymbol(c_v2f, v2f, sizeof v2f));
        FFTLB_CU(cudaMemcpyToSymbol(c_ring, ring, sizeof ring));
        FFTLB_CU(cudaMemcpyToSymbol(c_Fk, Fk, sizeof Fk));
        FFTLB_CU(cudaMemcpyToSymbol(c_Fkf, Fkf, sizeof Fkf));
        FFTLB_CU(cudaMemcpyToSymbol(c_Fkl, Fkl, sizeof Fkl));
        memcpy(vx_, vx, sizeof vx);
        memcpy(vy_, vy, sizeof vy);
        return Status::ok();
    }
    double vx_[Q], vy_[Q];

    Status alloc() {
        Status st;
        const size_t B = (size_t)B_;
        if (!(st = dalloc(&f0b_, B * Q * N_)).good()) return st;
        if (p_.integrator == 3 && !(st = dalloc(&f1b_, B * Q * N_)).good()) return st;
        if (!(st = dalloc(&specb_, B * NSLOT * ny_ * h_)).good()) return st;
        if (!(st = dalloc(&fieldsb_, B * 4 * N_)).good()) return st;
        if (!(st = dalloc(&auxb_, B * 3 * N_)).good()) return st;
        set_views(0);
        if (!(st = dalloc(&kxt_, (size_t)h_ + 1)).good()) return st;
        if (!(st = dalloc(&kyt_, (size_t)ny_)).good()) return st;
        if (!(st = dalloc(&Wr_, (size_t)h_)).good()) return st;
        if (!(st = dalloc(&Wp_, (size_t)h_)).good()) return st;
        if (!(st = dalloc(&Wc_, (size_t)ny_)).good()) return st;
        if (!(st = dalloc(&partial_, (size_t)ny_ * 8)).good()) return st;
        if (!(st = dalloc(&red_, 8)).good()) return st;
        if (!(st = dalloc(&err_, 4)).good()) return st;
        FFTLB_CU(cudaMemset(err_, 0, 4 * sizeof(int)));
        // fp64 staging for conversions: 33 N doubles (reuses nothing else)
        double *sc = nullptr;
        if (!(st = dalloc(&sc, Q * N_)).good()) return st;
        scratch_d_ = sc;
        return Status::ok();
    }

    // windowed wavenumber (Eqs. K1-K4) for bin index n in [-N/2, N/2 - 1];
    // the Nyquist bin is zeroed (the real part of the paper's inverse
    // transform of i k f~ receives nothing from it)
    long double kappa(int n, int Nlen) const {
        if (2 * n == -Nlen || 2 * n == Nlen) return 0.0L;
        const long double pi = 3.141592653589793238462643383279502884L;
        const long double dx = p_.dx;
        const long double k = 2.0L * pi * n / (Nlen * dx);
        if (p_.window == 0) return k;
        const long double s = sinl(pi * n / Nlen);
        // arcsin series coefficients (2j)! / (4^j (j!)^2 (2j+1))
        long double sum = 0, c = 1.0L, sp = s;
        for (int j = 0; j < p_.window; ++j) {
            if (j > 0) c = c * (2.0L * j - 1.0L) * (2.0L * j - 1.0L) / ((2.0L * j) * (2.0L * j + 1.0L));
            sum += c * sp;
            sp *= s * s;
        }
        return sum * 2.0L / dx;
    }

    static void twiddles(std::vector<C> &w, int n, int len) {
        // w[m] = exp(-2 pi i m / n), m < len
        const long double pi = 3.141592653589793238462643383279502884L;
        w.resize(len);
        for (int m = 0; m < len; ++m) {
            const long double a = 2.0L * pi * (long double)m / (long double)n;
            w[m].x = (real)cosl(a);
            w[m].y = (real)(-sinl(a));
        }
    }

    // per-pass twiddle tables of the power-of-two passes (see
    // pass_twiddle_len): T[t Ns + k] = exp(-2 pi i t k / (Ns R))
    static void pass_twiddles(std::vector<C> &T, int n, int maxlr) {
        T.clear();
        if (!is_pow2(n)) return;
        const long double pi = 3.141592653589793238462643383279502884L;
        int logn = 0;
        while ((1 << logn) < n) ++logn;
        int logNs = 0, rem = logn;
        while (rem > 0) {
            const int lr = rem >= maxlr ? maxlr : rem;
            if (logNs > 0) {
                const int Ns = 1 << logNs, R = 1 << lr;
                for (int t = 0; t < R; ++t)
                    for (int k = 0; k < Ns; ++k) {
                        const long double a = 2.0L * pi * (long double)(t * k) / (long double)(Ns * R);
                        C w;
                        w.x = (real)cosl(a);
                        w.y = (real)(-sinl(a));
                        T.push_back(w);
                    }
            }
            logNs += lr;
            rem -= lr;
        }
    }

    Status build_tables() {
        std::vector<real> kx(h_ + 1), ky(ny_);
        for (int j = 0; j <= h_; ++j) kx[j] = (real)kappa(j, nx_);   // j = h is the Nyquist bin
        for (int j = 0; j < ny_; ++j) ky[j] = (real)kappa(j < ny_ / 2 ? j : j - ny_, ny_);
        std::vector<C> wr, wp, wc;
        twiddles(wr, h_, h_);
        twiddles(wp, nx_, h_);
        twiddles(wc, ny_, ny_);
        FFTLB_CU(cudaMemcpy(kxt_, kx.data(), kx.size() * sizeof(real), cudaMemcpyHostToDevice));
        FFTLB_CU(cudaMemcpy(kyt_, ky.data(), ky.size() * sizeof(real), cudaMemcpyHostToDevice));
        FFTLB_CU(cudaMemcpy(Wr_, wr.data(), wr.size() * sizeof(C), cudaMemcpyHostToDevice));
        FFTLB_CU(cudaMemcpy(Wp_, wp.data(), wp.size() * sizeof(C), cudaMemcpyHostToDevice));
        FFTLB_CU(cudaMemcpy(Wc_, wc.data(), wc.size() * sizeof(C), cudaMemcpyHostToDevice));
        std::vector<C> tr, tr8, tc;
        pass_twiddles(tr, h_, 4);
        pass_twiddles(tr8, h_, 3);
        pass_twiddles(tc, ny_, 4);
        ntr_ = (int)tr.size();
        ntr8_ = (int)tr8.size();
        ntc_ = (int)tc.size();
        Status st;
        if (!(st = dalloc(&Tr_, std::max<size_t>(1, tr.size()))).good()) return st;
        if (!(st = dalloc(&Tr8_, std::max<size_t>(1, tr8.size()))).good()) return st;
        if (!(st = dalloc(&Tc_, std::max<size_t>(1, tc.size()))).good()) return st;
        if (ntr_) FFTLB_CU(cudaMemcpy(Tr_, tr.data(), tr.size() * sizeof(C), cudaMemcpyHostToDevice));
        if (ntr8_) FFTLB_CU(cudaMemcpy(Tr8_, tr8.data(), tr8.size() * sizeof(C), cudaMemcpyHostToDevice));
        if (ntc_) FFTLB_CU(cudaMemcpy(Tc_, tc.data(), tc.size() * sizeof(C), cudaMemcpyHostToDevice));
        if (wr_ok_ && (h_ == 512 || h_ == 256 || h_ == 128)) {
            // tw[k1 P + l] = exp(-2 pi i l k1 / h) for the row configuration of h
            const int P = h_ == 512 ? 32 : h_ == 256 ? 16 : 8, E = h_ / P;
            std::vector<C> t1((size_t)h_);
            const long double pi = 3.141592653589793238462643383279502884L;
            for (int k1 = 0; k1 < E; ++k1)
                for (int l = 0; l < P; ++l) {
                    const long double a = 2.0L * pi * (long double)(l * k1) / (long double)h_;
                    t1[(size_t)k1 * P + l].x = (real)cosl(a);
                    t1[(size_t)k1 * P + l].y = (real)(-sinl(a));
                }
            if (!(st = dalloc(&Tw1_, t1.size())).good()) return st;
            FFTLB_CU(cudaMemcpy(Tw1_, t1.data(), t1.size() * sizeof(C), cudaMemcpyHostToDevice));
        }
        if (wr_ok_ && (ny_ == 1024 || ny_ == 512 || ny_ == 256 || ny_ == 128)) {
            // twc[k1 P + l] = exp(-2 pi i l k1 / ny) for the column configuration of
            // ny, followed by the same values ordered [l][k1] (twc[ny + l E + k1])
            const int P = col_p_host(ny_), E = ny_ / P;
            std::vector<C> t1((size_t)2 * ny_);
            const long double pi = 3.141592653589793238462643383279502884L;
            for (int k1 = 0; k1 < E; ++k1)
                for (int l = 0; l < P; ++l) {
                    const long double a = 2.0L * pi * (long double)(l * k1) / (long double)ny_;
                    C w;
                    w.x = (real)cosl(a);
                    w.y = (real)(-sinl(a));
                    t1[(size_t)k1 * P + l] = w;
                    t1[(size_t)ny_ + (size_t)l * E + k1] = w;
                }
            if (!(st = dalloc(&Twc_, t1.size())).good()) return st;
            FFTLB_CU(cudaMemcpy(Twc_, t1.data(), t1.size() * sizeof(C), cudaMemcpyHostToDevice));
        }
        if (split_) {
            std::vector<uint4> fr;
            dft16_fragments(fr);
            if (!(st = dalloc(&tc16_, fr.size())).good()) return st;
            FFTLB_CU(cudaMemcpy(tc16_, fr.data(), fr.size() * sizeof(uint4), cudaMemcpyHostToDevice));
        }
        return Status::ok();
    }

    // bfloat16 nearest-even of a double (through float: the lo part of the
    // split absorbs any double rounding) and its value
    static uint16_t bf16_rne(double v) {
        const float f = (float)v;
        uint32_t u;
        memcpy(&u, &f, 4);
        u += 0x7fffu + ((u >> 16) & 1u);
        return (uint16_t)(u >> 16);
    }
    static double bf16_value(uint16_t b) {
        const uint32_t u = (uint32_t)b << 16;
        float f;
        memcpy(&f, &u, 4);
        return f;
    }

    // A fragments of the forward 16-point DFT matrix for tc_dft16_pass: for
    // lane (g, q) = (lane / 4, lane % 4), uint4 (a0, a1, a2, a3) of Wr_hi,
    // Wr_lo, Wi_hi, Wi_lo, with Wr = cos(2 pi m k / 16), Wi = -sin(...);
    // register r covers row m = g + 8 (r & 1) and columns k0, k0 + 1 with
    // k0 = 2q + 8 (r >> 1), column k0 in the lower half
    static void dft16_fragments(std::vector<uint4> &fr) {
        fr.assign(128, uint4{0, 0, 0, 0});
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, q = lane & 3;
            for (int part = 0; part < 4; ++part) {
                uint32_t r[4];
                for (int reg = 0; reg < 4; ++reg) {
                    const int m = g + 8 * (reg & 1), k0 = 2 * q + 8 * (reg >> 1);
                    uint32_t packed = 0;
                    for (int hlf = 0; hlf < 2; ++hlf) {
                        const double ang = 2.0 * M_PI * ((m * (k0 + hlf)) % 16) / 16.0;
                        double w = part < 2 ? std::cos(ang) : -std::sin(ang);
                        if (std::fabs(w) < 1e-12) w = 0.0;
                        const uint16_t hi = bf16_rne(w);
                        const uint16_t v = (part & 1) ? bf16_rne(w - bf16_value(hi)) : hi;
                        packed |= (uint32_t)v << (16 * hlf);
                    }
                    r[reg] = packed;
                }
                fr[4 * lane + part] = uint4{r[0], r[1], r[2], r[3]};
            }
        }
    }

    static GroupDesc group(int nin, int in0, int in1) {
        GroupDesc g;
        memset(&g, 0, sizeof g);
        g.nin = nin;
        g.in_slot[0] = in0;
        g.in_slot[1] = in1;
        g.add_slot = -1;
        return g;
    }
    // add output: term list of (input index, c0..c4)
    static void add_out(GroupDesc &g, int out_slot, int nterm, int t0, const double c0[5], int t1 = 0,
                        const double *c1 = nullptr) {
        const int o = g.nout++;
        g.out_slot[o] = out_slot;
        g.nterm[o] = nterm;
        g.term_in[o][0] = t0;
        g.term_in[o][1] = t1;
        for (int e = 0; e < 5; ++e) {
            g.c[o][0][e] = c0[e];
            g.c[o][1][e] = c1 ? c1[e] : 0.0;
        }
    }

    Status build_groups() {
        static const double DX[5] = {1, 0, 0, 0, 0}, DY[5] = {0, 1, 0, 0, 0};
        static const double DYY[5] = {0, 0, 0, -1, 0}, DXY[5] = {0, 0, 0, 0, -1};
        std::vector<GroupDesc> gs;
        // convection: i (v_x k_x + v_y k_y) f_i, in place, for the velocities
        // with v_y != 0 (the row kernel K1 writes i v_x k_x f_i^ / nx for the
        // others)
        conv_groups_ = (int)gs.size();
        nconv_ = 0;
        for (int i = 1; i < Q; ++i) {
            if (vy_[i] == 0.0) continue;
            ++nconv_;
            GroupDesc g = group(1, i - 1, 0);
            const double c[5] = {vx_[i], vy_[i], 0, 0, 0};
            add_out(g, i - 1, 1, 0, c);
            gs.push_back(g);
        }
        // level 1: the outputs that involve k_y (k3_src_slot: K3 forms the
        // rest).  Four of one input and one output (d_y T, d_y Pi, d_y g,
        // d_y u_y) run with the convection groups, in the same launch
        // (nconvl_ groups from conv_groups_: they fill its last round of
        // jobs); rho (d_y, d_yy) and u (d_y u_x, d_y div u) run as the
        // level-1 launch.
        {
            const int singles[4][2] = {{SLOT_T, D_TY}, {SLOT_PI, D_PIY}, {SLOT_G, D_GY}, {SLOT_UY, D_UYY}};
            for (auto &sgl : singles) {
                GroupDesc g = group(1, sgl[0], 0);
                add_out(g, SLOT_D1 + sgl[1], 1, 0, DY);
                gs.push_back(g);
            }
            nconvl_ = nconv_ + 4;
        }
        l1_groups_ = (int)gs.size();
        {
            GroupDesc g = group(1, SLOT_RHO, 0);
            add_out(g, SLOT_D1 + D_RY, 1, 0, DY);
            add_out(g, SLOT_D1 + D_LAP, 1, 0, DYY);   // K3 adds -k_x^2 rho^ / nx
            gs.push_back(g);
        }
        {
            GroupDesc g = group(2, SLOT_UX, SLOT_UY);
            add_out(g, SLOT_D1 + D_UXY, 1, 0, DY);
            add_out(g, SLOT_D1 + D_DIVY, 2, 0, DXY, 1, DYY);   // D_y (D_x u_x + D_y u_y)
            gs.push_back(g);
        }
        // level 2: d_y of Lambda_xy, Lambda_yy, Phi_y plus the d_x terms K3
        // wrote (k3_mul_slot): outputs in 53, 55, 56
        l2_groups_ = (int)gs.size();
        {
            const int l2[3][3] = {{SLOT_L2 + 1, SLOT_L2 + 0, SLOT_L2 + 0},          // in, out, add
                                  {SLOT_L2 + 2, SLOT_L2 + 2, SLOT_D1 + D_DIVX},
                                  {SLOT_L2 + 4, SLOT_L2 + 3, SLOT_L2 + 3}};
            for (auto &e : l2) {
                GroupDesc g = group(1, e[0], 0);
                add_out(g, e[1], 1, 0, DY);
                g.add_slot = e[2];
                gs.push_back(g);
            }
        }
        // gradient op: field i in slot i -> slots 20 + 2i, 21 + 2i
        grad_groups_ = (int)gs.size();
        for (int i = 0; i < 16; ++i) {
            GroupDesc g = group(1, i, 0);
            add_out(g, 20 + 2 * i, 1, 0, DX);
            add_out(g, 21 + 2 * i, 1, 0, DY);
            gs.push_back(g);
        }
        // invariants: rho in slot 0 -> D_y rho in slot 2 (one input, one
        // output: the convection kernels; D_x rho is formed in the row
        // spectrum by k_inv_rows)
        inv_groups_ = (int)gs.size();
        {
            GroupDesc g = group(1, 0, 0);
            add_out(g, 2, 1, 0, DY);
            gs.push_back(g);
        }
        Status st = dalloc(&groups_, gs.size());
        if (!st.good()) return st;
        FFTLB_CU(cudaMemcpy(groups_, gs.data(), gs.size() * sizeof(GroupDesc), cudaMemcpyHostToDevice));
        return Status::ok();
    }

    Status configure() {
        const size_t cs = sizeof(C);
        int dev = 0;
        FFTLB_CU(cudaGetDevice(&dev));
        int maxsm = 0;
        FFTLB_CU(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        const size_t budget = (size_t)maxsm - 2048;   // static shared memory headroom
        optin_ = (size_t)maxsm;
        // column tile width: largest of 8, 4, 2, 1 dividing h with the
        // batched column FFT fitting the registers (TW ny <= 16 NT) and
        // 3 tiles in shared memory
        TW_ = 1;
        for (int tw = 8; tw >= 1; tw >>= 1) {
            if (h_ % tw) continue;
            if ((size_t)tw * ny_ > 16 * NT) continue;
            if ((size_t)(ny_ + 3 * tw * ny_) * cs > budget) continue;
            TW_ = tw;
            break;
        }
        smem_col1_ = (size_t)(ny_ + 2 * TW_ * ny_) * cs;
        smem_col2_ = (size_t)(ny_ + 3 * TW_ * ny_) * cs;
        smem_rows1_ = (size_t)3 * h_ * cs;
        smem_inv_ = (size_t)4 * h_ * cs;
        if (smem_col2_ > budget || smem_inv_ > budget)
            return Status::err(FFTLB_ERR_ARG, "grid too large for shared-memory tiles");
        FFTLB_CU(cudaFuncSetAttribute(k_col<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
        FFTLB_CU(cudaFuncSetAttribute(k_inv_rows<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
        kp_.nx = nx_;
        kp_.ny = ny_;
        kp_.h = h_;
        kp_.nrun = B_;
        kp_.dx = (real)p_.dx;
        kp_.dt = (real)p_.dt;
        kp_.tau = (real)p_.tau;
        kp_.a = (real)p_.a;
        kp_.b = (real)p_.b;
        kp_.K = (real)p_.K;
        kp_.H = (real)p_.H;
        kp_.q = (real)p_.q;
        kp_.zeta = (real)p_.zeta;
        kp_.scale = (real)(1.0 / ((double)nx_ * (double)ny_));
        kp_.scale_x = (real)(1.0 / (double)nx_);
        kp_.tc16 = split_ ? tc16_ : nullptr;
        return configure_pipe(budget);
    }

    static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
        static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
        if (!fn) {
            void *p = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        }
        return fn;
    }

    // the spectrum arena as a 2-D tensor {2h reals, NSLOT ny rows}, boxes
    // of {2 TW reals, BOXR rows}
    Status make_tmap(CUtensorMap *m, int TW) {
        auto enc = tensor_map_encoder();
        if (!enc) return Status::err(FFTLB_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        cuuint64_t dims[2] = {(cuuint64_t)(2 * h_), (cuuint64_t)B_ * NSLOT * ny_};
        cuuint64_t strides[1] = {(cuuint64_t)(2 * h_) * sizeof(real)};
        cuuint32_t box[2] = {(cuuint32_t)(2 * TW), (cuuint32_t)BOXR_};
        cuuint32_t es[2] = {1, 1};
        CUresult r = enc(m, sizeof(real) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         (void *)specb_, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return Status::err(FFTLB_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
        return Status::ok();
    }

    // (the shared-memory opt-in is a per-function, process-wide attribute:
    // always the full budget, so that handles of different grids never
    // lower it below one another's needs)
    // (the budget leaves 2 KB for static shared memory; a kernel with more
    // gets the opt-in maximum less its own static part)
    template <typename K> Status occupancy(K kernel, int nthreads, size_t smem, int *blocks) {
        cudaFuncAttributes fa;
        FFTLB_CU(cudaFuncGetAttributes(&fa, kernel));
        const size_t lim = std::min(budget_, optin_ > fa.sharedSizeBytes ? optin_ - fa.sharedSizeBytes : (size_t)0);
        *blocks = 0;
        if (smem > lim) return Status::ok();
        FFTLB_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim));
        FFTLB_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kernel, nthreads, smem));
        return Status::ok();
    }

    size_t budget_ = 0, optin_ = 0;
    static constexpr int NT1 = KCfg<real, KS_K1>::NT, NTC = KCfg<real, KS_COL>::NT, NT5 = KCfg<real, KS_K5>::NT;
    int ntrmax() const { return std::max(ntr_, ntr8_); }
    // shared memory of the column kernel: twiddles, pass tables, k tables,
    // nbuf staged tiles of NIN inputs, NIN padded work tiles
    size_t col_smem(bool multi, int tw, int nbuf) const {
        const size_t cs = sizeof(C), rs = sizeof(real), pny = (size_t)padded_len(ny_);
        // staged input tiles are placed at 128-byte strides (tile_stride)
        const size_t tile = tile_stride<C>(tw, ny_) * cs, ptile = (size_t)tw * pny * cs, kt = (h_ + 1 + ny_) * rs;
        const size_t nin = multi ? 2 : 1;
        return nbuf > 1 ? (multi ? smem_bytes({ny_ * cs, ntc_ * cs, kt, nin * tile, nin * tile, ptile, ptile})
                                 : smem_bytes({ny_ * cs, ntc_ * cs, kt, nin * tile, nin * tile, ptile}))
                        : (multi ? smem_bytes({ny_ * cs, ntc_ * cs, kt, nin * tile, ptile, ptile})
                                 : smem_bytes({ny_ * cs, ntc_ * cs, kt, nin * tile, ptile}));
    }
    // shared memory of the final row kernel for chunk size ch, nhb head
    // buffers and nbuf chunk buffers
    size_t k5_smem(int ch, int nhb, int nbuf) const {
        const size_t cs = sizeof(C), rs = sizeof(real), ph = (size_t)padded_len(h_);
        const size_t head = (size_t)NHEAD * nx_ * rs, chunk = (size_t)ch * nx_ * rs;
        return smem_bytes({h_ * cs, h_ * cs, ntrmax() * cs, head, nhb > 1 ? head : 0, chunk, nbuf > 1 ? chunk : 0,
                           (size_t)std::max(ch, 3) * ph * cs});
    }
    // A column tile of width tw is staged as ny / BOXR_ tensor boxes of BOXR_
    // rows; every box needs a 128-byte aligned shared-memory destination
    // (the input tiles themselves sit at 128-byte strides, tile_stride).
    bool boxes_aligned(int tw) const { return ny_ <= BOXR_ || ((size_t)BOXR_ * tw * sizeof(C)) % 128 == 0; }
    // buffers for a column tile width: two unless one gives more blocks per SM
    Status col_nbuf(bool multi, int tw, int *nbuf, size_t *sm, int *grid) {
        int best = -1;
        for (int nb2 = 2; nb2 >= 1; --nb2) {
            const size_t s = col_smem(multi, tw, nb2);
            if (s > budget_) continue;
            int nb = 0;
            Status st = multi ? occupancy(kcol_pipe<real, true, SPLIT>, NTC, s, &nb) : occupancy(kcol_pipe<real, false, SPLIT>, NTC, s, &nb);
            if (!st.good()) return st;
            if (nb > best) {
                best = nb;
                *nbuf = nb2;
                *sm = s;
                *grid = std::max(1, nb) * nsm_;
            }
        }
        if (best < 1) return Status::err(FFTLB_ERR_ARG, "tuning parameters exceed shared memory");
        return Status::ok();
    }
    // largest row radix for a kernel transforming `rows` rows at a time with
    // nthr threads: radix 16 unless its passes would leave threads idle
    // radix-8-first rows when radix-16 passes would leave threads idle (the
    // split-BF16 mode keeps radix 16 first: its first pass is the DFT product)
    int row_maxlr(int rows, int nthr) const { return !split_ && rows * (h_ / 16) < nthr ? 3 : 4; }
    static int smax_for(int nx, int nt, int cap) {
        const int s = (nx + nt - 1) / nt;
        int r = 1;
        while (r < s) r *= 2;
        return r <= cap ? r : 0;
    }
    Status occ_k1(size_t sm, int *nb) {
        switch (SMAX1_) {
        case 1: return occupancy(k1_pipe<real, 1, SPLIT>, NT1, sm, nb);
        case 2: return occupancy(k1_pipe<real, 2, SPLIT>, NT1, sm, nb);
        case 4: return occupancy(k1_pipe<real, 4, SPLIT>, NT1, sm, nb);
        default: return occupancy(k1_pipe<real, 8, SPLIT>, NT1, sm, nb);
        }
    }
    Status occ_k5(size_t sm, int *nb) {
        switch (SMAX5_) {
        case 1: return occupancy(k5_pipe<real, 1, SPLIT>, NT5, sm, nb);
        case 2: return occupancy(k5_pipe<real, 2, SPLIT>, NT5, sm, nb);
        default: return occupancy(k5_pipe<real, 4, SPLIT>, NT5, sm, nb);
        }
    }


    Status configure_pipe(size_t budget) {
        budget_ = budget;
        const size_t cs = sizeof(C), rs = sizeof(real);
        if (((size_t)nx_ * rs) % 16 != 0)
            return Status::err(FFTLB_ERR_ARG, "rows must be a multiple of 16 bytes (fp32 needs nx divisible by 4)");
        int dev = 0;
        FFTLB_CU(cudaGetDevice(&dev));
        FFTLB_CU(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev));
        Status st;
        int nb = 0;
        const size_t ph = (size_t)padded_len(h_);
        SMAX1_ = smax_for(nx_, NT1, 8);
        SMAX5_ = smax_for(nx_, NT5, 4);
        if (!SMAX1_ || !SMAX5_) return Status::err(FFTLB_ERR_ARG, "grid row too long for the row kernels");
        // K1: chunks of 6..8 rows (>= 6 for the level-1 rows); most blocks
        // per SM first, then the largest chunk
        {
            int bestnb = 0;
            CH1_ = 0;
            for (int ch = 8; ch >= 6; --ch) {
                const size_t sm =
                    smem_bytes({h_ * cs, h_ * cs, ntr_ * cs, (size_t)ch * nx_ * rs, (size_t)ch * nx_ * rs, ch * ph * cs});
                if (sm > budget) continue;
                st = occ_k1(sm, &nb);
                if (!st.good()) return st;
                if (nb > bestnb) {
                    bestnb = nb;
                    CH1_ = ch;
                    smem1_ = sm;
                }
            }
            if (!CH1_) return Status::err(FFTLB_ERR_ARG, "grid too large for the row kernel");
            st = occ_k1(smem1_, &nb);
            if (!st.good()) return st;
            grid1_ = std::min(B_ * ny_, std::max(1, nb) * nsm_);
        }
        // column kernels: box height divides ny; most blocks per SM first,
        // then the widest tile
        BOXR_ = 1;
        for (int d = std::min(ny_, 256); d >= 1; --d)
            if (ny_ % d == 0) {
                BOXR_ = d;
                break;
            }
        const size_t pny = (size_t)padded_len(ny_);
        auto pick_tw = [&](bool multi, int *tw_out, int *nbuf_out, size_t *sm_out, int *grid_out) -> Status {
            int bestscore = -1;
            *tw_out = 0;
            for (int tw = 8; tw >= 1; tw >>= 1) {
                if (h_ % tw) continue;
                if ((2 * tw * rs) % 16) continue;   // tensor box row: whole 16-byte units
                if (!boxes_aligned(tw)) continue;
                for (int nbuf = 2; nbuf >= 1; --nbuf) {
                    int nb = 0;
                    const size_t sm = col_smem(multi, tw, nbuf);
                    if (sm > budget) continue;
                    Status s2 = multi ? occupancy(kcol_pipe<real, true, SPLIT>, NTC, sm, &nb)
                                      : occupancy(kcol_pipe<real, false, SPLIT>, NTC, sm, &nb);
                    if (!s2.good()) return s2;
                    // most blocks per SM, then the widest tile, then two buffers
                    const int score = nb * 1000 + tw * 10 + nbuf;
                    if (nb > 0 && score > bestscore) {
                        bestscore = score;
                        *tw_out = tw;
                        *nbuf_out = nbuf;
                        *sm_out = sm;
                        *grid_out = nb * nsm_;
                    }
                }
            }
            if (!*tw_out) return Status::err(FFTLB_ERR_ARG, "grid too large for the column kernel");
            return Status::ok();
        };
        if (!(st = pick_tw(false, &TWc_, &NBUFc_, &smemc_, &gridc_)).good()) return st;
        if (!(st = pick_tw(true, &TWl_, &NBUFl_, &smeml_, &gridl_)).good()) return st;
        if (!(st = make_tmap(&tmap_conv_, TWc_)).good()) return st;
        if (!(st = make_tmap(&tmap_l1_, TWl_)).good()) return st;
        // K3 (one row per block, not pipelined inside a block): most blocks
        // per SM first, so that one block's row loads overlap another's
        // transforms, then the most work rows
        {
            int bestnb = 0;
            WR3_ = 0;
            for (int wr = ND1; wr >= 1; --wr) {
                const size_t sm = smem_bytes({h_ * cs, h_ * cs, ntrmax() * cs, (size_t)ND1 * h_ * cs, (size_t)wr * ph * cs,
                                              (size_t)2 * nx_ * rs});
                if (sm > budget) continue;
                if (!(st = occupancy(k3_pipe<real, SPLIT>, NT3, sm, &nb)).good()) return st;
                if (nb > bestnb) {
                    bestnb = nb;
                    WR3_ = wr;
                    smem3_ = sm;
                }
            }
        }
        if (!WR3_) return Status::err(FFTLB_ERR_ARG, "grid too large for the level-1 row kernel");
        // K5: most blocks per SM first, then two head buffers, then the
        // largest chunk, then two chunk buffers
        {
            int bestscore = -1;
            CH5_ = 0;
            for (int nhb = 2; nhb >= 1; --nhb) {
                for (int ch = CHMAX5; ch >= 2; ch -= 2) {
                    for (int nbuf = 2; nbuf >= 1; --nbuf) {
                        const size_t sm = k5_smem(ch, nhb, nbuf);
                        if (sm > budget) continue;
                        if (!(st = occ_k5(sm, &nb)).good()) return st;
                        const int score = nb * 1000 + nhb * 100 + ch * 10 + nbuf;
                        if (nb > 0 && score > bestscore) {
                            bestscore = score;
                            CH5_ = ch;
                            NHB5_ = nhb;
                            NBUF5_ = nbuf;
                            smem5_ = sm;
                        }
                    }
                }
            }
        }
        if (!CH5_) return Status::err(FFTLB_ERR_ARG, "grid too large for the final row kernel");
        st = occ_k5(smem5_, &nb);
        if (!st.good()) return st;
        grid5_ = std::min(B_ * ny_, std::max(1, nb) * nsm_);
        return configure_wr();
    }

    // the warp-resident final row kernel where it applies (fp32, nx = 512 or
    // 1024, and its shared memory fits)
    Status configure_wr() {
        if constexpr (wr_ok_) {
            const bool rows = (h_ == 512 || h_ == 256 || h_ == 128) && Tw1_;
            const int NTr = nt_wr_host(h_);
            int nb = 0;
            Status st;
            if (rows && k5_wr_smem(h_) <= budget_) {
                smem5w_ = k5_wr_smem(h_);
                st = h_ == 512 ? occupancy(k5_wr<512>, nt_k5wr_host(h_), smem5w_, &nb)
                   : h_ == 256 ? occupancy(k5_wr<256>, NTr, smem5w_, &nb)
                               : occupancy(k5_wr<128>, NTr, smem5w_, &nb);
                if (!st.good()) return st;
                if (nb >= 1) {
                    k5wr_ = true;
                    grid5w_ = std::min(B_ * ny_, nb * nsm_);
                }
            }
            if (rows && k3_wr_smem(h_) <= budget_) {
                smem3w_ = k3_wr_smem(h_);
                st = h_ == 512 ? occupancy(k3_wr<512>, nt_k3wr_host(h_), smem3w_, &nb)
                   : h_ == 256 ? occupancy(k3_wr<256>, NTr, smem3w_, &nb)
                               : occupancy(k3_wr<128>, NTr, smem3w_, &nb);
                if (!st.good()) return st;
                if (nb >= 1) {
                    k3wr_ = true;
                    grid3w_ = std::min(B_ * ny_, nb * nsm_);
                }
            }
            if (rows && k1_wr_smem(h_) <= budget_) {
                smem1w_ = k1_wr_smem(h_);
                st = h_ == 512 ? occupancy(k1_wr<512>, nt_k1wr_host(h_), smem1w_, &nb)
                   : h_ == 256 ? occupancy(k1_wr<256>, NTr, smem1w_, &nb)
                               : occupancy(k1_wr<128>, NTr, smem1w_, &nb);
                if (!st.good()) return st;
                if (nb >= 1) {
                    k1wr_ = true;
                    grid1w_ = std::min(B_ * ny_, nb * nsm_);
                }
            }
            const int TWw = Twc_ ? col_tw_host(ny_) : 1, NTw = TWw * (Twc_ ? col_p_host(ny_) : 1);
            if (Twc_ && h_ % TWw == 0) {
                // one or two tile buffers: the most blocks per SM, then two
                // (FFTLB_COLWR_NBUF fixes the count at build time)
                int best = 0;
#ifdef FFTLB_COLWR_NBUF
                for (int nb2 = FFTLB_COLWR_NBUF; nb2 == FFTLB_COLWR_NBUF; --nb2) {
#else
                for (int nb2 = 2; nb2 >= 1; --nb2) {
#endif
                    const size_t sm = kcol_wr_smem(ny_, h_, nb2);
                    if (sm > budget_) continue;
                    st = ny_ == 1024 ? occupancy(kcol_wr<1024>, NTw, sm, &nb)
                       : ny_ == 512  ? occupancy(kcol_wr<512>, NTw, sm, &nb)
                       : ny_ == 256  ? occupancy(kcol_wr<256>, NTw, sm, &nb)
                                     : occupancy(kcol_wr<128>, NTw, sm, &nb);
                    if (!st.good()) return st;
                    if (nb > best) {
                        best = nb;
                        nbufcw_ = nb2;
                        smemcw_ = sm;
                    }
                }
                if (best > 0) {
                    st = make_tmap(&tmap_convw_, TWw);
                    if (!st.good()) return st;
                    colwr_ = true;
                    ntcw_ = NTw;
                    gridcw_ = best * nsm_;
                    const size_t sm = kcolm_wr_smem(ny_, h_);
                    nb = 0;
                    if (sm <= budget_) {
                        st = ny_ == 1024 ? occupancy(kcolm_wr<1024>, NTw, sm, &nb)
                           : ny_ == 512  ? occupancy(kcolm_wr<512>, NTw, sm, &nb)
                           : ny_ == 256  ? occupancy(kcolm_wr<256>, NTw, sm, &nb)
                                         : occupancy(kcolm_wr<128>, NTw, sm, &nb);
                        if (!st.good()) return st;
                    }
                    if (nb > 0) {
                        colmwr_ = true;
                        smemcmw_ = sm;
                        gridcmw_ = nb * nsm_;
                    }
                }
            }
        }
        return Status::ok();
    }

    // shared memory and tile width of the gradient kernels (first use)
    Status grad_config() {
        if (TWg_) return Status::ok();
        const size_t cs = sizeof(C), pny = (size_t)padded_len(ny_);
        smem_gr_ = smem_bytes({h_ * cs, h_ * cs, ntr_ * cs, h_ * cs, (size_t)padded_len(h_) * cs});
        int tw = 0;
        for (int t = 8; t >= 1; t >>= 1) {
            if (h_ % t) continue;
            const size_t sm = smem_bytes({ny_ * cs, ntc_ * cs, (size_t)t * ny_ * cs, t * pny * cs, t * pny * cs});
            if (sm > budget_) continue;
            tw = t;
            smem_gc_ = sm;
            break;
        }
        if (!tw || smem_gr_ > budget_) return Status::err(FFTLB_ERR_ARG, "grid too large for the gradient kernels");
        FFTLB_CU(cudaFuncSetAttribute(k_grad_rows_fwd<real, split_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget_));
        FFTLB_CU(cudaFuncSetAttribute(k_grad_rows_inv<real, split_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget_));
        FFTLB_CU(cudaFuncSetAttribute(k_grad_col<real, split_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget_));
        TWg_ = tw;
        return Status::ok();
    }

  public:
    Status enqueue_step() override {
        Status st;
        if (p_.integrator == 1) return stage(f0b_, nullptr, f0b_, real(0), real(1));
        if (!(st = stage(f0b_, nullptr, f1b_, real(0), real(1))).good()) return st;
        if (!(st = stage(f1b_, f0b_, f1b_, real(0.75), real(0.25))).good()) return st;
        return stage(f1b_, f0b_, f0b_, real(1.0 / 3.0), real(2.0 / 3.0));
    }

    cudaStream_t stream() const override { return stream_; }

    void get_tuning(int t[NTUNE]) const override {
        t[0] = TWc_;
        t[1] = TWl_;
        t[2] = CH1_;
        t[3] = CH5_;
        t[4] = NHB5_;
    }

    // apply explicit parameters (0 = keep): recompute shared-memory sizes,
    // grids and tensor maps; rejects values that do not fit
    Status set_tuning(const int t[NTUNE]) override {
        const size_t cs = sizeof(C), rs = sizeof(real);
        const size_t ph = (size_t)padded_len(h_), pny = (size_t)padded_len(ny_);
        const int twc = t[0] ? t[0] : TWc_, twl = t[1] ? t[1] : TWl_, ch1 = t[2] ? t[2] : CH1_;
        const int ch5 = t[3] ? t[3] : CH5_, nhb = t[4] ? t[4] : NHB5_;
        auto twok = [&](int tw) {
            return tw >= 1 && tw <= 8 && (tw & (tw - 1)) == 0 && h_ % tw == 0 && (2 * tw * rs) % 16 == 0 &&
                   boxes_aligned(tw);
        };
        if (!twok(twc) || !twok(twl) || ch1 < 6 || ch1 > 8 || ch5 < 2 || ch5 > CHMAX5 || (ch5 & 1) || nhb < 1 || nhb > 2)
            return Status::err(FFTLB_ERR_ARG, "tuning parameters out of range");
        const size_t sm1 = smem_bytes({h_ * cs, h_ * cs, ntr_ * cs, (size_t)ch1 * nx_ * rs, (size_t)ch1 * nx_ * rs, ch1 * ph * cs});
        size_t smc = 0, sml = 0;
        int nbc = 2, nbl = 2, gc = 1, gl = 1;
        // chunk buffers: two unless one gives more blocks per SM
        int nbuf5 = 0, best5 = -1;
        size_t sm5 = 0;
        for (int nb2 = 2; nb2 >= 1; --nb2) {
            const size_t s5 = k5_smem(ch5, nhb, nb2);
            if (s5 > budget_) continue;
            int nb5 = 0;
            Status s2 = occ_k5(s5, &nb5);
            if (!s2.good()) return s2;
            if (nb5 > best5) {
                best5 = nb5;
                nbuf5 = nb2;
                sm5 = s5;
            }
        }
        if (!nbuf5) return Status::err(FFTLB_ERR_ARG, "tuning parameters exceed shared memory");
        if (sm1 > budget_ || sm5 > budget_) return Status::err(FFTLB_ERR_ARG, "tuning parameters exceed shared memory");
        Status st;
        if (!(st = col_nbuf(false, twc, &nbc, &smc, &gc)).good()) return st;
        if (!(st = col_nbuf(true, twl, &nbl, &sml, &gl)).good()) return st;
        int nb = 0;
        st = occ_k1(sm1, &nb);
        if (!st.good()) return st;
        const int g1 = std::min(B_ * ny_, std::max(1, nb) * nsm_);
        st = occ_k5(sm5, &nb);
        if (!st.good()) return st;
        const int g5 = std::min(B_ * ny_, std::max(1, nb) * nsm_);
        CUtensorMap mc, ml;
        if (!(st = make_tmap(&mc, twc)).good()) return st;
        if (!(st = make_tmap(&ml, twl)).good()) return st;
        TWc_ = twc;
        TWl_ = twl;
        NBUFc_ = nbc;
        NBUFl_ = nbl;
        CH1_ = ch1;
        CH5_ = ch5;
        NHB5_ = nhb;
        NBUF5_ = nbuf5;
        smem1_ = sm1;
        smemc_ = smc;
        smeml_ = sml;
        smem5_ = sm5;
        grid1_ = g1;
        gridc_ = gc;
        gridl_ = gl;
        grid5_ = g5;
        tmap_conv_ = mc;
        tmap_l1_ = ml;
        return Status::ok();
    }

    Status autotune(double *stage_ms) override {
        // candidates time stages on the current state of every run, writing
        // to the RK stage buffer (or, for Euler, to a temporary one), so the
        // state itself is never changed
        real *out = f1b_;
        void *tmp = nullptr;
        if (!out) {
            if (cudaMalloc(&tmp, (size_t)B_ * Q * N_ * sizeof(real)) != cudaSuccess) {
                cudaGetLastError();
                return Status::err(FFTLB_ERR_OOM, "autotune: no room for a stage output buffer");
            }
            out = reinterpret_cast<real *>(tmp);
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        auto cleanup = [&]() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            if (tmp) cudaFree(tmp);
        };
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            cleanup();
            return Status::err(FFTLB_ERR_CUDA, "autotune: event creation failed");
        }
        auto time_stage = [&](double *ms) -> Status {
            Status st;
            for (int w = 0; w < 2; ++w)
                if (!(st = stage(f0b_, nullptr, out, real(0), real(1))).good()) return st;
            FFTLB_CU(cudaEventRecord(e0, stream_));
            for (int w = 0; w < 3; ++w)
                if (!(st = stage(f0b_, nullptr, out, real(0), real(1))).good()) return st;
            FFTLB_CU(cudaEventRecord(e1, stream_));
            FFTLB_CU(cudaEventSynchronize(e1));
            float t = 0;
            FFTLB_CU(cudaEventElapsedTime(&t, e0, e1));
            *ms = t / 3.0;
            return Status::ok();
        };
        int best[NTUNE];
        get_tuning(best);
        double best_ms = 0;
        Status st = time_stage(&best_ms);
        const int cand[NTUNE][4] = {{8, 4, 2, 1}, {8, 4, 2, 1}, {8, 7, 6, 0}, {8, 6, 4, 2}, {2, 1, 0, 0}};
        for (int p = 0; p < NTUNE && st.good(); ++p) {
            for (int c = 0; c < 4 && cand[p][c]; ++c) {
                int t[NTUNE];
                for (int q = 0; q < NTUNE; ++q) t[q] = best[q];
                if (cand[p][c] == best[p]) continue;
                t[p] = cand[p][c];
                if (!set_tuning(t).good()) continue;   // does not fit: skip
                double ms = 0;
                if (!(st = time_stage(&ms)).good()) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best[p] = t[p];
                }
            }
            Status s2 = set_tuning(best);
            if (st.good() && !s2.good()) st = s2;
        }
        if (st.good() && cudaStreamSynchronize(stream_) != cudaSuccess)
            st = Status::err(FFTLB_ERR_CUDA, "autotune: stream synchronisation failed");
        cleanup();
        if (!st.good()) return st;
        if (stage_ms) *stage_ms = best_ms;
        return Status::ok();
    }

  private:
    // Launch of a warp-resident kernel, with programmatic stream
    // serialization when built with FFTLB_PDL=1: its blocks may then start
    // their prologue while the kernel before it finishes (each of these
    // kernels calls grid_dep_wait before it touches memory that earlier
    // kernels wrote or read).  Off by default: measured at 1024^2, the step
    // took 1.230 ms with it against 1.077 ms without.
#ifndef FFTLB_PDL
#define FFTLB_PDL 0
#endif
    // The final row kernel alone (FFTLB_PDL_K5): it overlaps the level-2
    // launch's tail with its first convection chunk, and only its head copies
    // wait for that launch.
#ifndef FFTLB_PDL_K5
#define FFTLB_PDL_K5 0
#endif
    template <typename... KArgs, typename... Args>
    Status launch_pdl(const char *name, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                      Args &&...args) {
        return launch_ex(name, FFTLB_PDL, kernel, grid, block, smem, std::forward<Args>(args)...);
    }
    template <typename... KArgs, typename... Args>
    Status launch_ex(const char *name, int pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                     Args &&...args) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(block);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream_;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = pdl;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return Status::err(FFTLB_ERR_CUDA, std::string(name) + ": " + cudaGetErrorString(e));
        }
        return Status::ok();
    }

    Status launch_col(int first, int count, bool level1) {
        if constexpr (wr_ok_) {
            if (!level1 && colwr_) {
                if (count > kMaxColGroups) return Status::err(FFTLB_ERR_ARG, "too many column groups in one launch");
#define FFTLB_KCOLWR(NYV)                                                                                     \
    launch_pdl("kcol_wr", kcol_wr<NYV>, gridcw_, ntcw_, smemcw_, specb_, (const GroupDesc *)(groups_ + first),     \
               count, (const float *)kxt_, (const float *)kyt_, (const float2 *)Twc_, kp_, BOXR_, nbufcw_,          \
               tmap_convw_, err_)
                return ny_ == 1024 ? FFTLB_KCOLWR(1024)
                     : ny_ == 512  ? FFTLB_KCOLWR(512)
                     : ny_ == 256  ? FFTLB_KCOLWR(256)
                                   : FFTLB_KCOLWR(128);
#undef FFTLB_KCOLWR
            }
            if (level1 && colmwr_) {
                if (count > kMaxMGroups) return Status::err(FFTLB_ERR_ARG, "too many column groups in one launch");
#define FFTLB_KCOLMWR(NYV)                                                                                    \
    launch_pdl("kcolm_wr", kcolm_wr<NYV>, gridcmw_, ntcw_, smemcmw_, specb_, (const GroupDesc *)(groups_ + first), \
               count, (const float *)kxt_, (const float *)kyt_, (const float2 *)Twc_, kp_, BOXR_, tmap_convw_, err_)
                return ny_ == 1024 ? FFTLB_KCOLMWR(1024)
                     : ny_ == 512  ? FFTLB_KCOLMWR(512)
                     : ny_ == 256  ? FFTLB_KCOLMWR(256)
                                   : FFTLB_KCOLMWR(128);
#undef FFTLB_KCOLMWR
            }
        }
        if (level1)
            kcol_pipe<real, true, SPLIT><<<gridl_, NTC, smeml_, stream_>>>(specb_, groups_ + first, count, kxt_,
                                                                               kyt_, Wc_, Tc_, ntc_, kp_, TWl_, BOXR_,
                                                                               NBUFl_, tmap_l1_, err_);
        else
            kcol_pipe<real, false, SPLIT><<<gridc_, NTC, smemc_, stream_>>>(
                specb_, groups_ + first, count, kxt_, kyt_, Wc_, Tc_, ntc_, kp_, TWc_, BOXR_, NBUFc_, tmap_conv_, err_);
        FFTLB_LAUNCHED("kcol_pipe");
        return Status::ok();
    }

    Status stage(const real *cur, const real *base, real *out, real alpha, real beta) {
        Status st;
        if (wait_test_ns_) {
            k_wait_selftest<<<nsm_, 128, 0, stream_>>>(err_, wait_test_ns_);
            FFTLB_LAUNCHED("k_wait_selftest");
        }
        if (!(st = prof_begin(KK_ROW_FORWARD)).good()) return st;
        bool k1done = false;
        if constexpr (wr_ok_) {
            if (k1wr_) {
                const int nt = nt_k1wr_host(h_);
                auto *kern = h_ == 512 ? k1_wr<512> : h_ == 256 ? k1_wr<256> : k1_wr<128>;
                if (!(st = launch_pdl("k1_wr", kern, grid1w_, nt, smem1w_, cur, specb_, fieldsb_,
                                      (const float2 *)Tw1_, (const float2 *)Wp_, (const float *)kxt_, kp_, err_)).good())
                    return st;
                k1done = true;
            }
        }
        if (k1done) {
        } else if (SMAX1_ == 1)
            k1_pipe<real, 1, SPLIT><<<grid1_, NT1, smem1_, stream_>>>(cur, specb_, fieldsb_, Wr_, Wp_, Tr_, ntr_, kxt_, kp_,
                                                                                 CH1_, err_);
        else if (SMAX1_ == 2)
            k1_pipe<real, 2, SPLIT><<<grid1_, NT1, smem1_, stream_>>>(cur, specb_, fieldsb_, Wr_, Wp_, Tr_, ntr_, kxt_, kp_,
                                                                                 CH1_, err_);
        else if (SMAX1_ == 4)
            k1_pipe<real, 4, SPLIT><<<grid1_, NT1, smem1_, stream_>>>(cur, specb_, fieldsb_, Wr_, Wp_, Tr_, ntr_, kxt_, kp_, CH1_, err_);
        else
            k1_pipe<real, 8, SPLIT><<<grid1_, NT1, smem1_, stream_>>>(cur, specb_, fieldsb_, Wr_, Wp_, Tr_, ntr_, kxt_, kp_, CH1_, err_);
        FFTLB_LAUNCHED("k1_pipe");
        if (!(st = prof_end()).good()) return st;
        if (!(st = prof_begin(KK_COL_CONV)).good()) return st;
        if (!(st = launch_col(conv_groups_, nconvl_, false)).good()) return st;
        if (!(st = prof_end()).good()) return st;
        if (!(st = prof_begin(KK_COL_LEVEL1)).good()) return st;
        if (!(st = launch_col(l1_groups_, 2, true)).good()) return st;
        if (!(st = prof_end()).good()) return st;
        if (!(st = prof_begin(KK_ROW_LEVEL1)).good()) return st;
        bool k3done = false;
        if constexpr (wr_ok_) {
            if (k3wr_) {
                const int nt = nt_k3wr_host(h_);
                auto *kern = h_ == 512 ? k3_wr<512> : h_ == 256 ? k3_wr<256> : k3_wr<128>;
                if (!(st = launch_pdl("k3_wr", kern, grid3w_, nt, smem3w_, specb_, (const float *)fieldsb_, auxb_,
                                      (const float2 *)Tw1_, (const float2 *)Wp_, (const float *)kxt_, kp_, err_)).good())
                    return st;
                k3done = true;
            }
        }
        if (!k3done) {
            const int ml = row_maxlr(WR3_, NT3);
            k3_pipe<real, SPLIT><<<B_ * ny_, NT3, smem3_, stream_>>>(specb_, fieldsb_, auxb_, Wr_, Wp_, ml == 3 ? Tr8_ : Tr_,
                                                              ml == 3 ? ntr8_ : ntr_, kxt_, kp_, WR3_, ml, err_);
        }
        FFTLB_LAUNCHED("k3_pipe");
        if (!(st = prof_end()).good()) return st;
        if (!(st = prof_begin(KK_COL_LEVEL2)).good()) return st;
        if (!(st = launch_col(l2_groups_, 3, false)).good()) return st;   // one input, one output each
        if (!(st = prof_end()).good()) return st;
        if (!(st = prof_begin(KK_ROW_FINAL)).good()) return st;
        if constexpr (wr_ok_) {
            if (k5wr_) {
                const int nt = nt_k5wr_host(h_);
                auto *kern = h_ == 512 ? k5_wr<512> : h_ == 256 ? k5_wr<256> : k5_wr<128>;
                if (!(st = launch_ex("k5_wr", FFTLB_PDL || FFTLB_PDL_K5, kern, grid5w_, nt, smem5w_, (const float2 *)specb_,
                                      (const float *)fieldsb_, (const float *)auxb_, cur, base, out, alpha, beta,
                                      (const float2 *)Tw1_, (const float2 *)Wp_, kp_, err_)).good())
                    return st;
                return prof_end();
            }
        }
        const int ml5 = row_maxlr(CH5_, NT5);
        if (SMAX5_ == 1)
            k5_pipe<real, 1, SPLIT><<<grid5_, NT5, smem5_, stream_>>>(specb_, fieldsb_, auxb_, cur, base, out, alpha, beta, Wr_,
                                                               Wp_, ml5 == 3 ? Tr8_ : Tr_, ml5 == 3 ? ntr8_ : ntr_, kp_, CH5_, NHB5_, NBUF5_, ml5, err_);
        else if (SMAX5_ == 2)
            k5_pipe<real, 2, SPLIT><<<grid5_, NT5, smem5_, stream_>>>(specb_, fieldsb_, auxb_, cur, base, out, alpha, beta, Wr_,
                                                               Wp_, ml5 == 3 ? Tr8_ : Tr_, ml5 == 3 ? ntr8_ : ntr_, kp_, CH5_, NHB5_, NBUF5_, ml5, err_);
        else
            k5_pipe<real, 4, SPLIT><<<grid5_, NT5, smem5_, stream_>>>(specb_, fieldsb_, auxb_, cur, base, out, alpha, beta, Wr_,
                                                               Wp_, ml5 == 3 ? Tr8_ : Tr_, ml5 == 3 ? ntr8_ : ntr_, kp_, CH5_, NHB5_, NBUF5_, ml5, err_);
        FFTLB_LAUNCHED("k5_pipe");
        return prof_end();
    }

    // device error word (bounded waits that ran out)
    Status check_err() {
        int e = 0;
        FFTLB_CU(cudaMemcpyAsync(&e, err_, sizeof(int), cudaMemcpyDeviceToHost, stream_));
        FFTLB_CU(cudaStreamSynchronize(stream_));
        if (e) return Status::err(FFTLB_ERR_TIMEOUT, "a bounded device wait ran out (error word " + std::to_string(e) + ")");
        return Status::ok();
    }

    // (one synchronisation: the sums and the device error word of the steps
    // before them come back together)
    Status sums(bool with_grad, double out[6]) {
        k_inv_rows<real><<<ny_, NT, with_grad ? smem_rows1_ : 0, stream_>>>(f0_, fields_, spec_, partial_, Wr_, Wp_,
                                                                          kxt_, kp_, with_grad ? 1 : 0);
        FFTLB_LAUNCHED("k_inv_rows");
        if (with_grad) {
            Status st = launch_col(inv_groups_, 1, false);
            if (!st.good()) return st;
            k_inv_grad_y<real><<<ny_, NT, 0, stream_>>>(spec_, partial_, kp_);
            FFTLB_LAUNCHED("k_inv_grad_y");
        }
        k_reduce_partials<<<1, NT, 0, stream_>>>(partial_, ny_, (double)p_.K, red_);
        FFTLB_LAUNCHED("k_reduce_partials");
        int e = 0;
        FFTLB_CU(cudaMemcpyAsync(out, red_, 6 * sizeof(double), cudaMemcpyDeviceToHost, stream_));
        FFTLB_CU(cudaMemcpyAsync(&e, err_, sizeof(int), cudaMemcpyDeviceToHost, stream_));
        FFTLB_CU(cudaStreamSynchronize(stream_));
        if (e) return Status::err(FFTLB_ERR_TIMEOUT, "a bounded device wait ran out (error word " + std::to_string(e) + ")");
        return Status::ok();
    }
};

}  // namespace fftlb

// Learned warm start (include/fftlb_warmstart.h): a 4-layer periodic 3x3
// convolutional network trained on FFT-LB snapshots (arXiv:1011.3582,
// Sec. 4 phase separation) and applied to a handle's state.
//
// Every convolution is an implicit GEMM on the tensor cores: bfloat16
// operands staged in shared memory, mma.sync m16n8k16 with fp32
// accumulators.  Activations are NHWC bfloat16 (channels padded to 16 or
// 32), so one pixel's channels are contiguous 16-byte chunks.  A block
// owns 64-pixel row segments (4 warps x 16 pixels = the M dimension) and
// loops over them with its weights staged once:
//   k_conv<CIN, COUT, FWD_RELU | FWD_LAST | BWD>
//       out[p][n] = sum_tap sum_k w[tap][n][k] in[p + d(tap)][k]
//       FWD: + bias, ReLU (layers 1-3, bfloat16 out) or fp32 planar out
//       (layer 4).  BWD: the input gradient, using the weights transposed
//       and flipped (d -> -d), times the ReLU mask of the stored activation.
//   k_wgrad<CIN, GC>: dW[co][tap][ci] = sum_p G[p][co] A[p + d(tap)][ci]
//       (M = co, N = ci, K = pixels), fp32 atomics into the gradient.
// The parameter gradient, loss and Adam state are fp32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/fftlb_warmstart.h"
#include "engine.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int NL = 4;
// channels per layer l = 0..3 (functions so that host and device code share them)
__host__ __device__ constexpr int CIN_R(int l) { return l == 0 ? 3 : 32; }     // real input
__host__ __device__ constexpr int COUT_R(int l) { return l == 3 ? 2 : 32; }    // real output
__host__ __device__ constexpr int CINP(int l) { return l == 0 ? 16 : 32; }     // padded input (forward)
__host__ __device__ constexpr int COUTP(int l) { return l == 3 ? 8 : 32; }     // padded output (forward)
__host__ __device__ constexpr int GCH(int l) { return l == 3 ? 16 : 32; }      // stored gradient G_l
constexpr int TX = 64;                        // pixels per tile (one row segment)
constexpr int NTH = 128;                      // 4 warps x 16 pixels

enum { FWD_RELU = 0, FWD_LAST = 1, BWD = 2 };

__host__ __device__ constexpr int w_size(int l) { return COUT_R(l) * 9 * CIN_R(l); }
__host__ __device__ constexpr int w_off(int l) { return l == 0 ? 0 : w_off(l - 1) + w_size(l - 1) + COUT_R(l - 1); }
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + w_size(l); }
static_assert(b_off(NL - 1) + COUT_R(NL - 1) == FFTLB_CNN_NPARAMS, "parameter layout");

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// stage rows y-1..y+1, pixels x0-1..x0+TX of an NHWC bfloat16 tensor with C
// channels into s[3][TX + 2][C + 8] (periodic)
template <int C>
__device__ __forceinline__ void stage_rows(bf16 (*s)[TX + 2][C + 8], const bf16 *in, int y, int x0, int H, int W) {
    constexpr int CH = C / 8;
    for (int i = threadIdx.x; i < 3 * (TX + 2) * CH; i += NTH) {
        const int ch = i % CH, px = (i / CH) % (TX + 2), r = i / (CH * (TX + 2));
        const int yy = wrap(y + r - 1, H), xx = wrap(x0 + px - 1, W);
        *reinterpret_cast<uint4 *>(&s[r][px][ch * 8]) =
            *reinterpret_cast<const uint4 *>(in + ((size_t)yy * W + xx) * C + ch * 8);
    }
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(NTH) k_conv(const bf16 *__restrict__ in, const bf16 *__restrict__ w,
                                              const float *__restrict__ bias, void *out,
                                              const bf16 *__restrict__ mask, int H, int W) {
    constexpr int SC = CIN + 8;   // padded pixel stride: conflict-free fragment loads
    constexpr int NT = COUT / 8;
    __shared__ __align__(16) bf16 in_s[3][TX + 2][SC];
    __shared__ __align__(16) bf16 w_s[9][COUT][SC];
    for (int i = threadIdx.x; i < 9 * COUT * (CIN / 8); i += NTH) {
        const int row = i / (CIN / 8), ch = i % (CIN / 8);
        *reinterpret_cast<uint4 *>(&w_s[row / COUT][row % COUT][ch * 8]) =
            *reinterpret_cast<const uint4 *>(w + (size_t)row * CIN + ch * 8);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tpr = W / TX, ntiles = H * tpr;
    const size_t P = (size_t)H * W;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int y = tile / tpr, x0 = (tile - y * tpr) * TX;
        __syncthreads();   // previous tile's reads of in_s are done (and w_s is staged)
        stage_rows<CIN>(in_s, in, y, x0, H, W);
        __syncthreads();
        float acc[NT][4];
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap % 3;
            const bf16 *r0 = &in_s[ky][warp * 16 + g + kx][0];
            const bf16 *r1 = &in_s[ky][warp * 16 + g + 8 + kx][0];
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                const int k = kc * 16 + 2 * t;
                const uint32_t a0 = ld32(r0 + k), a1 = ld32(r1 + k), a2 = ld32(r0 + k + 8), a3 = ld32(r1 + k + 8);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const bf16 *rb = &w_s[tap][nt * 8 + g][k];
                    mma_bf16(acc[nt], a0, a1, a2, a3, ld32(rb), ld32(rb + 8));
                }
            }
        }
        const size_t pa = (size_t)y * W + x0 + warp * 16 + g, pb = pa + 8;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int co = nt * 8 + 2 * t;
            if (MODE == FWD_RELU) {
                bf16 *o = reinterpret_cast<bf16 *>(out);
                const float b0 = bias[co], b1 = bias[co + 1];
                *reinterpret_cast<__nv_bfloat162 *>(o + pa * COUT + co) =
                    __floats2bfloat162_rn(fmaxf(acc[nt][0] + b0, 0.f), fmaxf(acc[nt][1] + b1, 0.f));
                *reinterpret_cast<__nv_bfloat162 *>(o + pb * COUT + co) =
                    __floats2bfloat162_rn(fmaxf(acc[nt][2] + b0, 0.f), fmaxf(acc[nt][3] + b1, 0.f));
            } else if (MODE == FWD_LAST) {
                float *o = reinterpret_cast<float *>(out);
                if (co < 2) {   // two real output channels, planar
                    o[(size_t)co * P + pa] = acc[nt][0] + bias[co];
                    o[(size_t)(co + 1) * P + pa] = acc[nt][1] + bias[co + 1];
                    o[(size_t)co * P + pb] = acc[nt][2] + bias[co];
                    o[(size_t)(co + 1) * P + pb] = acc[nt][3] + bias[co + 1];
                }
            } else {
                bf16 *o = reinterpret_cast<bf16 *>(out);
                const __nv_bfloat162 ma = *reinterpret_cast<const __nv_bfloat162 *>(mask + pa * COUT + co);
                const __nv_bfloat162 mb = *reinterpret_cast<const __nv_bfloat162 *>(mask + pb * COUT + co);
                *reinterpret_cast<__nv_bfloat162 *>(o + pa * COUT + co) = __floats2bfloat162_rn(
                    __low2float(ma) > 0.f ? acc[nt][0] : 0.f, __high2float(ma) > 0.f ? acc[nt][1] : 0.f);
                *reinterpret_cast<__nv_bfloat162 *>(o + pb * COUT + co) = __floats2bfloat162_rn(
                    __low2float(mb) > 0.f ? acc[nt][2] : 0.f, __high2float(mb) > 0.f ? acc[nt][3] : 0.f);
            }
        }
    }
}

// dW[co][tap][ci] += sum_p G[p][co] A[p + d(tap)][ci]; warp w owns taps w,
// w + 4, w + 8.  G: NHWC with GC channels, A: NHWC with CIN channels.
template <int CIN, int GC>
__global__ void __launch_bounds__(NTH) k_wgrad(const bf16 *__restrict__ G, const bf16 *__restrict__ A,
                                               float *__restrict__ grad, int cout_r, int cin_r, int H, int W) {
    constexpr int SA = CIN + 8, SG = GC + 8;
    constexpr int MT = GC / 16, NT = CIN / 8;
    __shared__ __align__(16) bf16 a_s[3][TX + 2][SA];
    __shared__ __align__(16) bf16 g_s[TX][SG];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int tpr = W / TX, ntiles = H * tpr;
    float acc[3][MT][NT][4];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) acc[j][mt][nt][0] = acc[j][mt][nt][1] = acc[j][mt][nt][2] = acc[j][mt][nt][3] = 0.f;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int y = tile / tpr, x0 = (tile - y * tpr) * TX;
        __syncthreads();
        stage_rows<CIN>(a_s, A, y, x0, H, W);
        for (int i = threadIdx.x; i < TX * (GC / 8); i += NTH) {
            const int ch = i % (GC / 8), px = i / (GC / 8);
            *reinterpret_cast<uint4 *>(&g_s[px][ch * 8]) =
                *reinterpret_cast<const uint4 *>(G + ((size_t)y * W + x0 + px) * GC + ch * 8);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int tap = warp + 4 * j;
            if (tap < 9) {
                const int ky = tap / 3, kx = tap % 3;
#pragma unroll
                for (int ks = 0; ks < TX / 16; ++ks) {
                    const int p0 = ks * 16 + 2 * t;
                    uint32_t a[MT][4];
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        const int c0 = mt * 16 + g, c1 = c0 + 8;
                        a[mt][0] = pack2(g_s[p0][c0], g_s[p0 + 1][c0]);
                        a[mt][1] = pack2(g_s[p0][c1], g_s[p0 + 1][c1]);
                        a[mt][2] = pack2(g_s[p0 + 8][c0], g_s[p0 + 9][c0]);
                        a[mt][3] = pack2(g_s[p0 + 8][c1], g_s[p0 + 9][c1]);
                    }
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) {
                        const int ci = nt * 8 + g;
                        const uint32_t b0 = pack2(a_s[ky][p0 + kx][ci], a_s[ky][p0 + 1 + kx][ci]);
                        const uint32_t b1 = pack2(a_s[ky][p0 + 8 + kx][ci], a_s[ky][p0 + 9 + kx][ci]);
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
                            mma_bf16(acc[j][mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int tap = warp + 4 * j;
        if (tap >= 9) continue;
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int co = mt * 16 + g + (e >= 2 ? 8 : 0), ci = nt * 8 + 2 * t + (e & 1);
                    if (co < cout_r && ci < cin_r) atomicAdd(&grad[((size_t)co * 9 + tap) * cin_r + ci], acc[j][mt][nt][e]);
                }
    }
}

// db[co] += sum_p G[p][co] for co < cout_r
template <int GC>
__global__ void k_bgrad(const bf16 *__restrict__ G, float *__restrict__ db, int cout_r, size_t P) {
    __shared__ float red[256];
    const int c = threadIdx.x % GC, lane_p = threadIdx.x / GC;
    constexpr int PP = 256 / GC;
    float s = 0.f;
    for (size_t p = (size_t)blockIdx.x * PP + lane_p; p < P; p += (size_t)gridDim.x * PP) s += __bfloat162float(G[p * GC + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < GC) {
        float tot = 0.f;
        for (int k = 0; k < PP; ++k) tot += red[k * GC + threadIdx.x];
        if (threadIdx.x < cout_r) atomicAdd(&db[threadIdx.x], tot);
    }
}

// A0[p][c] = bf16(X[c][p]) for c < 3, channels 3..15 zero
__global__ void k_prep(const float *__restrict__ X, bf16 *__restrict__ A0, size_t P) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const bf16 z = __float2bfloat16_rn(0.f);
        uint4 lo;
        lo.x = pack2(__float2bfloat16_rn(X[p]), __float2bfloat16_rn(X[P + p]));
        lo.y = pack2(__float2bfloat16_rn(X[2 * P + p]), z);
        lo.z = lo.w = 0u;
        uint4 *d = reinterpret_cast<uint4 *>(A0 + p * 16);
        d[0] = lo;
        d[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// residual R = Y - (Xt - X[0:2]); loss += sum R^2; G4[p][c] = bf16(2 R / n)
__global__ void k_loss(const float *__restrict__ Y, const float *__restrict__ X, const float *__restrict__ Xt,
                       bf16 *__restrict__ G4, double *loss, size_t P) {
    __shared__ double red[256];
    const double inv_n = 1.0 / (2.0 * (double)P);
    double s = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const float r0 = Y[p] - (Xt[p] - X[p]);
        const float r1 = Y[P + p] - (Xt[P + p] - X[P + p]);
        s += (double)r0 * r0 + (double)r1 * r1;
        *reinterpret_cast<__nv_bfloat162 *>(G4 + p * 16) =
            __floats2bfloat162_rn((float)(2.0 * r0 * inv_n), (float)(2.0 * r1 * inv_n));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_n);
}

struct WeightPtrs {
    bf16 *wf[NL];   // [9][COUTP][CINP]
    bf16 *wb[NL];   // layers 2..4: [9][CIN_R = 32][GCH] (flipped taps, transposed)
    float *bias[NL];
};

// bfloat16 weight tiles for the forward and backward kernels from the fp32
// parameter vector (one thread per tile entry)
__global__ void k_weights(const float *__restrict__ prm, WeightPtrs wp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int r = i;
    for (int l = 0; l < NL; ++l) {
        const int nf = 9 * COUTP(l) * CINP(l);
        if (r < nf) {
            const int ci = r % CINP(l), co = (r / CINP(l)) % COUTP(l), tap = r / (CINP(l) * COUTP(l));
            const float v = (co < COUT_R(l) && ci < CIN_R(l)) ? prm[w_off(l) + (co * 9 + tap) * CIN_R(l) + ci] : 0.f;
            wp.wf[l][r] = __float2bfloat16_rn(v);
            return;
        }
        r -= nf;
        if (l > 0) {
            const int nb = 9 * CIN_R(l) * GCH(l);
            if (r < nb) {
                const int co = r % GCH(l), ci = (r / GCH(l)) % CIN_R(l), tp = r / (GCH(l) * CIN_R(l));
                const float v = co < COUT_R(l) ? prm[w_off(l) + (co * 9 + (8 - tp)) * CIN_R(l) + ci] : 0.f;
                wp.wb[l][r] = __float2bfloat16_rn(v);
                return;
            }
            r -= nb;
        }
        if (r < COUTP(l)) {
            wp.bias[l][r] = r < COUT_R(l) ? prm[b_off(l) + r] : 0.f;
            return;
        }
        r -= COUTP(l);
    }
}

int weight_entries() {
    int n = 0;
    for (int l = 0; l < NL; ++l) n += 9 * COUTP(l) * CINP(l) + (l > 0 ? 9 * CIN_R(l) * GCH(l) : 0) + COUTP(l);
    return n;
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int n, float lr, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

__global__ void k_encode(const double *__restrict__ rho, const double *__restrict__ T, float *__restrict__ X,
                         size_t P, double rho_c, double T_c, double s_rho, double s_T, double T_run) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        X[p] = (float)(s_rho * (rho[p] / rho_c - 1.0));
        X[P + p] = (float)(s_T * (T[p] / T_run - 1.0));
        X[2 * P + p] = (float)(T_run / T_c - 0.75);
    }
}

__global__ void k_decode(const float *__restrict__ X, const float *__restrict__ Y, double *__restrict__ rho,
                         double *__restrict__ u, double *__restrict__ T, size_t P, double rho_c, double s_rho,
                         double s_T, double T_run) {
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        rho[p] = rho_c * (1.0 + ((double)X[p] + (double)Y[p]) / s_rho);
        T[p] = T_run * (1.0 + ((double)X[P + p] + (double)Y[P + p]) / s_T);
        u[p] = 0.0;
    }
}

}  // namespace

struct fftlb_cnn_s {
    int H = 0, W = 0;
    size_t P = 0;
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    float *prm = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    float *X = nullptr, *Xt = nullptr, *Y = nullptr;
    bf16 *A[NL] = {nullptr};   // A_0 (16 ch), A_1..A_3 (32 ch)
    bf16 *G[NL] = {nullptr};   // G_1..G_3 (32 ch) in G[0..2], G_4 (16 ch) in G[3]
    double *loss = nullptr, *fields = nullptr;
    WeightPtrs wp{};
    int adam_k = 0;
    int grid_conv = 1, grid_wgrad = 1;
    long launches = 0;
    std::string err;
};

namespace {

fftlb_status fail(fftlb_cnn_t c, fftlb_status code, const std::string &msg) {
    if (c) c->err = msg;
    else fftlb::set_handleless_error(msg);
    return code;
}

#define CCU(c, call)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(c, FFTLB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CLAUNCH(c)                                                                                     \
    do {                                                                                               \
        cudaError_t e_ = cudaGetLastError();                                                           \
        if (e_ != cudaSuccess) return fail(c, FFTLB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
        ++(c)->launches;                                                                               \
    } while (0)

template <typename T> fftlb_status dalloc(fftlb_cnn_t c, T **p, size_t n) {
    void *q = nullptr;
    if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FFTLB_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    c->allocs.push_back(q);
    *p = reinterpret_cast<T *>(q);
    return FFTLB_OK;
}

void release(fftlb_cnn_t c) {
    for (void *p : c->allocs) cudaFree(p);
    c->allocs.clear();
}

int grid1d(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

fftlb_status refresh_weights(fftlb_cnn_t c) {
    const int n = weight_entries();
    k_weights<<<(n + 255) / 256, 256, 0, c->stream>>>(c->prm, c->wp);
    CLAUNCH(c);
    return FFTLB_OK;
}

fftlb_status upload(fftlb_cnn_t c, float *dst, const float *src, size_t n, int on_device) {
    if (!src) return fail(c, FFTLB_ERR_ARG, "NULL buffer");
    CCU(c, cudaMemcpyAsync(dst, src, n * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           c->stream));
    return FFTLB_OK;
}

// forward from c->X (device); output in c->Y
fftlb_status forward(fftlb_cnn_t c) {
    const int H = c->H, W = c->W, gc = c->grid_conv;
    k_prep<<<grid1d(c->P), 256, 0, c->stream>>>(c->X, c->A[0], c->P);
    CLAUNCH(c);
    k_conv<16, 32, FWD_RELU><<<gc, NTH, 0, c->stream>>>(c->A[0], c->wp.wf[0], c->wp.bias[0], c->A[1], nullptr, H, W);
    CLAUNCH(c);
    k_conv<32, 32, FWD_RELU><<<gc, NTH, 0, c->stream>>>(c->A[1], c->wp.wf[1], c->wp.bias[1], c->A[2], nullptr, H, W);
    CLAUNCH(c);
    k_conv<32, 32, FWD_RELU><<<gc, NTH, 0, c->stream>>>(c->A[2], c->wp.wf[2], c->wp.bias[2], c->A[3], nullptr, H, W);
    CLAUNCH(c);
    k_conv<32, 8, FWD_LAST><<<gc, NTH, 0, c->stream>>>(c->A[3], c->wp.wf[3], c->wp.bias[3], c->Y, nullptr, H, W);
    CLAUNCH(c);
    return FFTLB_OK;
}

// loss and parameter gradient (c->grad, c->loss) for c->X, c->Xt
fftlb_status backward(fftlb_cnn_t c) {
    const int H = c->H, W = c->W, gc = c->grid_conv, gw = c->grid_wgrad;
    fftlb_status s = forward(c);
    if (s != FFTLB_OK) return s;
    CCU(c, cudaMemsetAsync(c->grad, 0, FFTLB_CNN_NPARAMS * sizeof(float), c->stream));
    CCU(c, cudaMemsetAsync(c->loss, 0, sizeof(double), c->stream));
    k_loss<<<grid1d(c->P), 256, 0, c->stream>>>(c->Y, c->X, c->Xt, c->G[3], c->loss, c->P);
    CLAUNCH(c);
    const int gb = std::min<int>(1024, (int)((c->P + 255) / 256));
    // layer 4
    k_wgrad<32, 16><<<gw, NTH, 0, c->stream>>>(c->G[3], c->A[3], c->grad + w_off(3), COUT_R(3), CIN_R(3), H, W);
    CLAUNCH(c);
    k_bgrad<16><<<gb, 256, 0, c->stream>>>(c->G[3], c->grad + b_off(3), COUT_R(3), c->P);
    CLAUNCH(c);
    k_conv<16, 32, BWD><<<gc, NTH, 0, c->stream>>>(c->G[3], c->wp.wb[3], nullptr, c->G[2], c->A[3], H, W);
    CLAUNCH(c);
    // layers 3, 2
    for (int l = 2; l >= 1; --l) {
        k_wgrad<32, 32><<<gw, NTH, 0, c->stream>>>(c->G[l], c->A[l], c->grad + w_off(l), COUT_R(l), CIN_R(l), H, W);
        CLAUNCH(c);
        k_bgrad<32><<<gb, 256, 0, c->stream>>>(c->G[l], c->grad + b_off(l), COUT_R(l), c->P);
        CLAUNCH(c);
        k_conv<32, 32, BWD><<<gc, NTH, 0, c->stream>>>(c->G[l], c->wp.wb[l], nullptr, c->G[l - 1], c->A[l], H, W);
        CLAUNCH(c);
    }
    // layer 1
    k_wgrad<16, 32><<<gw, NTH, 0, c->stream>>>(c->G[0], c->A[0], c->grad + w_off(0), COUT_R(0), CIN_R(0), H, W);
    CLAUNCH(c);
    k_bgrad<32><<<gb, 256, 0, c->stream>>>(c->G[0], c->grad + b_off(0), COUT_R(0), c->P);
    CLAUNCH(c);
    return FFTLB_OK;
}

fftlb_status check_norm(fftlb_cnn_t c, const fftlb_cnn_norm *nm, double T_run) {
    if (!nm) return fail(c, FFTLB_ERR_ARG, "NULL norm");
    if (!(nm->rho_c > 0) || !(nm->T_c > 0) || !(nm->s_rho > 0) || !(nm->s_T > 0) || !(T_run > 0))
        return fail(c, FFTLB_ERR_ARG, "norm constants and T_run must be > 0");
    return FFTLB_OK;
}

fftlb_status encode_from(fftlb_cnn_t c, fftlb_t h, double T_run, const fftlb_cnn_norm *nm, float *X) {
    fftlb::Engine *e = fftlb::engine_of(h);
    if (!e) return fail(c, FFTLB_ERR_ARG, "NULL handle");
    if (e->params().nx != c->W || e->params().ny != c->H)
        return fail(c, FFTLB_ERR_ARG, "handle grid differs from the network's grid");
    fftlb_status s = check_norm(c, nm, T_run);
    if (s != FFTLB_OK) return s;
    double *rho = c->fields, *ux = rho + c->P, *uy = ux + c->P, *T = uy + c->P;
    fftlb::Status st = e->fields(rho, ux, uy, T, true);
    if (!st.good()) return fail(c, st.code, st.msg);
    // the engine works on its own stream: order ours after it
    CCU(c, cudaStreamSynchronize(e->stream()));
    k_encode<<<grid1d(c->P), 256, 0, c->stream>>>(rho, T, X, c->P, nm->rho_c, nm->T_c, nm->s_rho, nm->s_T, T_run);
    CLAUNCH(c);
    return FFTLB_OK;
}

}  // namespace

extern "C" {

fftlb_status fftlb_cnn_create(fftlb_cnn_t *out, int H, int W, void *cuda_stream) {
    if (!out) return fail(nullptr, FFTLB_ERR_ARG, "fftlb_cnn_create: out is NULL");
    *out = nullptr;
    if (H < 1 || W < TX || W > 4096 || W % TX != 0 || H > 4096)
        return fail(nullptr, FFTLB_ERR_ARG, "grid must have 1 <= H <= 4096 and W a multiple of 64 in [64, 4096]");
    fftlb_cnn_t c = new (std::nothrow) fftlb_cnn_s();
    if (!c) return fail(nullptr, FFTLB_ERR_OOM, "host allocation failed");
    c->H = H;
    c->W = W;
    c->P = (size_t)H * W;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    auto bad = [&](fftlb_status s) {
        const std::string m = c->err;
        release(c);
        delete c;
        return fail(nullptr, s, m);
    };
    const size_t P = c->P;
    fftlb_status s = FFTLB_OK;
    if ((s = dalloc(c, &c->prm, FFTLB_CNN_NPARAMS)) || (s = dalloc(c, &c->m, FFTLB_CNN_NPARAMS)) ||
        (s = dalloc(c, &c->v, FFTLB_CNN_NPARAMS)) || (s = dalloc(c, &c->grad, FFTLB_CNN_NPARAMS)) ||
        (s = dalloc(c, &c->X, 3 * P)) || (s = dalloc(c, &c->Xt, 2 * P)) || (s = dalloc(c, &c->Y, 2 * P)) ||
        (s = dalloc(c, &c->A[0], 16 * P)) || (s = dalloc(c, &c->A[1], 32 * P)) || (s = dalloc(c, &c->A[2], 32 * P)) ||
        (s = dalloc(c, &c->A[3], 32 * P)) || (s = dalloc(c, &c->G[0], 32 * P)) || (s = dalloc(c, &c->G[1], 32 * P)) ||
        (s = dalloc(c, &c->G[2], 32 * P)) || (s = dalloc(c, &c->G[3], 16 * P)) || (s = dalloc(c, &c->loss, 1)) ||
        (s = dalloc(c, &c->fields, 4 * P)))
        return bad(s);
    for (int l = 0; l < NL; ++l) {
        if ((s = dalloc(c, &c->wp.wf[l], (size_t)9 * COUTP(l) * CINP(l))) || (s = dalloc(c, &c->wp.bias[l], COUTP(l))))
            return bad(s);
        c->wp.wb[l] = nullptr;
        if (l > 0 && (s = dalloc(c, &c->wp.wb[l], (size_t)9 * CIN_R(l) * GCH(l)))) return bad(s);
    }
    if (cudaMemset(c->prm, 0, FFTLB_CNN_NPARAMS * sizeof(float)) != cudaSuccess ||
        cudaMemset(c->m, 0, FFTLB_CNN_NPARAMS * sizeof(float)) != cudaSuccess ||
        cudaMemset(c->v, 0, FFTLB_CNN_NPARAMS * sizeof(float)) != cudaSuccess ||
        cudaMemset(c->G[3], 0, 16 * P * sizeof(bf16)) != cudaSuccess) {
        c->err = "cudaMemset failed";
        return bad(FFTLB_ERR_CUDA);
    }
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = H * (W / TX);
    c->grid_conv = std::max(1, std::min(ntiles, 4 * nsm));
    c->grid_wgrad = std::max(1, std::min(ntiles, nsm));   // fewer blocks: fewer fp32 atomics per weight
    if ((s = refresh_weights(c)) != FFTLB_OK) return bad(s);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        c->err = "initial weight tiles failed";
        return bad(FFTLB_ERR_CUDA);
    }
    *out = c;
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_destroy(fftlb_cnn_t c) {
    if (!c) return FFTLB_OK;
    cudaStreamSynchronize(c->stream);
    release(c);
    delete c;
    return FFTLB_OK;
}

const char *fftlb_cnn_last_error(fftlb_cnn_t c) { return c ? c->err.c_str() : fftlb_last_error(nullptr); }

fftlb_status fftlb_cnn_set_params(fftlb_cnn_t c, const float *params, int reset_optimizer) {
    if (!c || !params) return fail(c, FFTLB_ERR_ARG, "NULL argument");
    CCU(c, cudaMemcpyAsync(c->prm, params, FFTLB_CNN_NPARAMS * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    if (reset_optimizer) {
        CCU(c, cudaMemsetAsync(c->m, 0, FFTLB_CNN_NPARAMS * sizeof(float), c->stream));
        CCU(c, cudaMemsetAsync(c->v, 0, FFTLB_CNN_NPARAMS * sizeof(float), c->stream));
        c->adam_k = 0;
    }
    fftlb_status s = refresh_weights(c);
    if (s != FFTLB_OK) return s;
    CCU(c, cudaStreamSynchronize(c->stream));
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_get_params(fftlb_cnn_t c, float *params) {
    if (!c || !params) return fail(c, FFTLB_ERR_ARG, "NULL argument");
    CCU(c, cudaMemcpyAsync(params, c->prm, FFTLB_CNN_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CCU(c, cudaStreamSynchronize(c->stream));
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_forward(fftlb_cnn_t c, const float *X, float *Y, int on_device) {
    if (!c || !Y) return fail(c, FFTLB_ERR_ARG, "NULL argument");
    c->launches = 0;
    fftlb_status s = upload(c, c->X, X, 3 * c->P, on_device);
    if (s != FFTLB_OK || (s = forward(c)) != FFTLB_OK) return s;
    CCU(c, cudaMemcpyAsync(Y, c->Y, 2 * c->P * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           c->stream));
    if (!on_device) CCU(c, cudaStreamSynchronize(c->stream));
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_gradient(fftlb_cnn_t c, const float *X, const float *Xt, float *grad, double *loss,
                                int on_device) {
    if (!c) return fail(c, FFTLB_ERR_ARG, "NULL network");
    c->launches = 0;
    fftlb_status s = upload(c, c->X, X, 3 * c->P, on_device);
    if (s != FFTLB_OK || (s = upload(c, c->Xt, Xt, 2 * c->P, on_device)) != FFTLB_OK || (s = backward(c)) != FFTLB_OK)
        return s;
    if (grad)
        CCU(c, cudaMemcpyAsync(grad, c->grad, FFTLB_CNN_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (loss) CCU(c, cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CCU(c, cudaStreamSynchronize(c->stream));
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_train_step(fftlb_cnn_t c, const float *X, const float *Xt, float lr, double *loss,
                                  int on_device) {
    if (!c) return fail(c, FFTLB_ERR_ARG, "NULL network");
    if (!(lr > 0)) return fail(c, FFTLB_ERR_ARG, "lr must be > 0");
    c->launches = 0;
    fftlb_status s = upload(c, c->X, X, 3 * c->P, on_device);
    if (s != FFTLB_OK || (s = upload(c, c->Xt, Xt, 2 * c->P, on_device)) != FFTLB_OK || (s = backward(c)) != FFTLB_OK)
        return s;
    ++c->adam_k;
    const float bc1 = 1.f - (float)std::pow(0.9, c->adam_k), bc2 = 1.f - (float)std::pow(0.999, c->adam_k);
    k_adam<<<(FFTLB_CNN_NPARAMS + 255) / 256, 256, 0, c->stream>>>(c->prm, c->m, c->v, c->grad, FFTLB_CNN_NPARAMS, lr,
                                                                   bc1, bc2);
    CLAUNCH(c);
    if ((s = refresh_weights(c)) != FFTLB_OK) return s;
    if (loss) {
        CCU(c, cudaMemcpyAsync(loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CCU(c, cudaStreamSynchronize(c->stream));
    }
    return FFTLB_OK;
}

fftlb_status fftlb_cnn_encode(fftlb_cnn_t c, fftlb_t h, double T_run, const fftlb_cnn_norm *norm, float *X_dev) {
    if (!c || !X_dev) return fail(c, FFTLB_ERR_ARG, "NULL argument");
    return encode_from(c, h, T_run, norm, X_dev);
}

fftlb_status fftlb_cnn_warm_start(fftlb_cnn_t c, fftlb_t h, double T_run, const fftlb_cnn_norm *norm) {
    if (!c) return fail(c, FFTLB_ERR_ARG, "NULL network");
    c->launches = 0;
    fftlb_status s = encode_from(c, h, T_run, norm, c->X);
    if (s != FFTLB_OK || (s = forward(c)) != FFTLB_OK) return s;
    double *rho = c->fields, *u = rho + c->P, *T = u + c->P;
    k_decode<<<grid1d(c->P), 256, 0, c->stream>>>(c->X, c->Y, rho, u, T, c->P, norm->rho_c, norm->s_rho, norm->s_T,
                                                  T_run);
    CLAUNCH(c);
    CCU(c, cudaStreamSynchronize(c->stream));
    fftlb::Engine *e = fftlb::engine_of(h);
    const long steps = e->steps();
    fftlb::Status st = e->set_fields(rho, u, u, T, true);
    if (!st.good()) return fail(c, st.code, st.msg);
    e->set_steps(steps);
    return FFTLB_OK;
}

long fftlb_cnn_launches(fftlb_cnn_t c) { return c ? c->launches : 0; }

}  // extern "C"

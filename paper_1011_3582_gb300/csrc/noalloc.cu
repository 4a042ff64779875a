// fftlb_gradient_static: the windowed spectral gradient of one fp64 field,
// computed without allocating any device memory.
//
// Who needs it: code that must not call cudaMalloc or cudaFree while it runs,
// for example a plug-in hosted by a framework whose caching allocator owns
// all device memory (a foreign cudaMalloc can fail once that pool has taken
// the GPU, and the framework cannot account for it), or a latency-critical
// loop in which an allocation's implicit device synchronisation is not
// acceptable.  Such a caller passes only its input and output buffers; the
// intermediate spectra and tables live in one fixed-size array in device
// global memory that this library defines at file scope.
//
// Cost of that choice: every GPU on which the library is loaded holds the
// array (kStaticBytes, about 1.6 MB) from module load until the process
// exits, and the grid is limited to nx * ny <= kMaxSites (nx, ny <= 1024).
// All calls share the one array and it keeps the last call's contents:
// calls that overlap on the GPU (several streams, several host threads)
// race on it and give wrong results; serialise them.
#include "engine_impl.cuh"

namespace fftlb {
void set_handleless_error(const std::string &msg);
}

namespace {

using fftlb::GroupDesc;
using fftlb::KP;
using fftlb::NT;

constexpr int kMaxLen = 1024;                 // nx, ny limit
constexpr int kMaxSites = 65536;              // nx * ny limit (e.g. 256 x 256)

// layout of the array, in doubles (each part 256-byte aligned)
constexpr size_t align32(size_t n) { return (n + 31) & ~size_t(31); }
constexpr size_t kOffSpec = 0;                                          // 3 one-sided spectra
constexpr size_t kOffKx = kOffSpec + align32(3 * (size_t)kMaxSites);     // kMaxLen/2 + 1
constexpr size_t kOffKy = kOffKx + align32(kMaxLen / 2 + 1);             // kMaxLen
constexpr size_t kOffWr = kOffKy + align32(kMaxLen);                     // kMaxLen/2 complex
constexpr size_t kOffWp = kOffWr + align32(kMaxLen);                     // kMaxLen/2 complex
constexpr size_t kOffWc = kOffWp + align32(kMaxLen);                     // kMaxLen complex
constexpr size_t kOffGrp = kOffWc + align32(2 * kMaxLen);                // one GroupDesc
constexpr size_t kTotalDoubles = kOffGrp + align32((sizeof(GroupDesc) + 7) / 8);
constexpr size_t kStaticBytes = kTotalDoubles * sizeof(double);
static_assert(kStaticBytes < 2 * 1024 * 1024, "static scratch stays below 2 MB");

static __device__ __align__(256) double g_static_scratch[kTotalDoubles];


bool valid_len(int n) {
    if (n < 4 || n > kMaxLen || (n & 1)) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// Tables of one call, written into the array: windowed wavenumbers
// (Eqs. K1-K4, Nyquist bins zeroed), twiddles, and the column-pass group
// {slot 0 -> D_x in slot 1, D_y in slot 2}.
__global__ void k_static_tables(double *base, int nx, int ny, double dx, int window) {
    const int h = nx / 2;
    double *kx = base + kOffKx, *ky = base + kOffKy;
    double2 *Wr = reinterpret_cast<double2 *>(base + kOffWr);
    double2 *Wp = reinterpret_cast<double2 *>(base + kOffWp);
    double2 *Wc = reinterpret_cast<double2 *>(base + kOffWc);
    const int total = (h + 1) + ny + h + h + ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int j = t;
        if (j < h + 1 + ny) {
            int n, N;
            double *dst;
            if (j <= h) {
                n = j;
                N = nx;
                dst = kx + j;
            } else {
                j -= h + 1;
                n = j < ny / 2 ? j : j - ny;
                N = ny;
                dst = ky + j;
            }
            double v = 0.0;
            if (2 * n != N && 2 * n != -N) {
                if (window == 0) {
                    v = 2.0 * 3.14159265358979323846 * n / (N * dx);
                } else {
                    const double s = sinpi((double)n / N);
                    double sum = 0, c = 1.0, sp = s;
                    for (int m = 0; m < window; ++m) {   // arcsin series coefficients
                        if (m > 0) c = c * (2.0 * m - 1.0) * (2.0 * m - 1.0) / ((2.0 * m) * (2.0 * m + 1.0));
                        sum += c * sp;
                        sp *= s * s;
                    }
                    v = sum * 2.0 / dx;
                }
            }
            *dst = v;
            continue;
        }
        j -= h + 1 + ny;
        double s, c;
        if (j < h) {   // Wr[m] = exp(-2 pi i m / h)
            sincospi(2.0 * j / h, &s, &c);
            Wr[j] = make_double2(c, -s);
        } else if (j < 2 * h) {   // Wp[k] = exp(-2 pi i k / nx)
            j -= h;
            sincospi(2.0 * j / nx, &s, &c);
            Wp[j] = make_double2(c, -s);
        } else {   // Wc[m] = exp(-2 pi i m / ny)
            j -= 2 * h;
            sincospi(2.0 * j / ny, &s, &c);
            Wc[j] = make_double2(c, -s);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        GroupDesc *g = reinterpret_cast<GroupDesc *>(base + kOffGrp);
        memset(g, 0, sizeof(GroupDesc));
        g->nin = 1;
        g->nout = 2;
        g->in_slot[0] = 0;
        g->out_slot[0] = 1;
        g->out_slot[1] = 2;
        g->nterm[0] = g->nterm[1] = 1;
        g->c[0][0][0] = 1.0;   // i k_x
        g->c[1][0][1] = 1.0;   // i k_y
    }
}

fftlb_status fail(fftlb_status code, const std::string &msg) {
    fftlb::set_handleless_error(msg);
    return code;
}

// With the caller's device current: the device address of the array (host
// code may not use the symbol itself as a device address) and the
// shared-memory opt-in of the column kernel.  Both are looked up again on
// every call: they are cheap, allocate nothing, and stay right after a
// device reset, which loads the module into a new context (a cached address
// would then name memory the array no longer occupies).
fftlb_status setup(int dev, double **addr, int *budget) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return fail(FFTLB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    int maxsm = 0;
    e = cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return fail(FFTLB_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    const int budget_b = maxsm - 2048;
    e = cudaFuncSetAttribute(fftlb::k_col<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget_b);
    if (e != cudaSuccess) return fail(FFTLB_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    *addr = reinterpret_cast<double *>(p);
    *budget = budget_b;
    return FFTLB_OK;
}

}  // namespace

extern "C" fftlb_status fftlb_gradient_static(const double *g, double *out, int nx, int ny, double dx, int window,
                                              void *cuda_stream) {
    if (!g || !out) return fail(FFTLB_ERR_ARG, "fftlb_gradient_static: NULL buffer");
    if (!valid_len(nx) || !valid_len(ny))
        return fail(FFTLB_ERR_ARG, "fftlb_gradient_static: nx, ny must be even 2^p 3^q in [4, 1024]");
    if ((long)nx * ny > kMaxSites)
        return fail(FFTLB_ERR_ARG, "fftlb_gradient_static: nx * ny = " + std::to_string((long)nx * ny) +
                                       " exceeds the static scratch limit of " + std::to_string(kMaxSites) + " sites");
    if (!(dx > 0) || window < 0 || window > 4)
        return fail(FFTLB_ERR_ARG, "fftlb_gradient_static: need dx > 0 and window in 0..4");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FFTLB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    double *base = nullptr;
    int budget = 0;
    fftlb_status st = setup(dev, &base, &budget);
    if (st != FFTLB_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    using C = double2;
    const int h = nx / 2;
    KP<double> kp{};
    kp.nx = nx;
    kp.ny = ny;
    kp.h = h;
    kp.dx = dx;
    kp.scale = 1.0 / ((double)nx * (double)ny);
    // column tile width, as in the handle path
    int TW = 1;
    for (int tw = 8; tw >= 1; tw >>= 1) {
        if (h % tw || tw * ny > 16 * NT || (size_t)(ny + 2 * tw * ny) * sizeof(C) > (size_t)budget) continue;
        TW = tw;
        break;
    }
    C *spec = reinterpret_cast<C *>(base + kOffSpec);
    C *Wr = reinterpret_cast<C *>(base + kOffWr), *Wp = reinterpret_cast<C *>(base + kOffWp);
    C *Wc = reinterpret_cast<C *>(base + kOffWc);
    const GroupDesc *grp = reinterpret_cast<const GroupDesc *>(base + kOffGrp);
    k_static_tables<<<8, 256, 0, s>>>(base, nx, ny, dx, window);
    const size_t smem_rows = (size_t)3 * h * sizeof(C);
    fftlb::k_rows_forward<double, double><<<dim3(ny, 1), NT, smem_rows, s>>>(g, spec, 0, Wr, Wp, kp);
    fftlb::k_col<double><<<dim3(h / TW, 1), NT, (size_t)(ny + 2 * TW * ny) * sizeof(C), s>>>(
        spec, grp, base + kOffKx, base + kOffKy, Wc, kp, TW, 1);
    fftlb::k_rows_inverse<double, double><<<dim3(ny, 2), NT, smem_rows, s>>>(spec, 1, out, Wr, Wp, kp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FFTLB_ERR_CUDA, std::string("fftlb_gradient_static launch: ") + cudaGetErrorString(e));
    return FFTLB_OK;
}

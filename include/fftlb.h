/*
 * fftlb.h - C ABI of libfftlb.so, a GB300 (sm_103a) implementation of the
 * windowed-FFT lattice-Boltzmann method for thermal liquid-vapour systems of
 * Gan, Xu, Zhang and Li, "FFT-LB modeling of thermal liquid-vapor systems"
 * (arXiv:1011.3582).
 *
 * The problem a handle holds is the paper's: a periodic nx x ny grid with
 * dx = dy (Sec. 3, periodic boundary conditions), the 33-velocity model of
 * Sec. 2.1 (Eq. 1), the BGK equation with the Gonnella-Lamura-Sofonea force
 * term of Sec. 2.2 (Eqs. 10-23) for the van der Waals EOS
 * P = rho T / (1 - b rho) - a rho^2 (Eq. 18 with general a, b), and every
 * spatial derivative taken by the windowed FFT of Sec. 3.6 (Eqs. FT, IFT,
 * FFT, K1-K4).
 *
 * Conventions shared by every call:
 *  - Fields are row-major [ny][nx] (x fastest).  The distribution function is
 *    [33][ny][nx], velocity j in the order of Eq. 1: j = 0 is v_0 = 0, and
 *    j = 1 + 8 (k-1) + (i-1) is v_ki = v_k (cos((i-1) pi/4), sin((i-1) pi/4)).
 *  - Host/device: a pointer argument is host memory unless the call's
 *    `on_device` flag is non-zero, in which case it is device memory on the
 *    handle's device.  The caller owns every buffer it passes; the library
 *    reads or writes it only during the call (asynchronously on the handle's
 *    stream for device pointers; host copies are complete when the call
 *    returns).
 *  - Streams: the handle works on the CUDA stream passed to fftlb_create
 *    (borrowed, not owned; NULL = the legacy default stream).
 *  - Errors: every call returns an fftlb_status; none aborts, traps or prints.
 *    fftlb_last_error(h) gives a message for the last failing call on h.
 *  - Memory: fftlb_create allocates all device memory the handle needs
 *    (cudaMalloc) and fftlb_destroy frees it; no other call allocates.
 */
#ifndef FFTLB_H
#define FFTLB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fftlb_s *fftlb_t;

typedef enum {
    FFTLB_OK = 0,
    FFTLB_ERR_ARG = 1,      /* invalid argument (sizes, parameters, NULL) */
    FFTLB_ERR_OOM = 2,      /* device allocation failed */
    FFTLB_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    FFTLB_ERR_UNSTABLE = 4, /* non-finite or unphysical state detected */
    FFTLB_ERR_TIMEOUT = 5,  /* a bounded device wait ran out */
    FFTLB_ERR_STATE = 6     /* call not valid in the handle's state */
} fftlb_status;

/* Problem parameters (Sec. 2.2, Sec. 3; paper defaults in brackets).
 *  nx, ny      grid; each an even 2^p 3^q with 4 <= n <= 1024 (fp64) or
 *              <= 2048 (fp32)
 *  dx          lattice spacing, dx = dy [1/256]
 *  dt          time step [1e-5]
 *  tau         BGK relaxation time (Eq. 2) [1e-2]
 *  a, b        vdW constants of P^w (Eq. 18) [9/8, 1/3]
 *  K, H        M = K + H T (Eq. 19) [1e-5, 0]
 *  q           heat-flux parameter of C_q (Eq. 23) [-0.004]
 *  zeta        bulk viscosity (Eqs. 21, 22) [0]
 *  window      0 = exact k; 1..4 = k_1..k_4 of Eqs. K1-K4 [4]
 *  integrator  1 = forward Euler, 3 = SSP-RK3 (Shu-Osher)
 *  precision   64 = everything in fp64; 32 = FFTs and pointwise in fp32
 *              (conservation sums still fp64); 32 | FFTLB_BF16SPLIT = fp32
 *              with the first radix-16 pass of every power-of-two row and
 *              column transform computed on the tensor cores as a DFT
 *              matrix product, operands split into bfloat16 hi + lo parts,
 *              fp32 accumulation (about 2^-16 relative error in that pass
 *              against 2^-24 in fp32; other lengths unchanged)
 *  check_every fftlb_step checks the state for non-finite or unphysical
 *              values every check_every steps (0 = never)
 */
#define FFTLB_BF16SPLIT 256

typedef struct {
    int nx, ny;
    double dx, dt, tau, a, b, K, H, q, zeta;
    int window, integrator, precision, check_every;
} fftlb_params;

/* Velocity set of Eq. 1: nspeeds rings of ndirs directions.  Only
 * nspeeds = 4, ndirs = 8 is supported; speeds = NULL selects the paper's
 * (1.0, 1.9, 2.9, 4.3).  The set lives in device constant memory shared by
 * all handles (and batches) of one precision in the process: while any of
 * them is alive, a create with other speeds fails with FFTLB_ERR_ARG. */
typedef struct {
    int nspeeds;
    const double *speeds;
    int ndirs;
} fftlb_velset;

/* Create a handle for problem *p on the current CUDA device.  velset may be
 * NULL (paper's set).  cuda_stream is a cudaStream_t (may be NULL).
 * Allocates ~ (2*33 + 38 + 15 + 5 + 7) nx ny values of the chosen precision.
 * Errors: FFTLB_ERR_ARG (sizes, tau <= 0, window, integrator, precision,
 * a velocity set other than that of live handles of the same precision),
 * FFTLB_ERR_OOM, FFTLB_ERR_CUDA.  On error *h is set to NULL. */
fftlb_status fftlb_create(fftlb_t *h, const fftlb_params *p,
                          const fftlb_velset *velset, void *cuda_stream);

/* Set f = f^eq(rho, u, T) (Eq. 3) from fp64 fields [ny][nx] and reset the
 * step counter.  Requires rho > 0, T > 0 and b rho < 1 where checked. */
fftlb_status fftlb_set_fields(fftlb_t h, const double *rho, const double *ux,
                              const double *uy, const double *T, int on_device);

/* Advance nsteps time steps (each: 1 stage for Euler, 3 for SSP-RK3),
 * asynchronously on the handle's stream, except that every check_every
 * steps the state is checked (which synchronises).  *steps_done (may be
 * NULL) receives the steps completed; on FFTLB_ERR_UNSTABLE it is the step
 * after which the bad state was seen. */
fftlb_status fftlb_step(fftlb_t h, long nsteps, long *steps_done);

/* Moments rho, u_x, u_y, T of the current f (Eqs. 7-9), as fp64 [ny][nx].
 * Any output pointer may be NULL.  Host outputs: synchronises. */
fftlb_status fftlb_fields(fftlb_t h, double *rho, double *ux, double *uy,
                          double *T, int on_device);

/* The full state f as fp64 [33][ny][nx] (get) or replace it (set). */
fftlb_status fftlb_get_f(fftlb_t h, double *f, int on_device);
fftlb_status fftlb_set_f(fftlb_t h, const double *f, int on_device);

/* Conservation sums in fp64 (Eqs. 12-17): out[0] = mass sum rho dx^2,
 * out[1], out[2] = momentum sum rho u dx^2, out[3] = total energy
 * sum e_T dx^2 with e_T = rho T - a rho^2 + K |grad rho|^2 / 2 + rho u^2 / 2
 * (grad rho by the windowed FFT), out[4] = max |u| (spurious velocity),
 * out[5] = simulated time steps * dt.  Synchronises the stream. */
fftlb_status fftlb_invariants(fftlb_t h, double out[6]);

/* Windowed spectral derivatives of caller fields (Sec. 3.6, Fig. 3; Eqs. FT,
 * IFT, FFT, K1-K4) using the handle's grid, dx and window: for each of
 * nfields real device fields g[nfields][ny][nx] (fp64) writes
 *   out[2*i]   = D_x g_i,   out[2*i+1] = D_y g_i   (device, fp64).
 * Uses the handle's scratch buffers (the handle's state f is untouched).
 * 1 <= nfields <= 16. */
fftlb_status fftlb_gradient(fftlb_t h, const double *g, double *out, int nfields);

/* Checkpoint: write / read f, the step count and the parameters (binary,
 * little-endian, with a format version).  fftlb_load requires a handle
 * created with the same nx, ny and precision. */
fftlb_status fftlb_save(fftlb_t h, const char *path);
fftlb_status fftlb_load(fftlb_t h, const char *path);

/* Free all device memory of h.  h may be NULL. */
fftlb_status fftlb_destroy(fftlb_t h);

/* Message of the last failing call on h (h may be NULL for errors from
 * fftlb_create).  Valid until the next call on the same thread. */
const char *fftlb_last_error(fftlb_t h);

/* Number of kernel launches issued by one time step (for accounting). */
int fftlb_launches_per_step(fftlb_t h);

/* Kernel timing.  fftlb_profile(h, 1) clears the counters and from then on
 * records a pair of CUDA events on the handle's stream around every launch
 * of a time step; fftlb_profile(h, 0) stops.  fftlb_profile_read fills, for
 * kernel kind k < nkinds (at most 6: see fftlb_kernel_name), the summed
 * device milliseconds ms[k], the launch count launches[k] and the
 * algorithmic bytes of one launch bytes[k] (each value the kernel must read
 * or write, counted once); any array may be NULL.  Synchronises. */
fftlb_status fftlb_profile(fftlb_t h, int enable);
fftlb_status fftlb_profile_read(fftlb_t h, double *ms, long *launches, double *bytes, int nkinds);
const char *fftlb_kernel_name(int kind);

/* Launch-parameter tuning of the pipelined stage kernels.  The runtime
 * parameters are tuning[5] = {column tile width of the convection pass,
 * column tile width of the level-1/2 passes, distribution rows per chunk of
 * the forward row kernel, convection rows per chunk of the final row kernel,
 * head buffers of the final row kernel (1 or 2)}.  fftlb_tuning reads them
 * (set = 0) or applies them (set = 1; 0 entries keep the current value;
 * FFTLB_ERR_ARG if a value is invalid or does not fit in shared memory).
 * fftlb_autotune times candidate values on the handle's current state
 * (saved and restored, so the state is unchanged) one parameter at a time,
 * keeps the fastest, and returns the best stage time in *stage_ms (may be
 * NULL).  Neither changes results: only the order of independent work. */
fftlb_status fftlb_autotune(fftlb_t h, double *stage_ms);
fftlb_status fftlb_tuning(fftlb_t h, int tuning[5], int set);

/* Test hook of the bounded device waits; the paper has no counterpart.  The
 * pipelined kernels wait for their staged copies on shared-memory barriers,
 * and every such wait gives up after a time limit (2 s), records a bit in the
 * handle's device error word and lets its block return, so that a stuck copy
 * cannot hang the GPU.  With ns > 0 (1e3 <= ns <= 1e9), every later stage
 * first launches one small kernel whose blocks wait, with the same code and
 * a limit of ns nanoseconds, on a barrier that nothing ever completes (no
 * copy is issued there); the wait runs out and sets the error word.  The
 * next call that reads the word (fftlb_step with check_every > 0,
 * fftlb_fields, fftlb_invariants) returns FFTLB_ERR_TIMEOUT, and every later
 * one does too: the word is not cleared, so the handle should be destroyed
 * (which works as usual).  ns = 0 turns the hook off.  FFTLB_ERR_ARG for
 * other values. */
fftlb_status fftlb_debug_wait_test(fftlb_t h, long long ns);

/* Batched sweep: nruns independent problems (each its own grid, parameters
 * and state; the same velocity set) advanced together.  Runs with identical
 * fftlb_params (check_every aside) form a group whose states are stored
 * back to back; every kernel of a stage is one persistent launch over the
 * rows / column tiles of all runs of the group.  One time step of every
 * group, the groups one after another on one internal stream, is captured
 * once into a CUDA graph; fftlb_batch_step(b, n) replays it n times on
 * cuda_stream (borrowed; NULL = legacy default stream).  With autotune != 0,
 * fftlb_batch_create tunes each group's launch parameters on a uniform
 * state.  check_every is ignored (no host checks inside replays); call
 * fftlb_batch_invariants to inspect a run.  Per-run calls take the run
 * index; they are ordered after the steps already launched.  Results of a
 * run are identical to those of a single handle with the same parameters.
 * Memory: as nruns single handles. */
typedef struct fftlb_batch_s *fftlb_batch_t;
fftlb_status fftlb_batch_create(fftlb_batch_t *b, int nruns, const fftlb_params *params,
                                const fftlb_velset *velset, int autotune, void *cuda_stream);
fftlb_status fftlb_batch_set_fields(fftlb_batch_t b, int run, const double *rho, const double *ux,
                                    const double *uy, const double *T, int on_device);
fftlb_status fftlb_batch_step(fftlb_batch_t b, long nsteps);
fftlb_status fftlb_batch_fields(fftlb_batch_t b, int run, double *rho, double *ux, double *uy,
                                double *T, int on_device);
fftlb_status fftlb_batch_get_f(fftlb_batch_t b, int run, double *f, int on_device);
fftlb_status fftlb_batch_invariants(fftlb_batch_t b, int run, double out[6]);
fftlb_status fftlb_batch_tuning(fftlb_batch_t b, int run, int tuning[5]);
long fftlb_batch_launches_per_step(fftlb_batch_t b);
fftlb_status fftlb_batch_destroy(fftlb_batch_t b);
const char *fftlb_batch_last_error(fftlb_batch_t b);

/* Windowed spectral gradient of one fp64 device field g[ny][nx] into
 * out[2][ny][nx] (out[0] = D_x g, out[1] = D_y g), like fftlb_gradient with
 * nfields = 1, but without a handle and without allocating device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * must not call cudaMalloc/cudaFree while they run (a plug-in inside a
 * framework whose caching allocator owns the GPU's memory, or a loop that
 * cannot afford an allocation's implicit device synchronisation).  Its
 * intermediate spectra and tables live in one fixed array in device global
 * memory (about 1.6 MB), defined by the library and held on every GPU that
 * loads it until the process exits.
 *  - Limits: nx, ny even 2^p 3^q in [4, 1024] and nx * ny <= 65536; larger
 *    grids return FFTLB_ERR_ARG with a message (fftlb_last_error(NULL)).
 *  - Every call looks up the array's device address and sets a kernel
 *    attribute, with the caller's device current (neither allocates), so a
 *    device reset between calls is harmless.  The first call on a device
 *    may also load the library's module there: make that first call before
 *    any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents:
 *    calls that overlap on the GPU (several streams or host threads) race
 *    and give wrong results.  Serialise them.
 *  - Asynchronous on cuda_stream (a cudaStream_t, may be NULL); g and out
 *    are caller-owned device buffers. */
fftlb_status fftlb_gradient_static(const double *g, double *out, int nx, int ny,
                                   double dx, int window, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FFTLB_H */

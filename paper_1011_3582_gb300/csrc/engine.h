// Precision-independent interface between the C ABI (api.cu) and the
// templated engine (engine_impl.cuh, instantiated in engine_f64.cu and
// engine_f32.cu).
#pragma once

#include <cuda_runtime.h>
#include <string>

#include "../../include/fftlb.h"

namespace fftlb {

struct Status {
    fftlb_status code = FFTLB_OK;
    std::string msg;
    static Status ok() { return Status(); }
    static Status err(fftlb_status c, const std::string &m) {
        Status s;
        s.code = c;
        s.msg = m;
        return s;
    }
    bool good() const { return code == FFTLB_OK; }
};

class Engine {
  public:
    virtual ~Engine() {}
    // nrun independent runs of the same grid and parameters, advanced
    // together by step / enqueue_step; per-run calls (set_fields, fields,
    // get_f, set_f, invariants, gradient) act on the run chosen by
    // select_run (run 0 after init)
    virtual Status init(const fftlb_params &p, const double speeds[4], cudaStream_t s, int nrun) = 0;
    virtual Status select_run(int run) = 0;
    virtual int nrun() const = 0;
    virtual Status set_fields(const double *rho, const double *ux, const double *uy, const double *T,
                              bool on_device) = 0;
    virtual Status step(long nsteps, long *done) = 0;
    virtual Status fields(double *rho, double *ux, double *uy, double *T, bool on_device) = 0;
    virtual Status get_f(double *f, bool on_device) = 0;
    virtual Status set_f(const double *f, bool on_device) = 0;
    virtual Status invariants(double out[6]) = 0;
    virtual Status gradient(const double *g, double *out, int nfields) = 0;
    virtual long steps() const = 0;
    virtual void set_steps(long s) = 0;
    virtual int launches_per_step() const = 0;
    virtual const fftlb_params &params() const = 0;
    // kernel timing: CUDA events around every stage launch, by kernel kind
    virtual Status profile(int enable) = 0;
    virtual Status profile_read(double *ms, long *launches, double *bytes, int nkinds) = 0;
    // one time step enqueued on the handle's stream with no host
    // synchronisation (no state checks): capturable in a CUDA graph
    virtual Status enqueue_step() = 0;
    virtual cudaStream_t stream() const = 0;
    // launch-parameter tuning: the runtime parameters of the pipelined
    // kernels (column tile widths, row-chunk sizes, head buffering)
    static constexpr int NTUNE = 5;
    virtual void get_tuning(int t[NTUNE]) const = 0;
    virtual Status set_tuning(const int t[NTUNE]) = 0;
    // times candidate parameters on the current state (saved and restored)
    // and keeps the fastest; *stage_ms receives the best stage time
    virtual Status autotune(double *stage_ms) = 0;
    // test hook of the bounded device waits: ns > 0 makes every stage start
    // with a kernel whose wait nothing completes (limit ns); 0 turns it off
    virtual Status set_wait_test(long long ns) = 0;
};

// kernel kinds of one stage (index into the profile arrays)
enum KernelKind {
    KK_ROW_FORWARD = 0,   // moments + forward row transforms
    KK_COL_CONV = 1,      // column pass, convection
    KK_COL_LEVEL1 = 2,    // column pass, level-1 derivatives
    KK_ROW_LEVEL1 = 3,    // level-1 row inverse + Lambda/Phi + forward rows
    KK_COL_LEVEL2 = 4,    // column pass, level-2 divergences
    KK_ROW_FINAL = 5,     // row inverse + force + BGK + RK combination
    KK_COUNT = 6
};
extern const char *const kKernelNames[KK_COUNT];

Engine *make_engine_f64();
Engine *make_engine_f32();
Engine *make_engine_f32_split();   // precision 32 | FFTLB_BF16SPLIT

// the engine behind a handle (NULL for a NULL handle); defined in api.cu
Engine *engine_of(fftlb_t h);
void set_handleless_error(const std::string &msg);

}  // namespace fftlb

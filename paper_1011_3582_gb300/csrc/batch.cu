// Batched sweep of independent FFT-LB runs (a phase-diagram sweep: many
// grids and temperatures, arXiv:1011.3582 Sec. 4.1) advanced together: one
// time step of every run, the runs one after another on one internal
// stream, is captured once into a CUDA graph, and every fftlb_batch_step
// replays the graph on the caller's stream (one graph launch per step
// instead of 18 kernel launches per run).  The persistent kernels of one
// run already spread over every SM, so the runs are not overlapped.  Runs
// of the same grid shape and precision share the launch parameters picked
// by the engine's autotuner.  Declarations and contracts: include/fftlb.h.
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace fftlb {
void set_handleless_error(const std::string &msg);
}

struct fftlb_batch_s {
    std::vector<fftlb::Engine *> eng;
    cudaStream_t origin = nullptr;   // every run's stream and the capture stream (owned)
    cudaStream_t user = nullptr;     // caller's stream (borrowed)
    cudaEvent_t ready = nullptr, done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long steps = 0;
    int graph_steps = 1;
    std::string err;
};

namespace {

fftlb_status fail(fftlb_batch_t b, fftlb_status code, const std::string &msg) {
    if (b) b->err = msg;
    else fftlb::set_handleless_error(msg);
    return code;
}

fftlb_status fail(fftlb_batch_t b, const fftlb::Status &st) { return fail(b, st.code, st.msg); }

#define BCU(b, call)                                                                             \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(b, FFTLB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void release(fftlb_batch_t b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto *e : b->eng) delete e;
    if (b->ready) cudaEventDestroy(b->ready);
    if (b->done) cudaEventDestroy(b->done);
    if (b->origin) cudaStreamDestroy(b->origin);
}

// the graph of graph_steps steps of every run, in run order
fftlb_status build_graph(fftlb_batch_t b) {
    if (b->exec) return FFTLB_OK;
    BCU(b, cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal));
    fftlb::Status st;
    for (size_t r = 0; r < b->eng.size() && st.good(); ++r)
        for (int s = 0; s < b->graph_steps && st.good(); ++s) st = b->eng[r]->enqueue_step();
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->origin, &g);
    if (!st.good()) {
        if (g) cudaGraphDestroy(g);
        return fail(b, st);
    }
    if (ee != cudaSuccess) return fail(b, FFTLB_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
    b->graph = g;
    BCU(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
    return FFTLB_OK;
}

// order the runs' stream after the graph launches on the caller's stream
fftlb_status after_graph(fftlb_batch_t b) {
    BCU(b, cudaEventRecord(b->done, b->user));
    BCU(b, cudaStreamWaitEvent(b->origin, b->done, 0));
    return FFTLB_OK;
}

}  // namespace

extern "C" {

fftlb_status fftlb_batch_create(fftlb_batch_t *out, int nruns, const fftlb_params *params, const fftlb_velset *vs,
                                int autotune, void *cuda_stream) {
    if (!out) return fail(nullptr, FFTLB_ERR_ARG, "fftlb_batch_create: out is NULL");
    *out = nullptr;
    if (nruns < 1 || nruns > 4096 || !params)
        return fail(nullptr, FFTLB_ERR_ARG, "fftlb_batch_create: need 1 <= nruns <= 4096 and params");
    double speeds[4] = {1.0, 1.9, 2.9, 4.3};   // Sec. 2.1, after Eq. 1
    if (vs) {
        if (vs->nspeeds != 4 || vs->ndirs != 8)
            return fail(nullptr, FFTLB_ERR_ARG, "velocity set: only 4 speeds x 8 directions is supported");
        if (vs->speeds)
            for (int i = 0; i < 4; ++i) speeds[i] = vs->speeds[i];
    }
    for (int r = 0; r < nruns; ++r)
        if (params[r].precision != 64 && params[r].precision != 32)
            return fail(nullptr, FFTLB_ERR_ARG, "run " + std::to_string(r) + ": precision must be 64 or 32");
    fftlb_batch_t b = new (std::nothrow) fftlb_batch_s();
    if (!b) return fail(nullptr, FFTLB_ERR_OOM, "host allocation failed");
    b->user = reinterpret_cast<cudaStream_t>(cuda_stream);
    auto bad = [&](fftlb_status code, const std::string &m) {
        release(b);
        delete b;
        return fail(nullptr, code, m);
    };
    if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
        return bad(FFTLB_ERR_CUDA, "stream / event creation failed");
    std::map<std::tuple<int, int, int, int>, std::vector<int>> shapes;
    for (int r = 0; r < nruns; ++r) {
        fftlb_params p = params[r];
        p.check_every = 0;   // steps are graph replays: no host-side checks inside
        fftlb::Engine *eng = p.precision == 64 ? fftlb::make_engine_f64() : fftlb::make_engine_f32();
        b->eng.push_back(eng);
        fftlb::Status st = eng->init(p, speeds, b->origin);
        if (!st.good()) return bad(st.code, "run " + std::to_string(r) + ": " + st.msg);
        shapes[std::make_tuple(p.nx, p.ny, p.precision, p.integrator)].push_back(r);
    }
    if (autotune) {
        // tune one run per shape on a uniform equilibrium state, share the choice
        for (auto &kv : shapes) {
            const int r0 = kv.second[0];
            const fftlb_params &p = b->eng[r0]->params();
            const size_t n = (size_t)p.nx * p.ny;
            std::vector<double> rho(n, 1.0 / (3.0 * (p.b > 0 ? p.b : 1.0 / 3.0))), z(n, 0.0);
            std::vector<double> T(n, p.b > 0 ? 0.9 * 8.0 * p.a / (27.0 * p.b) : 1.0);
            fftlb::Status st = b->eng[r0]->set_fields(rho.data(), z.data(), z.data(), T.data(), false);
            double ms = 0;
            if (st.good()) st = b->eng[r0]->autotune(&ms);
            if (!st.good()) return bad(st.code, "autotune: " + st.msg);
            int t[fftlb::Engine::NTUNE];
            b->eng[r0]->get_tuning(t);
            for (int r : kv.second) {
                st = b->eng[r]->set_tuning(t);
                if (!st.good()) return bad(st.code, "autotune: " + st.msg);
            }
        }
    }
    *out = b;
    return FFTLB_OK;
}

fftlb_status fftlb_batch_set_fields(fftlb_batch_t b, int run, const double *rho, const double *ux, const double *uy,
                                    const double *T, int on_device) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (run < 0 || run >= (int)b->eng.size()) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = b->eng[run]->set_fields(rho, ux, uy, T, on_device != 0);
    if (!st.good()) return fail(b, st);
    b->eng[run]->set_steps(b->steps);
    return FFTLB_OK;
}

fftlb_status fftlb_batch_step(fftlb_batch_t b, long nsteps) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (nsteps < 0) return fail(b, FFTLB_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return FFTLB_OK;
    fftlb_status s = build_graph(b);
    if (s != FFTLB_OK) return s;
    // make the graph start after anything the runs' stream still does
    BCU(b, cudaEventRecord(b->ready, b->origin));
    BCU(b, cudaStreamWaitEvent(b->user, b->ready, 0));
    for (long i = 0; i < nsteps; i += b->graph_steps) BCU(b, cudaGraphLaunch(b->exec, b->user));
    b->steps += nsteps;
    for (auto *e : b->eng) e->set_steps(b->steps);
    return FFTLB_OK;
}

fftlb_status fftlb_batch_fields(fftlb_batch_t b, int run, double *rho, double *ux, double *uy, double *T,
                                int on_device) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (run < 0 || run >= (int)b->eng.size()) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = b->eng[run]->fields(rho, ux, uy, T, on_device != 0);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_get_f(fftlb_batch_t b, int run, double *f, int on_device) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (run < 0 || run >= (int)b->eng.size()) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = b->eng[run]->get_f(f, on_device != 0);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_invariants(fftlb_batch_t b, int run, double out[6]) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (run < 0 || run >= (int)b->eng.size() || !out) return fail(b, FFTLB_ERR_ARG, "run out of range or out NULL");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = b->eng[run]->invariants(out);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_tuning(fftlb_batch_t b, int run, int tuning[5]) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    if (run < 0 || run >= (int)b->eng.size() || !tuning) return fail(b, FFTLB_ERR_ARG, "run out of range or NULL");
    b->eng[run]->get_tuning(tuning);
    return FFTLB_OK;
}

long fftlb_batch_launches_per_step(fftlb_batch_t b) {
    if (!b) return 0;
    long n = 0;
    for (auto *e : b->eng) n += e->launches_per_step();
    return n;
}

fftlb_status fftlb_batch_destroy(fftlb_batch_t b) {
    if (!b) return FFTLB_OK;
    cudaStreamSynchronize(b->user);
    release(b);
    delete b;
    return FFTLB_OK;
}

const char *fftlb_batch_last_error(fftlb_batch_t b) { return b ? b->err.c_str() : fftlb_last_error(nullptr); }

}  // extern "C"

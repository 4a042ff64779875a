// Batched sweep of independent FFT-LB runs (a phase-diagram sweep: many
// grids and temperatures, arXiv:1011.3582 Sec. 4.1) advanced together.
// Runs that share every parameter (grid, dx, dt, tau, EOS, K, H, q, zeta,
// window, integrator, precision) form one group, held by one engine whose
// arenas store the group's runs back to back: each pipelined kernel of a
// stage is one persistent launch over the rows or column tiles of all runs
// of the group.  One time step of every group is captured once into a CUDA
// graph on one internal stream (18 kernel nodes per group for SSP-RK3),
// and every fftlb_batch_step replays the graph on the caller's stream.
// Declarations and contracts: include/fftlb.h.
#include <map>
#include <string>
#include <vector>

#include "engine.h"

namespace fftlb {
void set_handleless_error(const std::string &msg);
}

struct fftlb_batch_s {
    std::vector<fftlb::Engine *> eng;          // one per parameter group
    std::vector<std::pair<int, int>> where;    // run -> (group, index in the group)
    cudaStream_t origin = nullptr;   // every group's stream and the capture stream (owned)
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
        if (params[r].precision != 64 && params[r].precision != 32 && params[r].precision != (32 | FFTLB_BF16SPLIT))
            return fail(nullptr, FFTLB_ERR_ARG,
                        "run " + std::to_string(r) + ": precision must be 64, 32 or 32 | FFTLB_BF16SPLIT");
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
    // group runs whose parameters are identical (check_every is ignored:
    // steps are graph replays, with no host-side checks inside)
    std::map<std::string, std::vector<int>> groups;
    std::vector<std::string> order;
    for (int r = 0; r < nruns; ++r) {
        fftlb_params p = params[r];
        p.check_every = 0;
        std::string key(reinterpret_cast<const char *>(&p), sizeof p);
        if (!groups.count(key)) order.push_back(key);
        groups[key].push_back(r);
    }
    b->where.assign(nruns, std::make_pair(0, 0));
    for (size_t gi = 0; gi < order.size(); ++gi) {
        const std::vector<int> &runs = groups[order[gi]];
        fftlb_params p = params[runs[0]];
        p.check_every = 0;
        fftlb::Engine *eng = p.precision == 64 ? fftlb::make_engine_f64()
                             : p.precision == 32 ? fftlb::make_engine_f32() : fftlb::make_engine_f32_split();
        b->eng.push_back(eng);
        fftlb::Status st = eng->init(p, speeds, b->origin, (int)runs.size());
        if (!st.good()) return bad(st.code, "run " + std::to_string(runs[0]) + ": " + st.msg);
        for (size_t i = 0; i < runs.size(); ++i) b->where[runs[i]] = std::make_pair((int)gi, (int)i);
        if (autotune) {
            // tune on a uniform state (rho_c, 0.9 T_c) in every run of the group
            const size_t n = (size_t)p.nx * p.ny;
            std::vector<double> rho(n, 1.0 / (3.0 * (p.b > 0 ? p.b : 1.0 / 3.0))), z(n, 0.0);
            std::vector<double> T(n, p.b > 0 ? 0.9 * 8.0 * p.a / (27.0 * p.b) : 1.0);
            for (size_t i = 0; i < runs.size() && st.good(); ++i) {
                st = eng->select_run((int)i);
                if (st.good()) st = eng->set_fields(rho.data(), z.data(), z.data(), T.data(), false);
            }
            double ms = 0;
            if (st.good()) st = eng->autotune(&ms);
            if (!st.good()) return bad(st.code, "autotune: " + st.msg);
        }
    }
    *out = b;
    return FFTLB_OK;
}

// the engine holding a run, with that run selected (NULL if out of range)
static fftlb::Engine *run_engine(fftlb_batch_t b, int run) {
    if (run < 0 || run >= (int)b->where.size()) return nullptr;
    fftlb::Engine *e = b->eng[b->where[run].first];
    return e->select_run(b->where[run].second).good() ? e : nullptr;
}

fftlb_status fftlb_batch_set_fields(fftlb_batch_t b, int run, const double *rho, const double *ux, const double *uy,
                                    const double *T, int on_device) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    fftlb::Engine *e = run_engine(b, run);
    if (!e) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = e->set_fields(rho, ux, uy, T, on_device != 0);
    if (!st.good()) return fail(b, st);
    e->set_steps(b->steps);
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
    fftlb::Engine *e = run_engine(b, run);
    if (!e) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = e->fields(rho, ux, uy, T, on_device != 0);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_get_f(fftlb_batch_t b, int run, double *f, int on_device) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    fftlb::Engine *e = run_engine(b, run);
    if (!e) return fail(b, FFTLB_ERR_ARG, "run out of range");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = e->get_f(f, on_device != 0);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_invariants(fftlb_batch_t b, int run, double out[6]) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    fftlb::Engine *e = out ? run_engine(b, run) : nullptr;
    if (!e) return fail(b, FFTLB_ERR_ARG, "run out of range or out NULL");
    fftlb_status s = after_graph(b);
    if (s != FFTLB_OK) return s;
    fftlb::Status st = e->invariants(out);
    return st.good() ? FFTLB_OK : fail(b, st);
}

fftlb_status fftlb_batch_tuning(fftlb_batch_t b, int run, int tuning[5]) {
    if (!b) return fail(nullptr, FFTLB_ERR_ARG, "NULL batch");
    fftlb::Engine *e = tuning ? run_engine(b, run) : nullptr;
    if (!e) return fail(b, FFTLB_ERR_ARG, "run out of range or NULL");
    e->get_tuning(tuning);
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

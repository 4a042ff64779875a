// C ABI of libfftlb.so (declarations and contracts in include/fftlb.h).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

struct fftlb_s {
    fftlb::Engine *eng = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

fftlb_status fail(fftlb_t h, const fftlb::Status &st) {
    if (h) h->err = st.msg;
    else g_create_err = st.msg;
    return st.code;
}

fftlb_status fail(fftlb_t h, fftlb_status code, const std::string &msg) {
    if (h) h->err = msg;
    else g_create_err = msg;
    return code;
}

const char kMagic[8] = {'F', 'F', 'T', 'L', 'B', 'C', 'K', 'P'};
const int32_t kFormat = 1;

}  // namespace

namespace fftlb {
// lets handle-less entry points in other translation units report a message
// through fftlb_last_error(NULL)
void set_handleless_error(const std::string &msg) { g_create_err = msg; }
Engine *engine_of(fftlb_t h) { return h ? h->eng : nullptr; }

const char *const kKernelNames[KK_COUNT] = {"row_forward_moments", "col_convection", "col_level1",
                                            "row_level1",          "col_level2",     "row_final"};
}  // namespace fftlb

extern "C" {

fftlb_status fftlb_create(fftlb_t *h, const fftlb_params *p, const fftlb_velset *vs, void *stream) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "fftlb_create: h is NULL");
    *h = nullptr;
    if (!p) return fail(nullptr, FFTLB_ERR_ARG, "fftlb_create: params is NULL");
    double speeds[4] = {1.0, 1.9, 2.9, 4.3};   // Sec. 2.1, after Eq. 1
    if (vs) {
        if (vs->nspeeds != 4 || vs->ndirs != 8)
            return fail(nullptr, FFTLB_ERR_ARG, "velocity set: only 4 speeds x 8 directions is supported");
        if (vs->speeds)
            for (int i = 0; i < 4; ++i) speeds[i] = vs->speeds[i];
    }
    if (p->precision != 64 && p->precision != 32 && p->precision != (32 | FFTLB_BF16SPLIT))
        return fail(nullptr, FFTLB_ERR_ARG, "precision must be 64, 32 or 32 | FFTLB_BF16SPLIT");
    fftlb_t hh = new (std::nothrow) fftlb_s();
    if (!hh) return fail(nullptr, FFTLB_ERR_OOM, "host allocation failed");
    hh->eng = p->precision == 64 ? fftlb::make_engine_f64()
              : p->precision == 32 ? fftlb::make_engine_f32() : fftlb::make_engine_f32_split();
    fftlb::Status st = hh->eng->init(*p, speeds, reinterpret_cast<cudaStream_t>(stream), 1);
    if (!st.good()) {
        delete hh->eng;
        delete hh;
        return fail(nullptr, st);
    }
    *h = hh;
    return FFTLB_OK;
}

fftlb_status fftlb_set_fields(fftlb_t h, const double *rho, const double *ux, const double *uy, const double *T,
                              int on_device) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->set_fields(rho, ux, uy, T, on_device != 0);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_step(fftlb_t h, long nsteps, long *steps_done) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->step(nsteps, steps_done);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_fields(fftlb_t h, double *rho, double *ux, double *uy, double *T, int on_device) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->fields(rho, ux, uy, T, on_device != 0);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_get_f(fftlb_t h, double *f, int on_device) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->get_f(f, on_device != 0);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_set_f(fftlb_t h, const double *f, int on_device) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->set_f(f, on_device != 0);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_invariants(fftlb_t h, double out[6]) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    if (!out) return fail(h, FFTLB_ERR_ARG, "out is NULL");
    fftlb::Status st = h->eng->invariants(out);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_gradient(fftlb_t h, const double *g, double *out, int nfields) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->gradient(g, out, nfields);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_save(fftlb_t h, const char *path) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    if (!path) return fail(h, FFTLB_ERR_ARG, "path is NULL");
    const fftlb_params &p = h->eng->params();
    const size_t n = (size_t)33 * p.nx * p.ny;
    std::vector<double> f(n);
    fftlb::Status st = h->eng->get_f(f.data(), false);
    if (!st.good()) return fail(h, st);
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(h, FFTLB_ERR_ARG, std::string("cannot open ") + path);
    const int64_t steps = h->eng->steps();
    bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(&kFormat, sizeof kFormat, 1, fp) == 1 &&
              fwrite(&p, sizeof p, 1, fp) == 1 && fwrite(&steps, sizeof steps, 1, fp) == 1 &&
              fwrite(f.data(), sizeof(double), n, fp) == n;
    ok = (fclose(fp) == 0) && ok;
    return ok ? FFTLB_OK : fail(h, FFTLB_ERR_ARG, std::string("write failed: ") + path);
}

fftlb_status fftlb_load(fftlb_t h, const char *path) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    if (!path) return fail(h, FFTLB_ERR_ARG, "path is NULL");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(h, FFTLB_ERR_ARG, std::string("cannot open ") + path);
    char magic[8];
    int32_t fmt = 0;
    fftlb_params q;
    int64_t steps = 0;
    bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(&fmt, sizeof fmt, 1, fp) == 1 &&
              fmt == kFormat && fread(&q, sizeof q, 1, fp) == 1 && fread(&steps, sizeof steps, 1, fp) == 1;
    const fftlb_params &p = h->eng->params();
    if (!ok || q.nx != p.nx || q.ny != p.ny || q.precision != p.precision) {
        fclose(fp);
        return fail(h, FFTLB_ERR_ARG, "checkpoint does not match the handle (format, nx, ny or precision)");
    }
    const size_t n = (size_t)33 * p.nx * p.ny;
    std::vector<double> f(n);
    ok = fread(f.data(), sizeof(double), n, fp) == n;
    fclose(fp);
    if (!ok) return fail(h, FFTLB_ERR_ARG, "checkpoint truncated");
    fftlb::Status st = h->eng->set_f(f.data(), false);
    if (!st.good()) return fail(h, st);
    h->eng->set_steps((long)steps);
    return FFTLB_OK;
}

fftlb_status fftlb_destroy(fftlb_t h) {
    if (!h) return FFTLB_OK;
    delete h->eng;
    delete h;
    return FFTLB_OK;
}

const char *fftlb_last_error(fftlb_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int fftlb_launches_per_step(fftlb_t h) { return h ? h->eng->launches_per_step() : 0; }

fftlb_status fftlb_profile(fftlb_t h, int enable) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->profile(enable);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_profile_read(fftlb_t h, double *ms, long *launches, double *bytes, int nkinds) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->profile_read(ms, launches, bytes, nkinds);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_autotune(fftlb_t h, double *stage_ms) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->autotune(stage_ms);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_tuning(fftlb_t h, int tuning[5], int set) {
    if (!h || !tuning) return fail(h, FFTLB_ERR_ARG, "NULL handle or tuning");
    if (!set) {
        h->eng->get_tuning(tuning);
        return FFTLB_OK;
    }
    fftlb::Status st = h->eng->set_tuning(tuning);
    return st.good() ? FFTLB_OK : fail(h, st);
}

fftlb_status fftlb_debug_wait_test(fftlb_t h, long long ns) {
    if (!h) return fail(nullptr, FFTLB_ERR_ARG, "NULL handle");
    fftlb::Status st = h->eng->set_wait_test(ns);
    return st.good() ? FFTLB_OK : fail(h, st);
}

const char *fftlb_kernel_name(int kind) {
    return (kind >= 0 && kind < fftlb::KK_COUNT) ? fftlb::kKernelNames[kind] : "";
}

}  // extern "C"

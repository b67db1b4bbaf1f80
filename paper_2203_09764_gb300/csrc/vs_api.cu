// vs_api.cu -- the C ABI (include/vs.h): contexts, fields, load, centrifuge,
// smoothing schedule, checks and read-back.  Serving lives in vs_serve.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/vs.h"
#include "vs_api_internal.h"

using namespace vs;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

static thread_local char g_err[512] = "";

vs_status vs::fail(vs_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

vs_status vs::cuda_fail(cudaError_t e, const char *what) {
    return fail(VS_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

extern "C" const char *vs_last_error(void) { return g_err; }

extern "C" const char *vs_version(void) { return "vs 1.0 (sm_103a)"; }

extern "C" int64_t vs_kernel_launches(void) { return (int64_t)launches(); }

// ---------------------------------------------------------------------------
// Context and device memory
// ---------------------------------------------------------------------------

void *vs::dev_alloc(vs_ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (c->opt.alloc) return c->opt.alloc(bytes, c->opt.alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void vs::dev_free(vs_ctx *c, void *p) {
    if (!p) return;
    if (c->opt.free_fn) c->opt.free_fn(p, c->opt.alloc_user);
    else cudaFree(p);
}

extern "C" vs_status vs_create(const vs_options *opt, vs_ctx **out) {
    if (!out) return fail(VS_EINVAL, "vs_create: out is NULL");
    *out = nullptr;
    vs_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    if ((o.alloc == nullptr) != (o.free_fn == nullptr))
        return fail(VS_EINVAL, "vs_create: alloc and free_fn must be given together");
    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (o.device < 0 || o.device >= ndev) return fail(VS_EINVAL, "vs_create: no CUDA device %d", o.device);
    CK(cudaSetDevice(o.device));
    vs_ctx *c = new (std::nothrow) vs_ctx();
    if (!c) return fail(VS_ENOMEM, "vs_create: out of host memory");
    c->opt = o;
    if (c->opt.max_slots <= 0) c->opt.max_slots = 8;
    if (c->opt.max_queue <= 0) c->opt.max_queue = 1024;
    c->t0 = std::chrono::steady_clock::now();
    // the one-time set-up of vs_vortex_check_noalloc on this device, so that
    // its later calls allocate nothing at all; a failure here is reported by
    // the first such call instead
    vs_noalloc_prepare(o.device);
    *out = c;
    return VS_OK;
}

extern "C" void vs_destroy(vs_ctx *c) {
    if (!c) return;
    serve_shutdown(c);
    delete c;
}

extern "C" double vs_now_ms(vs_ctx *c) {
    if (!c) return 0.0;
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c->t0).count();
}

// ---------------------------------------------------------------------------
// Fields
// ---------------------------------------------------------------------------

static size_t field_bytes(const vs_field *f) {
    return (size_t)4 * f->nc * (size_t)f->g.P * (f->prec == VS_FP64 ? 8 : 4);
}

// Extents: positive multiples of 4 (the colour classes), at most 2^30 plane
// positions (the sites and the layout's unused positions, make_geo) so that
// positions and per-site loop indices fit in 32-bit ints.
bool vs::valid_dims(const int32_t d[4]) {
    long long p = 1;
    for (int k = 0; k < 4; ++k) {
        if (d[k] < 4 || d[k] % 4 || d[k] > (1 << 30)) return false;
        p *= k == 0 ? 4 * ((d[0] / 4 == 5 || d[0] / 4 == 6 || d[0] / 4 == 7) ? 8 : d[0] / 4) : d[k];
        if (p > (1ll << 30)) return false;
    }
    return true;
}

uint64_t vs::field_footprint(const int32_t dims[4], int32_t precision, int32_t storage) {
    const long long P = make_geo(dims).P;   // plane stride, with the layout's unused positions
    int nc = storage == VS_LINK12 ? 12 : 18;
    uint64_t links = (uint64_t)4 * nc * P * (precision == VS_FP64 ? 8 : 4);
    return links + 8ull * P + 1216 * 8 + 4096 + (precision == VS_FP32 ? kDeferCap * sizeof(int) : 0);
}

extern "C" vs_status vs_field_create(vs_ctx *c, const int32_t dims[4], int32_t precision, int32_t storage,
                                     void *stream, vs_field **out) {
    if (!c || !dims || !out) return fail(VS_EINVAL, "vs_field_create: NULL argument");
    *out = nullptr;
    if (!valid_dims(dims))
        return fail(VS_EINVAL,
                    "vs_field_create: extents must be positive multiples of 4 with at most 2^30 layout positions "
                    "(got %d %d %d %d)", dims[0], dims[1], dims[2], dims[3]);
    if (precision != VS_FP64 && precision != VS_FP32) return fail(VS_EINVAL, "vs_field_create: bad precision");
    if (storage != VS_LINK18 && storage != VS_LINK12) return fail(VS_EINVAL, "vs_field_create: bad storage");
    if (precision == VS_FP64 && storage == VS_LINK12)
        return fail(VS_EUNSUPPORTED, "vs_field_create: 12-real storage is built for FP32 only");
    CK(cudaSetDevice(c->opt.device));
    vs_field *f = new (std::nothrow) vs_field();
    if (!f) return fail(VS_ENOMEM, "vs_field_create: out of host memory");
    f->ctx = c;
    f->prec = precision;
    f->nc = storage == VS_LINK12 ? 12 : 18;
    f->g = make_geo(dims);
    if (stream) {
        f->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete f; return cuda_fail(e, "cudaStreamCreate"); }
        f->own_stream = true;
    }
    f->U = dev_alloc(c, field_bytes(f));
    f->ref = (int8_t *)dev_alloc(c, 4 * (size_t)f->g.P);
    f->cur = (int8_t *)dev_alloc(c, 4 * (size_t)f->g.P);
    f->partials = (double *)dev_alloc(c, 1216 * sizeof(double) + 4096);
    if (precision == VS_FP32) f->defer_idx = (int *)dev_alloc(c, kDeferCap * sizeof(int));
    if (!f->U || !f->ref || !f->cur || !f->partials || (precision == VS_FP32 && !f->defer_idx)) {
        vs_field_destroy(f);
        return fail(VS_ENOMEM, "vs_field_create: device allocation of %zu bytes failed", field_bytes(f));
    }
    // scalars live after the partials: [1216 doubles][result double][counters...]
    f->d_result = f->partials + 1216;
    f->d_counts = (unsigned long long *)(f->d_result + 1);      // 8 slots
    f->d_sweep = f->d_counts + 8;                               // kSweepSlots slots
    f->defer_n = (unsigned *)(f->d_sweep + kSweepSlots);        // 2 counters
    cudaError_t e = cudaMemsetAsync(f->defer_n, 0, 2 * sizeof(unsigned), f->stream);
    if (e != cudaSuccess) {
        vs_field_destroy(f);
        return cuda_fail(e, "vs_field_create");
    }
    *out = f;
    return VS_OK;
}

extern "C" void vs_field_destroy(vs_field *f) {
    if (!f) return;
    cudaSetDevice(f->ctx->opt.device);
    if (f->stream) cudaStreamSynchronize(f->stream);
    dev_free(f->ctx, f->U);
    dev_free(f->ctx, f->ref);
    dev_free(f->ctx, f->cur);
    dev_free(f->ctx, f->G);
    dev_free(f->ctx, f->partials);
    dev_free(f->ctx, f->defer_idx);
    dev_free(f->ctx, f->scratch);
    dev_free(f->ctx, f->flowS);
    dev_free(f->ctx, f->sweep_counts);
    dev_free(f->ctx, f->sweep_actions);
    for (auto &e : f->events) cudaEventDestroy(e);
    if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
    delete f;
}

static vs_status ensure_scratch(vs_field *f, size_t bytes) {
    if (f->scratch_bytes >= bytes) return VS_OK;
    CK(cudaStreamSynchronize(f->stream));
    dev_free(f->ctx, f->scratch);
    f->scratch = dev_alloc(f->ctx, bytes);
    f->scratch_bytes = f->scratch ? bytes : 0;
    if (!f->scratch) return fail(VS_ENOMEM, "scratch allocation of %zu bytes failed", bytes);
    return VS_OK;
}

extern "C" vs_status vs_field_describe(const vs_field *f, vs_field_desc *d) {
    if (!f || !d) return fail(VS_EINVAL, "vs_field_describe: NULL argument");
    memset(d, 0, sizeof *d);
    for (int k = 0; k < 4; ++k) d->dims[k] = f->g.L[k];
    d->precision = f->prec;
    d->storage = f->nc == 12 ? VS_LINK12 : VS_LINK18;
    d->n_sites = f->g.V;
    d->plane_stride = f->g.P;
    d->n_components = f->nc;
    d->device = f->ctx->opt.device;
    d->links = f->U;
    d->labels = f->ref;
    d->stream = (void *)f->stream;
    d->gauge = f->gauge_on ? f->G : nullptr;
    return VS_OK;
}

extern "C" int64_t vs_layout_index(const int32_t dims[4], const int32_t x[4]) {
    const Geo g = make_geo(dims);
    return sidx(g, x[0], x[1], x[2], x[3]);
}

static vs_status check_device_error(vs_field *f) {
    CK(cudaGetLastError());
    return VS_OK;
}

extern "C" vs_status vs_synchronize(vs_field *f) {
    if (!f) return fail(VS_EINVAL, "vs_synchronize: NULL field");
    CK(cudaSetDevice(f->ctx->opt.device));
    CK(cudaStreamSynchronize(f->stream));
    return check_device_error(f);
}

// ---------------------------------------------------------------------------
// Load / read
// ---------------------------------------------------------------------------

// Host labels outside {-1, 0, 1} are rejected (branch-free scan, the
// position looked up only when there is a bad one).
static vs_status check_host_labels(const int8_t *labels, size_t n, const char *what) {
    unsigned bad = 0;
    for (size_t i = 0; i < n; ++i) bad |= (unsigned)(uint8_t)(labels[i] + 1) > 2u;
    if (bad)
        for (size_t i = 0; i < n; ++i)
            if (labels[i] < -1 || labels[i] > 1)
                return fail(VS_EINVAL, "%s: label %d at %zu outside {-1,0,1}", what, labels[i], i);
    return VS_OK;
}

extern "C" vs_status vs_load_field(vs_field *f, const double *links, const int8_t *labels, int32_t where) {
    if (!f) return fail(VS_EINVAL, "vs_load_field: NULL field");
    if ((links == nullptr) == (labels == nullptr))
        return fail(VS_EINVAL, "vs_load_field: exactly one of links / labels must be given");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_load_field: bad `where`");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t V = f->g.V;
    if (labels) {
        if (where == VS_HOST) {
            vs_status st = check_host_labels(labels, 4 * V, "vs_load_field");
            if (st) return st;
        }
        const int8_t *src = labels;
        if (where == VS_HOST) {
            vs_status st = ensure_scratch(f, 4 * V);
            if (st) return st;
            CK(cudaMemcpyAsync(f->scratch, labels, 4 * V, cudaMemcpyHostToDevice, f->stream));
            src = (const int8_t *)f->scratch;
        }
        CK(launch_load_labels(f->prec == VS_FP32, f->nc, f->g, src, f->U, f->ref, f->stream));
    } else {
        const double *src = links;
        if (where == VS_HOST) {
            vs_status st = ensure_scratch(f, 4 * V * 18 * sizeof(double));
            if (st) return st;
            CK(cudaMemcpyAsync(f->scratch, links, 4 * V * 18 * sizeof(double), cudaMemcpyHostToDevice, f->stream));
            src = (const double *)f->scratch;
        }
        CK(launch_load_links(f->prec == VS_FP32, f->nc, f->g, src, f->U, f->ref, f->stream));
    }
    if (where == VS_HOST) CK(cudaStreamSynchronize(f->stream));
    f->loaded = true;
    f->sweeps_done = 0;
    f->gauge_on = false;
    return VS_OK;
}

extern "C" vs_status vs_field_count_nonfinite(vs_field *f, int64_t *n_links) {
    if (!f || !n_links) return fail(VS_EINVAL, "vs_field_count_nonfinite: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_field_count_nonfinite: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    unsigned long long *cnt = f->d_counts + 7, h = 0;
    CK(cudaMemsetAsync(cnt, 0, sizeof h, f->stream));
    CK(launch_count_nonfinite(f->prec == VS_FP32, f->nc, f->g, f->U, cnt, f->stream));
    CK(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    *n_links = (int64_t)h;
    return VS_OK;
}

extern "C" vs_status vs_field_checkpoint(vs_field *f, double *links_out, int8_t *labels_out, int64_t *sweeps_done,
                                         int32_t where) {
    if (!f || !links_out || !labels_out || !sweeps_done) return fail(VS_EINVAL, "vs_field_checkpoint: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_field_checkpoint: field not loaded");
    if (f->gauge_on)
        return fail(VS_EUNSUPPORTED, "vs_field_checkpoint: the field is in a random gauge (checkpoint before "
                                     "vs_gauge_transform)");
    vs_status st = vs_read_field(f, links_out, where);
    if (st) return st;
    if ((st = vs_read_labels(f, labels_out, where))) return st;
    *sweeps_done = f->sweeps_done;
    return VS_OK;
}

extern "C" vs_status vs_field_restore(vs_field *f, const double *links, const int8_t *labels, int64_t sweeps_done,
                                      int32_t where) {
    if (!f || !links || !labels) return fail(VS_EINVAL, "vs_field_restore: NULL argument");
    if (sweeps_done < 0) return fail(VS_EINVAL, "vs_field_restore: sweeps_done < 0");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_field_restore: bad `where`");
    const size_t V = f->g.V;
    if (where == VS_HOST) {
        vs_status st = check_host_labels(labels, 4 * V, "vs_field_restore");
        if (st) return st;
    }
    vs_status st = vs_load_field(f, links, nullptr, where);   // links; labels recomputed, then replaced
    if (st) return st;
    const int8_t *src = labels;
    if (where == VS_HOST) {
        if ((st = ensure_scratch(f, 4 * V))) return st;
        CK(cudaMemcpyAsync(f->scratch, labels, 4 * V, cudaMemcpyHostToDevice, f->stream));
        src = (const int8_t *)f->scratch;
    }
    CK(launch_store_ref(f->g, src, f->ref, f->stream));
    if (where == VS_HOST) CK(cudaStreamSynchronize(f->stream));
    f->sweeps_done = sweeps_done;
    return VS_OK;
}

extern "C" vs_status vs_read_field(vs_field *f, double *out, int32_t where) {
    if (!f || !out) return fail(VS_EINVAL, "vs_read_field: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_read_field: field not loaded");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_read_field: bad `where`");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t bytes = 4 * (size_t)f->g.V * 18 * sizeof(double);
    if (where == VS_DEVICE) {
        CK(launch_read_links(f->prec == VS_FP32, f->nc, f->g, f->U, out, f->stream));
        return VS_OK;
    }
    vs_status st = ensure_scratch(f, bytes);
    if (st) return st;
    CK(launch_read_links(f->prec == VS_FP32, f->nc, f->g, f->U, (double *)f->scratch, f->stream));
    CK(cudaMemcpyAsync(out, f->scratch, bytes, cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    return VS_OK;
}

static vs_status read_labels_impl(vs_field *f, int8_t *out, int32_t where, bool current) {
    if (!f || !out) return fail(VS_EINVAL, "read labels: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "read labels: field not loaded");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "read labels: bad `where`");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t n = 4 * (size_t)f->g.V;
    int8_t *dst = out;
    if (where == VS_HOST) {
        vs_status st = ensure_scratch(f, n);
        if (st) return st;
        dst = (int8_t *)f->scratch;
    }
    if (current) CK(launch_current_labels(f->prec == VS_FP32, f->nc, f->g, f->U, dst, f->stream));
    else CK(launch_read_labels(f->g, f->ref, dst, f->stream));
    if (where == VS_HOST) {
        CK(cudaMemcpyAsync(out, dst, n, cudaMemcpyDeviceToHost, f->stream));
        CK(cudaStreamSynchronize(f->stream));
    }
    return VS_OK;
}

extern "C" vs_status vs_read_labels(vs_field *f, int8_t *out, int32_t where) {
    return read_labels_impl(f, out, where, false);
}

extern "C" vs_status vs_current_labels(vs_field *f, int8_t *out, int32_t where) {
    return read_labels_impl(f, out, where, true);
}

// ---------------------------------------------------------------------------
// Centrifuge, cooled hot start, re-unitarisation
// ---------------------------------------------------------------------------

extern "C" vs_status vs_centrifuge(vs_field *f, double omega, uint64_t seed) {
    if (!f) return fail(VS_EINVAL, "vs_centrifuge: NULL field");
    if (!(omega >= 0.0 && omega < 0.25))
        return fail(VS_EINVAL, "vs_centrifuge: omega = %g outside [0, 1/4)", omega);
    if (!f->loaded) return fail(VS_EINVAL, "vs_centrifuge: field not loaded");
    // the centrifuged links are built in the original gauge from the labels
    if (f->gauge_on) return fail(VS_EINVAL, "vs_centrifuge: field in a random gauge (centrifuge first)");
    CK(cudaSetDevice(f->ctx->opt.device));
    CK(launch_centrifuge(f->prec == VS_FP32, f->nc, f->g, f->ref, omega, seed, f->U, f->stream));
    return VS_OK;
}

static AusParams make_aus_params(vs_field *f, double alpha, double eps, double u0, int n_hits, int vp) {
    AusParams a;
    memset(&a, 0, sizeof a);
    a.g = f->g;
    a.U = f->U;
    a.ref = f->ref;
    a.G = f->gauge_on ? f->G : nullptr;
    a.n_threads = f->g.V / 4;
    a.alpha = alpha;
    a.c0 = (5.0 - 2.0 * eps) / 3.0;
    a.c1 = (eps - 1.0) / (12.0 * u0 * u0);
    a.alpha_f = (float)a.alpha;
    a.c0_f = (float)a.c0;
    a.c1_f = (float)a.c1;
    a.n_hits = n_hits;
    a.vp = vp ? 1 : 0;
    return a;
}

extern "C" vs_status vs_load_cooled(vs_field *f, uint64_t seed, int32_t n_cool) {
    if (!f) return fail(VS_EINVAL, "vs_load_cooled: NULL field");
    if (n_cool < 0) return fail(VS_EINVAL, "vs_load_cooled: n_cool < 0");
    CK(cudaSetDevice(f->ctx->opt.device));
    const int p = f->prec == VS_FP32;
    CK(launch_haar(p, f->nc, f->g, seed, f->U, f->stream));
    AusParams a = make_aus_params(f, 1.0, 1.0, 1.0, 3, 0);
    for (int s = 0; s < n_cool; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int c = 0; c < 4; ++c) {
                a.colour = c;
                CK(launch_aus_class(p, f->nc, false, mu, a, f->stream));
            }
    CK(launch_project(p, f->nc, f->g, f->U, f->ref, f->stream));
    f->loaded = true;
    f->sweeps_done = 0;
    f->gauge_on = false;
    return VS_OK;
}

extern "C" vs_status vs_gauge_transform(vs_field *f, const double *G, int32_t where) {
    if (!f || !G) return fail(VS_EINVAL, "vs_gauge_transform: NULL argument");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_gauge_transform: bad `where`");
    if (!f->loaded) return fail(VS_EINVAL, "vs_gauge_transform: field not loaded");
    if (f->gauge_on) return fail(VS_EINVAL, "vs_gauge_transform: field already transformed (reload first)");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t V = f->g.V;
    if (!f->G) {
        f->G = dev_alloc(f->ctx, (size_t)f->g.P * 18 * (f->prec == VS_FP64 ? 8 : 4));
        if (!f->G) return fail(VS_ENOMEM, "vs_gauge_transform: allocation failed");
    }
    const double *src = G;
    if (where == VS_HOST) {
        vs_status st = ensure_scratch(f, V * 18 * sizeof(double));
        if (st) return st;
        CK(cudaMemcpyAsync(f->scratch, G, V * 18 * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        src = (const double *)f->scratch;
    }
    CK(launch_gauge(f->prec == VS_FP32, f->nc, f->g, src, f->G, f->U, f->stream));
    if (where == VS_HOST) CK(cudaStreamSynchronize(f->stream));
    f->gauge_on = true;
    return VS_OK;
}

extern "C" vs_status vs_reunitarise(vs_field *f) {
    if (!f) return fail(VS_EINVAL, "vs_reunitarise: NULL field");
    if (!f->loaded) return fail(VS_EINVAL, "vs_reunitarise: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    CK(launch_reunit(f->prec == VS_FP32, f->nc, f->g, f->U, nullptr, f->stream));
    return VS_OK;
}

// ---------------------------------------------------------------------------
// Smoothing
// ---------------------------------------------------------------------------

// Angular margin from the smallest margin sine of a sweep (NaN: no candidate).
static double margin_of_sine_bits(unsigned long long bits) {
    if (bits == kMarginInit) return std::nan("");
    double v;
    memcpy(&v, &bits, sizeof v);
    return std::asin(std::min(v, 1.0));
}

// The vortex-preservation diagnostics of one sweep's counters.
static void fill_vp_stats(vs_sweep_stats &o, const unsigned long long *c) {
    o.n_label_diff = (int64_t)c[kCntLabelDiff];
    o.n_undecidable = (int64_t)c[kCntUndecidable];
    o.n_fp64_redecided = (int64_t)c[kCntRedecided];
    o.min_margin = margin_of_sine_bits(c[kCntMarginSine]);
}

cudaError_t vs::init_sweep_counters(unsigned long long *c, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t pitch = kSweepSlots * sizeof(unsigned long long);
    cudaError_t e = cudaMemset2DAsync(c, pitch, 0, pitch, n, st);
    if (e == cudaSuccess)
        e = cudaMemset2DAsync(c + kCntMarginSine, pitch, 0x7f, sizeof(unsigned long long), n, st);
    return e;
}

static cudaError_t subsweep_launch(vs_field *f, bool rect, int mu, const SubsweepParams &p) {
    if (f->prec == VS_FP64) return launch_subsweep_d18(rect, mu, p, f->stream);
    if (f->nc == 12) return launch_subsweep_f12(rect, mu, p, f->stream);
    return launch_subsweep_f18(rect, mu, p, f->stream);
}

static vs_status check_smooth_params(double rho, double eps, double u0) {
    if (!std::isfinite(rho) || !std::isfinite(eps) || !std::isfinite(u0) || !(u0 > 0))
        return fail(VS_EINVAL, "smoothing parameters must be finite with u0 > 0 (rho=%g eps=%g u0=%g)",
                    rho, eps, u0);
    double c0 = (5.0 - 2.0 * eps) / 3.0, c1 = (eps - 1.0) / (12.0 * u0 * u0);
    // |rho Q|_F <= rho sqrt(3) (6|c0| + 18|c1|); the exponential series is sized for <= 8
    if (std::fabs(rho) * std::sqrt(3.0) * (6 * std::fabs(c0) + 18 * std::fabs(c1)) > 8.0)
        return fail(VS_EINVAL, "rho = %g too large for eps = %g (|rho Q| may exceed 8)", rho, eps);
    return VS_OK;
}

// redecide: FP32 with vortex preservation, candidates within the FP32 band of
// a sector edge are decided again in FP64 (k_redecide).
static SubsweepParams make_params(vs_field *f, double rho, double eps, double u0, int vp, bool redecide) {
    SubsweepParams p;
    memset(&p, 0, sizeof p);
    p.g = f->g;
    p.U = f->U;
    p.Usrc = f->U;
    p.ref = f->ref;
    p.G = f->gauge_on ? f->G : nullptr;
    p.rho = rho;
    p.c0 = (5.0 - 2.0 * eps) / 3.0;
    p.c1 = (eps - 1.0) / (12.0 * u0 * u0);
    p.rho_f = (float)p.rho;
    p.c0_f = (float)p.c0;
    p.c1_f = (float)p.c1;
    p.vp = vp ? 1 : 0;
    if (redecide && vp && f->prec == VS_FP32 && f->defer_idx) {
        p.defer_idx = f->defer_idx;
        p.defer_n = f->defer_n;
        p.defer_done = f->defer_n + 1;
        p.defer_cap = kDeferCap;
    }
    return p;
}

extern "C" vs_status vs_subsweep(vs_field *f, int32_t mu, int32_t colour, double rho, double eps, double u0,
                                 int32_t vp) {
    if (!f) return fail(VS_EINVAL, "vs_subsweep: NULL field");
    if (!f->loaded) return fail(VS_EINVAL, "vs_subsweep: field not loaded");
    if (mu < 0 || mu > 3 || colour < 0 || colour > 3) return fail(VS_EINVAL, "vs_subsweep: bad mu/colour");
    vs_status st = check_smooth_params(rho, eps, u0);
    if (st) return st;
    CK(cudaSetDevice(f->ctx->opt.device));
    SubsweepParams p = make_params(f, rho, eps, u0, vp, false);
    p.colour = colour;
    p.n_threads = f->g.V / 4;
    p.counters = f->d_sweep;
    CK(init_sweep_counters(f->d_sweep, 1, f->stream));
    CK(subsweep_launch(f, eps != 1.0, mu, p));
    return VS_OK;
}

extern "C" vs_status vs_set_profiling(vs_field *f, int32_t on) {
    if (!f) return fail(VS_EINVAL, "vs_set_profiling: NULL field");
    f->profiling = on != 0;
    f->prof_ms = 0.0;
    f->prof_launches = 0;
    return VS_OK;
}

extern "C" vs_status vs_get_profile(vs_field *f, double *ms, int64_t *n) {
    if (!f || !ms || !n) return fail(VS_EINVAL, "vs_get_profile: NULL argument");
    *ms = f->prof_ms;
    *n = f->prof_launches;
    return VS_OK;
}

vs_status vs::smooth_enqueue(vs_field *f, int32_t n_sweeps, double rho, double eps, double u0,
                             const vs_anneal *sched, int32_t vp, bool want_stats,
                             unsigned long long *fixed_counters) {
    vs_anneal a;
    memset(&a, 0, sizeof a);
    a.kind = VS_ANNEALED;
    a.reunit_every = 10;
    if (sched) a = *sched;
    if (a.kind != VS_ANNEALED && a.kind != VS_SIMULTANEOUS) return fail(VS_EINVAL, "vs_smooth: bad schedule kind");
    if (n_sweeps < 0) return fail(VS_EINVAL, "vs_smooth: n_sweeps < 0");
    if (a.reunit_every < 0 || a.action_every < 0) return fail(VS_EINVAL, "vs_smooth: negative period");
    vs_status st = check_smooth_params(rho, eps, u0);
    if (st) return st;
    if (a.rho_per_sweep)
        for (int s = 0; s < n_sweeps; ++s) {
            st = check_smooth_params(a.rho_per_sweep[s], eps, u0);
            if (st) return st;
        }
    if (!f->loaded) return fail(VS_EINVAL, "vs_smooth: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    const bool rect = eps != 1.0;
    // per-sweep device counters and actions
    if (want_stats && f->sweep_cap < n_sweeps) {
        CK(cudaStreamSynchronize(f->stream));
        dev_free(f->ctx, f->sweep_counts);
        dev_free(f->ctx, f->sweep_actions);
        f->sweep_counts = (unsigned long long *)dev_alloc(f->ctx, kSweepSlots * sizeof(unsigned long long) * n_sweeps);
        f->sweep_actions = (double *)dev_alloc(f->ctx, sizeof(double) * n_sweeps);
        if (!f->sweep_counts || !f->sweep_actions) {
            f->sweep_cap = 0;
            return fail(VS_ENOMEM, "vs_smooth: stats allocation failed");
        }
        f->sweep_cap = n_sweeps;
    }
    if (want_stats) CK(init_sweep_counters(f->sweep_counts, n_sweeps, f->stream));
    if (a.kind == VS_SIMULTANEOUS) {
        st = ensure_scratch(f, field_bytes(f));
        if (st) return st;
    }
    if (f->profiling && (int)f->events.size() < 2 * n_sweeps) {
        CK(cudaStreamSynchronize(f->stream));
        while ((int)f->events.size() < 2 * n_sweeps) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            f->events.push_back(e);
        }
    }
    // Simultaneous schedule: every link from the previous field, so the field
    // and the scratch buffer alternate as source and destination (rejected
    // links are written with their old value); one copy at the end if the
    // last sweep wrote the scratch buffer.
    void *cur = f->U, *nxt = f->scratch;
    for (int s = 0; s < n_sweeps; ++s) {
        NvtxRange range("vs stout sweep");
        const double r = a.rho_per_sweep ? a.rho_per_sweep[s] : rho;
        SubsweepParams p = make_params(f, r, eps, u0, vp, a.fp64_redecide != 0);
        p.counters = fixed_counters ? fixed_counters : (want_stats ? f->sweep_counts + kSweepSlots * s : nullptr);
        if (f->profiling) CK(cudaEventRecord(f->events[2 * s], f->stream));
        if (a.kind == VS_ANNEALED) {
            p.n_threads = f->g.V / 4;
            for (int mu = 0; mu < 4; ++mu)
                for (int c = 0; c < 4; ++c) {
                    p.colour = c;
                    CK(subsweep_launch(f, rect, mu, p));
                }
        } else {
            p.Usrc = cur;
            p.U = nxt;
            p.colour = -1;
            p.n_threads = f->g.V;
            for (int mu = 0; mu < 4; ++mu) CK(subsweep_launch(f, rect, mu, p));
            std::swap(cur, nxt);
        }
        if (f->profiling) CK(cudaEventRecord(f->events[2 * s + 1], f->stream));
        if (f->prec == VS_FP32 && a.reunit_every > 0 && (f->sweeps_done + s + 1) % a.reunit_every == 0)
            CK(launch_reunit(1, f->nc, f->g, cur, vp ? f->ref : nullptr, f->stream,
                             f->gauge_on ? f->G : nullptr));
        if (want_stats && a.action_every > 0 && (s + 1) % a.action_every == 0)
            CK(launch_action(f->prec == VS_FP32, f->nc, f->g, cur, f->partials, f->sweep_actions + s, f->stream));
    }
    if (cur != f->U) CK(cudaMemcpyAsync(f->U, cur, field_bytes(f), cudaMemcpyDeviceToDevice, f->stream));
    if (f->profiling && n_sweeps > 0) {
        CK(cudaEventSynchronize(f->events[2 * n_sweeps - 1]));
        for (int s = 0; s < n_sweeps; ++s) {
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, f->events[2 * s], f->events[2 * s + 1]));
            f->prof_ms += ms;
            f->prof_launches += a.kind == VS_ANNEALED ? 16 : 4;
        }
    }
    f->last_action_every = a.action_every;
    f->sweeps_done += n_sweeps;
    return VS_OK;
}

extern "C" vs_status vs_smooth(vs_field *f, int32_t n_sweeps, double rho, double eps, double u0,
                               const vs_anneal *sched, int32_t vp, vs_sweep_stats *stats) {
    if (!f) return fail(VS_EINVAL, "vs_smooth: NULL field");
    vs_status st = smooth_enqueue(f, n_sweeps, rho, eps, u0, sched, vp, stats != nullptr);
    if (st || !stats) return st;
    std::vector<unsigned long long> cnt(kSweepSlots * (size_t)n_sweeps);
    std::vector<double> act(n_sweeps);
    if (n_sweeps > 0) {
        CK(cudaMemcpyAsync(cnt.data(), f->sweep_counts, cnt.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, f->stream));
        CK(cudaMemcpyAsync(act.data(), f->sweep_actions, act.size() * sizeof(double), cudaMemcpyDeviceToHost,
                           f->stream));
    }
    CK(cudaStreamSynchronize(f->stream));
    const long long per_sweep = 4ll * f->g.V;
    for (int s = 0; s < n_sweeps; ++s) {
        vs_sweep_stats &o = stats[s];
        const unsigned long long *c = &cnt[kSweepSlots * (size_t)s];
        memset(&o, 0, sizeof o);
        o.n_reject = (int64_t)c[kCntReject];
        o.n_accept = per_sweep - o.n_reject;
        o.n_fp64_exp = (int64_t)c[kCntSecond];
        fill_vp_stats(o, c);
        int ae = f->last_action_every;
        if (ae > 0 && (s + 1) % ae == 0) {
            o.has_action = 1;
            o.action = act[s];
        }
    }
    return check_device_error(f);
}

extern "C" vs_status vs_smooth_aus(vs_field *f, int32_t n_sweeps, double alpha, double epsilon, double u0,
                                   int32_t n_hits, int32_t reunit_every, int32_t vortex_preserve,
                                   vs_sweep_stats *stats) {
    if (!f) return fail(VS_EINVAL, "vs_smooth_aus: NULL field");
    if (n_sweeps < 0 || n_hits < 1 || reunit_every < 0) return fail(VS_EINVAL, "vs_smooth_aus: bad count");
    if (!std::isfinite(alpha) || !(alpha >= 0.0 && alpha <= 1.0) || !std::isfinite(epsilon) || !(u0 > 0))
        return fail(VS_EINVAL, "vs_smooth_aus: need 0 <= alpha <= 1, finite eps, u0 > 0");
    if (!f->loaded) return fail(VS_EINVAL, "vs_smooth_aus: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    const bool rect = epsilon != 1.0;
    const int p = f->prec == VS_FP32;
    if (stats && f->sweep_cap < n_sweeps) {
        CK(cudaStreamSynchronize(f->stream));
        dev_free(f->ctx, f->sweep_counts);
        dev_free(f->ctx, f->sweep_actions);
        f->sweep_counts = (unsigned long long *)dev_alloc(f->ctx, kSweepSlots * sizeof(unsigned long long) * n_sweeps);
        f->sweep_actions = (double *)dev_alloc(f->ctx, sizeof(double) * n_sweeps);
        if (!f->sweep_counts || !f->sweep_actions) {
            f->sweep_cap = 0;
            return fail(VS_ENOMEM, "vs_smooth_aus: stats allocation failed");
        }
        f->sweep_cap = n_sweeps;
    }
    if (stats) CK(init_sweep_counters(f->sweep_counts, n_sweeps, f->stream));
    AusParams a = make_aus_params(f, alpha, epsilon, u0, n_hits, vortex_preserve);
    for (int s = 0; s < n_sweeps; ++s) {
        NvtxRange range("vs AUS sweep");
        a.counters = stats ? f->sweep_counts + kSweepSlots * s : nullptr;
        for (int mu = 0; mu < 4; ++mu)
            for (int c = 0; c < 4; ++c) {
                a.colour = c;
                CK(launch_aus_class(p, f->nc, rect, mu, a, f->stream));
            }
        if (f->prec == VS_FP32 && reunit_every > 0 && (f->sweeps_done + s + 1) % reunit_every == 0)
            CK(launch_reunit(1, f->nc, f->g, f->U, vortex_preserve ? f->ref : nullptr, f->stream,
                             f->gauge_on ? f->G : nullptr));
    }
    f->sweeps_done += n_sweeps;
    if (!stats) return VS_OK;
    std::vector<unsigned long long> cnt(kSweepSlots * (size_t)n_sweeps);
    if (n_sweeps > 0)
        CK(cudaMemcpyAsync(cnt.data(), f->sweep_counts, cnt.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    for (int s = 0; s < n_sweeps; ++s) {
        memset(&stats[s], 0, sizeof stats[s]);
        stats[s].n_reject = (int64_t)cnt[kSweepSlots * s + kCntReject];
        stats[s].n_accept = 4ll * f->g.V - stats[s].n_reject;
        fill_vp_stats(stats[s], &cnt[kSweepSlots * s]);
    }
    return check_device_error(f);
}

// ---------------------------------------------------------------------------
// APE / AUS with unit circle projection, Runge-Kutta Wilson flow
// ---------------------------------------------------------------------------

static cudaError_t ape_launch(vs_field *f, bool rect, int mu, const ApeParams &p) {
    if (f->prec == VS_FP64) return launch_ape_d18(rect, mu, p, f->stream);
    if (f->nc == 12) return launch_ape_f12(rect, mu, p, f->stream);
    return launch_ape_f18(rect, mu, p, f->stream);
}

static cudaError_t flow_launch(vs_field *f, bool rect, int mu, const FlowParams &p) {
    if (f->prec == VS_FP64) return launch_flow_d18(rect, mu, p, f->stream);
    if (f->nc == 12) return launch_flow_f12(rect, mu, p, f->stream);
    return launch_flow_f18(rect, mu, p, f->stream);
}

// per-sweep counter blocks (kSweepSlots each) in the field's stats buffer
static vs_status ensure_sweep_counts(vs_field *f, int32_t n, const char *who) {
    if (f->sweep_cap >= n) return VS_OK;
    CK(cudaStreamSynchronize(f->stream));
    dev_free(f->ctx, f->sweep_counts);
    dev_free(f->ctx, f->sweep_actions);
    f->sweep_counts = (unsigned long long *)dev_alloc(f->ctx, kSweepSlots * sizeof(unsigned long long) * n);
    f->sweep_actions = (double *)dev_alloc(f->ctx, sizeof(double) * n);
    if (!f->sweep_counts || !f->sweep_actions) {
        f->sweep_cap = 0;
        return fail(VS_ENOMEM, "%s: stats allocation failed", who);
    }
    f->sweep_cap = n;
    return VS_OK;
}

extern "C" vs_status vs_smooth_ape(vs_field *f, int32_t n_sweeps, double alpha, double epsilon, double u0,
                                   int32_t schedule, int32_t reunit_every, int32_t vortex_preserve,
                                   vs_sweep_stats *stats) {
    if (!f) return fail(VS_EINVAL, "vs_smooth_ape: NULL field");
    if (n_sweeps < 0 || reunit_every < 0) return fail(VS_EINVAL, "vs_smooth_ape: bad count");
    if (schedule != VS_ANNEALED && schedule != VS_SIMULTANEOUS) return fail(VS_EINVAL, "vs_smooth_ape: bad schedule");
    if (!std::isfinite(alpha) || !(alpha >= 0.0 && alpha <= 1.0) || !std::isfinite(epsilon) || !(u0 > 0))
        return fail(VS_EINVAL, "vs_smooth_ape: need 0 <= alpha <= 1, finite eps, u0 > 0");
    if (!f->loaded) return fail(VS_EINVAL, "vs_smooth_ape: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    const bool rect = epsilon != 1.0;
    vs_status st;
    if (stats) {
        if ((st = ensure_sweep_counts(f, n_sweeps, "vs_smooth_ape"))) return st;
        CK(init_sweep_counters(f->sweep_counts, n_sweeps, f->stream));
    }
    if (schedule == VS_SIMULTANEOUS && (st = ensure_scratch(f, field_bytes(f)))) return st;
    ApeParams a;
    memset(&a, 0, sizeof a);
    a.g = f->g;
    a.U = f->U;
    a.ref = f->ref;
    a.G = f->gauge_on ? f->G : nullptr;
    a.alpha = alpha;
    a.c0 = (5.0 - 2.0 * epsilon) / 3.0;
    a.c1 = (epsilon - 1.0) / (12.0 * u0 * u0);
    a.alpha_f = (float)a.alpha;
    a.c0_f = (float)a.c0;
    a.c1_f = (float)a.c1;
    a.vp = vortex_preserve ? 1 : 0;
    void *cur = f->U, *nxt = f->scratch;   // simultaneous: alternating buffers, as in vs_smooth
    for (int s = 0; s < n_sweeps; ++s) {
        NvtxRange range("vs APE/UCP sweep");
        a.counters = stats ? f->sweep_counts + kSweepSlots * s : nullptr;
        if (schedule == VS_ANNEALED) {
            a.U = f->U;
            a.Usrc = f->U;
            a.n_threads = f->g.V / 4;
            for (int mu = 0; mu < 4; ++mu)
                for (int c = 0; c < 4; ++c) {
                    a.colour = c;
                    CK(ape_launch(f, rect, mu, a));
                }
        } else {
            a.Usrc = cur;
            a.U = nxt;
            a.colour = -1;
            a.n_threads = f->g.V;
            for (int mu = 0; mu < 4; ++mu) CK(ape_launch(f, rect, mu, a));
            std::swap(cur, nxt);
        }
        if (f->prec == VS_FP32 && reunit_every > 0 && (f->sweeps_done + s + 1) % reunit_every == 0)
            CK(launch_reunit(1, f->nc, f->g, cur, vortex_preserve ? f->ref : nullptr, f->stream,
                             f->gauge_on ? f->G : nullptr));
    }
    if (cur != f->U) CK(cudaMemcpyAsync(f->U, cur, field_bytes(f), cudaMemcpyDeviceToDevice, f->stream));
    f->sweeps_done += n_sweeps;
    if (!stats) return VS_OK;
    std::vector<unsigned long long> cnt(kSweepSlots * (size_t)n_sweeps);
    if (n_sweeps > 0)
        CK(cudaMemcpyAsync(cnt.data(), f->sweep_counts, cnt.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    for (int s = 0; s < n_sweeps; ++s) {
        memset(&stats[s], 0, sizeof stats[s]);
        stats[s].n_reject = (int64_t)cnt[kSweepSlots * s + kCntReject];
        stats[s].n_accept = 4ll * f->g.V - stats[s].n_reject;
        stats[s].n_singular = (int32_t)cnt[kSweepSlots * s + kCntSecond];
        fill_vp_stats(stats[s], &cnt[kSweepSlots * s]);
    }
    return check_device_error(f);
}

extern "C" vs_status vs_flow_rk3(vs_field *f, int32_t n_steps, double step, double epsilon, double u0,
                                 int32_t reunit_every, vs_sweep_stats *stats) {
    if (!f) return fail(VS_EINVAL, "vs_flow_rk3: NULL field");
    if (n_steps < 0 || reunit_every < 0) return fail(VS_EINVAL, "vs_flow_rk3: bad count");
    vs_status st = check_smooth_params(step, epsilon, u0);
    if (st) return st;
    if (!(step >= 0.0)) return fail(VS_EINVAL, "vs_flow_rk3: step must be >= 0");
    if (!f->loaded) return fail(VS_EINVAL, "vs_flow_rk3: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    const bool rect = epsilon != 1.0;
    if ((st = ensure_scratch(f, field_bytes(f)))) return st;
    const size_t sbytes = 4ull * 9 * f->g.P * (f->prec == VS_FP32 ? sizeof(float) : sizeof(double));
    if (f->flowS_bytes < sbytes) {
        CK(cudaStreamSynchronize(f->stream));
        dev_free(f->ctx, f->flowS);
        f->flowS = dev_alloc(f->ctx, sbytes);
        f->flowS_bytes = f->flowS ? sbytes : 0;
        if (!f->flowS) return fail(VS_ENOMEM, "vs_flow_rk3: exponent buffer of %zu bytes failed", sbytes);
    }
    if (stats) {
        if ((st = ensure_sweep_counts(f, n_steps, "vs_flow_rk3"))) return st;
        CK(init_sweep_counters(f->sweep_counts, n_steps, f->stream));
    }
    // Luscher's third-order scheme in the low-storage form: stage k uses
    // H_S <- a_k H_Z + b_k H_S and W <- exp(i c_k H_S) W with
    // (a, b, c) = (1, 0, 1/4), (8/9, -17/36, 1), (3/4, -1, 1).
    static const double A[3] = {1.0, 8.0 / 9.0, 0.75}, B[3] = {0.0, -17.0 / 36.0, -1.0}, C[3] = {0.25, 1.0, 1.0};
    FlowParams p;
    memset(&p, 0, sizeof p);
    p.g = f->g;
    p.U = f->U;
    p.Usrc = f->scratch;
    p.S = f->flowS;
    p.n_threads = f->g.V;
    p.h = step;
    p.c0 = (5.0 - 2.0 * epsilon) / 3.0;
    p.c1 = (epsilon - 1.0) / (12.0 * u0 * u0);
    p.h_f = (float)p.h;
    p.c0_f = (float)p.c0;
    p.c1_f = (float)p.c1;
    // Every link of a stage is computed from the previous stage's field, so the
    // field and the scratch buffer alternate as source and destination (every
    // link of the destination is written); one copy at the end if the last
    // stage wrote the scratch buffer.
    void *cur = f->U, *nxt = f->scratch;
    for (int s = 0; s < n_steps; ++s) {
        NvtxRange range("vs RK3 step");
        p.counters = stats ? f->sweep_counts + kSweepSlots * s : nullptr;
        for (int k = 0; k < 3; ++k) {
            p.a = A[k];
            p.b = B[k];
            p.c = C[k];
            p.a_f = (float)p.a;
            p.b_f = (float)p.b;
            p.c_f = (float)p.c;
            p.Usrc = cur;
            p.U = nxt;
            for (int mu = 0; mu < 4; ++mu) CK(flow_launch(f, rect, mu, p));
            std::swap(cur, nxt);
        }
        if (f->prec == VS_FP32 && reunit_every > 0 && (f->sweeps_done + s + 1) % reunit_every == 0)
            CK(launch_reunit(1, f->nc, f->g, cur, nullptr, f->stream, nullptr));
    }
    if (cur != f->U) CK(cudaMemcpyAsync(f->U, cur, field_bytes(f), cudaMemcpyDeviceToDevice, f->stream));
    f->sweeps_done += n_steps;
    if (!stats) return VS_OK;
    std::vector<unsigned long long> cnt(kSweepSlots * (size_t)n_steps);
    if (n_steps > 0)
        CK(cudaMemcpyAsync(cnt.data(), f->sweep_counts, cnt.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    for (int s = 0; s < n_steps; ++s) {
        memset(&stats[s], 0, sizeof stats[s]);
        stats[s].n_accept = 4ll * f->g.V;
        stats[s].n_fp64_exp = (int64_t)cnt[kSweepSlots * s + kCntSecond];
        stats[s].n_label_diff = -1;
        stats[s].n_undecidable = -1;
        stats[s].min_margin = std::nan("");
    }
    return check_device_error(f);
}

// ---------------------------------------------------------------------------
// Observables
// ---------------------------------------------------------------------------

extern "C" vs_status vs_action(vs_field *f, double *mean_S) {
    if (!f || !mean_S) return fail(VS_EINVAL, "vs_action: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_action: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    CK(launch_action(f->prec == VS_FP32, f->nc, f->g, f->U, f->partials, f->d_result, f->stream));
    CK(cudaMemcpyAsync(mean_S, f->d_result, sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    return VS_OK;
}

extern "C" vs_status vs_observables(vs_field *f, vs_observables_out *out, double *S_site, double *SR_site,
                                    double *q_site, int32_t where) {
    if (!f || !out) return fail(VS_EINVAL, "vs_observables: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_observables: field not loaded");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_observables: bad `where`");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t V = f->g.V;
    double *dS = S_site, *dSR = SR_site, *dq = q_site;
    if (where == VS_HOST && (S_site || SR_site || q_site)) {
        vs_status st = ensure_scratch(f, 3 * V * sizeof(double));
        if (st) return st;
        double *sc = (double *)f->scratch;
        dS = S_site ? sc : nullptr;
        dSR = SR_site ? sc + V : nullptr;
        dq = q_site ? sc + 2 * V : nullptr;
    }
    // 3 x 400 partials fit in the 1216 + 512 doubles after f->partials; results after them
    double *res = f->partials + 1200;
    CK(launch_observables(f->prec == VS_FP32, f->nc, f->g, f->U, f->partials, res, dS, dSR, dq, f->stream));
    double h[3];
    CK(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, f->stream));
    if (where == VS_HOST) {
        if (S_site) CK(cudaMemcpyAsync(S_site, dS, V * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        if (SR_site) CK(cudaMemcpyAsync(SR_site, dSR, V * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        if (q_site) CK(cudaMemcpyAsync(q_site, dq, V * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
    }
    CK(cudaStreamSynchronize(f->stream));
    out->mean_S = h[0];
    out->mean_SR = h[1];
    out->Q = h[2];
    return VS_OK;
}

extern "C" vs_status vs_correlation(vs_field *f, const double *a, const double *b, int32_t where, double *C) {
    if (!f || !a || !b || !C) return fail(VS_EINVAL, "vs_correlation: NULL argument");
    if (where != VS_HOST && where != VS_DEVICE) return fail(VS_EINVAL, "vs_correlation: bad `where`");
    CK(cudaSetDevice(f->ctx->opt.device));
    const size_t V = f->g.V;
    const double *da = a, *db = b;
    if (where == VS_HOST) {
        vs_status st = ensure_scratch(f, 2 * V * sizeof(double));
        if (st) return st;
        double *sc = (double *)f->scratch;
        CK(cudaMemcpyAsync(sc, a, V * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        CK(cudaMemcpyAsync(sc + V, b, V * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        da = sc;
        db = sc + V;
    }
    // 3 x 400 partials, then the result and the three sums
    double *res = f->partials + 1200;
    CK(launch_correlation(da, db, (long long)V, f->partials, res, f->stream));
    double h[4];
    CK(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    if (!(h[2] > 0) || !(h[3] > 0)) return fail(VS_EINVAL, "vs_correlation: a density is zero on every site");
    *C = h[0];
    return VS_OK;
}

extern "C" vs_status vs_vortex_check(vs_field *f, vs_vortex_report *out) {
    if (!f || !out) return fail(VS_EINVAL, "vs_vortex_check: NULL argument");
    if (!f->loaded) return fail(VS_EINVAL, "vs_vortex_check: field not loaded");
    CK(cudaSetDevice(f->ctx->opt.device));
    unsigned long long *cnt = f->d_counts + 2;      // [3] counts, [1] margin bits
    CK(cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), f->stream));
    CK(cudaMemsetAsync(cnt + 3, 0x7f, sizeof(unsigned long long), f->stream));
    CK(launch_vortex(f->prec == VS_FP32, f->nc, f->g, f->U, f->ref, f->cur, cnt, cnt + 3, f->stream,
                     f->gauge_on ? f->G : nullptr));
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    out->n_links = 4ll * f->g.V;
    out->n_label_diff = (int64_t)h[0];
    out->n_charge_diff = (int64_t)h[1];
    out->n_near_boundary = (int64_t)h[2];
    double m;
    memcpy(&m, &h[3], sizeof m);
    out->min_margin = m;
    return VS_OK;
}

extern "C" vs_status vs_debug_expm(vs_ctx *c, const double *X, int32_t n, int32_t precision, double *E) {
    if (!c || !X || !E || n < 0) return fail(VS_EINVAL, "vs_debug_expm: bad argument");
    if (precision != VS_FP32 && precision != VS_FP64) return fail(VS_EINVAL, "vs_debug_expm: bad precision");
    if (n == 0) return VS_OK;
    CK(cudaSetDevice(c->opt.device));
    size_t bytes = (size_t)n * 18 * sizeof(double);
    double *dX = (double *)dev_alloc(c, bytes), *dE = (double *)dev_alloc(c, bytes);
    if (!dX || !dE) {
        dev_free(c, dX);
        dev_free(c, dE);
        return fail(VS_ENOMEM, "vs_debug_expm: allocation failed");
    }
    cudaError_t e = cudaMemcpy(dX, X, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_debug_expm(precision == VS_FP32, dX, n, dE, 0);
    if (e == cudaSuccess) e = cudaMemcpy(E, dE, bytes, cudaMemcpyDeviceToHost);
    dev_free(c, dX);
    dev_free(c, dE);
    if (e != cudaSuccess) return cuda_fail(e, "vs_debug_expm");
    return VS_OK;
}

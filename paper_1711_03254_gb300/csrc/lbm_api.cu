// Host runtime behind the C ABI of include/lbm.h: context, device buffers,
// argument checks, kernel dispatch, read-back and checkpoints.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

std::mutex g_alloc_mu;
void *(*g_alloc)(size_t, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
thread_local std::string g_last_error;

// |u_F| beyond the lattice speed of sound sqrt(T0) is outside the scheme's range
constexpr double kMaxSpeed = 0.57735026918962576;

size_t storage_bytes(lbm_precision p) {
    switch (p) {
    case LBM_FP64: return 8;
    case LBM_FP32: return 4;
    default: return 2;
    }
}

}  // namespace

struct lbm_ctx {
    lbm_config cfg{};
    std::vector<lbm_instance_params> par;
    Grid g{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    void *(*alloc)(size_t, void *) = nullptr;
    void (*release)(void *, void *) = nullptr;
    std::vector<void *> owned;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t *link = nullptr;
    void *psi = nullptr, *macro = nullptr, *usnap = nullptr, *dpar = nullptr;
    double *partial = nullptr, *red_out = nullptr;
    int nblk = 0;
    bool has_geometry = false, has_fields = false;
    long long step = 0, since_snap = 0;
    long long launches = 0;
    lbm_kernel kernel = LBM_KERNEL_AUTO;
    int tile = -1, zchunk = -1;  // fused-kernel tiling; -1 = heuristic
    std::string err;

    bool fp64() const { return cfg.precision == LBM_FP64; }
    size_t tbytes() const { return fp64() ? 8 : 4; }
    size_t cells() const { return (size_t)cfg.batch * (size_t)g.n; }
    size_t f_bytes() const { return cells() * 2 * 19 * storage_bytes(cfg.precision); }

    lbm_status fail(lbm_status s, const std::string &m) {
        err = m;
        g_last_error = m;
        return s;
    }
    lbm_status cuda_fail(cudaError_t e, const char *what) {
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                    std::string(what) + ": " + cudaGetErrorString(e));
    }
    void *dalloc(size_t bytes) {
        void *p = nullptr;
        if (alloc) {
            p = alloc(bytes, (void *)stream);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            p = nullptr;
        }
        if (p) owned.push_back(p);
        return p;
    }
    void dfree(void *p) {
        if (!p) return;
        for (size_t k = 0; k < owned.size(); ++k)
            if (owned[k] == p) {
                owned.erase(owned.begin() + k);
                break;
            }
        if (release)
            release(p, (void *)stream);
        else
            cudaFree(p);
    }
};

#define LBM_CUDA(call, what)                              \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return ctx->cuda_fail(e__, what); \
    } while (0)

namespace {

template <class T> void fill_params(const lbm_ctx *ctx, std::vector<InstParam<T>> &out) {
    const double T0 = 1.0 / 3.0;
    out.resize(ctx->par.size());
    for (size_t b = 0; b < ctx->par.size(); ++b) {
        const lbm_instance_params &p = ctx->par[b];
        InstParam<T> &q = out[b];
        q.nu[0] = (T)(T0 * (p.tau[0] - 0.5));
        q.nu[1] = (T)(T0 * (p.tau[1] - 0.5));
        q.G = (T)p.G;
        q.rs[0] = (T)(p.rho_s < 0.0 ? -p.rho_s : 0.0);
        q.rs[1] = (T)(p.rho_s > 0.0 ? p.rho_s : 0.0);
        for (int a = 0; a < 3; ++a) {
            q.g[a] = (T)p.g[a];
            q.u_in[a] = (T)p.u_in[a];
        }
        q.rho_in[0] = (T)p.rho_in[0];
        q.rho_in[1] = (T)p.rho_in[1];
    }
}

lbm_status upload_params(lbm_ctx *ctx) {
    if (ctx->fp64()) {
        std::vector<InstParam<double>> h;
        fill_params(ctx, h);
        LBM_CUDA(cudaMemcpyAsync(ctx->dpar, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, ctx->stream),
                 "upload parameters");
        LBM_CUDA(cudaStreamSynchronize(ctx->stream), "upload parameters");
    } else {
        std::vector<InstParam<float>> h;
        fill_params(ctx, h);
        LBM_CUDA(cudaMemcpyAsync(ctx->dpar, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, ctx->stream),
                 "upload parameters");
        LBM_CUDA(cudaStreamSynchronize(ctx->stream), "upload parameters");
    }
    return LBM_OK;
}

// Fused-kernel tiling when none was set: 32x8 columns (32x4 in FP64, whose
// ring buffers are twice as large), z chunks sized for about eight CTAs per SM.
void default_tiling(const lbm_ctx *ctx, int &tile, int &zchunk) {
    if (tile < 0) tile = ctx->cfg.precision == LBM_FP64 ? 1 : 0;
    if (zchunk < 0) {
        const int tx = tile == 2 ? 64 : 32;
        const int ty = tile == 0 ? 8 : (tile == 3 ? 16 : 4);
        const long long cols = (long long)((ctx->g.nx + tx - 1) / tx) * ((ctx->g.ny + ty - 1) / ty) * ctx->cfg.batch;
        int sms = 152;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long want = 8LL * sms;
        long long chunks = (want + cols - 1) / cols;
        if (chunks < 1) chunks = 1;
        zchunk = (int)((ctx->g.nz + chunks - 1) / chunks);
        if (zchunk < 8) zchunk = ctx->g.nz < 8 ? ctx->g.nz : 8;
    }
}

StepArgs step_args(lbm_ctx *ctx, int write_macro) {
    StepArgs a{};
    a.precision = ctx->cfg.precision;
    a.eq_order = ctx->cfg.eq_order;
    a.wall_model = ctx->cfg.wall_model;
    a.write_macro = write_macro;
    a.batch = ctx->cfg.batch;
    a.g = ctx->g;
    a.f_in = ctx->f[ctx->cur];
    a.f_out = ctx->f[ctx->cur ^ 1];
    a.link = ctx->link;
    a.psi = ctx->psi;
    a.macro = ctx->macro;
    a.par = ctx->dpar;
    a.rho0[0] = ctx->cfg.rho0_shift[0];
    a.rho0[1] = ctx->cfg.rho0_shift[1];
    a.stream = ctx->stream;
    return a;
}

}  // namespace

extern "C" {

lbm_status lbm_set_allocator(void *(*alloc)(size_t, void *), void (*release)(void *, void *)) {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if ((alloc == nullptr) != (release == nullptr)) {
        g_last_error = "lbm_set_allocator: give both functions or neither";
        return LBM_ERR_ARG;
    }
    g_alloc = alloc;
    g_free = release;
    return LBM_OK;
}

lbm_status lbm_create(const lbm_config *cfg, const lbm_instance_params *per_instance, lbm_ctx **out) {
    if (out) *out = nullptr;
    if (!cfg || !per_instance || !out) {
        g_last_error = "lbm_create: null argument";
        return LBM_ERR_ARG;
    }
    if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || cfg->batch < 1) {
        g_last_error = "lbm_create: every dimension and the batch must be >= 1";
        return LBM_ERR_ARG;
    }
    if ((long long)cfg->nx * cfg->ny * cfg->nz >= (1LL << 31)) {
        g_last_error = "lbm_create: more than 2^31 cells per instance";
        return LBM_ERR_ARG;
    }
    if (cfg->precision < LBM_FP64 || cfg->precision > LBM_FP32_BF16S || cfg->eq_order < 0 || cfg->eq_order > 1 ||
        cfg->wall_model < 0 || cfg->wall_model > 1) {
        g_last_error = "lbm_create: precision, eq_order or wall_model out of range";
        return LBM_ERR_ARG;
    }
    for (int b = 0; b < cfg->batch; ++b) {
        const lbm_instance_params &p = per_instance[b];
        if (!(p.tau[0] > 0.5) || !(p.tau[1] > 0.5)) {
            g_last_error = "lbm_create: tau must exceed 1/2";
            return LBM_ERR_ARG;
        }
        const double vals[] = {p.G, p.rho_s, p.g[0], p.g[1], p.g[2], p.rho_in[0], p.rho_in[1], p.u_in[0], p.u_in[1],
                               p.u_in[2], p.tau[0], p.tau[1]};
        for (double v : vals)
            if (!std::isfinite(v)) {
                g_last_error = "lbm_create: non-finite parameter";
                return LBM_ERR_ARG;
            }
    }
    lbm_ctx *ctx = new lbm_ctx();
    ctx->cfg = *cfg;
    ctx->par.assign(per_instance, per_instance + cfg->batch);
    ctx->g.nx = cfg->nx;
    ctx->g.ny = cfg->ny;
    ctx->g.nz = cfg->nz;
    ctx->g.nxy = cfg->nx * cfg->ny;
    ctx->g.n = (long long)cfg->nx * cfg->ny * cfg->nz;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        ctx->alloc = g_alloc;
        ctx->release = g_free;
    }
    if (cudaGetDevice(&ctx->dev) != cudaSuccess) {
        g_last_error = "lbm_create: no CUDA device";
        delete ctx;
        return LBM_ERR_CUDA;
    }
    const size_t cells = ctx->cells();
    ctx->nblk = reduce_blocks(ctx->g.n);
    ctx->f[0] = ctx->dalloc(ctx->f_bytes());
    ctx->f[1] = ctx->dalloc(ctx->f_bytes());
    ctx->link = (uint32_t *)ctx->dalloc(cells * 4);
    ctx->psi = ctx->dalloc(cells * 2 * ctx->tbytes());
    ctx->macro = ctx->dalloc(cells * 5 * ctx->tbytes());
    ctx->usnap = ctx->dalloc(cells * 3 * ctx->tbytes());
    ctx->dpar = ctx->dalloc((size_t)cfg->batch * sizeof(InstParam<double>));
    ctx->partial = (double *)ctx->dalloc((size_t)cfg->batch * ctx->nblk * 9 * sizeof(double));
    ctx->red_out = (double *)ctx->dalloc((size_t)cfg->batch * 9 * sizeof(double));
    if (!ctx->f[0] || !ctx->f[1] || !ctx->link || !ctx->psi || !ctx->macro || !ctx->usnap || !ctx->dpar ||
        !ctx->partial || !ctx->red_out) {
        g_last_error = "lbm_create: device allocation failed";
        lbm_destroy(ctx);
        return LBM_ERR_OOM;
    }
    lbm_status s = upload_params(ctx);
    if (s != LBM_OK) {
        lbm_destroy(ctx);
        return s;
    }
    *out = ctx;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    std::vector<void *> own = ctx->owned;
    for (void *p : own) ctx->dfree(p);
    delete ctx;
}

lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return LBM_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_ctx *ctx, lbm_kernel kernel) {
    if (!ctx) return LBM_ERR_ARG;
    if (kernel != LBM_KERNEL_AUTO && kernel != LBM_KERNEL_TWO_PASS && kernel != LBM_KERNEL_FUSED)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: strategy not available for this configuration");
    ctx->kernel = kernel;
    return LBM_OK;
}

long long lbm_launch_count(const lbm_ctx *ctx) { return ctx ? ctx->launches : 0; }

lbm_status lbm_set_tiling(lbm_ctx *ctx, int tile, int zchunk) {
    if (!ctx) return LBM_ERR_ARG;
    if (tile < -1 || tile >= fused_tile_count() || zchunk == 0 || zchunk < -1)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_tiling: tile or zchunk out of range");
    ctx->tile = tile;
    ctx->zchunk = zchunk;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx *ctx, const uint8_t *cell_type) {
    if (!ctx || !cell_type) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_set_geometry: null argument") : LBM_ERR_ARG;
    const size_t cells = ctx->cells();
    for (int b = 0; b < ctx->cfg.batch; ++b) {
        bool any_fluid = false;
        for (long long k = 0; k < ctx->g.n; ++k) {
            const uint8_t t = cell_type[(size_t)b * ctx->g.n + k];
            if (t > 3) return ctx->fail(LBM_ERR_ARG, "lbm_set_geometry: cell type above 3");
            any_fluid |= t == 0;
        }
        if (!any_fluid) return ctx->fail(LBM_ERR_ARG, "lbm_set_geometry: an instance has no FLUID cell");
    }
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    uint8_t *dt = (uint8_t *)ctx->dalloc(cells);
    if (!dt) return ctx->fail(LBM_ERR_OOM, "lbm_set_geometry: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(dt, cell_type, cells, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_links(dt, ctx->link, ctx->g, ctx->cfg.batch, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(dt);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_set_geometry");
    ctx->launches += 1;
    ctx->has_geometry = true;
    ctx->has_fields = false;
    return LBM_OK;
}

lbm_status lbm_set_fields(lbm_ctx *ctx, const double *rho1, const double *rho2, const double *u) {
    if (!ctx || !rho1 || !rho2 || !u) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_set_fields: null argument") : LBM_ERR_ARG;
    if (!ctx->has_geometry) return ctx->fail(LBM_ERR_STATE, "lbm_set_fields: call lbm_set_geometry first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const size_t cells = ctx->cells();
    double *d = (double *)ctx->dalloc(cells * 5 * sizeof(double));
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_set_fields: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(d, rho1, cells * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + cells, rho2, cells * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 2 * cells, u, cells * 24, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) {
        InitArgs a{};
        a.precision = ctx->cfg.precision;
        a.eq_order = ctx->cfg.eq_order;
        a.batch = ctx->cfg.batch;
        a.g = ctx->g;
        a.r1 = d;
        a.r2 = d + cells;
        a.u = d + 2 * cells;
        a.link = ctx->link;
        a.f_out = ctx->f[ctx->cur];
        a.macro = ctx->macro;
        a.usnap = ctx->usnap;
        a.par = ctx->dpar;
        a.rho0[0] = ctx->cfg.rho0_shift[0];
        a.rho0[1] = ctx->cfg.rho0_shift[1];
        a.stream = ctx->stream;
        e = launch_init(a);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(d);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_set_fields");
    ctx->launches += 1;
    ctx->has_fields = true;
    ctx->since_snap = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int n) {
    if (!ctx) return LBM_ERR_ARG;
    if (n < 0) return ctx->fail(LBM_ERR_ARG, "lbm_step: negative step count");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_step: call lbm_set_fields first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const bool fused = ctx->kernel != LBM_KERNEL_TWO_PASS;
    int tile = ctx->tile, zchunk = ctx->zchunk;
    if (fused) default_tiling(ctx, tile, zchunk);
    for (int s = 0; s < n; ++s) {
        StepArgs a = step_args(ctx, s == n - 1);
        cudaError_t e = fused ? launch_fused(a, tile, zchunk) : launch_two_pass(a);
        if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_step launch");
        ctx->launches += fused ? 1 : 2;
        ctx->cur ^= 1;
    }
    ctx->step += n;
    ctx->since_snap += n;
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_ctx *ctx, double *rho1, double *rho2, double *u) {
    if (!ctx) return LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_get_fields: no fields yet");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const size_t cells = ctx->cells();
    double *d = (double *)ctx->dalloc(cells * 5 * sizeof(double));
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_get_fields: device allocation failed");
    cudaError_t e = launch_macro_to_f64(ctx->macro, ctx->fp64(), d, d + cells, d + 2 * cells, ctx->g,
                                        ctx->cfg.batch, ctx->stream);
    if (e == cudaSuccess && rho1) e = cudaMemcpyAsync(rho1, d, cells * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && rho2) e = cudaMemcpyAsync(rho2, d + cells, cells * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, d + 2 * cells, cells * 24, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(d);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_get_fields");
    ctx->launches += 1;
    return LBM_OK;
}

lbm_status lbm_reduce(lbm_ctx *ctx, double *out) {
    if (!ctx || !out) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_reduce: null argument") : LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_reduce: no fields yet");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    ReduceArgs a{};
    a.fp64 = ctx->fp64();
    a.batch = ctx->cfg.batch;
    a.g = ctx->g;
    a.macro = ctx->macro;
    a.usnap = ctx->usnap;
    a.link = ctx->link;
    a.partial = ctx->partial;
    a.nblk = ctx->nblk;
    a.out = ctx->red_out;
    a.k = ctx->since_snap;
    a.stream = ctx->stream;
    int nl = 0;
    LBM_CUDA(launch_reduce(a, &nl), "lbm_reduce launch");
    ctx->launches += nl;
    std::vector<double> h((size_t)ctx->cfg.batch * 9);
    LBM_CUDA(cudaMemcpyAsync(h.data(), ctx->red_out, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream),
             "lbm_reduce copy");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "lbm_reduce sync");
    bool bad = false;
    for (int b = 0; b < ctx->cfg.batch; ++b) {
        const double *r = &h[(size_t)b * 9];
        double *o = out + (size_t)b * 7;
        for (int c = 0; c < 5; ++c) o[c] = r[c];
        const long long k = ctx->since_snap;
        o[5] = k > 0 ? std::sqrt(r[5]) / ((double)k * std::sqrt(r[6]) + 1e-30) : 0.0;
        o[6] = r[8] > 0 ? NAN : r[7];
        if (r[8] > 0 || r[7] > kMaxSpeed || !std::isfinite(r[0]) || !std::isfinite(r[1])) bad = true;
    }
    ctx->since_snap = 0;
    if (bad) return ctx->fail(LBM_ERR_DIVERGED, "lbm_reduce: non-finite value or |u_F| above the lattice sound speed");
    return LBM_OK;
}

lbm_status lbm_get_distributions(lbm_ctx *ctx, double *f) {
    if (!ctx || !f) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_get_distributions: null argument") : LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_get_distributions: no fields yet");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const size_t vals = ctx->cells() * 2 * 19;
    double *d = (double *)ctx->dalloc(vals * 8);
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_get_distributions: device allocation failed");
    cudaError_t e = launch_f_convert(ctx->cfg.precision, ctx->f[ctx->cur], d, nullptr, nullptr, ctx->g,
                                     ctx->cfg.batch, ctx->cfg.rho0_shift, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, vals * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(d);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_get_distributions");
    ctx->launches += 1;
    return LBM_OK;
}

lbm_status lbm_set_distributions(lbm_ctx *ctx, const double *f) {
    if (!ctx || !f) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_set_distributions: null argument") : LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_set_distributions: call lbm_set_fields first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const size_t vals = ctx->cells() * 2 * 19;
    double *d = (double *)ctx->dalloc(vals * 8);
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_set_distributions: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(d, f, vals * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = launch_f_convert(ctx->cfg.precision, nullptr, nullptr, d, ctx->f[ctx->cur], ctx->g, ctx->cfg.batch,
                             ctx->cfg.rho0_shift, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(d);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_set_distributions");
    ctx->launches += 1;
    return LBM_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    uint32_t version;
    uint32_t pad;
    lbm_config cfg;
    long long step, since_snap;
    uint64_t f_bytes, link_bytes, macro_bytes, usnap_bytes;
};
}  // namespace

lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t *bytes) {
    if (!ctx || !bytes) return LBM_ERR_ARG;
    const size_t cells = ctx->cells();
    StateHeader h{};
    std::memcpy(h.magic, "LBMSTATE", 8);
    h.version = 1;
    h.cfg = ctx->cfg;
    h.step = ctx->step;
    h.since_snap = ctx->since_snap;
    h.f_bytes = ctx->f_bytes();
    h.link_bytes = cells * 4;
    h.macro_bytes = cells * 5 * ctx->tbytes();
    h.usnap_bytes = cells * 3 * ctx->tbytes();
    const size_t need = sizeof(h) + h.f_bytes + h.link_bytes + h.macro_bytes + h.usnap_bytes;
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) return ctx->fail(LBM_ERR_ARG, "lbm_get_state: buffer too small");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_get_state: no fields yet");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    char *p = (char *)buf;
    std::memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    LBM_CUDA(cudaMemcpyAsync(p, ctx->f[ctx->cur], h.f_bytes, cudaMemcpyDeviceToHost, ctx->stream), "get_state f");
    p += h.f_bytes;
    LBM_CUDA(cudaMemcpyAsync(p, ctx->link, h.link_bytes, cudaMemcpyDeviceToHost, ctx->stream), "get_state link");
    p += h.link_bytes;
    LBM_CUDA(cudaMemcpyAsync(p, ctx->macro, h.macro_bytes, cudaMemcpyDeviceToHost, ctx->stream), "get_state macro");
    p += h.macro_bytes;
    LBM_CUDA(cudaMemcpyAsync(p, ctx->usnap, h.usnap_bytes, cudaMemcpyDeviceToHost, ctx->stream), "get_state usnap");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "get_state sync");
    *bytes = need;
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx *ctx, const void *buf, size_t bytes) {
    if (!ctx || !buf) return LBM_ERR_ARG;
    StateHeader h;
    if (bytes < sizeof(h)) return ctx->fail(LBM_ERR_ARG, "lbm_set_state: buffer too small");
    std::memcpy(&h, buf, sizeof(h));
    const lbm_config &c = ctx->cfg;
    if (std::memcmp(h.magic, "LBMSTATE", 8) != 0 || h.version != 1 || h.cfg.nx != c.nx || h.cfg.ny != c.ny ||
        h.cfg.nz != c.nz || h.cfg.batch != c.batch || h.cfg.precision != c.precision ||
        h.cfg.eq_order != c.eq_order || h.cfg.wall_model != c.wall_model ||
        h.cfg.rho0_shift[0] != c.rho0_shift[0] || h.cfg.rho0_shift[1] != c.rho0_shift[1])
        return ctx->fail(LBM_ERR_ARG, "lbm_set_state: configuration mismatch");
    const size_t cells = ctx->cells();
    if (h.f_bytes != ctx->f_bytes() || h.link_bytes != cells * 4 || h.macro_bytes != cells * 5 * ctx->tbytes() ||
        h.usnap_bytes != cells * 3 * ctx->tbytes() ||
        bytes < sizeof(h) + h.f_bytes + h.link_bytes + h.macro_bytes + h.usnap_bytes)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_state: size mismatch");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const char *p = (const char *)buf + sizeof(h);
    LBM_CUDA(cudaMemcpyAsync(ctx->f[ctx->cur], p, h.f_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state f");
    p += h.f_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->link, p, h.link_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state link");
    p += h.link_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->macro, p, h.macro_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state macro");
    p += h.macro_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->usnap, p, h.usnap_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state usnap");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "set_state sync");
    ctx->step = h.step;
    ctx->since_snap = h.since_snap;
    ctx->has_geometry = ctx->has_fields = true;
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) {
    if (ctx) return ctx->err.c_str();
    return g_last_error.c_str();
}

}  // extern "C"

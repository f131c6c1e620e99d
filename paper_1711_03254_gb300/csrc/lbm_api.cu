// Host runtime behind the C ABI of include/lbm.h: context, device buffers,
// argument checks, kernel dispatch, read-back and checkpoints.
#include <algorithm>
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
// the persistent cluster kernel loops each thread over cells of its instance
constexpr long long kClusterMaxCells = 65536;
// AUTO runs problems of at most this many non-solid cells (summed over the
// batch) with the persistent update: stepped from the host, and inside the
// steady loop's CUDA graphs
constexpr long long kPersistAutoItems = 65536, kPersistGraphItems = 32768;
constexpr int kMaxBatch = 32767;

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
    Ref *ref[2] = {nullptr, nullptr};  // reference densities, swapped with f (not used in FP64)
    int cur = 0;
    uint32_t *link = nullptr;
    uint32_t *list = nullptr;  // non-solid cells of each instance, in cell order [batch][n]
    int *list_count = nullptr; // entries per instance
    long long list_max = 0;
    long long nonsolid = 0;    // non-solid cells over all instances
    // compact layout: 0 = f, ref dense; 1 = compact (LBM_KERNEL_COMPACT, LBM_KERNEL_FUSED_COMPACT)
    int layout = 0;
    bool compact_ok = false;   // grid within the packed-coordinate limits
    uint32_t *cxyz = nullptr, *clink = nullptr;
    uint2 *rowtab = nullptr;
    int words = 0;
    bool in_graph = false;     // lbm_run_to_steady is resolving and capturing its updates
    unsigned *bar = nullptr;   // persistent update: barrier counter, give-up flag
    bool persist_used = false; // a persistent launch ran since the flag was last read
    long long bar_cycles = 4000000000LL;  // bound on a barrier wait (about 2 s of SM clock)
    unsigned bar_missing = 0;  // failure test: arrivals the barriers wait for that never come
    FcPlan fplan{};  // single-read fused update on the compact layout (ok when it fits)
    std::vector<uint32_t> plane_start;  // compact index of each plane's first cell (instance 0), nz + 1
    bool half_step = false;             // the density pass of a split update has run
    void *psi = nullptr, *macro = nullptr, *usnap = nullptr, *dpar = nullptr;
    double *partial = nullptr, *red_out = nullptr;
    int nblk = 0;
    bool has_geometry = false, has_fields = false;
    long long step = 0, since_snap = 0;
    long long launches = 0;
    lbm_kernel kernel = LBM_KERNEL_AUTO;
    int tile = -1, zchunk = -1;  // fused-kernel tiling; -1 = heuristic
    std::string err;

    // per-kernel event timing (lbm_timing_begin / lbm_timing_end)
    struct TimedLaunch {
        lbm_kernel kind;
        int first;  // index of its first event
    };
    bool timing = false;
    int timing_max = 0, timing_launches = 0;
    std::vector<cudaEvent_t> tev;
    int tev_used = 0;
    std::vector<TimedLaunch> timed;

    void drop_events() {
        for (cudaEvent_t e : tev) cudaEventDestroy(e);
        tev.clear();
        timed.clear();
        tev_used = 0;
        timing_launches = 0;
        timing = false;
    }
    // events for one launcher call of `kind`, or NULL when it is not timed
    cudaEvent_t *events_for(lbm_kernel kind) {
        if (!timing) return nullptr;
        const int kernels = (kind == LBM_KERNEL_TWO_PASS || kind == LBM_KERNEL_COMPACT) ? 2 : 1;
        const int nev = kernels + 1;
        if (timing_launches + kernels > timing_max || tev_used + nev > (int)tev.size()) return nullptr;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
        timed.push_back({kind, tev_used});
        cudaEvent_t *ev = &tev[tev_used];
        tev_used += nev;
        timing_launches += kernels;
        return ev;
    }

    bool fp64() const { return cfg.precision == LBM_FP64; }
    bool slip_on() const {
        for (const lbm_instance_params &p : par)
            if (p.slip != 0.0) return true;
        return false;
    }
    // the third-order regularisation and wall slip are built into the two-pass
    // strategies (TWO_PASS, COMPACT) only
    bool single_read_ok() const { return cfg.reg_order != 3 && !slip_on(); }
    size_t tbytes() const { return fp64() ? 8 : 4; }
    size_t cells() const { return (size_t)cfg.batch * (size_t)g.n; }
    size_t f_bytes() const { return cells() * 2 * 19 * storage_bytes(cfg.precision); }
    size_t ref_bytes() const { return fp64() ? 0 : cells() * 2 * sizeof(Ref); }

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
        q.slip = (T)p.slip;
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

// NULL if every instance's parameters are valid, else what is wrong.
const char *check_params(const lbm_instance_params *per_instance, int batch) {
    for (int b = 0; b < batch; ++b) {
        const lbm_instance_params &p = per_instance[b];
        if (!(p.tau[0] > 0.5) || !(p.tau[1] > 0.5)) return "tau must exceed 1/2";
        const double vals[] = {p.G, p.rho_s, p.g[0], p.g[1], p.g[2], p.rho_in[0], p.rho_in[1], p.u_in[0], p.u_in[1],
                               p.u_in[2], p.tau[0], p.tau[1]};
        for (double v : vals)
            if (!std::isfinite(v)) return "non-finite parameter";
        if (!(p.slip >= 0.0 && p.slip <= 1.0)) return "slip must lie in [0, 1]";
    }
    return nullptr;
}

// Strategy for an n-update call.  AUTO: the compact two-pass update when the
// grid fits its packed coordinates, the dense two-pass one otherwise.
lbm_kernel resolve_kernel(const lbm_ctx *ctx, int n) {
    // the fused compact update needs its rows and lag buffer to fit in shared
    // memory; where they do not, its layout's two-pass update runs
    if (ctx->kernel == LBM_KERNEL_FUSED_COMPACT) return ctx->fplan.ok ? LBM_KERNEL_FUSED_COMPACT : LBM_KERNEL_COMPACT;
    if (ctx->kernel != LBM_KERNEL_AUTO) return ctx->kernel;
    // small problems: one cooperative launch for the n updates, each thread
    // keeping its cell, beats two launches per update (GB300, FP32, us per
    // update, stepped from the host: 16^3 5.6 against 12.3, 16 x 16^3 9.3
    // against 14.4, even at 4 x 32^3; in the steady loop's CUDA graphs, where
    // launches are cheap: 16^3 6.2 against 7.0, 8 x 16^3 7.3 against 8.0, even
    // at 16 x 16^3; FP64, stepped: 16^3 28.1 against 34.8, the 16-instance
    // channel sweep 53.2 against 57.4)
    const long long items = (long long)ctx->cfg.batch * ctx->list_max;
    if (ctx->compact_ok && !ctx->slip_on() && n >= 8 &&
        items <= (ctx->in_graph ? kPersistGraphItems : kPersistAutoItems))
        return LBM_KERNEL_PERSISTENT;
    // measured on GB300: the two-pass update on the compact layout beats the
    // dense two-pass one on porous (1.5x) and all-fluid (1.1x) grids, the fused
    // one (2-4x), and the persistent cluster kernel on every small case tried
    // (16^3 to 32^3, 1 to 16 instances: 1.4-10x)
    return ctx->compact_ok ? LBM_KERNEL_COMPACT : LBM_KERNEL_TWO_PASS;
}

bool uses_compact_layout(lbm_kernel k) {
    return k == LBM_KERNEL_COMPACT || k == LBM_KERNEL_FUSED_COMPACT || k == LBM_KERNEL_PERSISTENT;
}

// the strategies whose kernels read f once per update (no slip, no
// third-order regularisation)
bool single_read(lbm_kernel k) {
    return k == LBM_KERNEL_FUSED || k == LBM_KERNEL_CLUSTER || k == LBM_KERNEL_FUSED_COMPACT;
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

// Plan of the single-read fused update on the compact layout: its lag buffer
// holds the non-solid cells of one group of rows of one plane, so the largest
// such count over the geometry (from the rows' first compact indices) sizes it.
lbm_status plan_fused_compact(lbm_ctx *ctx) {
    ctx->fplan = FcPlan{};
    ctx->plane_start.clear();
    if (!ctx->compact_ok) return LBM_OK;
    const int B = ctx->cfg.batch, ny = ctx->g.ny, nz = ctx->g.nz, rc = fusedc_rows_per_cta();
    const size_t rows = (size_t)ny * nz;
    std::vector<uint32_t> start((size_t)B * (rows + 1));
    for (int b = 0; b < B; ++b) {
        const uint2 *src = ctx->rowtab + (size_t)b * (rows + 1) * ctx->words;
        LBM_CUDA(cudaMemcpy2DAsync(start.data() + (size_t)b * (rows + 1), sizeof(uint32_t), src,
                                   sizeof(uint2) * ctx->words, sizeof(uint32_t), rows + 1, cudaMemcpyDeviceToHost,
                                   ctx->stream),
                 "fused plan: row starts");
    }
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "fused plan: row starts");
    ctx->plane_start.resize((size_t)nz + 1);
    for (int z = 0; z <= nz; ++z) ctx->plane_start[z] = start[(size_t)z * ny];
    if (ctx->fp64()) return LBM_OK;
    long long cap = 0;
    for (int b = 0; b < B; ++b) {
        const uint32_t *st = start.data() + (size_t)b * (rows + 1);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; y += rc) {
                const size_t r0 = (size_t)z * ny + y, r1 = (size_t)z * ny + std::min(y + rc, ny);
                cap = std::max<long long>(cap, (long long)st[r1] - (long long)st[r0]);
            }
    }
    LBM_CUDA(fusedc_plan(ctx->cfg.precision, ctx->cfg.eq_order, ctx->g, B, (int)std::max<long long>(cap, 1),
                         ctx->fplan),
             "fused plan");
    return LBM_OK;
}

// Lists of the non-solid cells of every instance (in cell order) for the
// two-pass kernels, and the static pseudo-potential of the SOLID cells, built
// on the device from the geometry words in ctx->link.  With the compact layout
// available, also the packed coordinates of the listed cells, their geometry
// words and the per-row occupancy words.  One read-back of the per-instance
// counts sets the compact stride kmax (the largest count).
lbm_status build_cell_lists(lbm_ctx *ctx) {
    const int B = ctx->cfg.batch;
    const size_t rows = (size_t)ctx->g.ny * ctx->g.nz;
    uint32_t *rowcnt = (uint32_t *)ctx->dalloc((size_t)B * rows * 4);
    if (!rowcnt) return ctx->fail(LBM_ERR_OOM, "cell lists: device allocation failed");
    uint2 *tab = ctx->compact_ok ? ctx->rowtab : nullptr;
    std::vector<int> cnt(B);
    cudaError_t e = launch_row_counts(ctx->link, ctx->g, B, rowcnt, ctx->list_count, tab, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt.data(), ctx->list_count, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost,
                            ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ctx->dfree(rowcnt);
        return ctx->cuda_fail(e, "cell lists");
    }
    long long mx = 0, total = 0;
    for (int b = 0; b < B; ++b) {
        total += cnt[b];
        if ((long long)cnt[b] > mx) mx = cnt[b];
    }
    ctx->list_max = mx;
    ctx->nonsolid = total;
    const size_t cells = ctx->cells();
    e = cudaMemsetAsync(ctx->list, 0, cells * 4, ctx->stream);
    if (e == cudaSuccess && ctx->compact_ok) e = cudaMemsetAsync(ctx->cxyz, 0, cells * 4, ctx->stream);
    if (e == cudaSuccess)
        e = launch_row_fill(ctx->link, ctx->g, B, rowcnt, ctx->list, ctx->compact_ok ? ctx->cxyz : nullptr, tab,
                            (uint32_t)mx, ctx->stream);
    if (e == cudaSuccess) e = launch_psi_solid(ctx->link, ctx->psi, ctx->fp64(), ctx->g, B, ctx->dpar, ctx->stream);
    if (e == cudaSuccess && ctx->compact_ok)
        e = launch_compact_links(ctx->list, ctx->list_count, ctx->link, ctx->clink, ctx->g, B, (uint32_t)mx,
                                 ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(rowcnt);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "cell lists");
    ctx->launches += ctx->compact_ok ? 5 : 4;
    return plan_fused_compact(ctx);
}

// Bring f and the reference densities of the current state into `want`
// (0 dense, 1 compact), through the other buffer.  Leaving the compact layout
// also restores psi of the SOLID cells, which compact updates overwrite.
lbm_status ensure_layout(lbm_ctx *ctx, int want) {
    if (ctx->layout == want) return LBM_OK;
    LBM_CUDA(launch_layout(ctx->cfg.precision, want == 1, ctx->f[ctx->cur], ctx->f[ctx->cur ^ 1], ctx->ref[ctx->cur],
                           ctx->ref[ctx->cur ^ 1], ctx->list, ctx->list_count, ctx->g, ctx->cfg.batch,
                           (uint32_t)ctx->list_max, ctx->stream),
             "layout conversion");
    ctx->launches += 1;
    if (want == 0) {
        LBM_CUDA(launch_psi_solid(ctx->link, ctx->psi, ctx->fp64(), ctx->g, ctx->cfg.batch, ctx->dpar, ctx->stream),
                 "solid psi");
        ctx->launches += 1;
    }
    ctx->cur ^= 1;
    ctx->layout = want;
    return LBM_OK;
}

StepArgs step_args(lbm_ctx *ctx, int write_macro) {
    StepArgs a{};
    a.precision = ctx->cfg.precision;
    a.eq_order = ctx->cfg.eq_order;
    a.reg_order = ctx->cfg.reg_order;
    a.slip = ctx->slip_on() ? 1 : 0;
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
    a.ref_in = ctx->ref[ctx->cur];
    a.ref_out = ctx->ref[ctx->cur ^ 1];
    a.list = ctx->list;
    a.list_count = ctx->list_count;
    a.list_max = ctx->list_max;
    a.cxyz = ctx->cxyz;
    a.clink = ctx->clink;
    a.rowtab = ctx->rowtab;
    a.words = ctx->words;
    a.kmax = (uint32_t)ctx->list_max;
    a.stream = ctx->stream;
    a.bar = ctx->bar;
    a.bar_cycles = ctx->bar_cycles;
    a.bar_missing = ctx->bar_missing;
    return a;
}

// After persistent launches: LBM_ERR_TIMEOUT if a grid-wide barrier gave up
// (its blocks then left the launch early and the state is not an update).
lbm_status check_barrier(lbm_ctx *ctx) {
    if (!ctx->persist_used) return LBM_OK;
    unsigned h[2] = {0, 0};
    LBM_CUDA(cudaMemcpyAsync(h, ctx->bar, sizeof h, cudaMemcpyDeviceToHost, ctx->stream), "barrier flag");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "barrier flag");
    ctx->persist_used = false;
    if (h[1]) return ctx->fail(LBM_ERR_TIMEOUT, "persistent update: a grid-wide barrier gave up waiting");
    return LBM_OK;
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
    // instances run along gridDim.y (at most 65535), the layout conversion
    // along 2 * batch of it
    if (cfg->batch > kMaxBatch) {
        g_last_error = "lbm_create: at most 32767 instances per context";
        return LBM_ERR_ARG;
    }
    // kernels index one component's 19 planes with 32-bit offsets
    if (19LL * cfg->nx * cfg->ny * cfg->nz >= (1LL << 32)) {
        g_last_error = "lbm_create: more than 226 million cells per instance";
        return LBM_ERR_ARG;
    }
    if (cfg->precision < LBM_FP64 || cfg->precision > LBM_FP32_BF16S || cfg->eq_order < 0 || cfg->eq_order > 1 ||
        cfg->wall_model < 0 || cfg->wall_model > 3 ||
        (cfg->reg_order != 0 && cfg->reg_order != 2 && cfg->reg_order != 3)) {
        g_last_error = "lbm_create: precision, eq_order, wall_model or reg_order out of range";
        return LBM_ERR_ARG;
    }
    if (const char *bad = check_params(per_instance, cfg->batch)) {
        g_last_error = std::string("lbm_create: ") + bad;
        return LBM_ERR_ARG;
    }
    lbm_ctx *ctx = new lbm_ctx();
    ctx->cfg = *cfg;
    ctx->cfg.reg_order = cfg->reg_order == 3 ? 3 : 2;
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
    if (!ctx->fp64()) {
        ctx->ref[0] = (Ref *)ctx->dalloc(ctx->ref_bytes());
        ctx->ref[1] = (Ref *)ctx->dalloc(ctx->ref_bytes());
    }
    ctx->link = (uint32_t *)ctx->dalloc(cells * 4);
    ctx->list = (uint32_t *)ctx->dalloc(cells * 4);
    ctx->compact_ok = cfg->nx <= kCompactMaxX && cfg->ny <= kCompactMaxY && cfg->nz <= kCompactMaxZ;
    if (ctx->compact_ok) {
        ctx->words = (cfg->nx + 31) / 32;
        ctx->cxyz = (uint32_t *)ctx->dalloc(cells * 4);
        ctx->clink = (uint32_t *)ctx->dalloc(cells * 4);
        ctx->rowtab = (uint2 *)ctx->dalloc((size_t)cfg->batch * ((size_t)cfg->ny * cfg->nz + 1) * ctx->words *
                                           sizeof(uint2));
        if (!ctx->cxyz || !ctx->clink || !ctx->rowtab) {
            g_last_error = "lbm_create: device allocation failed";
            lbm_destroy(ctx);
            return LBM_ERR_OOM;
        }
    }
    ctx->list_count = (int *)ctx->dalloc((size_t)cfg->batch * sizeof(int));
    if (!ctx->list || !ctx->list_count) {
        g_last_error = "lbm_create: device allocation failed";
        lbm_destroy(ctx);
        return LBM_ERR_OOM;
    }
    ctx->psi = ctx->dalloc(cells * 2 * ctx->tbytes());
    ctx->macro = ctx->dalloc(cells * 5 * ctx->tbytes());
    ctx->usnap = ctx->dalloc(cells * 3 * ctx->tbytes());
    ctx->dpar = ctx->dalloc((size_t)cfg->batch * sizeof(InstParam<double>));
    ctx->partial = (double *)ctx->dalloc((size_t)cfg->batch * ctx->nblk * 9 * sizeof(double));
    ctx->red_out = (double *)ctx->dalloc((size_t)cfg->batch * 9 * sizeof(double));
    ctx->bar = (unsigned *)ctx->dalloc(4 * sizeof(unsigned));
    if (!ctx->f[0] || !ctx->f[1] || (!ctx->fp64() && (!ctx->ref[0] || !ctx->ref[1])) || !ctx->link || !ctx->psi || !ctx->macro || !ctx->usnap || !ctx->dpar ||
        !ctx->partial || !ctx->red_out || !ctx->bar) {
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
    ctx->drop_events();
    std::vector<void *> own = ctx->owned;
    for (void *p : own) ctx->dfree(p);
    delete ctx;
}

lbm_status lbm_set_params(lbm_ctx *ctx, const lbm_instance_params *per_instance) {
    if (!ctx || !per_instance) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_set_params: null argument") : LBM_ERR_ARG;
    if (ctx->half_step) return ctx->fail(LBM_ERR_STATE, "lbm_set_params: finish the split update first");
    if (const char *bad = check_params(per_instance, ctx->cfg.batch))
        return ctx->fail(LBM_ERR_ARG, std::string("lbm_set_params: ") + bad);
    if (single_read(ctx->kernel) || ctx->kernel == LBM_KERNEL_PERSISTENT)
        for (int b = 0; b < ctx->cfg.batch; ++b)
            if (per_instance[b].slip != 0.0)
                return ctx->fail(LBM_ERR_ARG, "lbm_set_params: wall slip needs the TWO_PASS or COMPACT strategy");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    ctx->par.assign(per_instance, per_instance + ctx->cfg.batch);
    const lbm_status s = upload_params(ctx);
    if (s != LBM_OK) return s;
    // the dense layout keeps psi of the SOLID cells, which follows from rho^s
    if (ctx->has_geometry && ctx->layout == 0) {
        LBM_CUDA(launch_psi_solid(ctx->link, ctx->psi, ctx->fp64(), ctx->g, ctx->cfg.batch, ctx->dpar, ctx->stream),
                 "lbm_set_params: solid psi");
        ctx->launches += 1;
    }
    return LBM_OK;
}

lbm_status lbm_set_barrier_test(lbm_ctx *ctx, long long wait_cycles, unsigned missing) {
    if (!ctx) return LBM_ERR_ARG;
    if (wait_cycles < 1000) return ctx->fail(LBM_ERR_ARG, "lbm_set_barrier_test: wait_cycles below 1000");
    ctx->bar_cycles = wait_cycles;
    ctx->bar_missing = missing;
    return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return LBM_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_ctx *ctx, lbm_kernel kernel) {
    if (!ctx) return LBM_ERR_ARG;
    if (kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_PERSISTENT)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: unknown strategy");
    if (kernel == LBM_KERNEL_CLUSTER && ctx->g.n > kClusterMaxCells)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: CLUSTER needs at most 65536 cells per instance");
    if (kernel == LBM_KERNEL_COMPACT && !ctx->compact_ok)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: COMPACT needs nx <= 2048, ny <= 2048, nz <= 1024");
    if (kernel == LBM_KERNEL_FUSED_COMPACT && (!ctx->compact_ok || ctx->fp64()))
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: FUSED_COMPACT needs the compact layout and FP32 arithmetic");
    if (!ctx->single_read_ok() && single_read(kernel))
        return ctx->fail(LBM_ERR_ARG,
                         "lbm_set_kernel: reg_order 3 and wall slip run in the TWO_PASS and COMPACT strategies");
    if (kernel == LBM_KERNEL_PERSISTENT && (!ctx->compact_ok || ctx->slip_on()))
        return ctx->fail(LBM_ERR_ARG, "lbm_set_kernel: PERSISTENT needs the compact layout and no wall slip");
    ctx->kernel = kernel;
    return LBM_OK;
}

long long lbm_launch_count(const lbm_ctx *ctx) { return ctx ? ctx->launches : 0; }

int lbm_resolved_kernel(const lbm_ctx *ctx, int n) { return ctx ? (int)resolve_kernel(ctx, n) : -1; }

lbm_status lbm_timing_begin(lbm_ctx *ctx, int max_launches) {
    if (!ctx) return LBM_ERR_ARG;
    if (max_launches < 1 || max_launches > 65536)
        return ctx->fail(LBM_ERR_ARG, "lbm_timing_begin: max_launches must be in 1..65536");
    if (ctx->timing) return ctx->fail(LBM_ERR_STATE, "lbm_timing_begin: timing is already on");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    // at most 3 events per 2 launches (two-pass) or 2 per launch (fused, cluster)
    const int nev = 2 * max_launches + 1;
    ctx->tev.reserve((size_t)nev);
    for (int k = 0; k < nev; ++k) {
        cudaEvent_t e;
        const cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            ctx->drop_events();
            return ctx->cuda_fail(err, "lbm_timing_begin: cudaEventCreate");
        }
        ctx->tev.push_back(e);
    }
    ctx->timing_max = max_launches;
    ctx->timing = true;
    return LBM_OK;
}

lbm_status lbm_timing_end(lbm_ctx *ctx, double *ms, long long *launches) {
    if (!ctx) return LBM_ERR_ARG;
    if (!ms || !launches) return ctx->fail(LBM_ERR_ARG, "lbm_timing_end: null output array");
    if (!ctx->timing) return ctx->fail(LBM_ERR_STATE, "lbm_timing_end: timing is not on");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    for (int p = 0; p < LBM_PART_COUNT; ++p) {
        ms[p] = 0.0;
        launches[p] = 0;
    }
    cudaError_t e = cudaSuccess;
    if (ctx->tev_used > 0) e = cudaEventSynchronize(ctx->tev[ctx->tev_used - 1]);
    for (size_t k = 0; k < ctx->timed.size() && e == cudaSuccess; ++k) {
        const auto &t = ctx->timed[k];
        cudaEvent_t *ev = &ctx->tev[t.first];
        float a = 0.f, b = 0.f;
        if (t.kind == LBM_KERNEL_TWO_PASS || t.kind == LBM_KERNEL_COMPACT) {
            e = cudaEventElapsedTime(&a, ev[0], ev[1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
            ms[LBM_PART_PSI] += a;
            ms[LBM_PART_COLLIDE] += b;
            launches[LBM_PART_PSI] += 1;
            launches[LBM_PART_COLLIDE] += 1;
        } else {
            e = cudaEventElapsedTime(&a, ev[0], ev[1]);
            const int p = (t.kind == LBM_KERNEL_FUSED || t.kind == LBM_KERNEL_FUSED_COMPACT) ? LBM_PART_FUSED
                                                                                         : LBM_PART_CLUSTER;
            ms[p] += a;
            launches[p] += 1;
        }
    }
    ctx->drop_events();
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_timing_end: event query");
    return LBM_OK;
}

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
    const int B = ctx->cfg.batch;
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    // the types are checked on the device, before anything of the context changes
    uint8_t *dt = (uint8_t *)ctx->dalloc(cells + sizeof(int) * (size_t)(B + 1) + 16);
    if (!dt) return ctx->fail(LBM_ERR_OOM, "lbm_set_geometry: device allocation failed");
    int *dflags = (int *)(dt + ((cells + 15) / 16) * 16);
    std::vector<int> flags((size_t)B + 1);
    cudaError_t e = cudaMemcpyAsync(dt, cell_type, cells, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dflags, 0, flags.size() * sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_check_types(dt, ctx->g, B, dflags, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flags.data(), dflags, flags.size() * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ctx->dfree(dt);
        return ctx->cuda_fail(e, "lbm_set_geometry");
    }
    ctx->launches += 1;
    const char *bad = flags[0] ? "lbm_set_geometry: cell type above 3" : nullptr;
    for (int b = 0; b < B && !bad; ++b)
        if (!flags[1 + b]) bad = "lbm_set_geometry: an instance has no FLUID cell";
    if (bad) {
        ctx->dfree(dt);
        return ctx->fail(LBM_ERR_ARG, bad);
    }
    e = launch_links(dt, ctx->link, ctx->g, B, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(dt);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_set_geometry");
    ctx->launches += 1;
    lbm_status s = build_cell_lists(ctx);
    if (s != LBM_OK) return s;
    ctx->has_geometry = true;
    ctx->has_fields = false;
    ctx->half_step = false;
    ctx->layout = 0;
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
        a.ref_out = ctx->ref[ctx->cur];
        a.macro = ctx->macro;
        a.usnap = ctx->usnap;
        a.par = ctx->dpar;
        a.stream = ctx->stream;
        e = launch_init(a);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    ctx->dfree(d);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_set_fields");
    // the shifted storages first write the reference densities (k_init_ref)
    ctx->launches += (ctx->cfg.precision == LBM_FP32_F16S || ctx->cfg.precision == LBM_FP32_BF16S) ? 2 : 1;
    ctx->layout = 0;
    ctx->has_fields = true;
    ctx->half_step = false;
    ctx->since_snap = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *ctx, int n) {
    if (!ctx) return LBM_ERR_ARG;
    if (n < 0) return ctx->fail(LBM_ERR_ARG, "lbm_step: negative step count");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_step: call lbm_set_fields first");
    if (ctx->half_step) return ctx->fail(LBM_ERR_STATE, "lbm_step: finish the split update (lbm_step_part 1) first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const lbm_kernel k = resolve_kernel(ctx, n);
    if (n > 0) {
        const lbm_status ls = ensure_layout(ctx, uses_compact_layout(k) ? 1 : 0);
        if (ls != LBM_OK) return ls;
    }
    if (k == LBM_KERNEL_CLUSTER || k == LBM_KERNEL_PERSISTENT) {
        if (n > 0) {
            StepArgs a = step_args(ctx, 1);
            a.ev = ctx->events_for(k);
            cudaError_t e = k == LBM_KERNEL_CLUSTER ? launch_cluster(a, n) : launch_persist(a, n);
            if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_step persistent launch");
            if (k == LBM_KERNEL_PERSISTENT) ctx->persist_used = true;
            ctx->launches += 1;
            ctx->cur ^= (n & 1);
        }
        ctx->step += n;
        ctx->since_snap += n;
        return LBM_OK;
    }
    const bool fused = k == LBM_KERNEL_FUSED;
    const bool one_launch = fused || k == LBM_KERNEL_FUSED_COMPACT;
    int tile = ctx->tile, zchunk = ctx->zchunk;
    if (fused) default_tiling(ctx, tile, zchunk);
    for (int s = 0; s < n; ++s) {
        StepArgs a = step_args(ctx, s == n - 1);
        a.ev = ctx->events_for(k);
        cudaError_t e = fused ? launch_fused(a, tile, zchunk)
                        : k == LBM_KERNEL_FUSED_COMPACT ? launch_fusedc(a, ctx->fplan)
                        : (k == LBM_KERNEL_COMPACT ? launch_compact(a) : launch_two_pass(a));
        if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_step launch");
        ctx->launches += one_launch ? 1 : 2;
        ctx->cur ^= 1;
    }
    ctx->step += n;
    ctx->since_snap += n;
    return LBM_OK;
}

lbm_status lbm_step_part(lbm_ctx *ctx, int part) {
    if (!ctx) return LBM_ERR_ARG;
    if (part != 0 && part != 1) return ctx->fail(LBM_ERR_ARG, "lbm_step_part: part must be 0 or 1");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_step_part: call lbm_set_fields first");
    if (!ctx->compact_ok) return ctx->fail(LBM_ERR_ARG, "lbm_step_part: needs the compact layout's limits");
    if ((part == 1) != ctx->half_step)
        return ctx->fail(LBM_ERR_STATE, part ? "lbm_step_part: run the density pass (part 0) first"
                                             : "lbm_step_part: the collision pass (part 1) is pending");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const lbm_status ls = ensure_layout(ctx, 1);
    if (ls != LBM_OK) return ls;
    StepArgs a = step_args(ctx, 1);
    LBM_CUDA(launch_compact(a, part == 0 ? 1 : 2), "lbm_step_part launch");
    ctx->launches += 1;
    if (part == 1) {
        ctx->cur ^= 1;
        ctx->step += 1;
        ctx->since_snap += 1;
    }
    ctx->half_step = part == 0;
    return LBM_OK;
}

// D3Q19 directions (this library's order) with c_z = +1 and c_z = -1
static const int kUpDirs[5] = {5, 11, 14, 15, 18};
static const int kDownDirs[5] = {6, 12, 13, 16, 17};

static lbm_status plane_args(lbm_ctx *ctx, int what, int z, size_t &cells, size_t &unit) {
    if (ctx->cfg.batch != 1) return ctx->fail(LBM_ERR_ARG, "plane copy: one instance per context only");
    if (what < LBM_PLANE_F_UP || what > LBM_PLANE_PSI) return ctx->fail(LBM_ERR_ARG, "plane copy: unknown part");
    if (z < 0 || z >= ctx->g.nz) return ctx->fail(LBM_ERR_ARG, "plane copy: plane out of range");
    if (!ctx->compact_ok || ctx->plane_start.size() != (size_t)ctx->g.nz + 1)
        return ctx->fail(LBM_ERR_STATE, "plane copy: needs a geometry within the compact layout's limits");
    cells = ctx->plane_start[z + 1] - ctx->plane_start[z];
    const size_t pair_f = 2 * storage_bytes(ctx->cfg.precision), pair_psi = 2 * ctx->tbytes();
    unit = what == LBM_PLANE_PSI ? pair_psi : 5 * pair_f;
    return LBM_OK;
}

lbm_status lbm_plane_bytes(lbm_ctx *ctx, int what, int z, size_t *bytes) {
    if (!ctx || !bytes) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_plane_bytes: null argument") : LBM_ERR_ARG;
    size_t cells = 0, unit = 0;
    const lbm_status s = plane_args(ctx, what, z, cells, unit);
    if (s != LBM_OK) return s;
    *bytes = cells * unit;
    return LBM_OK;
}

lbm_status lbm_plane_copy(lbm_ctx *ctx, int what, int z, void *buf, int to_buf) {
    if (!ctx || !buf) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_plane_copy: null argument") : LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_plane_copy: call lbm_set_fields first");
    size_t cells = 0, unit = 0;
    const lbm_status s = plane_args(ctx, what, z, cells, unit);
    if (s != LBM_OK) return s;
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const lbm_status ls = ensure_layout(ctx, 1);
    if (ls != LBM_OK) return ls;
    const size_t k0 = ctx->plane_start[z];
    char *b = (char *)buf;
    if (what == LBM_PLANE_PSI) {
        char *d = (char *)ctx->psi + k0 * unit;
        LBM_CUDA(cudaMemcpyAsync(to_buf ? (void *)b : (void *)d, to_buf ? (const void *)d : (const void *)b,
                                 cells * unit, cudaMemcpyDefault, ctx->stream),
                 "lbm_plane_copy");
    } else {
        const size_t pair = unit / 5, kmax = (size_t)ctx->list_max;
        const int *dirs = what == LBM_PLANE_F_UP ? kUpDirs : kDownDirs;
        for (int m = 0; m < 5; ++m) {
            char *d = (char *)ctx->f[ctx->cur] + ((size_t)dirs[m] * kmax + k0) * pair;
            char *h = b + (size_t)m * cells * pair;
            LBM_CUDA(cudaMemcpyAsync(to_buf ? (void *)h : (void *)d, to_buf ? (const void *)d : (const void *)h,
                                     cells * pair, cudaMemcpyDefault, ctx->stream),
                     "lbm_plane_copy");
        }
    }
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "lbm_plane_copy");
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
    return check_barrier(ctx);
}

lbm_status lbm_reduce(lbm_ctx *ctx, double *out) {
    if (!ctx || !out) return ctx ? ctx->fail(LBM_ERR_ARG, "lbm_reduce: null argument") : LBM_ERR_ARG;
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_reduce: no fields yet");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    {
        const lbm_status bs = check_barrier(ctx);
        if (bs != LBM_OK) return bs;
    }
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
    if (ensure_layout(ctx, 0) != LBM_OK) return LBM_ERR_CUDA;
    const size_t vals = ctx->cells() * 2 * 19;
    double *d = (double *)ctx->dalloc(vals * 8);
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_get_distributions: device allocation failed");
    cudaError_t e = launch_f_convert(ctx->cfg.precision, ctx->f[ctx->cur], d, nullptr, nullptr, ctx->ref[ctx->cur],
                                     ctx->link, ctx->g, ctx->cfg.batch, ctx->stream);
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
    if (ensure_layout(ctx, 0) != LBM_OK) return LBM_ERR_CUDA;
    const size_t vals = ctx->cells() * 2 * 19;
    double *d = (double *)ctx->dalloc(vals * 8);
    if (!d) return ctx->fail(LBM_ERR_OOM, "lbm_set_distributions: device allocation failed");
    cudaError_t e = cudaMemcpyAsync(d, f, vals * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = launch_f_convert(ctx->cfg.precision, nullptr, nullptr, d, ctx->f[ctx->cur], ctx->ref[ctx->cur],
                             ctx->link, ctx->g, ctx->cfg.batch, ctx->stream);
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
    uint32_t layout;  // 0 dense, 1 compact
    lbm_config cfg;
    long long step, since_snap;
    uint64_t f_bytes, ref_bytes, link_bytes, macro_bytes, usnap_bytes;
};
}  // namespace

lbm_status lbm_get_state(lbm_ctx *ctx, void *buf, size_t *bytes) {
    if (!ctx || !bytes) return LBM_ERR_ARG;
    const size_t cells = ctx->cells();
    StateHeader h{};
    std::memcpy(h.magic, "LBMSTATE", 8);
    h.version = 3;
    h.cfg = ctx->cfg;
    h.layout = (uint32_t)ctx->layout;
    h.step = ctx->step;
    h.since_snap = ctx->since_snap;
    h.f_bytes = ctx->f_bytes();
    h.ref_bytes = ctx->ref_bytes();
    h.link_bytes = cells * 4;
    h.macro_bytes = cells * 5 * ctx->tbytes();
    h.usnap_bytes = cells * 3 * ctx->tbytes();
    const size_t need = sizeof(h) + h.f_bytes + h.ref_bytes + h.link_bytes + h.macro_bytes + h.usnap_bytes;
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
    if (h.ref_bytes)
        LBM_CUDA(cudaMemcpyAsync(p, ctx->ref[ctx->cur], h.ref_bytes, cudaMemcpyDeviceToHost, ctx->stream),
                 "get_state ref");
    p += h.ref_bytes;
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
    if (std::memcmp(h.magic, "LBMSTATE", 8) != 0 || h.version != 3 || h.cfg.nx != c.nx || h.cfg.ny != c.ny ||
        h.cfg.nz != c.nz || h.cfg.batch != c.batch || h.cfg.precision != c.precision ||
        h.cfg.eq_order != c.eq_order || h.cfg.wall_model != c.wall_model || h.cfg.reg_order != c.reg_order)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_state: configuration mismatch");
    const size_t cells = ctx->cells();
    if (h.f_bytes != ctx->f_bytes() || h.ref_bytes != ctx->ref_bytes() || h.link_bytes != cells * 4 ||
        h.macro_bytes != cells * 5 * ctx->tbytes() || h.usnap_bytes != cells * 3 * ctx->tbytes() ||
        bytes < sizeof(h) + h.f_bytes + h.ref_bytes + h.link_bytes + h.macro_bytes + h.usnap_bytes)
        return ctx->fail(LBM_ERR_ARG, "lbm_set_state: size mismatch");
    if (h.layout > 1 || (h.layout == 1 && !ctx->compact_ok))
        return ctx->fail(LBM_ERR_ARG, "lbm_set_state: layout mismatch");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    const char *p = (const char *)buf + sizeof(h);
    LBM_CUDA(cudaMemcpyAsync(ctx->f[ctx->cur], p, h.f_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state f");
    p += h.f_bytes;
    if (h.ref_bytes)
        LBM_CUDA(cudaMemcpyAsync(ctx->ref[ctx->cur], p, h.ref_bytes, cudaMemcpyHostToDevice, ctx->stream),
                 "set_state ref");
    p += h.ref_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->link, p, h.link_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state link");
    p += h.link_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->macro, p, h.macro_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state macro");
    p += h.macro_bytes;
    LBM_CUDA(cudaMemcpyAsync(ctx->usnap, p, h.usnap_bytes, cudaMemcpyHostToDevice, ctx->stream), "set_state usnap");
    LBM_CUDA(cudaStreamSynchronize(ctx->stream), "set_state sync");
    {
        // the geometry words are on the device now
        lbm_status s = build_cell_lists(ctx);
        if (s != LBM_OK) return s;
    }
    ctx->step = h.step;
    ctx->since_snap = h.since_snap;
    ctx->layout = (int)h.layout;
    ctx->has_geometry = ctx->has_fields = true;
    ctx->half_step = false;
    return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *ctx, int steps_per_trial, const char *cache_path, int chosen[3]) {
    if (!ctx) return LBM_ERR_ARG;
    if (steps_per_trial < 1) return ctx->fail(LBM_ERR_ARG, "lbm_autotune: steps_per_trial < 1");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_autotune: call lbm_set_fields first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    cudaDeviceProp prop;
    LBM_CUDA(cudaGetDeviceProperties(&prop, ctx->dev), "cudaGetDeviceProperties");
    char key[512];
    std::snprintf(key, sizeof key, "%dx%dx%d b%d p%d e%d w%d r%d %s", ctx->cfg.nx, ctx->cfg.ny, ctx->cfg.nz,
                  ctx->cfg.batch, (int)ctx->cfg.precision, ctx->cfg.eq_order, ctx->cfg.wall_model,
                  ctx->cfg.reg_order, prop.name);
    for (char *c = key; *c; ++c)
        if (*c == '"' || *c == '\\') *c = '_';
    auto apply = [&](int k, int t, int z) {
        ctx->kernel = (lbm_kernel)k;
        ctx->tile = t;
        ctx->zchunk = z;
        if (chosen) {
            chosen[0] = k;
            chosen[1] = t;
            chosen[2] = z;
        }
    };
    if (cache_path) {
        if (FILE *fp = std::fopen(cache_path, "r")) {
            char line[1024];
            int hit = 0, k = 0, t = 0, z = 0;
            while (std::fgets(line, sizeof line, fp)) {
                char kbuf[512];
                int kk, tt, zz;
                double ms;
                if (std::sscanf(line, "{\"key\": \"%511[^\"]\", \"kernel\": %d, \"tile\": %d, \"zchunk\": %d, \"ms\": %lf",
                                kbuf, &kk, &tt, &zz, &ms) == 5 &&
                    std::strcmp(kbuf, key) == 0) {
                    hit = 1;
                    k = kk;
                    t = tt;
                    z = zz;
                }
            }
            std::fclose(fp);
            if (hit) {
                apply(k, t, z);
                return LBM_OK;
            }
        }
    }
    // save the state: both f and reference buffers of the current side, fields
    const size_t fb = ctx->f_bytes(), rb = ctx->ref_bytes(), mb = ctx->cells() * 5 * ctx->tbytes();
    void *sf = ctx->dalloc(fb);
    void *sr = rb ? ctx->dalloc(rb) : nullptr;
    void *smac = ctx->dalloc(mb);
    if (!sf || (rb && !sr) || !smac) {
        ctx->dfree(sf);
        ctx->dfree(sr);
        ctx->dfree(smac);
        return ctx->fail(LBM_ERR_OOM, "lbm_autotune: no room to save the state");
    }
    const int cur0 = ctx->cur, layout0 = ctx->layout;
    const long long step0 = ctx->step, snap0 = ctx->since_snap, launches0 = ctx->launches;
    const lbm_kernel k_save = ctx->kernel;
    const int t_save = ctx->tile, z_save = ctx->zchunk;
    cudaError_t e = cudaMemcpyAsync(sf, ctx->f[cur0], fb, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && rb) e = cudaMemcpyAsync(sr, ctx->ref[cur0], rb, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(smac, ctx->macro, mb, cudaMemcpyDeviceToDevice, ctx->stream);
    struct Cand {
        int k, t, z;
    };
    std::vector<Cand> cands;
    cands.push_back({LBM_KERNEL_TWO_PASS, -1, -1});
    if (ctx->compact_ok) cands.push_back({LBM_KERNEL_COMPACT, -1, -1});
    const bool single_read_ok = ctx->single_read_ok();
    if (ctx->fplan.ok && single_read_ok) cands.push_back({LBM_KERNEL_FUSED_COMPACT, -1, -1});
    if (ctx->g.n <= kClusterMaxCells && single_read_ok) cands.push_back({LBM_KERNEL_CLUSTER, -1, -1});
    if (ctx->compact_ok && !ctx->slip_on()) cands.push_back({LBM_KERNEL_PERSISTENT, -1, -1});
    for (int t = 0; single_read_ok && t < fused_tile_count(); ++t) {
        cands.push_back({LBM_KERNEL_FUSED, t, -1});
        for (int z : {8, 16, 32, 64})
            if (z < ctx->g.nz) cands.push_back({LBM_KERNEL_FUSED, t, z});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    Cand pick = cands.front();
    lbm_status st = LBM_OK;
    for (const Cand &c : cands) {
        if (e != cudaSuccess) break;
        ctx->kernel = (lbm_kernel)c.k;
        ctx->tile = c.t;
        ctx->zchunk = c.z;
        st = lbm_step(ctx, steps_per_trial);  // warm-up (also compiles nothing: all code is ahead-of-time)
        if (st != LBM_OK) break;
        e = cudaEventRecord(e0, ctx->stream);
        if (e != cudaSuccess) break;
        st = lbm_step(ctx, steps_per_trial);
        if (st != LBM_OK) break;
        e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
            best = ms;
            pick = c;
        }
        // restore the saved state for the next candidate (a compact trial
        // overwrote psi of the SOLID cells, which the dense kernels read)
        ctx->cur = cur0;
        if (ctx->layout != layout0 && layout0 == 0 && e == cudaSuccess)
            e = launch_psi_solid(ctx->link, ctx->psi, ctx->fp64(), ctx->g, ctx->cfg.batch, ctx->dpar, ctx->stream);
        ctx->layout = layout0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->f[cur0], sf, fb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess && rb)
            e = cudaMemcpyAsync(ctx->ref[cur0], sr, rb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->macro, smac, mb, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    ctx->dfree(sf);
    ctx->dfree(sr);
    ctx->dfree(smac);
    ctx->cur = cur0;
    ctx->layout = layout0;
    ctx->step = step0;
    ctx->since_snap = snap0;
    (void)launches0;
    if (st != LBM_OK || e != cudaSuccess) {
        ctx->kernel = k_save;
        ctx->tile = t_save;
        ctx->zchunk = z_save;
        return st != LBM_OK ? st : ctx->cuda_fail(e, "lbm_autotune");
    }
    if (pick.k == LBM_KERNEL_FUSED) default_tiling(ctx, pick.t, pick.z);
    apply(pick.k, pick.t, pick.z);
    if (cache_path) {
        if (FILE *fp = std::fopen(cache_path, "a")) {
            std::fprintf(fp, "{\"key\": \"%s\", \"kernel\": %d, \"tile\": %d, \"zchunk\": %d, \"ms\": %.6f}\n", key,
                         pick.k, pick.t, pick.z, best / steps_per_trial);
            std::fclose(fp);
        }
    }
    return LBM_OK;
}

lbm_status lbm_run_to_steady(lbm_ctx *ctx, int check_every, double tol, int max_steps, int *steps_done,
                             double *residual) {
    if (!ctx) return LBM_ERR_ARG;
    if (check_every < 1 || max_steps < 0) return ctx->fail(LBM_ERR_ARG, "lbm_run_to_steady: bad counts");
    if (!ctx->has_fields) return ctx->fail(LBM_ERR_STATE, "lbm_run_to_steady: call lbm_set_fields first");
    LBM_CUDA(cudaSetDevice(ctx->dev), "cudaSetDevice");
    // AUTO resolves for graph replay while this call runs
    struct InGraph {
        lbm_ctx *c;
        explicit InGraph(lbm_ctx *c_) : c(c_) { c->in_graph = true; }
        ~InGraph() { c->in_graph = false; }
    } in_graph(ctx);
    const int B = ctx->cfg.batch;
    {
        // convert the layout now: a conversion must not be captured into the graphs
        const lbm_status ls = ensure_layout(ctx, uses_compact_layout(resolve_kernel(ctx, check_every)) ? 1 : 0);
        if (ls != LBM_OK) return ls;
    }
    // capture on a private stream ordered after the context's stream
    cudaStream_t cs = nullptr;
    LBM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    double *hres = nullptr;
    cudaError_t e = cudaMallocHost(&hres, (size_t)B * 9 * sizeof(double));
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t user = ctx->stream;
    const int cur0 = ctx->cur;
    auto capture = [&](int parity) -> cudaError_t {
        // record check_every updates + reduction + read-back starting from side `parity`
        cudaGraph_t gph = nullptr;
        const long long st0 = ctx->step, sn0 = ctx->since_snap, la0 = ctx->launches;
        ctx->stream = cs;
        ctx->cur = parity;
        cudaError_t ee = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ee != cudaSuccess) return ee;
        lbm_status s1 = lbm_step(ctx, check_every);
        ReduceArgs a{};
        a.fp64 = ctx->fp64();
        a.batch = B;
        a.g = ctx->g;
        a.macro = ctx->macro;
        a.usnap = ctx->usnap;
        a.link = ctx->link;
        a.partial = ctx->partial;
        a.nblk = ctx->nblk;
        a.out = ctx->red_out;
        a.stream = cs;
        int nl = 0;
        cudaError_t e2 = s1 == LBM_OK ? launch_reduce(a, &nl) : cudaErrorUnknown;
        if (e2 == cudaSuccess)
            e2 = cudaMemcpyAsync(hres, ctx->red_out, (size_t)B * 9 * sizeof(double), cudaMemcpyDeviceToHost, cs);
        ee = cudaStreamEndCapture(cs, &gph);
        if (ee == cudaSuccess) ee = e2;
        if (ee == cudaSuccess) ee = cudaGraphInstantiate(&exec[parity], gph, 0);
        if (gph) cudaGraphDestroy(gph);
        ctx->stream = user;
        ctx->cur = cur0;
        ctx->step = st0;
        ctx->since_snap = sn0;
        ctx->launches = la0;
        return ee;
    };
    if (e == cudaSuccess) e = capture(cur0);
    if (e == cudaSuccess && (check_every & 1)) e = capture(cur0 ^ 1);
    // order the private stream after work already queued on the user stream
    cudaEvent_t ev = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    int done = 0;
    bool diverged = false, conv = false;
    const lbm_kernel kres = resolve_kernel(ctx, check_every);
    const long long launches_per_replay =
        ((kres == LBM_KERNEL_CLUSTER || kres == LBM_KERNEL_PERSISTENT) ? 1
         : (kres == LBM_KERNEL_FUSED || kres == LBM_KERNEL_FUSED_COMPACT) ? check_every
                                                                         : 2LL * check_every) + 2;
    ctx->since_snap = 0;  // the first replay measures against the current snapshot
    while (e == cudaSuccess && done + check_every <= max_steps) {
        e = cudaGraphLaunch(exec[ctx->cur], cs);  // graphs are indexed by the side holding the state
        if (e != cudaSuccess) break;
        e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) break;
        done += check_every;
        ctx->cur ^= (check_every & 1);
        ctx->step += check_every;
        ctx->launches += launches_per_replay;
        conv = true;
        for (int b = 0; b < B; ++b) {
            const double *r = hres + (size_t)b * 9;
            const double res = std::sqrt(r[5]) / ((double)check_every * std::sqrt(r[6]) + 1e-30);
            if (residual) residual[b] = res;
            // the same divergence test as lbm_reduce: a non-finite value, or
            // |u_F| above the lattice sound speed
            if (r[8] > 0 || !std::isfinite(res) || r[7] > kMaxSpeed) diverged = true;
            if (!(res <= tol)) conv = false;
        }
        if (diverged || conv) break;
    }
    ctx->since_snap = 0;
    if (steps_done) *steps_done = done;
    if (ev) cudaEventDestroy(ev);
    for (auto &x : exec)
        if (x) cudaGraphExecDestroy(x);
    if (hres) cudaFreeHost(hres);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return ctx->cuda_fail(e, "lbm_run_to_steady");
    if (kres == LBM_KERNEL_PERSISTENT) {
        ctx->persist_used = true;
        const lbm_status bs = check_barrier(ctx);
        if (bs != LBM_OK) return bs;
    }
    if (diverged)
        return ctx->fail(LBM_ERR_DIVERGED, "lbm_run_to_steady: non-finite value or |u_F| above the lattice sound speed");
    if (!conv) return ctx->fail(LBM_ERR_TIMEOUT, "lbm_run_to_steady: max_steps used up before the tolerance");
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *ctx) {
    if (ctx) return ctx->err.c_str();
    return g_last_error.c_str();
}

}  // extern "C"

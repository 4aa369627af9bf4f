// C-ABI layer of libvlasov: descriptor validation, workspace layout and the
// entry points declared in include/vlasov.h. Every compute call only
// enqueues kernels on the caller's stream.
#include <nvtx3/nvToolsExt.h>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "mlp_common.cuh"

struct vl_ctx {
    vl_desc d;
    void* f[VL_MAX_SPECIES];
    double* fluid;
    double* yee;
    double* eb;
    vl::Workspace ws;
    vl::MomConv conv[VL_MAX_SPECIES];
    // MLP warm start (workspace sections)
    float* mlp_w;           // [NPARAM] FP32 parameters
    float* mlp_m;           // Adam first moments
    float* mlp_v;           // Adam second moments
    float* mlp_g;           // gradient accumulator
    double* mlp_acc;        // [45] sample statistics, then [1] loss
    double* mlp_loss;
    int* mlp_err;
    float* mlp_pred;        // [ncell][2][10] predictions of the current species
    unsigned long long* harvest_count;
    bool mlp_ready;
    int adam_step;
    float* harvest;
    long long harvest_cap;
    int fit_mode[VL_MAX_SPECIES];   // moment_fit_wide: -1 chosen on the device, 0 common, 1 wide
    int* status_host;               // status word: pinned host memory mapped into the device
    int* status_dev;                // its device-side address
    char err[512];
};

static_assert(VL_MLP_NPARAM == vl::mlp::kNParam, "parameter blob size");
static_assert(VL_MLP_SAMPLE == vl::mlp::kSample, "sample size");

namespace vl {
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n); }
}  // namespace vl

namespace {

// errors of calls without a context (per host thread)
thread_local char g_err[512] = "";

// NVTX range around a compute entry point, named after the call, so that a
// profiler can select the kernels one call launched (ncu --nvtx
// --nvtx-include "moment_fit_solve/"); a no-op unless a tool is attached.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

vl_status fail(vl_ctx* ctx, vl_status st, const char* fmt, ...) {
    char* buf = ctx ? ctx->err : g_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    return st;
}

vl_status cuda_check(vl_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return VL_OK;
    return fail(ctx, VL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

long long ncell_of(const vl_desc& d) { return (long long)d.nx * d.ny; }

long long vblock_of(const vl_desc& d, int s) {
    return d.nvdim == 1 ? d.nv[s][0] : (long long)d.nv[s][0] * d.nv[s][1] * d.nv[s][2];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t cellwork, coef_v, coef_f, status, u1, u2, cur, fluid_f, counters, select;
    size_t mlp_w, mlp_m, mlp_v, mlp_g, mlp_acc, mlp_err, mlp_pred, harvest_count, total;
};

Layout layout_of(const vl_desc& d) {
    Layout L;
    const size_t nc = (size_t)ncell_of(d);
    size_t off = 0;
    L.cellwork = off; off = align256(off + nc * 20 * sizeof(double));
    L.coef_v = off; off = align256(off + nc * 16 * sizeof(double));
    L.coef_f = off; off = align256(off + nc * 16 * sizeof(double));
    L.status = off; off = align256(off + nc * 2 * sizeof(int));
    L.u1 = off; off = align256(off + nc * 10 * sizeof(double));
    L.u2 = off; off = align256(off + nc * 10 * sizeof(double));
    L.cur = off; off = align256(off + nc * 3 * sizeof(double));
    L.fluid_f = off; off = align256(off + 2 * nc * 10 * sizeof(float));
    L.counters = off; off = align256(off + VL_NSTATS * sizeof(unsigned long long));
    L.select = off; off = align256(off + 2 * sizeof(unsigned long long));
    const size_t np = (size_t)VL_MLP_NPARAM * sizeof(float);
    L.mlp_w = off; off = align256(off + np);
    L.mlp_m = off; off = align256(off + np);
    L.mlp_v = off; off = align256(off + np);
    L.mlp_g = off; off = align256(off + np);
    L.mlp_acc = off; off = align256(off + 56 * sizeof(double));
    L.mlp_err = off; off = align256(off + sizeof(int));
    L.mlp_pred = off; off = align256(off + nc * 20 * sizeof(float));
    L.harvest_count = off; off = align256(off + sizeof(unsigned long long));
    L.total = off;
    return L;
}

bool supported_block(int n) { return n == 8 || n == 12 || n == 16 || n == 20 || n == 24; }

vl_status validate(const vl_desc* d, vl_ctx* ctx) {
    if (!d) return fail(ctx, VL_EINVAL, "descriptor is NULL");
    if (d->nvdim != 1 && d->nvdim != 3) return fail(ctx, VL_EINVAL, "nvdim must be 1 or 3 (got %d)", d->nvdim);
    if (d->nx < 1 || d->ny < 1 || d->nx > 65535 || d->ny > 65535)
        return fail(ctx, VL_EINVAL, "nx, ny must be in [1, 65535]");
    if (d->nvdim == 1 && d->ny != 1) return fail(ctx, VL_EINVAL, "1D1V needs ny = 1");
    if (!(d->dx > 0.0) || !(d->dy > 0.0)) return fail(ctx, VL_EINVAL, "dx, dy must be positive");
    if (d->bc_y != 0 && d->bc_y != 1) return fail(ctx, VL_EINVAL, "bc_y must be 0 or 1");
    if (d->bc_y == 1 && (d->nvdim != 3 || d->ny < 3)) return fail(ctx, VL_EINVAL, "walls in y need 2D3V and ny >= 3");
    if (d->nspecies < 1 || d->nspecies > VL_MAX_SPECIES)
        return fail(ctx, VL_EINVAL, "nspecies must be in [1, %d]", VL_MAX_SPECIES);
    if (d->precision != 32 && d->precision != 64) return fail(ctx, VL_EINVAL, "precision must be 32 or 64");
    if (d->nshear != 3 && d->nshear != 5) return fail(ctx, VL_EINVAL, "nshear must be 3 or 5");
    if (!(d->fit_tol > 0.0) || d->fit_max_iter < 1 || d->fit_max_iter > 1000)
        return fail(ctx, VL_EINVAL, "fit_tol must be > 0 and fit_max_iter in [1, 1000]");
    if (d->nvdim == 3 && !(d->c > 0.0)) return fail(ctx, VL_EINVAL, "2D3V needs the speed of light c > 0");
    for (int s = 0; s < d->nspecies; ++s) {
        if (!(d->m[s] > 0.0) || !std::isfinite(d->q[s])) return fail(ctx, VL_EINVAL, "species %d: bad q or m", s);
        int na = d->nvdim == 1 ? 1 : 3;
        for (int a = 0; a < na; ++a) {
            if (d->nv[s][a] < 1) return fail(ctx, VL_EINVAL, "species %d: nv must be positive", s);
            if (!(d->vmax[s][a] > d->vmin[s][a])) return fail(ctx, VL_EINVAL, "species %d: vmax <= vmin", s);
        }
        if (d->nvdim == 1) {
            if (d->nv[s][0] > 64) return fail(ctx, VL_ENOTSUP, "1D1V supports nv <= 64");
        } else {
            if (d->nv[s][0] != d->nv[s][1] || d->nv[s][0] != d->nv[s][2])
                return fail(ctx, VL_ENOTSUP, "species %d: the velocity block must be cubic", s);
            if (!supported_block(d->nv[s][0]))
                return fail(ctx, VL_ENOTSUP, "species %d: nv = %d not compiled (8, 12, 16, 20, 24)", s, d->nv[s][0]);
            if (d->bc_y == 1) {
                double lo = d->vmin[s][1], hi = d->vmax[s][1];
                if (std::fabs(lo + hi) > 1e-12 * (hi - lo))
                    return fail(ctx, VL_EINVAL, "species %d: reflecting walls need a v_y box symmetric about 0", s);
            }
        }
    }
    return VL_OK;
}

double dv_of(const vl_desc& d, int s, int a) {
    return (d.vmax[s][a] - d.vmin[s][a]) / d.nv[s][a];
}

void fill_box(const vl_desc& d, int s, double* vmin, double* dv) {
    for (int a = 0; a < 3; ++a) {
        bool used = d.nvdim == 3 || a == 0;
        vmin[a] = used ? d.vmin[s][a] : 0.0;
        dv[a] = used ? dv_of(d, s, a) : 1.0;
    }
}

// The status word: a kernel that finds a numeric error (non-finite or
// negative fit targets) writes VL_ENUMERIC there; the next compute call on
// the context reports it (and clears it) instead of enqueueing its work.
vl_status pending_numeric(vl_ctx* ctx) {
    volatile int* w = ctx->status_host;
    const int v = *w;
    if (v == VL_OK) return VL_OK;
    *w = VL_OK;
    return fail(ctx, (vl_status)v,
                "a kernel of an earlier call found non-finite or negative fit targets (moments of f or fluid state)");
}

vl_status check_ctx(vl_ctx* ctx) {
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    return pending_numeric(ctx);
}

vl_status check_species(vl_ctx* ctx, int s) {
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    vl_status st = pending_numeric(ctx);
    if (st != VL_OK) return st;
    if (s < 0 || s >= ctx->d.nspecies) return fail(ctx, VL_EINVAL, "species %d out of range", s);
    if (!ctx->f[s]) return fail(ctx, VL_EINVAL, "species %d has no distribution function (fluid-only context)", s);
    return VL_OK;
}

}  // namespace

extern "C" {

size_t vlasov_work_bytes(const vl_desc* desc) {
    if (validate(desc, nullptr) != VL_OK) return 0;
    return layout_of(*desc).total;
}

vl_status vlasov_init(const vl_desc* desc, void* const* f_dev, double* fluid_dev, double* yee_dev, double* eb_dev,
                      void* work_dev, size_t work_bytes, vl_ctx** out) {
    if (!out) return fail(nullptr, VL_EINVAL, "out is NULL");
    *out = nullptr;
    vl_status st = validate(desc, nullptr);
    if (st != VL_OK) return st;
    // f_dev (or an entry) may be NULL for a fluid-only context: the calls
    // that touch f then fail with VL_EINVAL
    if (!fluid_dev || !eb_dev) return fail(nullptr, VL_EINVAL, "fluid and eb buffers are required");
    if (desc->nvdim == 3 && !yee_dev) return fail(nullptr, VL_EINVAL, "2D3V needs the Yee field buffer");
    Layout L = layout_of(*desc);
    if (!work_dev || work_bytes < L.total)
        return fail(nullptr, VL_EINVAL, "workspace too small: %zu bytes given, %zu needed", work_bytes, L.total);
    if (((uintptr_t)work_dev & 255u) != 0) return fail(nullptr, VL_EINVAL, "workspace must be 256-byte aligned");
    int* word = nullptr;
    int* word_dev = nullptr;
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&word), sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *word = VL_OK;
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&word_dev), word, 0);
        if (e != cudaSuccess) cudaFreeHost(word);
    }
    if (e != cudaSuccess) return fail(nullptr, VL_ECUDA, "status word: %s", cudaGetErrorString(e));
    vl_ctx* c = new vl_ctx();
    c->d = *desc;
    c->status_host = word;
    c->status_dev = word_dev;
    for (int s = 0; s < VL_MAX_SPECIES; ++s) c->f[s] = (f_dev && s < desc->nspecies) ? f_dev[s] : nullptr;
    c->fluid = fluid_dev;
    c->yee = yee_dev;
    c->eb = eb_dev;
    char* w = static_cast<char*>(work_dev);
    c->ws.cellwork = reinterpret_cast<double*>(w + L.cellwork);
    c->ws.coef_v = reinterpret_cast<double*>(w + L.coef_v);
    c->ws.coef_f = reinterpret_cast<double*>(w + L.coef_f);
    c->ws.fit_status = reinterpret_cast<int*>(w + L.status);
    c->ws.fluid_u1 = reinterpret_cast<double*>(w + L.u1);
    c->ws.fluid_u2 = reinterpret_cast<double*>(w + L.u2);
    c->ws.fluid_l = nullptr;
    c->ws.cur = reinterpret_cast<double*>(w + L.cur);
    c->ws.fluid_f = reinterpret_cast<float*>(w + L.fluid_f);
    c->ws.counters = reinterpret_cast<unsigned long long*>(w + L.counters);
    c->ws.fit_select = reinterpret_cast<unsigned long long*>(w + L.select);
    c->ws.mlp = nullptr;
    c->mlp_w = reinterpret_cast<float*>(w + L.mlp_w);
    c->mlp_m = reinterpret_cast<float*>(w + L.mlp_m);
    c->mlp_v = reinterpret_cast<float*>(w + L.mlp_v);
    c->mlp_g = reinterpret_cast<float*>(w + L.mlp_g);
    c->mlp_acc = reinterpret_cast<double*>(w + L.mlp_acc);
    c->mlp_loss = c->mlp_acc + 55;
    c->mlp_err = reinterpret_cast<int*>(w + L.mlp_err);
    c->mlp_pred = reinterpret_cast<float*>(w + L.mlp_pred);
    c->harvest_count = reinterpret_cast<unsigned long long*>(w + L.harvest_count);
    c->mlp_ready = false;
    c->adam_step = 0;
    c->harvest = nullptr;
    c->harvest_cap = 0;
    for (int s = 0; s < desc->nspecies; ++s) {
        double vmin[3], dv[3];
        fill_box(*desc, s, vmin, dv);
        vl::make_mom_conv(vmin, dv, desc->nv[s][0], &c->conv[s]);
    }
    for (int s = 0; s < VL_MAX_SPECIES; ++s) c->fit_mode[s] = -1;
    c->err[0] = 0;
    e = cudaMemset(c->ws.counters, 0, VL_NSTATS * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFreeHost(c->status_host);
        delete c;
        return fail(nullptr, VL_ECUDA, "clearing counters: %s", cudaGetErrorString(e));
    }
    *out = c;
    return VL_OK;
}

vl_status vlasov_free(vl_ctx* ctx) {
    if (ctx && ctx->status_host) cudaFreeHost(ctx->status_host);
    delete ctx;
    return VL_OK;
}

vl_status vl_sync_status(vl_ctx* ctx, vl_stream_t stream) {
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    vl_status st = cuda_check(ctx, cudaStreamSynchronize((cudaStream_t)stream), "vl_sync_status");
    if (st != VL_OK) return st;
    return pending_numeric(ctx);
}

const char* vl_last_error(const vl_ctx* ctx) { return ctx ? ctx->err : g_err; }

vl_status pfc_advect_x(vl_ctx* ctx, int s, int axis, double dt, vl_stream_t stream) {
    Range nvtx_("pfc_advect_x");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    const vl_desc& d = ctx->d;
    if (axis != 0 && axis != 1) return fail(ctx, VL_EINVAL, "axis must be 0 or 1");
    if (axis == 1 && d.nvdim != 3) return fail(ctx, VL_EINVAL, "1D1V has no y axis");
    if (!std::isfinite(dt)) return fail(ctx, VL_EINVAL, "dt is not finite");
    const long long V = vblock_of(d, s);
    const int es = d.precision == 64 ? 8 : 4;
    vl::SpaceSweepArgs a;
    a.f = ctx->f[s];
    a.V = V;
    a.nvx = d.nv[s][0];
    a.nvy = d.nvdim == 3 ? d.nv[s][1] : 1;
    const int wall = axis == 1 && d.bc_y == 1;
    a.wall = wall;
    if (axis == 0) {
        a.n = d.nx;
        a.row_stride = V;
        a.line_stride = (long long)d.nx * V;
        a.nlines = d.ny;
        a.axis_div = 1;
        a.axis_mod = d.nv[s][0];
        a.vmin_a = d.vmin[s][0];
        a.dv_a = dv_of(d, s, 0);
        a.dt_over_h = dt / d.dx;
    } else {
        a.n = d.ny;
        a.row_stride = (long long)d.nx * V;
        a.line_stride = V;
        a.nlines = d.nx;
        a.axis_div = d.nv[s][0];
        a.axis_mod = d.nv[s][1];
        a.vmin_a = d.vmin[s][1];
        a.dv_a = dv_of(d, s, 1);
        a.dt_over_h = dt / d.dy;
    }
    // largest displacement in cells, checked in floating point (no int overflow)
    {
        int ax = axis;
        double vmax = std::fmax(std::fabs(d.vmin[s][ax]), std::fabs(d.vmax[s][ax]));
        double dmax = vmax * std::fabs(dt) / (ax == 0 ? d.dx : d.dy);
        if (!(dmax < 1.0e6)) return fail(ctx, VL_EINVAL, "displacement of %g cells is not supported", dmax);
        if (wall && !(dmax + 3.0 <= (double)d.ny))
            return fail(ctx, VL_EINVAL, "y sweep: |v_y| dt / dy = %g too large for %d rows between walls", dmax, d.ny);
    }
    if (wall && a.nvy % 4 == 0) {
        a.mode = 2;
        a.ncol = 4 * a.nvx;
        a.nchunks = d.nv[s][2] * (a.nvy / 4);
    } else if (wall) {
        a.mode = 1;
        a.ncol = 2 * a.nvx;
        a.nchunks = d.nv[s][2] * ((a.nvy + 1) / 2);
    } else {
        a.mode = 0;
        a.ncol = 32;
        while (a.ncol > 8 && (size_t)a.n * a.ncol * es > 64 * 1024) a.ncol /= 2;
        a.nchunks = (int)((V + a.ncol - 1) / a.ncol);
    }
    // cp.async staging needs every column run (V, nvx and the tile width in
    // bytes) to be a multiple of 16 bytes; the base of f is 256-byte aligned
    {
        const long long run = wall ? a.nvx : V;
        a.vec = (run * es) % 16 == 0 && ((long long)a.ncol * es) % 16 == 0 && (V * es) % 16 == 0;
    }
    if ((long long)a.nchunks * a.nlines >= (1LL << 31) - (1LL << 20))
        return fail(ctx, VL_ENOTSUP, "too many sweep tiles (%d x %d)", a.nchunks, a.nlines);
    const size_t tile_bytes = (size_t)a.n * a.ncol * es;
    a.nbuf = 2 * tile_bytes <= 200 * 1024 ? 2 : 1;
    if (tile_bytes > 200 * 1024 || a.ncol > 256)
        return fail(ctx, VL_ENOTSUP, "spatial line too long for one shared-memory tile (%d cells)", a.n);
    return cuda_check(ctx, vl::launch_pfc_space(a, d.precision, (cudaStream_t)stream), "pfc_advect_x");
}

vl_status pfc_advect_xy(vl_ctx* ctx, int s, double dt, void* f_out, vl_stream_t stream) {
    Range nvtx_("pfc_advect_xy");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    const vl_desc& d = ctx->d;
    if (d.nvdim != 3) return fail(ctx, VL_EINVAL, "pfc_advect_xy needs a 2D3V descriptor");
    if (!std::isfinite(dt)) return fail(ctx, VL_EINVAL, "dt is not finite");
    if (!f_out) return fail(ctx, VL_EINVAL, "f_out is NULL");
    const long long V = vblock_of(d, s);
    const int es = d.precision == 64 ? 8 : 4;
    const size_t bytes = (size_t)ncell_of(d) * (size_t)V * es;
    {
        const char* a0 = static_cast<const char*>(ctx->f[s]);
        const char* b0 = static_cast<const char*>(f_out);
        if (b0 < a0 + bytes && a0 < b0 + bytes) return fail(ctx, VL_EINVAL, "f_out overlaps the species' f");
        if (reinterpret_cast<uintptr_t>(f_out) % es != 0) return fail(ctx, VL_EINVAL, "f_out is not aligned to its element size");
    }
    // the single-axis sweeps' limits, so that both paths accept the same calls
    for (int ax = 0; ax < 2; ++ax) {
        const double h = ax == 0 ? d.dx : d.dy;
        const double vmax = std::fmax(std::fabs(d.vmin[s][ax]), std::fabs(d.vmax[s][ax]));
        const double dmax = vmax * std::fabs(dt) / h;
        if (!(dmax < 1.0e6)) return fail(ctx, VL_EINVAL, "displacement of %g cells is not supported", dmax);
        if (ax == 1 && d.bc_y == 1 && !(dmax + 3.0 <= (double)d.ny))
            return fail(ctx, VL_EINVAL, "y sweep: |v_y| dt / dy = %g too large for %d rows between walls", dmax, d.ny);
    }
    vl::SpaceXYArgs a;
    a.f_in = ctx->f[s];
    a.f_out = f_out;
    a.nx = d.nx;
    a.ny = d.ny;
    a.V = V;
    a.nvx = d.nv[s][0];
    a.nvy = d.nv[s][1];
    a.wall = d.bc_y == 1;
    a.ncol = 128 / es;
    a.nchunks = (int)((V + a.ncol - 1) / a.ncol);
    a.vminx = d.vmin[s][0];
    a.dvx = dv_of(d, s, 0);
    a.cx = dt / d.dx;
    a.vminy = d.vmin[s][1];
    a.dvy = dv_of(d, s, 1);
    a.cy = dt / d.dy;
    // halos: the largest shift along each axis (as the kernels compute it) + 2
    auto halo = [](double vmin, double dv, double c, int nv, int n, bool periodic) {
        int smax = 0;
        for (int i = 0; i < nv; ++i) {
            double ca = std::fabs((vmin + (i + 0.5) * dv) * c);
            if (periodic) ca = std::fmod(ca, (double)n);
            if (!(ca <= (double)n)) ca = (double)n;
            smax = std::max(smax, (int)std::floor(ca));
        }
        return smax + 2;
    };
    a.hx = halo(a.vminx, a.dvx, a.cx, a.nvx, d.nx, true);
    a.hy = halo(a.vminy, a.dvy, a.cy, a.nvy, d.ny, !a.wall);
    a.counters = ctx->ws.counters;
    a.tx = d.nx % 32 == 0 ? 32 : (d.nx % 16 == 0 ? 16 : (d.nx % 8 == 0 ? 8 : 0));
    a.ty = d.ny % 16 == 0 ? 16 : (d.ny % 8 == 0 ? 8 : 0);
    const long long ntiles = a.tx && a.ty ? (long long)a.nchunks * (d.nx / a.tx) * (d.ny / a.ty) : 0;
    const bool fused = a.tx && a.ty && a.hy <= 8 && a.hy <= d.ny && ntiles < (1LL << 31);
    cudaStream_t cs = (cudaStream_t)stream;
    if (fused) {
        st = cuda_check(ctx, vl::launch_pfc_space_xy(a, d.precision, cs), "pfc_advect_xy");
    } else {
        // grids without 8-cell tiles or with long y shifts: the two in-place
        // sweeps, then the result moves to f_out
        st = pfc_advect_x(ctx, s, 0, dt, stream);
        if (st == VL_OK) st = pfc_advect_x(ctx, s, 1, dt, stream);
        if (st == VL_OK)
            st = cuda_check(ctx, cudaMemcpyAsync(f_out, ctx->f[s], bytes, cudaMemcpyDeviceToDevice, cs), "pfc_advect_xy copy");
    }
    if (st == VL_OK) ctx->f[s] = f_out;
    return st;
}

vl_status pfc_advect_v(vl_ctx* ctx, int s, double dt, double* mom_out, vl_stream_t stream) {
    Range nvtx_("pfc_advect_v");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    const vl_desc& d = ctx->d;
    if (!std::isfinite(dt)) return fail(ctx, VL_EINVAL, "dt is not finite");
    vl::VelocityArgs a;
    a.f = ctx->f[s];
    a.eb = ctx->eb;
    a.shears = ctx->ws.cellwork;
    a.mom_out = mom_out;
    a.ncell = ncell_of(d);
    a.nv = d.nv[s][0];
    a.nshear = d.nshear;
    a.qm = d.q[s] / d.m[s];
    a.dt = dt;
    fill_box(d, s, a.vmin, a.dv);
    a.conv = ctx->conv[s];
    return cuda_check(ctx, vl::launch_velocity(a, d.nvdim, d.precision, (cudaStream_t)stream), "pfc_advect_v");
}

vl_status pfc_advect_v_static(const vl_desc* desc, int s, void* f_dev, const double* eb_dev, long long ncell,
                              double dt, double* mom_out, vl_stream_t stream) {
    Range nvtx_("pfc_advect_v_static");
    vl_status st = validate(desc, nullptr);
    if (st != VL_OK) return st;
    const vl_desc& d = *desc;
    if (s < 0 || s >= d.nspecies) return fail(nullptr, VL_EINVAL, "species %d out of range", s);
    if (ncell < 0) return fail(nullptr, VL_EINVAL, "ncell must be >= 0 (got %lld)", ncell);
    if (ncell > VL_STATIC_SCRATCH_CELLS)
        return fail(nullptr, VL_EINVAL,
                    "pfc_advect_v_static: %lld cells exceed the static scratch (%d cells); split the call",
                    ncell, VL_STATIC_SCRATCH_CELLS);
    if (ncell == 0) return VL_OK;
    if (!f_dev || !eb_dev) return fail(nullptr, VL_EINVAL, "f_dev and eb_dev are required");
    if (!std::isfinite(dt)) return fail(nullptr, VL_EINVAL, "dt is not finite");
    {
        // misaligned pointers would fault in the kernels' element and FP64
        // accesses; overlapping outputs would corrupt f
        const size_t es = d.precision == 64 ? 8 : 4;
        const uintptr_t fp = reinterpret_cast<uintptr_t>(f_dev);
        if (fp % es != 0) return fail(nullptr, VL_EINVAL, "f_dev is not aligned to its element size (%zu bytes)", es);
        if (reinterpret_cast<uintptr_t>(eb_dev) % 8 != 0) return fail(nullptr, VL_EINVAL, "eb_dev is not 8-byte aligned");
        if (mom_out) {
            const uintptr_t mp = reinterpret_cast<uintptr_t>(mom_out);
            if (mp % 8 != 0) return fail(nullptr, VL_EINVAL, "mom_out is not 8-byte aligned");
            const uintptr_t fbytes = (uintptr_t)ncell * (uintptr_t)vblock_of(d, s) * es;
            const uintptr_t mbytes = (uintptr_t)ncell * (d.nvdim == 1 ? 4 : 20) * sizeof(double);
            if (mp < fp + fbytes && fp < mp + mbytes) return fail(nullptr, VL_EINVAL, "mom_out overlaps f_dev");
        }
    }
    void* scratch = nullptr;
    st = cuda_check(nullptr, vl::static_scratch_address(&scratch), "pfc_advect_v_static (scratch address)");
    if (st != VL_OK) return st;
    vl::VelocityArgs a;
    a.f = f_dev;
    a.eb = eb_dev;
    a.shears = static_cast<double*>(scratch);
    a.mom_out = mom_out;
    a.ncell = ncell;
    a.nv = d.nv[s][0];
    a.nshear = d.nshear;
    a.qm = d.q[s] / d.m[s];
    a.dt = dt;
    fill_box(d, s, a.vmin, a.dv);
    vl::make_mom_conv(a.vmin, a.dv, d.nv[s][0], &a.conv);
    return cuda_check(nullptr, vl::launch_velocity(a, d.nvdim, d.precision, (cudaStream_t)stream),
                      "pfc_advect_v_static");
}

vl_status moments(vl_ctx* ctx, int s, double* mom_out, vl_stream_t stream) {
    Range nvtx_("moments");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    if (!mom_out) return fail(ctx, VL_EINVAL, "mom_out is NULL");
    const vl_desc& d = ctx->d;
    vl::MomentArgs a;
    a.f = ctx->f[s];
    a.mom_out = mom_out;
    a.ncell = ncell_of(d);
    a.nv = d.nv[s][0];
    fill_box(d, s, a.vmin, a.dv);
    a.conv = ctx->conv[s];
    return cuda_check(ctx, vl::launch_moments(a, d.nvdim, d.precision, (cudaStream_t)stream), "moments");
}

vl_status moment_fit_wide(vl_ctx* ctx, int s, int wide) {
    if (!ctx) return VL_EINVAL;
    if (s < 0 || s >= ctx->d.nspecies) return fail(ctx, VL_EINVAL, "species out of range");
    ctx->fit_mode[s] = wide < 0 ? -1 : (wide != 0 ? 1 : 0);
    return VL_OK;
}

vl_status moment_fit_solve(vl_ctx* ctx, int s, const double* vmom, int use_mlp, double* theta_v, double* theta_f,
                           vl_stream_t stream) {
    Range nvtx_("moment_fit_solve");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    if (!vmom) return fail(ctx, VL_EINVAL, "vmom is NULL");
    const vl_desc& d = ctx->d;
    if (use_mlp && !ctx->mlp_ready) return fail(ctx, VL_EINVAL, "use_mlp: no MLP weights on this context");
    if (use_mlp && d.nvdim != 3) return fail(ctx, VL_ENOTSUP, "the MLP warm start serves the 2D3V fit");
    const int ncomp = d.nvdim == 1 ? 3 : 10;
    vl::FitArgs a;
    a.vmom = vmom;
    a.fluid = ctx->fluid + (size_t)s * ncell_of(d) * ncomp;
    a.coef_v = ctx->ws.coef_v;
    a.coef_f = ctx->ws.coef_f;
    a.status = ctx->ws.fit_status;
    a.counters = ctx->ws.counters;
    a.warm = nullptr;
    a.harvest = d.nvdim == 3 ? ctx->harvest : nullptr;
    a.harvest_cap = ctx->harvest_cap;
    a.harvest_count = ctx->harvest_count;
    a.ncell = ncell_of(d);
    a.nv = d.nv[s][0];
    fill_box(d, s, a.vmin, a.dv);
    for (int q = 0; q < 3; ++q) a.vmax[q] = a.vmin[q] + a.dv[q] * (d.nvdim == 3 || q == 0 ? d.nv[s][q] : 1);
    a.tol = d.fit_tol;
    a.max_iter = d.fit_max_iter;
    a.fp64 = d.precision == 64 ? 1 : 0;
    a.numeric = ctx->status_dev;
    a.wide = a.fp64 ? 0 : ctx->fit_mode[s];
    a.select = nullptr;
    cudaStream_t cs = (cudaStream_t)stream;
    if (d.nvdim == 3 && a.wide < 0) {
        // the double-float kernel is chosen on the device from the targets
        st = cuda_check(ctx, cudaMemsetAsync(ctx->ws.fit_select, 0, 2 * sizeof(unsigned long long), cs),
                        "moment_fit (kernel choice)");
        if (st != VL_OK) return st;
        st = cuda_check(ctx, vl::launch_fit_select(a, ctx->ws.fit_select, cs), "moment_fit (kernel choice)");
        if (st != VL_OK) return st;
        a.select = ctx->ws.fit_select;
    }
    if (use_mlp) {
        vl::MlpInferArgs m;
        m.w = ctx->mlp_w;
        m.mode = 0;
        m.vmom = vmom;
        m.fluid = a.fluid;
        m.nmom = 20;
        m.x = nullptr;
        m.nfit = 2 * a.ncell;
        for (int q = 0; q < 3; ++q) {
            m.vmin[q] = a.vmin[q];
            m.dv[q] = a.dv[q];
            m.vmax[q] = a.vmax[q];
        }
        m.y = ctx->mlp_pred;
        m.err = ctx->mlp_err;
        st = cuda_check(ctx, vl::launch_mlp_infer(m, cs), "moment_fit (MLP warm start)");
        if (st != VL_OK) return st;
        a.warm = ctx->mlp_pred;
    }
    st = cuda_check(ctx, vl::launch_fit(a, d.nvdim, cs), "moment_fit (Newton)");
    if (st != VL_OK) return st;
    if (theta_v) {
        st = cuda_check(ctx, vl::launch_theta(a.coef_v, a.status, 0, theta_v, a.ncell, d.nvdim, cs), "theta");
        if (st != VL_OK) return st;
    }
    if (theta_f) st = cuda_check(ctx, vl::launch_theta(a.coef_f, a.status, 1, theta_f, a.ncell, d.nvdim, cs), "theta");
    return st;
}

vl_status moment_fit_exchange(vl_ctx* ctx, int s, const double* vmom, double* mom_out, vl_stream_t stream) {
    Range nvtx_("moment_fit_exchange");
    vl_status st = check_species(ctx, s);
    if (st != VL_OK) return st;
    if (!vmom) return fail(ctx, VL_EINVAL, "vmom is NULL");
    const vl_desc& d = ctx->d;
    vl::ExchangeArgs x;
    x.f = ctx->f[s];
    x.vmom = vmom;
    x.coef_v = ctx->ws.coef_v;
    x.coef_f = ctx->ws.coef_f;
    x.status = ctx->ws.fit_status;
    x.mom_out = mom_out;
    x.counters = ctx->ws.counters;
    x.ncell = ncell_of(d);
    x.nv = d.nv[s][0];
    fill_box(d, s, x.vmin, x.dv);
    x.conv = ctx->conv[s];
    x.par = ctx->ws.cellwork;
    return cuda_check(ctx, vl::launch_exchange(x, d.nvdim, d.precision, (cudaStream_t)stream),
                      "moment_fit (exchange)");
}

vl_status moment_fit(vl_ctx* ctx, int s, const double* vmom, int use_mlp, double* theta_v, double* theta_f,
                     double* mom_out, vl_stream_t stream) {
    Range nvtx_("moment_fit");
    vl_status st = moment_fit_solve(ctx, s, vmom, use_mlp, theta_v, theta_f, stream);
    if (st != VL_OK) return st;
    return moment_fit_exchange(ctx, s, vmom, mom_out, stream);
}

vl_status fluid_step_closure(vl_ctx* ctx, double dt, vl_stream_t stream) {
    Range nvtx_("fluid_step_closure");
    {
        const vl_status st0 = check_ctx(ctx);
        if (st0 != VL_OK) return st0;
    }
    const vl_desc& d = ctx->d;
    if (d.nvdim != 3) return fail(ctx, VL_EINVAL, "the gradient-closure fluid model is 2D3V");
    if (!std::isfinite(dt)) return fail(ctx, VL_EINVAL, "dt is not finite");
    const double chi = 2.0 * std::sqrt(2.0 / 3.14159265358979323846);
    cudaStream_t cs = (cudaStream_t)stream;
    for (int s = 0; s < d.nspecies; ++s) {
        double* U = ctx->fluid + (size_t)s * ncell_of(d) * 10;
        vl::FluidArgs a;
        a.U = U;
        a.eb = ctx->eb;
        a.nx = d.nx;
        a.ny = d.ny;
        a.bc_y = d.bc_y;
        a.nvdim = 3;
        a.nmom = 20;
        a.precision = d.precision;
        a.dx = d.dx;
        a.dy = d.dy;
        a.qm = d.q[s] / d.m[s];
        a.dt = dt;
        a.q0 = nullptr;
        a.q1 = nullptr;
        a.wq0 = 0.0;
        a.wq1 = 0.0;
        a.closure = 1;
        a.Usf = ctx->ws.fluid_f;
        a.Qf = nullptr;
        // chi / k_s0 with k_s0 = 1/d_s, d_s = sqrt(m_s / (n0 q_s^2)) at n0 = 1 (mu0 = 1)
        if (d.q[s] == 0.0) return fail(ctx, VL_EINVAL, "species %d: the closure needs a charged species", s);
        a.chi_k0 = chi * std::sqrt(d.m[s] / (d.q[s] * d.q[s]));
        a.Us = U; a.U0 = U; a.Uout = ctx->ws.fluid_u1; a.a0 = 0.0; a.a1 = 1.0;
        vl_status e = cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step_closure");
        if (e != VL_OK) return e;
        a.Us = ctx->ws.fluid_u1; a.Uout = ctx->ws.fluid_u2; a.a0 = 0.75; a.a1 = 0.25;
        e = cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step_closure");
        if (e != VL_OK) return e;
        a.Us = ctx->ws.fluid_u2; a.Uout = U; a.a0 = 1.0 / 3.0; a.a1 = 2.0 / 3.0;
        e = cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step_closure");
        if (e != VL_OK) return e;
    }
    return VL_OK;
}

}  // extern "C"

namespace {
// One SSP-RK3 step of species s's fluid state (the body of fluid_step).
vl_status fluid_one(vl_ctx* ctx, int s, double dt, const double* q0, const double* q1, cudaStream_t cs) {
    const vl_desc& d = ctx->d;
    const int ncomp = d.nvdim == 1 ? 3 : 10;
    const int nmom = d.nvdim == 1 ? 4 : 20;
    if (!q0 || !q1) return fail(ctx, VL_EINVAL, "moments of species %d are NULL", s);
    double* U = ctx->fluid + (size_t)s * ncell_of(d) * ncomp;
    vl::FluidArgs a;
    a.U = U;
    a.eb = ctx->eb;
    a.nx = d.nx;
    a.ny = d.ny;
    a.bc_y = d.bc_y;
    a.nvdim = d.nvdim;
    a.nmom = nmom;
    a.precision = d.precision;
    a.dx = d.dx;
    a.dy = d.dy;
    a.qm = d.q[s] / d.m[s];
    a.dt = dt;
    a.q0 = q0;
    a.q1 = q1;
    a.closure = 0;
    a.chi_k0 = 0.0;
    a.Usf = ctx->ws.fluid_f;
    a.Qf = ctx->ws.fluid_f + (size_t)ncell_of(d) * 10;
    // stage 1: U1 = U + dt L(U; Q^t)
    a.Us = U; a.U0 = U; a.Uout = ctx->ws.fluid_u1; a.wq0 = 1.0; a.wq1 = 0.0; a.a0 = 0.0; a.a1 = 1.0;
    vl_status e = cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step");
    if (e != VL_OK) return e;
    // stage 2: U2 = 3/4 U + 1/4 (U1 + dt L(U1; Q^t+1))
    a.Us = ctx->ws.fluid_u1; a.Uout = ctx->ws.fluid_u2; a.wq0 = 0.0; a.wq1 = 1.0; a.a0 = 0.75; a.a1 = 0.25;
    e = cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step");
    if (e != VL_OK) return e;
    // stage 3: U = 1/3 U + 2/3 (U2 + dt L(U2; Q^t+1/2))
    a.Us = ctx->ws.fluid_u2; a.Uout = U; a.wq0 = 0.5; a.wq1 = 0.5; a.a0 = 1.0 / 3.0; a.a1 = 2.0 / 3.0;
    return cuda_check(ctx, vl::launch_fluid_stage(a, cs), "fluid_step");
}
}  // namespace

extern "C" {

vl_status fluid_step(vl_ctx* ctx, double dt, const double* const* mom_t, const double* const* mom_t1,
                     vl_stream_t stream) {
    Range nvtx_("fluid_step");
    {
        const vl_status st0 = check_ctx(ctx);
        if (st0 != VL_OK) return st0;
    }
    if (!mom_t || !mom_t1) return fail(ctx, VL_EINVAL, "moment arrays are NULL");
    for (int s = 0; s < ctx->d.nspecies; ++s) {
        const vl_status e = fluid_one(ctx, s, dt, mom_t[s], mom_t1[s], (cudaStream_t)stream);
        if (e != VL_OK) return e;
    }
    return VL_OK;
}

vl_status fluid_step_species(vl_ctx* ctx, int s, double dt, const double* mom_t, const double* mom_t1,
                             vl_stream_t stream) {
    Range nvtx_("fluid_step_species");
    {
        const vl_status st0 = check_ctx(ctx);
        if (st0 != VL_OK) return st0;
    }
    if (s < 0 || s >= ctx->d.nspecies) return fail(ctx, VL_EINVAL, "species %d out of range", s);
    return fluid_one(ctx, s, dt, mom_t, mom_t1, (cudaStream_t)stream);
}

vl_status maxwell_step(vl_ctx* ctx, double h, const double* const* mom, vl_stream_t stream) {
    Range nvtx_("maxwell_step");
    {
        const vl_status st0 = check_ctx(ctx);
        if (st0 != VL_OK) return st0;
    }
    const vl_desc& d = ctx->d;
    const int ncomp = d.nvdim == 1 ? 3 : 10;
    const int nmom = d.nvdim == 1 ? 4 : 20;
    const long long nc = ncell_of(d);
    const double* src[VL_MAX_SPECIES];
    for (int s = 0; s < d.nspecies; ++s) {
        if (mom && !mom[s]) return fail(ctx, VL_EINVAL, "moments of species %d are NULL", s);
        src[s] = mom ? mom[s] : ctx->fluid + (size_t)s * nc * ncomp;
    }
    const int stride = mom ? nmom : ncomp;
    cudaStream_t cs = (cudaStream_t)stream;
    if (d.nvdim == 1) {
        vl_status e = cuda_check(ctx, vl::launch_current(ctx->ws.cur, src, d.q, d.nspecies, stride, 0, nc, 1,
                                                         d.ion_background, cs), "maxwell_step (charge)");
        if (e != VL_OK) return e;
        return cuda_check(ctx, vl::launch_poisson(ctx->ws.cur, ctx->eb, d.nx, d.dx, cs), "maxwell_step (Poisson)");
    }
    if (!std::isfinite(h)) return fail(ctx, VL_EINVAL, "h is not finite");
    vl_status e = cuda_check(ctx, vl::launch_current(ctx->ws.cur, src, d.q, d.nspecies, stride, 1, nc, 3, 0.0, cs),
                             "maxwell_step (current)");
    if (e != VL_OK) return e;
    vl::FieldArgs a;
    a.yee = ctx->yee;
    a.eb = ctx->eb;
    a.cur = ctx->ws.cur;
    a.nx = d.nx;
    a.ny = d.ny;
    a.wall = d.bc_y == 1;
    a.dx = d.dx;
    a.dy = d.dy;
    a.c2 = d.c * d.c;
    a.h = h;
    return cuda_check(ctx, vl::launch_maxwell(a, cs), "maxwell_step (FDTD)");
}

// ---------------------------------------------------------------- MLP warm start

namespace {
unsigned long long splitmix64(unsigned long long& s) {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
vl_status mlp_check_err(vl_ctx* ctx, cudaStream_t cs, const char* what) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->mlp_err, sizeof(int), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_check(ctx, e, what);
    if (h) return fail(ctx, VL_ECUDA, "%s: a tensor-core wait timed out", what);
    return VL_OK;
}
}  // namespace

vl_status mlp_init(vl_ctx* ctx, unsigned long long seed) {
    Range nvtx_("mlp_init");
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    std::vector<float> w(VL_MLP_NPARAM, 0.f);
    // unit normalisation until mlp_normalize sets it from samples
    for (int q = 0; q < 12; ++q) w[vl::mlp::kOffXs + q] = 1.f;
    for (int q = 0; q < 10; ++q) w[vl::mlp::kOffYs + q] = 1.f;
    for (int q = 0; q < 10; ++q) w[vl::mlp::kOffYsc + q] = 1.f;
    unsigned long long st = seed;
    auto uniform = [&]() { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); };
    // Glorot-uniform weights, zero biases
    const int fan[3][2] = {{12, 128}, {128, 128}, {128, 10}};
    const int off[3] = {vl::mlp::kOffW1, vl::mlp::kOffW2, vl::mlp::kOffW3};
    for (int l = 0; l < 3; ++l) {
        const double lim = std::sqrt(6.0 / (fan[l][0] + fan[l][1]));
        for (int q = 0; q < fan[l][0] * fan[l][1]; ++q) w[off[l] + q] = (float)((2.0 * uniform() - 1.0) * lim);
    }
    cudaError_t e = cudaMemcpy(ctx->mlp_w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_m, 0, VL_MLP_NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_v, 0, VL_MLP_NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_init");
    ctx->adam_step = 0;
    ctx->mlp_ready = true;
    return VL_OK;
}

vl_status mlp_set_weights(vl_ctx* ctx, const float* w_host) {
    if (!ctx || !w_host) return fail(ctx, VL_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(ctx->mlp_w, w_host, VL_MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->mlp_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_set_weights");
    ctx->mlp_ready = true;
    return VL_OK;
}

vl_status mlp_get_weights(vl_ctx* ctx, float* w_host) {
    if (!ctx || !w_host) return fail(ctx, VL_EINVAL, "NULL argument");
    if (!ctx->mlp_ready) return fail(ctx, VL_EINVAL, "no MLP weights on this context");
    return cuda_check(ctx, cudaMemcpy(w_host, ctx->mlp_w, VL_MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost),
                      "mlp_get_weights");
}

vl_status mlp_set_harvest(vl_ctx* ctx, float* samples_dev, long long capacity, vl_stream_t stream) {
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    if (capacity < 0 || (capacity > 0 && !samples_dev)) return fail(ctx, VL_EINVAL, "bad harvest buffer");
    ctx->harvest = capacity > 0 ? samples_dev : nullptr;
    ctx->harvest_cap = capacity;
    return cuda_check(ctx, cudaMemsetAsync(ctx->harvest_count, 0, sizeof(unsigned long long), (cudaStream_t)stream),
                      "mlp_set_harvest");
}

vl_status mlp_harvest_count(vl_ctx* ctx, long long* n, vl_stream_t stream) {
    if (!ctx || !n) return fail(ctx, VL_EINVAL, "NULL argument");
    unsigned long long h = 0;
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, ctx->harvest_count, sizeof(h), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_harvest_count");
    *n = (long long)(h < (unsigned long long)ctx->harvest_cap ? h : (unsigned long long)ctx->harvest_cap);
    return VL_OK;
}

vl_status mlp_normalize(vl_ctx* ctx, const float* samples_dev, long long n, vl_stream_t stream) {
    Range nvtx_("mlp_normalize");
    if (!ctx || !samples_dev || n <= 0) return fail(ctx, VL_EINVAL, "bad samples");
    if (!ctx->mlp_ready) return fail(ctx, VL_EINVAL, "call mlp_init first");
    return cuda_check(ctx, vl::launch_mlp_stats(samples_dev, n, ctx->mlp_acc, ctx->mlp_w, (cudaStream_t)stream),
                      "mlp_normalize");
}

vl_status mlp_train(vl_ctx* ctx, const float* samples_dev, long long n, int steps, int batch, float lr,
                    unsigned long long seed, double* loss_host, vl_stream_t stream) {
    Range nvtx_("mlp_train");
    if (!ctx || !samples_dev || n <= 0) return fail(ctx, VL_EINVAL, "bad samples");
    if (!ctx->mlp_ready) return fail(ctx, VL_EINVAL, "call mlp_init first");
    if (steps < 0 || batch < 128 || batch % 128 != 0 || batch > (1 << 24) || !(lr > 0.f))
        return fail(ctx, VL_EINVAL, "steps >= 0, batch a positive multiple of 128 and lr > 0 are required");
    cudaStream_t cs = (cudaStream_t)stream;
    for (int k = 0; k < steps; ++k) {
        cudaError_t e = cudaMemsetAsync(ctx->mlp_g, 0, VL_MLP_NPARAM * sizeof(float), cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(double), cs);
        if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_train");
        vl::MlpTrainArgs a;
        a.w = ctx->mlp_w;
        a.grad = ctx->mlp_g;
        a.loss = ctx->mlp_loss;
        a.samples = samples_dev;
        a.n = n;
        a.mode = 0;
        a.rows = batch;
        a.row0 = 0;
        unsigned long long sk = seed ^ (0xD1B54A32D192ED03ull * (unsigned long long)(ctx->adam_step + 1));
        a.seed = splitmix64(sk);
        a.inv_count = 1.f / (float)(batch * 10);
        a.err = ctx->mlp_err;
        vl_status st = cuda_check(ctx, vl::launch_mlp_train_step(a, cs), "mlp_train (step)");
        if (st != VL_OK) return st;
        ctx->adam_step += 1;
        st = cuda_check(ctx, vl::launch_mlp_adam(ctx->mlp_w, ctx->mlp_m, ctx->mlp_v, ctx->mlp_g, lr, ctx->adam_step, cs),
                        "mlp_train (Adam)");
        if (st != VL_OK) return st;
        if (loss_host) {
            double l = 0.0;
            e = cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost, cs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
            if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_train (loss)");
            loss_host[k] = l / (double)(batch * 10);
        }
    }
    return mlp_check_err(ctx, cs, "mlp_train");
}

vl_status mlp_forward(vl_ctx* ctx, const float* x_dev, long long n, float* y_dev, vl_stream_t stream) {
    Range nvtx_("mlp_forward");
    if (!ctx || n < 0 || (n > 0 && (!x_dev || !y_dev))) return fail(ctx, VL_EINVAL, "bad arguments");
    if (!ctx->mlp_ready) return fail(ctx, VL_EINVAL, "no MLP weights on this context");
    vl::MlpInferArgs m = {};
    m.w = ctx->mlp_w;
    m.mode = 1;
    m.x = x_dev;
    m.nfit = n;
    m.y = y_dev;
    m.err = ctx->mlp_err;
    cudaStream_t cs = (cudaStream_t)stream;
    vl_status st = cuda_check(ctx, vl::launch_mlp_infer(m, cs), "mlp_forward");
    if (st != VL_OK) return st;
    return mlp_check_err(ctx, cs, "mlp_forward");
}

vl_status mlp_grad(vl_ctx* ctx, const float* samples_dev, long long n, float* grad_dev, double* loss_host,
                   vl_stream_t stream) {
    Range nvtx_("mlp_grad");
    if (!ctx || !samples_dev || n <= 0 || !grad_dev) return fail(ctx, VL_EINVAL, "bad arguments");
    if (!ctx->mlp_ready) return fail(ctx, VL_EINVAL, "no MLP weights on this context");
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(grad_dev, 0, VL_MLP_NPARAM * sizeof(float), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->mlp_loss, 0, sizeof(double), cs);
    if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_grad");
    for (long long r0 = 0; r0 < n; r0 += 128 * 1024) {
        vl::MlpTrainArgs a;
        a.w = ctx->mlp_w;
        a.grad = grad_dev;
        a.loss = ctx->mlp_loss;
        a.samples = samples_dev;
        a.n = n;
        a.mode = 1;
        a.row0 = r0;
        a.rows = n - r0 < 128 * 1024 ? n - r0 : 128 * 1024;
        a.seed = 0;
        a.inv_count = 1.f / (float)(n * 10);
        a.err = ctx->mlp_err;
        vl_status st = cuda_check(ctx, vl::launch_mlp_train_step(a, cs), "mlp_grad");
        if (st != VL_OK) return st;
    }
    if (loss_host) {
        double l = 0.0;
        e = cudaMemcpyAsync(&l, ctx->mlp_loss, sizeof(double), cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (e != cudaSuccess) return cuda_check(ctx, e, "mlp_grad (loss)");
        *loss_host = l / (double)(n * 10);
    }
    return mlp_check_err(ctx, cs, "mlp_grad");
}

vl_status vl_read_stats(vl_ctx* ctx, long long out[VL_NSTATS], vl_stream_t stream) {
    if (!ctx || !out) return fail(ctx, VL_EINVAL, "NULL argument");
    unsigned long long h[VL_NSTATS];
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h, ctx->ws.counters, sizeof(h), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_check(ctx, e, "vl_read_stats");
    for (int q = 0; q < VL_NSTATS; ++q) out[q] = (long long)h[q];
    return VL_OK;
}

vl_status vl_reset_stats(vl_ctx* ctx, vl_stream_t stream) {
    if (!ctx) return fail(nullptr, VL_EINVAL, "context is NULL");
    return cuda_check(ctx, cudaMemsetAsync(ctx->ws.counters, 0, VL_NSTATS * sizeof(unsigned long long), (cudaStream_t)stream),
                      "vl_reset_stats");
}

long long vl_launch_count(void) { return vl::g_launches.load(); }

vl_status vl_fma_peak(int precision, double* ops_per_s, void* sink_dev, vl_stream_t stream) {
    if (precision != 32 && precision != 64) return fail(nullptr, VL_EINVAL, "precision must be 32 or 64");
    if (!ops_per_s || !sink_dev) return fail(nullptr, VL_EINVAL, "NULL argument");
    if (reinterpret_cast<uintptr_t>(sink_dev) % 8 != 0) return fail(nullptr, VL_EINVAL, "sink_dev is not 8-byte aligned");
    *ops_per_s = 0.0;
    return cuda_check(nullptr, vl::fma_peak(precision, ops_per_s, sink_dev, (cudaStream_t)stream), "vl_fma_peak");
}

}  // extern "C"

// C ABI of the library: context lifetime, options, stepping, convergence,
// field and population I/O, checkpoints.  Every entry point returns a status;
// the message of the last failure is kept per thread.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <string>
#include <vector>

#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_error = "no error";

lbm_status fail(lbm_status s, const std::string &msg)
{
    g_error = msg;
    return s;
}

}  // namespace

lbm_status lbm::set_error(lbm_status s, const std::string &msg) { return fail(s, msg); }

namespace {

lbm_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

lbm_allocator g_alloc = {nullptr, nullptr, nullptr};

void *dev_alloc(size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (g_alloc.alloc) return g_alloc.alloc(bytes, g_alloc.user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p)
{
    if (!p) return;
    if (g_alloc.release) g_alloc.release(p, g_alloc.user);
    else cudaFree(p);
}

}  // namespace

struct lbm_ctx {
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;
    double nu = 0, gamma = 1, U = 0;
    double omega[9] = {0, 0, 0, 1, 1, 1, 1, 1, 1};
    int gi_mode = LBM_GI_FULL;
    int storage = LBM_STORAGE_F32;
    int guard = 0;
    int fd_iso = 0;  // density gradient: 0 central differences, 1 isotropic stencil
    int sround = 1;  // 16-bit storage: stochastic rounding of the stored deviations
    lbm_side sides[4];
    double Fx = 0, Fy = 0;
    int Ly_option = 0;  // 0 = automatic
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    uint8_t *d_solid = nullptr;
    std::vector<long> hist_steps;     // lbm_run_to_steady's checks: step count after each
    std::vector<double> hist_r;       // and its residual
    float *d_force = nullptr;
    double *d_snap_ux = nullptr, *d_snap_uy = nullptr, *d_partials = nullptr, *d_result = nullptr;
    unsigned long long *d_guard = nullptr;
    int *d_err = nullptr;        // set by a step kernel whose bounded wait expired
    unsigned int *d_work = nullptr;  // step-kernel work counters (zero between launches)
    CUtensorMap tload[2];        // TMA load descriptors of f[0], f[1]
    CUtensorMap tstore[2];       // TMA store descriptors of f[0], f[1]
    double *h_result = nullptr;  // pinned, 5 doubles
    void *d_ghost[2] = {nullptr, nullptr};  // convective outlet ghost column of f[0], f[1] ([5][ny])
    void *d_stage = nullptr;     // grow-only device staging for field and population transfers
    size_t stage_bytes = 0;
    int res_blocks = 1;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    long steps = 0, launches = 0;
    int num_sms = 1;
};

namespace {

size_t pop_bytes(const lbm_ctx *c) { return (size_t)9 * (size_t)c->plane * storage_bytes(c->storage); }

// Resident blocks per SM of the step-kernel variant p launches.
int step_blocks_per_sm(const lbm_ctx *c, const StepParams &p)
{
    const bool forced = p.force != nullptr || p.Fx != 0.0 || p.Fy != 0.0;
    switch (c->storage) {
    case LBM_STORAGE_F16: return blocks_per_sm_f16(c->gi_mode, forced);
    case LBM_STORAGE_BF16: return blocks_per_sm_bf16(c->gi_mode, forced);
    case LBM_STORAGE_F64: return blocks_per_sm_f64(c->gi_mode, forced);
    default: return blocks_per_sm_f32(c->gi_mode, forced);
    }
}

StepParams make_params(const lbm_ctx *c)
{
    StepParams p;
    memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.pitch = c->pitch;
    p.plane = c->plane;
    p.perx = c->sides[0].kind == LBM_SIDE_PERIODIC;
    p.pery = c->sides[2].kind == LBM_SIDE_PERIODIC;
    p.gi_mode = c->gi_mode;
    p.guard = c->guard;
    p.fd_iso = c->fd_iso;
    p.sround = c->sround;
    p.step = (unsigned int)c->steps;
    p.gamma = c->gamma;
    p.w3 = c->omega[3];
    p.w4 = c->omega[4];
    p.w5 = c->omega[5];
    p.w6 = c->omega[6];
    p.w7 = c->omega[7];
    p.w8 = c->omega[8];
    for (int s = 0; s < 4; ++s) {
        const bool moving = c->sides[s].kind == LBM_SIDE_MOVING_WALL;
        p.side_u[s][0] = moving ? c->sides[s].ux : 0.0;
        p.side_u[s][1] = moving ? c->sides[s].uy : 0.0;
    }
    // open sides: the inlet's peak speed rides in side_u[west]
    p.inlet = c->sides[0].kind == LBM_SIDE_INLET;
    p.outlet = c->sides[1].kind == LBM_SIDE_OUTLET;
    if (p.inlet) p.side_u[0][0] = c->sides[0].ux;
    p.ghost_in = c->d_ghost[c->cur];
    p.ghost_out = c->d_ghost[1 - c->cur];
    p.Fx = c->Fx;
    p.Fy = c->Fy;
    p.force = c->d_force;
    p.solid = c->d_solid;
    p.guard_count = c->d_guard;
    p.error = c->d_err;
    p.work = c->d_work;
    p.cf.set(c->gamma, c->omega, c->gi_mode, c->Fx, c->Fy, p.side_u);
    p.cd.set(c->gamma, c->omega, c->gi_mode, c->Fx, c->Fy, p.side_u);
    const double out_u = p.outlet ? c->sides[1].ux : 0.0;
    p.cf.set_open(c->ny, out_u);
    p.cd.set_open(c->ny, out_u);
    p.c2.set(p.cf);
    p.nstrips = (c->nx + strip_width(c->storage) - 1) / strip_width(c->storage);
    const int bps = step_blocks_per_sm(c, p);
    const int resident = c->num_sms * bps * WARPS;  // resident warps
    int Ly = c->Ly_option;
    if (Ly <= 0) {
        // at least four items per resident warp (handed out dynamically) and
        // segments of at most 14 rows: a warp works through an item's rows one
        // after another, so short items keep the latency of a small domain's
        // step and the tail short, while each item re-reads four halo source
        // rows (4096^2 FP32 on GB300, phase-ordered items: 8 rows 76.8, 12 rows
        // 78.4, 14 rows 78.5, 16 rows 77.7, 24 rows 76.2 GLUPS; FP16 14 and 16
        // rows 75.3)
        int nseg = (4 * resident + p.nstrips - 1) / p.nstrips;
        if (nseg < 1) nseg = 1;
        Ly = (c->ny + nseg - 1) / nseg;
        if (Ly > 14) Ly = 14;
        if (Ly < 1) Ly = 1;
    }
    if (Ly > c->ny) Ly = c->ny;
    p.Ly = Ly;
    const int nseg = (c->ny + Ly - 1) / Ly;
    p.nseg = nseg;
    p.nwave = 1;
    p.nseg_phase = nseg;
    p.nitems = p.nstrips * nseg;
    if (c->storage != LBM_STORAGE_F64) {
        // one phase of segments per wave of resident warps (see StepParams)
        const int waves = (int)((double)p.nitems / resident + 0.5);
        if (waves > 1 && waves < nseg) {
            p.nwave = waves;
            p.nseg_phase = (nseg + waves - 1) / waves;
            p.nitems = p.nstrips * p.nseg_phase * waves;
        }
    }
    return p;
}

int step_grid(const lbm_ctx *c, const StepParams &p)
{
    const int bps = step_blocks_per_sm(c, p);
    const int resident = c->num_sms * bps;
    const int blocks = (p.nitems + WARPS - 1) / WARPS;
    return blocks < resident ? blocks : resident;
}

cudaError_t launch_step(const lbm_ctx *c, const StepParams &p, int grid)
{
    const CUtensorMap &tin = c->tload[c->cur];
    const CUtensorMap &tout = c->tstore[1 - c->cur];
    const void *fin = c->f[c->cur];
    void *fout = c->f[1 - c->cur];
    switch (c->storage) {
    case LBM_STORAGE_F16: return launch_step_f16(p, tin, tout, fin, fout, grid, c->stream);
    case LBM_STORAGE_BF16: return launch_step_bf16(p, tin, tout, fin, fout, grid, c->stream);
    case LBM_STORAGE_F64: return launch_step_f64(p, tin, tout, fin, fout, grid, c->stream);
    default: return launch_step_f32(p, tin, tout, fin, fout, grid, c->stream);
    }
}

cudaError_t build_tensor_maps(lbm_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        cudaError_t e =
            make_tensor_maps(&c->tload[k], &c->tstore[k], c->storage, c->f[k], c->nx, c->ny, c->pitch, c->plane);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// A step kernel that gave up on a bounded wait leaves a flag; report it once.
lbm_status check_device_error(lbm_ctx *c)
{
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error flag");
    if (v) {
        // on the context's stream: later kernels there see the cleared counters
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        cudaMemsetAsync(c->d_work, 0, 2 * sizeof(unsigned int), c->stream);
        cudaStreamSynchronize(c->stream);
        if (v == 2) return fail(LBM_ERR_CUDA, "debug bounds check: a kernel index was out of range (device error flag 2)");
        return fail(LBM_ERR_CUDA, "a kernel's bounded wait expired (device error flag raised)");
    }
    return LBM_OK;
}

bool valid_omega(double w) { return w > 0.0 && w < 2.0 && isfinite(w); }

lbm_status check_ctx(const lbm_ctx *c)
{
    if (!c) return fail(LBM_ERR_INVALID, "null context");
    return LBM_OK;
}

void free_ctx(lbm_ctx *c)
{
    if (!c) return;
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    if (c->stream && c->stream != c->own_stream) cudaStreamSynchronize(c->stream);
    dev_free(c->f[0]);
    dev_free(c->f[1]);
    dev_free(c->d_solid);
    dev_free(c->d_force);
    dev_free(c->d_snap_ux);
    dev_free(c->d_snap_uy);
    dev_free(c->d_partials);
    dev_free(c->d_result);
    dev_free(c->d_guard);
    dev_free(c->d_err);
    dev_free(c->d_work);
    dev_free(c->d_stage);
    dev_free(c->d_ghost[0]);
    dev_free(c->d_ghost[1]);
    if (c->h_result) cudaFreeHost(c->h_result);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

// Device staging buffer of at least `bytes` (kept for the context's lifetime).
void *stage_buffer(lbm_ctx *c, size_t bytes)
{
    if (bytes <= c->stage_bytes) return c->d_stage;
    if (c->d_stage) {
        cudaStreamSynchronize(c->stream);
        dev_free(c->d_stage);
    }
    c->d_stage = dev_alloc(bytes);
    c->stage_bytes = c->d_stage ? bytes : 0;
    return c->d_stage;
}

// Outlet ghost column of the current state from its last column (a no-op
// without an outlet).
lbm_status outlet_reseed(lbm_ctx *c)
{
    if (!c->d_ghost[0]) return LBM_OK;
    StepParams p = make_params(c);
    LBM_CUDA(launch_outlet_seed(p, c->storage, c->f[c->cur], c->d_ghost[c->cur], c->stream));
    return LBM_OK;
}

lbm_status snapshot_reset(lbm_ctx *c)
{
    StepParams p = make_params(c);
    LBM_CUDA(launch_residual(p, c->storage, c->f[c->cur], c->d_snap_ux, c->d_snap_uy, c->d_partials,
                             c->res_blocks, c->d_result, c->stream));
    return LBM_OK;
}

}  // namespace

extern "C" {

const char *lbm_last_error(void) { return g_error.c_str(); }

lbm_status lbm_set_allocator(const lbm_allocator *a)
{
    if (a && (!a->alloc || !a->release)) return fail(LBM_ERR_INVALID, "allocator needs alloc and release");
    if (a) g_alloc = *a;
    else g_alloc = lbm_allocator{nullptr, nullptr, nullptr};
    return LBM_OK;
}

lbm_status lbm_create(int nx, int ny, double nu, double gamma, double U, const lbm_boundaries *bnd,
                      lbm_ctx **out)
{
    if (!out) return fail(LBM_ERR_INVALID, "out is null");
    *out = nullptr;
    if (nx < 3 || ny < 3) return fail(LBM_ERR_INVALID, "nx and ny must be >= 3");
    if (ny > 65535) return fail(LBM_ERR_INVALID, "ny must be <= 65535");
    if ((long long)nx * ny > (1LL << 31) / 9) return fail(LBM_ERR_INVALID, "domain too large");
    if (!(nu > 0.0) || !isfinite(nu)) return fail(LBM_ERR_INVALID, "nu must be > 0");
    if (!(gamma > 0.0 && gamma <= 1.0)) return fail(LBM_ERR_INVALID, "gamma must be in (0, 1]");
    if (!(U >= 0.0) || !isfinite(U)) return fail(LBM_ERR_INVALID, "U must be >= 0");
    const double w = 1.0 / (3.0 * nu / gamma + 0.5);
    if (!valid_omega(w)) return fail(LBM_ERR_INVALID, "omega4 out of (0, 2)");

    lbm_side sides[4];
    if (bnd) {
        sides[0] = bnd->west;
        sides[1] = bnd->east;
        sides[2] = bnd->south;
        sides[3] = bnd->north;
        for (int s = 0; s < 4; ++s)
            if (sides[s].kind < 0 || sides[s].kind > 4) return fail(LBM_ERR_INVALID, "bad side kind");
        if ((sides[0].kind == LBM_SIDE_PERIODIC) != (sides[1].kind == LBM_SIDE_PERIODIC) ||
            (sides[2].kind == LBM_SIDE_PERIODIC) != (sides[3].kind == LBM_SIDE_PERIODIC))
            return fail(LBM_ERR_INVALID, "opposite sides must both be periodic or both walls");
        for (int s = 0; s < 4; ++s) {
            if (sides[s].kind == LBM_SIDE_INLET && s != 0)
                return fail(LBM_ERR_INVALID, "an inlet must be the west side");
            if (sides[s].kind == LBM_SIDE_OUTLET && s != 1)
                return fail(LBM_ERR_INVALID, "an outlet must be the east side");
        }
        if (sides[0].kind == LBM_SIDE_INLET && !(fabs(sides[0].ux) < 0.5))
            return fail(LBM_ERR_INVALID, "inlet peak speed must be below 0.5");
        if (sides[1].kind == LBM_SIDE_OUTLET && !(sides[1].ux >= 0.0 && sides[1].ux <= 1.0))
            return fail(LBM_ERR_INVALID, "outlet convection speed must be in [0, 1]");
    } else {
        sides[0] = sides[1] = sides[2] = lbm_side{LBM_SIDE_WALL, 0.0, 0.0};
        sides[3] = lbm_side{LBM_SIDE_MOVING_WALL, U, 0.0};
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ERR_OOM, "host allocation failed");
    c->nx = nx;
    c->ny = ny;
    c->pitch = (nx + 63) / 64 * 64;
    c->plane = (long long)c->pitch * ny;
    c->nu = nu;
    c->gamma = gamma;
    c->U = U;
    c->omega[4] = c->omega[5] = w;
    for (int s = 0; s < 4; ++s) c->sides[s] = sides[s];
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (c->num_sms < 1) c->num_sms = 1;

    e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "cudaStreamCreate");
    }
    c->stream = c->own_stream;
    const size_t N = (size_t)nx * ny;
    c->f[0] = dev_alloc(pop_bytes(c));
    c->f[1] = dev_alloc(pop_bytes(c));
    c->d_snap_ux = (double *)dev_alloc(N * sizeof(double));
    c->d_snap_uy = (double *)dev_alloc(N * sizeof(double));
    StepParams p0 = make_params(c);
    c->res_blocks = residual_blocks(p0);
    c->d_partials = (double *)dev_alloc((size_t)c->res_blocks * 5 * sizeof(double));
    c->d_result = (double *)dev_alloc(8 * sizeof(double));
    c->d_guard = (unsigned long long *)dev_alloc(sizeof(unsigned long long));
    c->d_err = (int *)dev_alloc(sizeof(int));
    c->d_work = (unsigned int *)dev_alloc(2 * sizeof(unsigned int));
    if (sides[1].kind == LBM_SIDE_OUTLET) {
        c->d_ghost[0] = dev_alloc((size_t)5 * ny * sizeof(double));
        c->d_ghost[1] = dev_alloc((size_t)5 * ny * sizeof(double));
    }
    if (!c->f[0] || !c->f[1] || !c->d_snap_ux || !c->d_snap_uy || !c->d_partials || !c->d_result || !c->d_guard ||
        !c->d_err || !c->d_work || (sides[1].kind == LBM_SIDE_OUTLET && (!c->d_ghost[0] || !c->d_ghost[1]))) {
        free_ctx(c);
        return fail(LBM_ERR_OOM, "device allocation failed");
    }
    if (cudaMallocHost((void **)&c->h_result, 8 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return fail(LBM_ERR_OOM, "pinned host allocation failed");
    }
    if (bnd && bnd->solid) {
        // the mask [ny][pitch] and, after it, its row table (make_solid_rows)
        const std::vector<uint8_t> h = mask_with_row_table(bnd->solid, nx, ny, c->pitch,
                                                           sides[0].kind == LBM_SIDE_PERIODIC,
                                                           sides[2].kind == LBM_SIDE_PERIODIC);
        c->d_solid = (uint8_t *)dev_alloc(h.size());
        if (!c->d_solid) {
            free_ctx(c);
            return fail(LBM_ERR_OOM, "device allocation failed (mask)");
        }
        e = cudaMemcpy(c->d_solid, h.data(), h.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_ctx(c);
            return cuda_fail(e, "cudaMemcpy(mask)");
        }
    }
    e = build_tensor_maps(c);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "cuTensorMapEncodeTiled");
    }
    e = cudaMemsetAsync(c->d_guard, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_work, 0, 2 * sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, pop_bytes(c), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_snap_ux, 0, N * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_snap_uy, 0, N * sizeof(double), c->stream);
    if (e != cudaSuccess) {
        free_ctx(c);
        return cuda_fail(e, "cudaMemset");
    }
    *out = c;
    lbm_status s = lbm_init_fields(c, nullptr, nullptr, nullptr);
    if (s != LBM_OK) {
        free_ctx(c);
        *out = nullptr;
        return s;
    }
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *ctx) { free_ctx(ctx); }

lbm_status lbm_set_stream(lbm_ctx *c, void *stream)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    cudaStream_t s = stream ? (cudaStream_t)stream : c->own_stream;
    if (s != c->stream) {
        // order the new stream after everything queued on the old one
        cudaEvent_t ev;
        LBM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaEventRecord(ev, c->stream);
        cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        c->stream = s;
    }
    return LBM_OK;
}

lbm_status lbm_set_option(lbm_ctx *c, const char *key, double v)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!key) return fail(LBM_ERR_INVALID, "null option key");
    const std::string k(key);
    if (k == "omega3" || k == "omega6" || k == "omega7" || k == "omega8") {
        if (!valid_omega(v)) return fail(LBM_ERR_INVALID, k + " must be in (0, 2)");
        c->omega[k[5] - '0'] = v;
    } else if (k == "gi_mode") {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(LBM_ERR_INVALID, "gi_mode must be 0, 1 or 2");
        c->gi_mode = (int)v;
    } else if (k == "guard") {
        c->guard = v != 0.0;
    } else if (k == "fd") {
        if (v != 0.0 && v != 1.0) return fail(LBM_ERR_INVALID, "fd must be 0 (central) or 1 (isotropic)");
        c->fd_iso = (int)v;
    } else if (k == "stochastic_rounding") {
        c->sround = v != 0.0;
    } else if (k == "fx" || k == "fy") {
        if (!isfinite(v)) return fail(LBM_ERR_INVALID, "force must be finite");
        (k == "fx" ? c->Fx : c->Fy) = v;
    } else if (k == "cells_per_item") {
        if (!(v >= 1.0) || v > 65535.0) return fail(LBM_ERR_INVALID, "cells_per_item must be >= 1");
        c->Ly_option = (int)v;
    } else if (k == "storage") {
        const int ns = (int)v;
        if (v != (double)ns || ns < 0 || ns > 3) return fail(LBM_ERR_INVALID, "storage must be 0..3");
        if (ns == c->storage) return LBM_OK;
        const int old = c->storage;
        StepParams p = make_params(c);
        c->storage = ns;
        void *nf0 = dev_alloc(pop_bytes(c));
        void *nf1 = dev_alloc(pop_bytes(c));
        if (!nf0 || !nf1) {
            dev_free(nf0);
            dev_free(nf1);
            c->storage = old;
            return fail(LBM_ERR_OOM, "device allocation failed (storage change)");
        }
        cudaError_t e = launch_convert(p, old, c->f[c->cur], ns, nf0, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(nf1, 0, pop_bytes(c), c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            dev_free(nf0);
            dev_free(nf1);
            c->storage = old;
            return cuda_fail(e, "storage conversion");
        }
        dev_free(c->f[0]);
        dev_free(c->f[1]);
        c->f[0] = nf0;
        c->f[1] = nf1;
        c->cur = 0;
        e = build_tensor_maps(c);
        if (e != cudaSuccess) return cuda_fail(e, "cuTensorMapEncodeTiled");
        // the ghost column holds the compute precision of the new storage
        lbm_status so = outlet_reseed(c);
        if (so != LBM_OK) return so;
    } else {
        return fail(LBM_ERR_INVALID, "unknown option: " + k);
    }
    return LBM_OK;
}

lbm_status lbm_get_option(lbm_ctx *c, const char *key, double *v)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!key || !v) return fail(LBM_ERR_INVALID, "null argument");
    const std::string k(key);
    if (k.size() == 6 && k.compare(0, 5, "omega") == 0 && k[5] >= '3' && k[5] <= '8') *v = c->omega[k[5] - '0'];
    else if (k == "gi_mode") *v = c->gi_mode;
    else if (k == "guard") *v = c->guard;
    else if (k == "fd") *v = c->fd_iso;
    else if (k == "stochastic_rounding") *v = c->sround;
    else if (k == "fx") *v = c->Fx;
    else if (k == "fy") *v = c->Fy;
    else if (k == "storage") *v = c->storage;
    else if (k == "gamma") *v = c->gamma;
    else if (k == "nu") *v = c->nu;
    else if (k == "cells_per_item") *v = make_params(c).Ly;
    else if (k == "work_items") *v = make_params(c).nitems;
    else if (k == "grid") {
        StepParams p = make_params(c);
        *v = step_grid(c, p);
    } else if (k == "pitch") *v = c->pitch;
    else return fail(LBM_ERR_INVALID, "unknown option: " + k);
    return LBM_OK;
}

lbm_status lbm_set_force_field(lbm_ctx *c, const double *fx, const double *fy)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!fx && !fy) {
        LBM_CUDA(cudaStreamSynchronize(c->stream));
        dev_free(c->d_force);
        c->d_force = nullptr;
        return LBM_OK;
    }
    if (!fx || !fy) return fail(LBM_ERR_INVALID, "fx and fy must both be given");
    if (!c->d_force) {
        c->d_force = (float *)dev_alloc((size_t)2 * c->plane * sizeof(float));
        if (!c->d_force) return fail(LBM_ERR_OOM, "device allocation failed (force)");
    }
    std::vector<float> h((size_t)2 * c->plane, 0.0f);
    for (int y = 0; y < c->ny; ++y)
        for (int x = 0; x < c->nx; ++x) {
            h[(size_t)y * c->pitch + x] = (float)fx[(size_t)y * c->nx + x];
            h[(size_t)c->plane + (size_t)y * c->pitch + x] = (float)fy[(size_t)y * c->nx + x];
        }
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    LBM_CUDA(cudaMemcpy(c->d_force, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
    return LBM_OK;
}

lbm_status lbm_init_fields(lbm_ctx *c, const double *rho, const double *ux, const double *uy)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    const size_t N = (size_t)c->nx * c->ny;
    const double *src[3] = {rho, ux, uy};
    const double *dptr[3] = {nullptr, nullptr, nullptr};
    if (rho || ux || uy) {
        double *stage = (double *)stage_buffer(c, 3 * N * sizeof(double));
        if (!stage) return fail(LBM_ERR_OOM, "device allocation failed (init staging)");
        for (int i = 0; i < 3; ++i) {
            if (!src[i]) continue;
            LBM_CUDA(cudaMemcpyAsync(stage + i * N, src[i], N * 8, cudaMemcpyHostToDevice, c->stream));
            dptr[i] = stage + i * N;
        }
    }
    StepParams p = make_params(c);
    LBM_CUDA(launch_init_eq(p, c->storage, dptr[0], dptr[1], dptr[2], c->f[c->cur], c->stream));
    lbm_status s = outlet_reseed(c);
    if (s != LBM_OK) return s;
    s = snapshot_reset(c);
    if (s != LBM_OK) return s;
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    c->steps = 0;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *c, long n)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (n < 0) return fail(LBM_ERR_INVALID, "n must be >= 0");
    if (n == 0) return LBM_OK;
    StepParams p = make_params(c);
    const int grid = step_grid(c, p);
    for (long i = 0; i < n; ++i) {
        p.step = (unsigned int)c->steps;  // seeds the stochastic rounding of 16-bit storage
        p.ghost_in = c->d_ghost[c->cur];
        p.ghost_out = c->d_ghost[1 - c->cur];
        cudaError_t e = launch_step(c, p, grid);
        if (e != cudaSuccess) return cuda_fail(e, "stream_collide launch");
        c->cur = 1 - c->cur;
        c->steps += 1;
        c->launches += 1;
    }
    return LBM_OK;
}

lbm_status lbm_residual(lbm_ctx *c, double *residual, double sums[5])
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    lbm_status s = snapshot_reset(c);
    if (s != LBM_OK) return s;
    LBM_CUDA(cudaMemcpyAsync(c->h_result, c->d_result, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    s = check_device_error(c);
    if (s != LBM_OK) return s;
    const double du2 = c->h_result[0], u2 = c->h_result[1];
    double r;
    if (!isfinite(du2) || !isfinite(u2)) r = NAN;
    else if (u2 == 0.0) r = du2 == 0.0 ? 0.0 : INFINITY;
    else r = sqrt(du2 / u2);
    if (residual) *residual = r;
    if (sums)
        for (int k = 0; k < 5; ++k) sums[k] = c->h_result[k];
    return LBM_OK;
}

lbm_status lbm_run_to_steady(lbm_ctx *c, double tol, long check_every, long max_steps, double wall_seconds,
                             long *steps_done, double *final_residual)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!(tol > 0.0)) return fail(LBM_ERR_INVALID, "tol must be > 0");
    if (check_every < 1) return fail(LBM_ERR_INVALID, "check_every must be >= 1");
    if (max_steps < 0) return fail(LBM_ERR_INVALID, "max_steps must be >= 0");
    const auto t0 = std::chrono::steady_clock::now();
    long done = 0;
    double r = INFINITY;
    lbm_status st = LBM_ERR_NOT_CONVERGED;
    c->hist_steps.clear();
    c->hist_r.clear();
    // fresh snapshot at the starting state
    lbm_status s = lbm_residual(c, nullptr, nullptr);
    if (s != LBM_OK) return s;
    while (done < max_steps) {
        const long n = check_every < max_steps - done ? check_every : max_steps - done;
        s = lbm_step(c, n);
        if (s != LBM_OK) return s;
        done += n;
        s = lbm_residual(c, &r, nullptr);
        if (s != LBM_OK) return s;
        c->hist_steps.push_back(c->steps);
        c->hist_r.push_back(r);
        if (!isfinite(r)) {
            st = fail(LBM_ERR_DIVERGED, "non-finite velocity after step " + std::to_string(c->steps));
            break;
        }
        if (r < tol) {
            st = LBM_OK;
            break;
        }
        if (wall_seconds > 0.0) {
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > wall_seconds) {
                st = fail(LBM_ERR_TIMEOUT, "wall-clock limit reached");
                break;
            }
        }
    }
    if (st == LBM_ERR_NOT_CONVERGED) {
        char buf[64];
        snprintf(buf, sizeof(buf), "%.3e", r);
        fail(st, std::string("max_steps reached with residual ") + buf);
    }
    if (steps_done) *steps_done = done;
    if (final_residual) *final_residual = r;
    return st;
}

lbm_status lbm_residual_history(lbm_ctx *c, long *steps, double *residuals, long capacity, long *count)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!count || capacity < 0) return fail(LBM_ERR_INVALID, "count is null or capacity < 0");
    const long n = (long)c->hist_r.size();
    const long m = capacity < n ? capacity : n;
    for (long i = 0; i < m; ++i) {
        if (steps) steps[i] = c->hist_steps[(size_t)i];
        if (residuals) residuals[i] = c->hist_r[(size_t)i];
    }
    *count = n;
    return LBM_OK;
}

lbm_status lbm_fields(lbm_ctx *c, double *rho, double *ux, double *uy)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    const size_t N = (size_t)c->nx * c->ny;
    double *d = (double *)stage_buffer(c, 3 * N * sizeof(double));
    if (!d) return fail(LBM_ERR_OOM, "device allocation failed (fields staging)");
    StepParams p = make_params(c);
    LBM_CUDA(launch_fields(p, c->storage, c->f[c->cur], d, d + N, d + 2 * N, c->stream));
    if (rho) LBM_CUDA(cudaMemcpyAsync(rho, d, N * 8, cudaMemcpyDeviceToHost, c->stream));
    if (ux) LBM_CUDA(cudaMemcpyAsync(ux, d + N, N * 8, cudaMemcpyDeviceToHost, c->stream));
    if (uy) LBM_CUDA(cudaMemcpyAsync(uy, d + 2 * N, N * 8, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

lbm_status lbm_get_populations(lbm_ctx *c, double *f)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!f) return fail(LBM_ERR_INVALID, "null output");
    const size_t N = (size_t)c->nx * c->ny;
    double *d = (double *)stage_buffer(c, 9 * N * sizeof(double));
    if (!d) return fail(LBM_ERR_OOM, "device allocation failed (population staging)");
    StepParams p = make_params(c);
    LBM_CUDA(launch_pops_to_f64(p, c->storage, c->f[c->cur], d, c->stream));
    LBM_CUDA(cudaMemcpyAsync(f, d, 9 * N * 8, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

lbm_status lbm_set_populations(lbm_ctx *c, const double *f)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!f) return fail(LBM_ERR_INVALID, "null input");
    const size_t N = (size_t)c->nx * c->ny;
    double *d = (double *)stage_buffer(c, 9 * N * sizeof(double));
    if (!d) return fail(LBM_ERR_OOM, "device allocation failed (population staging)");
    LBM_CUDA(cudaMemcpyAsync(d, f, 9 * N * 8, cudaMemcpyHostToDevice, c->stream));
    StepParams p = make_params(c);
    LBM_CUDA(launch_pops_from_f64(p, c->storage, d, c->f[c->cur], c->stream));
    lbm_status s = outlet_reseed(c);
    if (s != LBM_OK) return s;
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_drag(lbm_ctx *c, double force[2])
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!force) return fail(LBM_ERR_INVALID, "null output");
    StepParams p = make_params(c);
    LBM_CUDA(launch_drag(p, c->storage, c->f[c->cur], c->d_partials, c->res_blocks, c->d_result, c->stream));
    LBM_CUDA(cudaMemcpyAsync(c->h_result, c->d_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    force[0] = c->h_result[0];
    force[1] = c->h_result[1];
    return check_device_error(c);
}

lbm_status lbm_steps_done(lbm_ctx *c, long *steps)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!steps) return fail(LBM_ERR_INVALID, "null output");
    *steps = c->steps;
    return LBM_OK;
}

lbm_status lbm_kernel_launches(lbm_ctx *c, long *launches)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!launches) return fail(LBM_ERR_INVALID, "null output");
    *launches = c->launches;
    return LBM_OK;
}

lbm_status lbm_guard_count(lbm_ctx *c, long *count)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!count) return fail(LBM_ERR_INVALID, "null output");
    unsigned long long v = 0;
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    LBM_CUDA(cudaMemcpy(&v, c->d_guard, sizeof(v), cudaMemcpyDeviceToHost));
    *count = (long)v;
    return LBM_OK;
}

lbm_status lbm_bounded_wait_selftest(lbm_ctx *c, double *waited_s)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    // the kernel writes the time it waited into the last slot of the result scratch
    unsigned long long *d_ns = reinterpret_cast<unsigned long long *>(c->d_result + 7);
    unsigned long long ns = 0;
    cudaError_t e = launch_bounded_wait_selftest(c->d_err, d_ns, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    if (waited_s) *waited_s = (double)ns * 1e-9;
    return check_device_error(c);
}

// Checkpoint layout: 8-byte magic, then int32 {version, nx, ny, storage, gi_mode},
// int64 steps, double {gamma, nu, omega3..8, Fx, Fy}, then nine planes of
// nx*ny stored elements (rows packed); version 2 (domains with a convective
// outlet) appends the outlet ghost column, 5 * ny values in the compute type.
static const char kMagic[8] = {'L', 'B', 'M', 'G', 'B', '3', '0', '0'};

lbm_status lbm_save(lbm_ctx *c, const char *path)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!path) return fail(LBM_ERR_INVALID, "null path");
    const size_t es = storage_bytes(c->storage);
    std::vector<unsigned char> h((size_t)9 * c->nx * c->ny * es);
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    LBM_CUDA(cudaMemcpy2D(h.data(), (size_t)c->nx * es, c->f[c->cur], (size_t)c->pitch * es, (size_t)c->nx * es,
                          (size_t)9 * c->ny, cudaMemcpyDeviceToHost));
    const size_t gbytes = (size_t)5 * c->ny * (c->storage == LBM_STORAGE_F64 ? sizeof(double) : sizeof(float));
    std::vector<unsigned char> gh(c->d_ghost[0] ? gbytes : 0);
    if (!gh.empty()) LBM_CUDA(cudaMemcpy(gh.data(), c->d_ghost[c->cur], gbytes, cudaMemcpyDeviceToHost));
    FILE *fp = fopen(path, "wb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    int hdr[5] = {gh.empty() ? 1 : 2, c->nx, c->ny, c->storage, c->gi_mode};
    long long steps = c->steps;
    double par[10] = {c->gamma, c->nu, c->omega[3], c->omega[4], c->omega[5], c->omega[6], c->omega[7], c->omega[8], c->Fx, c->Fy};
    bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(hdr, sizeof(int), 5, fp) == 5 &&
              fwrite(&steps, sizeof(steps), 1, fp) == 1 && fwrite(par, sizeof(double), 10, fp) == 10 &&
              fwrite(h.data(), 1, h.size(), fp) == h.size() &&
              (gh.empty() || fwrite(gh.data(), 1, gh.size(), fp) == gh.size());
    ok = (fclose(fp) == 0) && ok;
    if (!ok) return fail(LBM_ERR_IO, std::string("write failed: ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx *c, const char *path)
{
    if (check_ctx(c)) return LBM_ERR_INVALID;
    if (!path) return fail(LBM_ERR_INVALID, "null path");
    FILE *fp = fopen(path, "rb");
    if (!fp) return fail(LBM_ERR_IO, std::string("cannot open ") + path);
    char magic[8];
    int hdr[5];
    long long steps;
    double par[10];
    bool ok = fread(magic, 1, 8, fp) == 8 && memcmp(magic, kMagic, 8) == 0 &&
              fread(hdr, sizeof(int), 5, fp) == 5 && fread(&steps, sizeof(steps), 1, fp) == 1 &&
              fread(par, sizeof(double), 10, fp) == 10;
    if (!ok || (hdr[0] != 1 && hdr[0] != 2)) {
        fclose(fp);
        return fail(LBM_ERR_IO, "not a checkpoint of this library");
    }
    if ((hdr[0] == 2) != (c->d_ghost[0] != nullptr)) {
        fclose(fp);
        return fail(LBM_ERR_INVALID, "checkpoint and context differ in their outlet side");
    }
    if (hdr[1] != c->nx || hdr[2] != c->ny) {
        fclose(fp);
        return fail(LBM_ERR_INVALID, "checkpoint size differs from the context");
    }
    if (hdr[3] < 0 || hdr[3] > 3 || hdr[4] < 0 || hdr[4] > 2) {
        fclose(fp);
        return fail(LBM_ERR_IO, "corrupt checkpoint header");
    }
    lbm_status s = lbm_set_option(c, "storage", hdr[3]);
    if (s != LBM_OK) {
        fclose(fp);
        return s;
    }
    const size_t es = storage_bytes(c->storage);
    std::vector<unsigned char> h((size_t)9 * c->nx * c->ny * es);
    ok = fread(h.data(), 1, h.size(), fp) == h.size();
    const size_t gbytes = (size_t)5 * c->ny * (c->storage == LBM_STORAGE_F64 ? sizeof(double) : sizeof(float));
    std::vector<unsigned char> gh(hdr[0] == 2 ? gbytes : 0);
    if (ok && !gh.empty()) ok = fread(gh.data(), 1, gh.size(), fp) == gh.size();
    fclose(fp);
    if (!ok) return fail(LBM_ERR_IO, "truncated checkpoint");
    c->gi_mode = hdr[4];
    c->gamma = par[0];
    c->nu = par[1];
    for (int k = 0; k < 6; ++k) c->omega[3 + k] = par[2 + k];
    c->Fx = par[8];
    c->Fy = par[9];
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    LBM_CUDA(cudaMemcpy2D(c->f[c->cur], (size_t)c->pitch * es, h.data(), (size_t)c->nx * es, (size_t)c->nx * es,
                          (size_t)9 * c->ny, cudaMemcpyHostToDevice));
    if (!gh.empty()) LBM_CUDA(cudaMemcpy(c->d_ghost[c->cur], gh.data(), gh.size(), cudaMemcpyHostToDevice));
    c->steps = (long)steps;
    return snapshot_reset(c);
}

}  // extern "C"

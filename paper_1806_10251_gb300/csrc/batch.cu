// Batches of steady solves and the serving loop (continuous batching).
//
// A batch owns up to max_slots resident domains.  Every engine tick admits
// queued requests whose device footprint fits the budget (FIFO), advances all
// running domains K steps by replaying one captured CUDA graph of K launches
// of the batched step kernel (all domains in lockstep), then checks each
// running domain's FP64 convergence residual and retires the converged,
// diverged and exhausted ones.  Per-domain tables (parameters, TMA
// descriptors, active list, item prefix sums, active count) live in device
// memory, so the graph stays valid while domains join and retire.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lbm_internal.h"

namespace lbm {
cudaError_t launch_batch_f32(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s);
cudaError_t launch_batch_f16(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s);
cudaError_t launch_batch_bf16(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s);
cudaError_t launch_batch_f64(int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s);
int batch_blocks_f32(int gi_mode, bool forced);
int batch_blocks_f16(int gi_mode, bool forced);
int batch_blocks_bf16(int gi_mode, bool forced);
int batch_blocks_f64(int gi_mode, bool forced);

cudaError_t launch_batch_step(int storage, int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s)
{
    switch (storage) {
    case LBM_STORAGE_F16: return launch_batch_f16(gi_mode, forced, a, grid, s);
    case LBM_STORAGE_BF16: return launch_batch_bf16(gi_mode, forced, a, grid, s);
    case LBM_STORAGE_F64: return launch_batch_f64(gi_mode, forced, a, grid, s);
    default: return launch_batch_f32(gi_mode, forced, a, grid, s);
    }
}

int batch_blocks_per_sm(int storage, int gi_mode, bool forced)
{
    switch (storage) {
    case LBM_STORAGE_F16: return batch_blocks_f16(gi_mode, forced);
    case LBM_STORAGE_BF16: return batch_blocks_bf16(gi_mode, forced);
    case LBM_STORAGE_F64: return batch_blocks_f64(gi_mode, forced);
    default: return batch_blocks_f32(gi_mode, forced);
    }
}
}  // namespace lbm

using namespace lbm;

namespace {

struct Slot {
    bool used = false;
    long id = 0;
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;
    void *f[2] = {nullptr, nullptr};
    double *snap = nullptr;  // 2 * nx * ny: ux then uy
    uint8_t *solid = nullptr;
    size_t bytes = 0;
    StepParams p{};
    bool forced = false;  // uniform body force: stepped by the forced kernel variant
    bool running = false;
    double tol = 0;
    long max_steps = 0;
    int res_blocks = 1;
    int check_mult = 1;         // convergence check every check_mult ticks
    int ticks_since_check = 0;
    bool check_due = false;     // this tick ends with a check
    double *acc = nullptr;      // velocity sums of the current check window ([2][N]), or null
    int samples = 0;            // samples in acc
};

struct Pending {
    long id;
    lbm_request req;
    std::vector<uint8_t> solid;
};

struct Record {
    int slot = -1;
    int readers = 0;  // lbm_batch_fields calls reading the slot's buffers; release waits for 0
    bool cancel = false;  // lbm_batch_cancel on a running request: stop at the next tick
    int state = LBM_REQ_QUEUED;
    long steps = 0;
    double residual = INFINITY;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct lbm_batch {
    int storage = LBM_STORAGE_F16;
    int gi_mode = LBM_GI_FULL;
    size_t budget = 0, used = 0;
    int max_slots = 1024;
    int check_every = 1000;
    int avg_samples = -1;  // velocity samples per check interval (-1: 16 for 16-bit storage, else 0)
    int Ly_option = 0;
    int Ly = 24;
    bool tuned = false;
    double tuned_strip_rows = 0;  // active strip-rows when the rows per item were last chosen
    int parity = 0;
    int num_sms = 1;
    std::vector<Slot> slots;
    std::vector<DomainDesc> h_desc;
    DomainDesc *d_desc = nullptr;
    int *d_active = nullptr, *d_prefix = nullptr;
    unsigned int *d_step0 = nullptr, *h_step0 = nullptr;  // per active index: steps done (h_ pinned)
    int sround = 1;
    BatchState *d_state = nullptr;
    int *h_active = nullptr, *h_prefix = nullptr;  // pinned
    BatchState *h_state = nullptr;                 // pinned
    unsigned int *d_work = nullptr;
    unsigned int *d_ctl = nullptr;  // persistent kernel: item counters, barrier arrivals and generation
    int persistent_option = -1;     // -1: chosen by the autotuner, 0: per-step launches, 1: persistent
    int admission = 0;              // 0: first come first served, 1: smallest domain first
    double max_running_cells = 0;   // admit while the running domains hold fewer cells (0: no cap)
    int mode = 0;                   // current: 0 per-step launches, 1 persistent kernel
    int *d_err = nullptr;
    double *d_sums = nullptr, *d_partials = nullptr, *h_sums = nullptr;
    cudaStream_t stream = nullptr, io_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_K = 0;
    int graph_M = 0;
    int graph_variants = 0;                 // bit 0: unforced launch captured, bit 1: forced launch
    int variants = 0;                       // the same bits for the current active set
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;      // queue, records, slot bookkeeping
    std::mutex run_mu;  // one tick at a time
    std::deque<Pending> queue;
    std::unordered_map<long, Record> records;
    long next_id = 1;
    std::thread engine;
    std::atomic<bool> stop{false};
    std::condition_variable cv;
    bool engine_on = false;
    double cell_updates = 0;
    long launches = 0, ticks = 0;
    std::string engine_error;
};

namespace {

double seconds(const lbm_batch *b)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - b->t0).count();
}

lbm_status bfail(lbm_status s, const std::string &m) { return set_error(s, m); }

// Velocity samples per check interval: a reduced-precision batch averages the
// velocity over the interval (stochastic rounding leaves an unbiased noise on
// the state that the average takes out of the residual and the result).
int samples_per_tick(const lbm_batch *b)
{
    const int m = b->avg_samples >= 0
                      ? b->avg_samples
                      : ((b->storage == LBM_STORAGE_F16 || b->storage == LBM_STORAGE_BF16) ? 16 : 0);
    return m < b->check_every ? m : b->check_every;
}

size_t footprint(const lbm_batch *b, int nx, int ny, bool solid)
{
    const size_t pitch = (size_t)(nx + 63) / 64 * 64;
    const size_t plane = pitch * ny;
    const size_t snaps = samples_per_tick(b) > 0 ? 4 : 2;  // snapshot (+ window sums) in FP64
    return 2 * 9 * plane * storage_bytes(b->storage) + snaps * (size_t)nx * ny * sizeof(double) +
           (solid ? plane + (size_t)ny * ((nx + 31) / 32) : 0);  // mask + its row table
}

void free_slot(Slot &s)
{
    if (s.f[0]) cudaFree(s.f[0]);
    if (s.f[1]) cudaFree(s.f[1]);
    if (s.snap) cudaFree(s.snap);
    if (s.solid) cudaFree(s.solid);
    if (s.acc) cudaFree(s.acc);
    s = Slot();
}

void set_geometry(StepParams &p, int Ly, int storage)
{
    p.nstrips = (p.nx + strip_width(storage) - 1) / strip_width(storage);
    p.Ly = Ly < p.ny ? Ly : p.ny;
    p.nseg = (p.ny + p.Ly - 1) / p.Ly;
    p.nwave = 1;  // segment-major order inside a batch
    p.nseg_phase = p.nseg;
    p.nitems = p.nstrips * p.nseg;
}

// Allocate and initialise one admitted request (rest state, lid or walls).
lbm_status admit(lbm_batch *b, int si, const Pending &q)
{
    Slot &s = b->slots[si];
    const lbm_request &r = q.req;
    s.used = true;
    s.id = q.id;
    s.nx = r.nx;
    s.ny = r.ny;
    s.pitch = (r.nx + 63) / 64 * 64;
    s.plane = (long long)s.pitch * r.ny;
    s.bytes = footprint(b, r.nx, r.ny, !q.solid.empty());
    const size_t pb = 9 * (size_t)s.plane * storage_bytes(b->storage);
    const size_t N = (size_t)r.nx * r.ny;
    const bool avg = samples_per_tick(b) > 0;
    // the mask [ny][pitch] and, after it, its row table (make_solid_rows)
    std::vector<uint8_t> mask;
    if (!q.solid.empty())
        mask = mask_with_row_table(q.solid.data(), r.nx, r.ny, s.pitch, r.use_bnd && r.bnd.west.kind == LBM_SIDE_PERIODIC,
                                   r.use_bnd && r.bnd.south.kind == LBM_SIDE_PERIODIC);
    if (cudaMalloc(&s.f[0], pb) != cudaSuccess || cudaMalloc(&s.f[1], pb) != cudaSuccess ||
        cudaMalloc((void **)&s.snap, 2 * N * sizeof(double)) != cudaSuccess ||
        (avg && cudaMalloc((void **)&s.acc, 2 * N * sizeof(double)) != cudaSuccess) ||
        (!mask.empty() && cudaMalloc((void **)&s.solid, mask.size()) != cudaSuccess)) {
        cudaGetLastError();
        free_slot(s);
        return LBM_ERR_OOM;
    }
    if (s.solid && cudaMemcpy(s.solid, mask.data(), mask.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        free_slot(s);
        return LBM_ERR_CUDA;
    }
    // parameters (the same derivation as lbm_create / make_params)
    lbm_side sides[4];
    if (r.use_bnd) {
        sides[0] = r.bnd.west;
        sides[1] = r.bnd.east;
        sides[2] = r.bnd.south;
        sides[3] = r.bnd.north;
    } else {
        sides[0] = sides[1] = sides[2] = lbm_side{LBM_SIDE_WALL, 0.0, 0.0};
        sides[3] = lbm_side{LBM_SIDE_MOVING_WALL, r.U, 0.0};
    }
    StepParams &p = s.p;
    memset(&p, 0, sizeof(p));
    p.nx = r.nx;
    p.ny = r.ny;
    p.pitch = s.pitch;
    p.plane = s.plane;
    p.perx = sides[0].kind == LBM_SIDE_PERIODIC;
    p.pery = sides[2].kind == LBM_SIDE_PERIODIC;
    p.gi_mode = b->gi_mode;
    p.gamma = r.gamma;
    double w[9] = {0, 0, 0, 1, 1, 1, 1, 1, 1};
    w[4] = w[5] = 1.0 / (3.0 * r.nu / r.gamma + 0.5);
    p.w3 = w[3];
    p.w4 = w[4];
    p.w5 = w[5];
    p.w6 = w[6];
    p.w7 = w[7];
    p.w8 = w[8];
    for (int k = 0; k < 4; ++k) {
        const bool moving = sides[k].kind == LBM_SIDE_MOVING_WALL;
        p.side_u[k][0] = moving ? sides[k].ux : 0.0;
        p.side_u[k][1] = moving ? sides[k].uy : 0.0;
    }
    p.Fx = r.fx;
    p.Fy = r.fy;
    p.solid = s.solid;
    p.sround = b->sround;
    p.cf.set(r.gamma, w, b->gi_mode, r.fx, r.fy, p.side_u);
    p.cd.set(r.gamma, w, b->gi_mode, r.fx, r.fy, p.side_u);
    p.c2.set(p.cf);
    set_geometry(p, b->Ly, b->storage);
    s.tol = r.tol;
    s.max_steps = r.max_steps;
    s.check_mult = r.check_every > b->check_every ? (int)((r.check_every + b->check_every - 1) / b->check_every) : 1;
    s.ticks_since_check = 0;
    s.res_blocks = residual_blocks(p);
    // descriptor table entry
    DomainDesc &d = b->h_desc[si];
    memset(&d, 0, sizeof(d));
    for (int k = 0; k < 2; ++k)
        if (make_tensor_maps(&d.tload[k], &d.tstore[k], b->storage, s.f[k], r.nx, r.ny, s.pitch, s.plane) !=
            cudaSuccess) {
            free_slot(s);
            return LBM_ERR_CUDA;
        }
    d.p = p;
    d.f[0] = s.f[0];
    d.f[1] = s.f[1];
    d.forced = r.fx != 0.0 || r.fy != 0.0;
    s.forced = d.forced != 0;
    d.acc = s.acc;
    s.samples = 0;
    cudaError_t e = cudaMemcpyAsync(b->d_desc + si, &d, sizeof(DomainDesc), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && s.acc) e = cudaMemsetAsync(s.acc, 0, 2 * N * sizeof(double), b->stream);
    if (e == cudaSuccess)
        e = launch_init_eq(p, b->storage, nullptr, nullptr, nullptr, s.f[b->parity], b->stream);
    if (e == cudaSuccess)
        e = launch_residual(p, b->storage, s.f[b->parity], s.snap, s.snap + N, b->d_partials, s.res_blocks,
                            b->d_sums + 5 * si, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // h_desc entry may change later
    if (e != cudaSuccess) {
        free_slot(s);
        return LBM_ERR_CUDA;
    }
    s.running = true;
    return LBM_OK;
}

void admit_pending(lbm_batch *b)
{
    for (;;) {
        Pending q;
        int si = -1;
        {
            std::lock_guard<std::mutex> lk(b->mu);
            if (b->queue.empty()) return;
            // the next request: the oldest, or the oldest of the smallest domains
            size_t pick = 0;
            if (b->admission == 1)
                for (size_t i = 1; i < b->queue.size(); ++i)
                    if ((long long)b->queue[i].req.nx * b->queue[i].req.ny <
                        (long long)b->queue[pick].req.nx * b->queue[pick].req.ny)
                        pick = i;
            const Pending &head = b->queue[pick];
            if (b->max_running_cells > 0) {
                double run = 0;
                for (const Slot &s : b->slots)
                    if (s.used && s.running) run += (double)s.nx * s.ny;
                // the cap bounds the step time (so the tick, admission and
                // cancellation latency); an empty batch admits any request
                if (run > 0 && run + (double)head.req.nx * head.req.ny > b->max_running_cells) return;
            }
            const size_t need = footprint(b, head.req.nx, head.req.ny, !head.solid.empty());
            if (b->used + need > b->budget) return;  // the pick waits for memory
            for (int k = 0; k < b->max_slots; ++k)
                if (!b->slots[k].used) {
                    si = k;
                    break;
                }
            if (si < 0) return;
            q = std::move(b->queue[pick]);
            b->queue.erase(b->queue.begin() + (long)pick);
            b->slots[si].used = true;  // reserve
            b->used += need;
        }
        const lbm_status st = admit(b, si, q);
        std::lock_guard<std::mutex> lk(b->mu);
        Record &rec = b->records[q.id];
        if (st != LBM_OK) {
            b->used -= footprint(b, q.req.nx, q.req.ny, !q.solid.empty());
            b->slots[si] = Slot();
            rec.state = LBM_REQ_FAILED;
            rec.t_admit = rec.t_done = seconds(b);
        } else {
            rec.slot = si;
            rec.state = LBM_REQ_RUNNING;
            rec.t_admit = seconds(b);
        }
    }
}

// Upload the active list and the item prefix sums; returns the active count.
int build_active(lbm_batch *b, double &cells)
{
    int n = 0, total = 0, split = 0;
    cells = 0;
    b->variants = 0;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        // the unforced domains first, then the forced ones: each group is one
        // launch of its own kernel variant over a contiguous item range
        // cancelled requests leave the active set here, between ticks
        for (int k = 0; k < b->max_slots; ++k) {
            Slot &s = b->slots[k];
            if (!s.used || !s.running) continue;
            Record &rec = b->records[s.id];
            if (rec.cancel) {
                s.running = false;
                rec.state = LBM_REQ_CANCELLED;
                rec.t_done = seconds(b);
            }
        }
        for (int pass = 0; pass < 2; ++pass) {
            for (int k = 0; k < b->max_slots; ++k) {
                const Slot &s = b->slots[k];
                if (!s.used || !s.running || (int)s.forced != pass) continue;
                b->h_active[n] = k;
                b->h_prefix[n] = total;
                b->h_step0[n] = (unsigned int)b->records[s.id].steps;
                total += s.p.nitems;
                cells += (double)s.nx * s.ny;
                b->variants |= 1 << pass;
                ++n;
            }
            if (pass == 0) split = total;
        }
    }
    b->h_prefix[n] = total;
    b->h_state->n_active = n;
    b->h_state->total_items = total;
    b->h_state->split_items = split;
    cudaMemcpyAsync(b->d_active, b->h_active, (size_t)(n > 0 ? n : 1) * sizeof(int), cudaMemcpyHostToDevice,
                    b->stream);
    cudaMemcpyAsync(b->d_prefix, b->h_prefix, (size_t)(n + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    cudaMemcpyAsync(b->d_step0, b->h_step0, (size_t)(n > 0 ? n : 1) * sizeof(unsigned int), cudaMemcpyHostToDevice,
                    b->stream);
    cudaMemcpyAsync(b->d_state, b->h_state, sizeof(BatchState), cudaMemcpyHostToDevice, b->stream);
    return n;
}

BatchArgs batch_args(const lbm_batch *b, int parity, int k, bool forced)
{
    BatchArgs a;
    a.domains = b->d_desc;
    a.active = b->d_active;
    a.prefix = b->d_prefix;
    a.state = b->d_state;
    a.work = b->d_work;
    a.error = b->d_err;
    a.parity = parity;
    a.step0 = b->d_step0;
    a.k = k;
    a.forced = forced;
    a.ctl = b->d_ctl;
    return a;
}

int batch_grid(const lbm_batch *b, bool forced)
{
    return b->num_sms * batch_blocks_per_sm(b->storage, b->gi_mode, forced);
}

// One step of all running domains: a launch per force variant present.
void launch_batch_all(lbm_batch *b, int parity, int k, const int grid[2])
{
    for (int v = 0; v < 2; ++v)
        if (b->variants >> v & 1)
            launch_batch_step(b->storage, b->gi_mode, v == 1, batch_args(b, parity, k, v == 1), grid[v], b->stream);
}

// The persistent kernel serves the full GI kernel in the packed storages when
// the running domains are all of one force variant.
bool persistent_possible(const lbm_batch *b)
{
    return b->persistent_option != 0 && batch_persistent_supported(b->storage, b->gi_mode) &&
           (b->variants == 1 || b->variants == 2);
}

int persistent_grid(const lbm_batch *b)
{
    return b->num_sms * batch_persistent_blocks_per_sm(b->storage, b->variants == 2);
}

// Steps k0 .. k0 + n - 1 of a tick that starts on buffer `parity`, in the
// current mode: one persistent launch, or a launch per step and force variant.
cudaError_t launch_steps(lbm_batch *b, int parity, int k0, int n, const int grid[2], int pgrid)
{
    if (b->mode == 1) {
        const bool forced = b->variants == 2;
        return launch_batch_persistent(b->storage, forced, batch_args(b, parity, k0, forced), k0, n, pgrid,
                                       b->stream);
    }
    for (int k = k0; k < k0 + n; ++k) launch_batch_all(b, (parity + k) & 1, k, grid);
    return cudaGetLastError();
}

// Set the rows per item of every running domain and re-upload their descriptors.
void apply_Ly(lbm_batch *b, int Ly)
{
    b->Ly = Ly;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        for (int k = 0; k < b->max_slots; ++k) {
            Slot &s = b->slots[k];
            if (!s.used || !s.running) continue;
            set_geometry(s.p, Ly, b->storage);
            b->h_desc[k].p = s.p;
            cudaMemcpyAsync(&b->d_desc[k].p, &b->h_desc[k].p, sizeof(StepParams), cudaMemcpyHostToDevice,
                            b->stream);
        }
    }
    cudaStreamSynchronize(b->stream);
}

// Strip-rows of the running domains (one warp-strip row is the unit of work
// of the step kernel).
double active_strip_rows(lbm_batch *b)
{
    std::lock_guard<std::mutex> lk(b->mu);
    double n = 0;
    const int w = strip_width(b->storage);
    for (int k = 0; k < b->max_slots; ++k) {
        const Slot &s = b->slots[k];
        if (s.used && s.running) n += (double)((s.nx + w - 1) / w) * s.ny;
    }
    return n;
}

// Pick the rows per item (the tile height of a warp's work item).  A warp
// works through its item's rows one after another, so the item height bounds
// the latency of a launch when there is little work, while short items re-read
// more halo rows when there is much.  The starting point gives about four
// items per resident warp over the whole active set (1..16 rows); the
// candidates h/2, h, 2h are then timed on a few steps of the current batch
// (the steps count) and the fastest kept.  Chosen again whenever the active
// work has changed by more than a factor of two.
lbm_status autotune(lbm_batch *b)
{
    const double rows = active_strip_rows(b);
    const int resident = b->num_sms * batch_blocks_per_sm(b->storage, b->gi_mode, false) * WARPS;
    int h = (int)ceil(rows / (4.0 * resident));
    h = h < 1 ? 1 : (h > 16 ? 16 : h);
    int cand[3] = {h > 1 ? (h + 1) / 2 : 1, h, h < 16 ? 2 * h : 24};
    float best_ms = 1e30f;
    int best = h, best_mode = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LBM_ERR_CUDA;
    const int reps = 4;  // even: the parity is unchanged
    const int grid[2] = {batch_grid(b, false), batch_grid(b, true)};
    {
        double cells;
        build_active(b, cells);  // the force variants present
    }
    const bool can_persist = persistent_possible(b);
    const int pgrid = can_persist ? persistent_grid(b) : 0;
    int last = -1;
    for (int c : cand) {
        if (c == last) continue;
        last = c;
        apply_Ly(b, c);
        for (int mode = 0; mode < 2; ++mode) {
            if (mode == 1 && !can_persist) continue;
            if (b->persistent_option >= 0 && mode != b->persistent_option) continue;
            b->mode = mode;
            double cells;
            build_active(b, cells);
            cudaEventRecord(e0, b->stream);
            cudaError_t le = launch_steps(b, b->parity, 0, reps, grid, pgrid);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return LBM_ERR_CUDA;
            }
            if (le != cudaSuccess) {  // a cooperative launch the device refuses: not a candidate
                cudaGetLastError();
                continue;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            std::lock_guard<std::mutex> lk(b->mu);
            b->launches += reps;
            b->cell_updates += cells * reps;
            for (int k = 0; k < b->max_slots; ++k)
                if (b->slots[k].used && b->slots[k].running) b->records[b->slots[k].id].steps += reps;
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
                best_mode = mode;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_Ly(b, best);
    b->mode = best_mode;
    b->tuned = true;
    b->tuned_strip_rows = rows;
    return LBM_OK;
}

// The steps of one tick in segments that end at the velocity sample points
// (a launch per step, or one persistent launch per segment), each sample an
// accumulate launch over the active domains; recorded into the tick's graph
// (per-step launches) or launched directly (persistent launches: a
// cooperative launch is never recorded into a graph).
cudaError_t issue_tick(lbm_batch *b, const int grid[2], int pgrid)
{
    const int M = samples_per_tick(b), K = b->check_every;
    const int every = M > 0 ? K / M : K;  // steps between velocity samples
    const int gacc = b->num_sms * 8;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < K && le == cudaSuccess;) {
        const int n = (M > 0 && k / every < M) ? every : K - k;
        le = launch_steps(b, b->parity, k, n, grid, pgrid);
        k += n;
        if (le == cudaSuccess && M > 0 && k % every == 0 && k / every <= M)
            le = launch_batch_accumulate(b->storage, batch_args(b, (b->parity + k) & 1, k, false), gacc, b->stream);
    }
    return le;
}

lbm_status capture_graph(lbm_batch *b)
{
    // occupancy queries (and shared-memory attributes) before the capture starts
    const int grid[2] = {batch_grid(b, false), batch_grid(b, true)};
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ERR_CUDA;
    const cudaError_t le = issue_tick(b, grid, 0);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

// The graph of per-step launches for the current K, force variants and
// samples (the persistent mode needs none).
lbm_status ensure_graph(lbm_batch *b)
{
    const int M = samples_per_tick(b);
    if (b->mode == 1 && !persistent_possible(b)) b->mode = 0;  // the active set no longer allows it
    if (b->mode == 1) return LBM_OK;
    if (b->graph && b->graph_K == b->check_every && b->graph_variants == b->variants && b->graph_M == M)
        return LBM_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    const lbm_status st = capture_graph(b);
    if (st != LBM_OK) return st;
    b->graph_K = b->check_every;
    b->graph_variants = b->variants;
    b->graph_M = M;
    return LBM_OK;
}

// One engine tick; *busy tells whether anything was running or admitted.
lbm_status tick(lbm_batch *b, bool *busy)
{
    std::lock_guard<std::mutex> run_lock(b->run_mu);
    admit_pending(b);
    double cells = 0;
    int n = build_active(b, cells);
    *busy = n > 0;
    if (n == 0) return LBM_OK;
    if (b->Ly_option <= 0) {
        const double rows = active_strip_rows(b);
        if (!b->tuned || rows > 2.0 * b->tuned_strip_rows || rows < 0.5 * b->tuned_strip_rows) b->tuned = false;
    }
    if (!b->tuned && b->Ly_option <= 0) {
        lbm_status st = autotune(b);
        if (st != LBM_OK) return bfail(st, "batch autotune failed");
        n = build_active(b, cells);
    }
    if (ensure_graph(b) != LBM_OK) return bfail(LBM_ERR_CUDA, "batch graph capture failed");
    cudaError_t e;
    if (b->mode == 1) {
        const int grid[2] = {batch_grid(b, false), batch_grid(b, true)};
        e = issue_tick(b, grid, persistent_grid(b));
        if (e != cudaSuccess) return bfail(LBM_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
    } else {
        e = cudaGraphLaunch(b->graph, b->stream);
        if (e != cudaSuccess) return bfail(LBM_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    }
    // convergence residual (FP64) of every running domain whose check is due:
    // its own interval has passed, or its step budget ends with this tick
    for (int i = 0; i < n; ++i) {
        const int k = b->h_active[i];
        Slot &s = b->slots[k];
        long steps_after;
        {
            std::lock_guard<std::mutex> lk(b->mu);
            steps_after = b->records[s.id].steps + b->check_every;
        }
        s.ticks_since_check += 1;
        if (s.acc) s.samples += samples_per_tick(b);
        s.check_due = s.ticks_since_check >= s.check_mult || steps_after >= s.max_steps;
        if (!s.check_due) continue;
        s.ticks_since_check = 0;
        const size_t N = (size_t)s.nx * s.ny;
        // a reduced-precision domain compares window averages (and keeps the
        // last one in its snapshot as its result)
        const bool avg = s.acc && s.samples > 0;
        e = launch_residual(s.p, b->storage, s.f[b->parity], s.snap, s.snap + N, b->d_partials, s.res_blocks,
                            b->d_sums + 5 * k, b->stream, avg ? s.acc : nullptr, avg ? 1.0 / s.samples : 0.0);
        if (avg) s.samples = 0;
        if (e != cudaSuccess) return bfail(LBM_ERR_CUDA, "batch residual launch failed");
    }
    cudaMemcpyAsync(b->h_sums, b->d_sums, (size_t)b->max_slots * 5 * sizeof(double), cudaMemcpyDeviceToHost,
                    b->stream);
    int err = 0;
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(LBM_ERR_CUDA, std::string("batch tick: ") + cudaGetErrorString(e));
    cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) {
        // on the batch stream: later launches there see the cleared counters
        cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
        cudaMemsetAsync(b->d_work, 0, 2 * sizeof(unsigned int), b->stream);
        cudaMemsetAsync(b->d_ctl, 0, 4 * sizeof(unsigned int), b->stream);
        cudaStreamSynchronize(b->stream);
        if (err == 2) return bfail(LBM_ERR_CUDA, "debug bounds check: a batched kernel index was out of range");
        return bfail(LBM_ERR_CUDA, "a batched step kernel's bounded wait expired");
    }
    const double t = seconds(b);
    std::lock_guard<std::mutex> lk(b->mu);  // counters and records are read by other threads
    b->launches += b->check_every;
    b->cell_updates += cells * b->check_every;
    b->ticks += 1;
    for (int i = 0; i < n; ++i) {
        const int k = b->h_active[i];
        Slot &s = b->slots[k];
        Record &rec = b->records[s.id];
        rec.steps += b->check_every;
        if (!s.check_due) continue;
        const double du2 = b->h_sums[5 * k], u2 = b->h_sums[5 * k + 1];
        double r;
        if (!isfinite(du2) || !isfinite(u2)) r = NAN;
        else if (u2 == 0.0) r = du2 == 0.0 ? 0.0 : INFINITY;
        else r = sqrt(du2 / u2);
        rec.residual = r;
        int state = LBM_REQ_RUNNING;
        if (!isfinite(r) && !(r == INFINITY)) state = LBM_REQ_DIVERGED;
        else if (r < s.tol) state = LBM_REQ_CONVERGED;
        else if (rec.steps >= s.max_steps) state = LBM_REQ_NOT_CONVERGED;
        if (state != LBM_REQ_RUNNING) {
            s.running = false;
            rec.state = state;
            rec.t_done = t;
        }
    }
    return LBM_OK;
}

void engine_loop(lbm_batch *b)
{
    while (!b->stop.load()) {
        bool busy = false;
        const lbm_status st = tick(b, &busy);
        if (st != LBM_OK) {
            std::lock_guard<std::mutex> lk(b->mu);
            b->engine_error = lbm_last_error();
            for (auto &kv : b->records)
                if (kv.second.state == LBM_REQ_RUNNING || kv.second.state == LBM_REQ_QUEUED) {
                    kv.second.state = LBM_REQ_FAILED;
                    kv.second.t_done = seconds(b);
                }
            return;
        }
        if (!busy) {
            std::unique_lock<std::mutex> lk(b->mu);
            b->cv.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(size_t hbm_budget_bytes, int storage, int gi_mode, lbm_batch **out)
{
    if (!out) return bfail(LBM_ERR_INVALID, "out is null");
    *out = nullptr;
    if (storage < 0 || storage > 3) return bfail(LBM_ERR_INVALID, "storage must be 0..3");
    if (gi_mode < 0 || gi_mode > 2) return bfail(LBM_ERR_INVALID, "gi_mode must be 0..2");
    if (hbm_budget_bytes == 0) return bfail(LBM_ERR_INVALID, "budget must be > 0");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return bfail(LBM_ERR_CUDA, "no usable CUDA device");
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(LBM_ERR_OOM, "host allocation failed");
    b->storage = storage;
    b->gi_mode = gi_mode;
    b->budget = hbm_budget_bytes;
    b->t0 = std::chrono::steady_clock::now();
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    b->slots.resize(b->max_slots);
    b->h_desc.resize(b->max_slots);
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->io_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc((void **)&b->d_desc, (size_t)b->max_slots * sizeof(DomainDesc)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_active, (size_t)b->max_slots * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_prefix, (size_t)(b->max_slots + 1) * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_step0, (size_t)b->max_slots * sizeof(unsigned int)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_step0, (size_t)b->max_slots * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_state, sizeof(BatchState)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_work, 2 * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_ctl, 4 * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_err, sizeof(int)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_sums, (size_t)b->max_slots * 5 * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void **)&b->d_partials, 1024 * 5 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_sums, (size_t)b->max_slots * 5 * sizeof(double)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_active, (size_t)b->max_slots * sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_prefix, (size_t)(b->max_slots + 1) * sizeof(int)) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_state, sizeof(BatchState)) == cudaSuccess;
    if (ok) {
        ok = cudaMemset(b->d_work, 0, 2 * sizeof(unsigned int)) == cudaSuccess &&
             cudaMemset(b->d_ctl, 0, 4 * sizeof(unsigned int)) == cudaSuccess &&
             cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess &&
             cudaMemset(b->d_sums, 0, (size_t)b->max_slots * 5 * sizeof(double)) == cudaSuccess;
        b->h_state->n_active = 0;
        b->h_state->total_items = 0;
    }
    if (!ok) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return bfail(LBM_ERR_OOM, "batch allocation failed");
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_set_option(lbm_batch *b, const char *key, double v)
{
    if (!b || !key) return bfail(LBM_ERR_INVALID, "null argument");
    const std::string k(key);
    std::lock_guard<std::mutex> run_lock(b->run_mu);
    if (k == "persistent") {
        if (v != -1.0 && v != 0.0 && v != 1.0) return bfail(LBM_ERR_INVALID, "persistent must be -1, 0 or 1");
        b->persistent_option = (int)v;  // run_mu held: not during a tick
        b->mode = v == 1.0 ? 1 : 0;
        b->tuned = false;
        return LBM_OK;
    }
    if (k == "admission") {
        if (v != 0.0 && v != 1.0) return bfail(LBM_ERR_INVALID, "admission must be 0 or 1");
        std::lock_guard<std::mutex> lk(b->mu);
        b->admission = (int)v;
        return LBM_OK;
    }
    if (k == "max_running_cells") {
        if (!(v >= 0) || !isfinite(v)) return bfail(LBM_ERR_INVALID, "max_running_cells must be >= 0");
        std::lock_guard<std::mutex> lk(b->mu);
        b->max_running_cells = v;
        return LBM_OK;
    }
    if (k == "average_samples") {
        if (v < 0 || v > 1024 || v != (double)(int)v) return bfail(LBM_ERR_INVALID, "average_samples must be 0..1024");
        std::lock_guard<std::mutex> lk(b->mu);
        if (!b->records.empty()) return bfail(LBM_ERR_INVALID, "average_samples must be set before the first submit");
        b->avg_samples = (int)v;
        return LBM_OK;
    }
    if (k == "check_every") {
        const int K = (int)v;
        if (K < 2 || K % 2 || K > 100000) return bfail(LBM_ERR_INVALID, "check_every must be even, 2..100000");
        b->check_every = K;
    } else if (k == "stochastic_rounding") {
        b->sround = v != 0.0;  // domains admitted from now on
    } else if (k == "rows_per_item") {
        if (v < 0 || v > 65535) return bfail(LBM_ERR_INVALID, "rows_per_item must be 0..65535");
        b->Ly_option = (int)v;
        if (b->Ly_option > 0) {
            apply_Ly(b, b->Ly_option);
            b->tuned = true;
        } else {
            b->tuned = false;
        }
    } else {
        return bfail(LBM_ERR_INVALID, "unknown batch option: " + k);
    }
    return LBM_OK;
}

lbm_status lbm_batch_submit(lbm_batch *b, const lbm_request *req, long *id)
{
    if (!b || !req) return bfail(LBM_ERR_INVALID, "null argument");
    if (req->nx < 3 || req->ny < 3 || req->ny > 65535) return bfail(LBM_ERR_INVALID, "bad domain size");
    if (!(req->nu > 0) || !(req->gamma > 0 && req->gamma <= 1)) return bfail(LBM_ERR_INVALID, "bad nu or gamma");
    const double w = 1.0 / (3.0 * req->nu / req->gamma + 0.5);
    if (!(w > 0 && w < 2)) return bfail(LBM_ERR_INVALID, "omega4 out of (0, 2)");
    if (!(req->tol > 0) || req->max_steps <= 0) return bfail(LBM_ERR_INVALID, "tol and max_steps must be > 0");
    if (req->check_every < 0) return bfail(LBM_ERR_INVALID, "check_every must be >= 0");
    if (req->use_bnd) {
        const lbm_side *sd[4] = {&req->bnd.west, &req->bnd.east, &req->bnd.south, &req->bnd.north};
        for (int k = 0; k < 4; ++k)
            if (sd[k]->kind < 0 || sd[k]->kind > 2)
                return bfail(LBM_ERR_INVALID, "bad side kind (a batch takes periodic, wall and moving-wall sides)");
        if ((sd[0]->kind == LBM_SIDE_PERIODIC) != (sd[1]->kind == LBM_SIDE_PERIODIC) ||
            (sd[2]->kind == LBM_SIDE_PERIODIC) != (sd[3]->kind == LBM_SIDE_PERIODIC))
            return bfail(LBM_ERR_INVALID, "opposite sides must both be periodic or both walls");
    }
    Pending q;
    q.req = *req;
    if (req->use_bnd && req->bnd.solid)
        q.solid.assign(req->bnd.solid, req->bnd.solid + (size_t)req->nx * req->ny);
    q.req.bnd.solid = nullptr;
    if (footprint(b, req->nx, req->ny, !q.solid.empty()) > b->budget)
        return bfail(LBM_ERR_INVALID, "request larger than the batch budget");
    {
        std::lock_guard<std::mutex> lk(b->mu);
        // an engine thread that stopped on an error admits nothing any more
        if (!b->engine_error.empty()) return bfail(LBM_ERR_CUDA, "batch engine stopped: " + b->engine_error);
        q.id = b->next_id++;
        Record &rec = b->records[q.id];
        rec.t_submit = seconds(b);
        if (id) *id = q.id;
        b->queue.push_back(std::move(q));
    }
    b->cv.notify_all();
    return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch *b, long id, int *done, lbm_result *res)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->records.find(id);
    if (it == b->records.end()) return bfail(LBM_ERR_INVALID, "unknown request id");
    const Record &r = it->second;
    if (done) *done = r.state >= LBM_REQ_CONVERGED;
    if (res) {
        res->state = r.state;
        res->steps = r.steps;
        res->residual = r.residual;
        res->t_submit = r.t_submit;
        res->t_admit = r.t_admit;
        res->t_done = r.t_done;
    }
    return LBM_OK;
}

lbm_status lbm_batch_fields(lbm_batch *b, long id, double *rho, double *ux, double *uy)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    Slot s;
    int parity;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        auto it = b->records.find(id);
        if (it == b->records.end()) return bfail(LBM_ERR_INVALID, "unknown request id");
        if (it->second.state < LBM_REQ_CONVERGED || it->second.slot < 0)
            return bfail(LBM_ERR_INVALID, "request not finished (or released)");
        s = b->slots[it->second.slot];
        parity = b->parity;
        // pin the slot: a concurrent lbm_batch_release waits until the read ends
        ++it->second.readers;
    }
    const size_t N = (size_t)s.nx * s.ny;
    double *d = nullptr;
    cudaError_t e = cudaMalloc((void **)&d, 3 * N * sizeof(double));
    lbm_status st = LBM_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        st = bfail(LBM_ERR_OOM, "device allocation failed (fields)");
    } else {
        e = launch_fields(s.p, b->storage, s.f[parity], d, d + N, d + 2 * N, b->io_stream);
        // a window-averaged domain returns the velocity average of its last check
        // (held in the snapshot; solid cells keep the fields kernel's NaN)
        const double *vu = s.acc ? s.snap : d + N, *vv = s.acc ? s.snap + N : d + 2 * N;
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, d, N * 8, cudaMemcpyDeviceToHost, b->io_stream);
        if (e == cudaSuccess && ux) e = cudaMemcpyAsync(ux, vu, N * 8, cudaMemcpyDeviceToHost, b->io_stream);
        if (e == cudaSuccess && uy) e = cudaMemcpyAsync(uy, vv, N * 8, cudaMemcpyDeviceToHost, b->io_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->io_stream);
        cudaFree(d);
        if (e != cudaSuccess) st = bfail(LBM_ERR_CUDA, std::string("batch fields: ") + cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> lk(b->mu);
        auto it = b->records.find(id);
        if (it != b->records.end()) --it->second.readers;
    }
    b->cv.notify_all();
    return st;
}

lbm_status lbm_batch_cancel(lbm_batch *b, long id)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    {
        std::lock_guard<std::mutex> lk(b->mu);
        auto it = b->records.find(id);
        if (it == b->records.end()) return bfail(LBM_ERR_INVALID, "unknown request id");
        Record &rec = it->second;
        if (rec.state >= LBM_REQ_CONVERGED) return bfail(LBM_ERR_INVALID, "request already finished");
        bool dequeued = false;
        if (rec.state == LBM_REQ_QUEUED)
            for (auto q = b->queue.begin(); q != b->queue.end(); ++q)
                if (q->id == id) {
                    b->queue.erase(q);
                    dequeued = true;
                    break;
                }
        if (dequeued) {
            rec.state = LBM_REQ_CANCELLED;
            rec.t_done = seconds(b);
        } else {
            rec.cancel = true;  // running, or being admitted: the engine retires it between ticks
        }
    }
    b->cv.notify_all();
    return LBM_OK;
}

lbm_status lbm_batch_release(lbm_batch *b, long id)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    Slot s;
    {
        std::unique_lock<std::mutex> lk(b->mu);
        auto it = b->records.find(id);
        if (it == b->records.end()) return bfail(LBM_ERR_INVALID, "unknown request id");
        if (it->second.state < LBM_REQ_CONVERGED) return bfail(LBM_ERR_INVALID, "request not finished");
        // buffers being read by lbm_batch_fields stay until those reads end
        b->cv.wait(lk, [&] {
            auto jt = b->records.find(id);
            return jt == b->records.end() || jt->second.readers == 0;
        });
        it = b->records.find(id);
        if (it == b->records.end()) return bfail(LBM_ERR_INVALID, "unknown request id");
        const int si = it->second.slot;
        if (si >= 0) {
            s = b->slots[si];
            b->slots[si] = Slot();
            b->used -= s.bytes;
        }
        b->records.erase(it);
    }
    free_slot(s);
    b->cv.notify_all();
    return LBM_OK;
}

lbm_status lbm_batch_run(lbm_batch *b, double wall_seconds)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    if (b->engine_on) return bfail(LBM_ERR_INVALID, "the background engine is running");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        bool busy = false;
        const lbm_status st = tick(b, &busy);
        if (st != LBM_OK) return st;
        if (!busy) {
            std::lock_guard<std::mutex> lk(b->mu);
            if (b->queue.empty()) return LBM_OK;
            // the queue head does not fit and nothing runs: it never will
            return bfail(LBM_ERR_OOM, "queued request cannot be admitted (release finished requests)");
        }
        if (wall_seconds > 0 &&
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > wall_seconds)
            return bfail(LBM_ERR_TIMEOUT, "wall-clock limit reached");
    }
}

lbm_status lbm_batch_start(lbm_batch *b)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    if (b->engine_on) return LBM_OK;
    b->stop = false;
    b->engine = std::thread(engine_loop, b);
    b->engine_on = true;
    return LBM_OK;
}

lbm_status lbm_batch_stop(lbm_batch *b)
{
    if (!b) return bfail(LBM_ERR_INVALID, "null batch");
    if (!b->engine_on) return LBM_OK;
    b->stop = true;
    b->cv.notify_all();
    b->engine.join();
    b->engine_on = false;
    if (!b->engine_error.empty()) return bfail(LBM_ERR_CUDA, b->engine_error);
    return LBM_OK;
}

lbm_status lbm_batch_stats(lbm_batch *b, double stats[6])
{
    if (!b || !stats) return bfail(LBM_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lk(b->mu);
    int running = 0;
    for (const auto &kv : b->records) running += kv.second.state == LBM_REQ_RUNNING;
    stats[0] = b->cell_updates;
    stats[1] = (double)b->launches;
    stats[2] = (double)b->ticks;
    stats[3] = running;
    stats[4] = (double)b->queue.size();
    stats[5] = (double)b->used;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    lbm_batch_stop(b);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &s : b->slots)
        if (s.used) free_slot(s);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_desc);
    cudaFree(b->d_active);
    cudaFree(b->d_prefix);
    cudaFree(b->d_step0);
    if (b->h_step0) cudaFreeHost(b->h_step0);
    cudaFree(b->d_state);
    cudaFree(b->d_work);
    cudaFree(b->d_ctl);
    cudaFree(b->d_err);
    cudaFree(b->d_sums);
    cudaFree(b->d_partials);
    if (b->h_sums) cudaFreeHost(b->h_sums);
    if (b->h_active) cudaFreeHost(b->h_active);
    if (b->h_prefix) cudaFreeHost(b->h_prefix);
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->io_stream) cudaStreamDestroy(b->io_stream);
    delete b;
}

}  // extern "C"

// Internal types shared by the translation units of the CUDA library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"

// Debug build (compiled with LBM_DEBUG_BOUNDS=1: build(debug=True)): the step
// kernels check every computed index of their global-memory accesses (and the
// general pull's ring columns) against the buffer it addresses; a violation
// sets the device error flag to 2 and skips the access, and the host reports
// it at the next synchronising call.
#ifndef LBM_DEBUG_BOUNDS
#define LBM_DEBUG_BOUNDS 0
#endif
#define LBM_IN_BOUNDS(idx, extent, err) \
    (!LBM_DEBUG_BOUNDS || ::lbm::debug_in_bounds((long long)(idx), (long long)(extent), (err)))

namespace lbm {

#ifdef __CUDACC__
__device__ __forceinline__ bool debug_in_bounds(long long i, long long n, int *err)
{
    if (i >= 0 && i < n) return true;
    if (err) atomicExch(err, 2);
    return false;
}
#endif

// Columns of one warp strip of the stream-collide kernel (one per lane), warps
// per block.
constexpr int WS = 32;  // one cell per lane (FP64 storage)
constexpr int WARPS = 4;
constexpr int THREADS = 32 * WARPS;  // threads per block of the step kernel

// Columns of a warp strip for a storage type: the FP32/FP16/BF16 kernels give a
// lane two neighbouring cells (packed FP32 arithmetic), the FP64 kernel one.
inline int strip_width(int storage) { return storage == LBM_STORAGE_F64 ? WS : 2 * WS; }

// FP16 storage holds 2^14 g rather than g (an exact power-of-two scale): the
// deviations of slow regions (|g| down to about 1e-8) then stay in the normal
// FP16 range, where rounding has the full 11-bit precision and stochastic
// rounding is exact; |2^14 g| stays far below the FP16 maximum 65504 for any
// stable flow (|g| < 4).
constexpr float F16_SCALE = 16384.0f;
constexpr float F16_INV_SCALE = 1.0f / 16384.0f;

// Collision constants in the compute precision, filled on the host once per
// launch (no FP64 arithmetic in the FP32 kernels).
template <typename R>
struct Consts {
    R ig, half_ig;                 // 1/gamma, 1/(2 gamma)
    R ig2;                         // 1/gamma^2
    R w3_12, w4_4, w5_4, w6_4, w7_4, w8_4;
    R c6;                          // third-order factor: 2 (Eq. 4) or 3/g - 1/g^2 (Sec. 5)
    R A, B, C3;                    // A_gamma, B_gamma, C_gamma/3 (after Eq. 53)
    R k3, k4, k5;                  // 1/omega_j - 1/2
    R a3, a4;                      // 2/(3 omega3), 2/(3 omega4)
    R Fx, Fy;                      // uniform force
    R wall6[4][2];                 // 6 u_wall of each side (west, east, south, north)
    R c4;                          // 3 - 6/gamma + 4/gamma^2 (raw fourth-order equilibrium, u^4 term)
    R inlet_k, H;                  // parabolic inlet: 4 / ny^2 and ny
    R out_u;                       // convective outlet: convection speed

    void set(double g, const double w[9], int gi_mode, double fx, double fy, const double side_u[4][2])
    {
        ig = R(1.0 / g);
        half_ig = R(0.5 / g);
        ig2 = R(1.0 / (g * g));
        w3_12 = R(w[3] / 12.0);
        w4_4 = R(w[4] / 4.0);
        w5_4 = R(w[5] / 4.0);
        w6_4 = R(w[6] / 4.0);
        w7_4 = R(w[7] / 4.0);
        w8_4 = R(w[8] / 4.0);
        c6 = gi_mode == LBM_GI_UNCORRECTED ? R(2.0) : R(3.0 / g - 1.0 / (g * g));
        A = R(4.0 / (g * g) - 1.0 / g);
        B = R(1.0 / (g * g) - 1.0 / g);
        C3 = R((1.0 / g - 1.0) / 3.0);
        k3 = R(1.0 / w[3] - 0.5);
        k4 = R(1.0 / w[4] - 0.5);
        k5 = R(1.0 / w[5] - 0.5);
        a3 = R(2.0 / (3.0 * w[3]));
        a4 = R(2.0 / (3.0 * w[4]));
        Fx = R(fx);
        Fy = R(fy);
        for (int s = 0; s < 4; ++s)
            for (int d = 0; d < 2; ++d) wall6[s][d] = R(6.0 * side_u[s][d]);
        c4 = R(3.0 - 6.0 / g + 4.0 / (g * g));
        inlet_k = R(0);
        H = R(0);
        out_u = R(0);
    }

    // open sides (Sec. 6, square cylinder): channel height ny, outlet speed
    void set_open(int ny, double outlet_u)
    {
        inlet_k = R(4.0 / ((double)ny * (double)ny));
        H = R((double)ny);
        out_u = R(outlet_u);
    }
};

// The collision constants of the packed-FP32 kernel (two cells per lane), each
// duplicated into a pair, so that a packed instruction reads the pair as one
// operand instead of the kernel building it from a scalar.
struct Consts2 {
    float2 one, half, two, three, four, m_two, third, two_thirds, ninth;
    float2 ig, half_ig, ig2;
    float2 w3_12, w4_4, w5_4, w6_4, w7_4, w8_4, c6;
    float2 hA, hB, B, C3, a3, a4, k3x2, k4x2, mk5;  // -A/2, -B/2, B, C/3, a3, a4, 2 k3, 2 k4, -k5
    float2 Fx, Fy;

    void set(const Consts<float> &c)
    {
        auto p = [](float v) { return make_float2(v, v); };
        one = p(1.f);
        half = p(0.5f);
        two = p(2.f);
        three = p(3.f);
        four = p(4.f);
        m_two = p(-2.f);
        third = p(1.f / 3.f);
        two_thirds = p(2.f / 3.f);
        ninth = p(1.f / 9.f);
        ig = p(c.ig);
        half_ig = p(c.half_ig);
        ig2 = p(c.ig2);
        w3_12 = p(c.w3_12);
        w4_4 = p(c.w4_4);
        w5_4 = p(c.w5_4);
        w6_4 = p(c.w6_4);
        w7_4 = p(c.w7_4);
        w8_4 = p(c.w8_4);
        c6 = p(c.c6);
        hA = p(-0.5f * c.A);
        hB = p(-0.5f * c.B);
        B = p(c.B);
        C3 = p(c.C3);
        a3 = p(c.a3);
        a4 = p(c.a4);
        k3x2 = p(2.f * c.k3);
        k4x2 = p(2.f * c.k4);
        mk5 = p(-c.k5);
        Fx = p(c.Fx);
        Fy = p(c.Fy);
    }
};

// Everything one launch of the step kernel needs, passed by value.
struct StepParams {
    int nx, ny;
    int pitch;              // row stride in elements (multiple of 32)
    long long plane;        // elements per population plane (pitch * ny)
    int perx, pery;         // periodic in x / y
    int gi_mode;            // LBM_GI_*
    int guard;              // strain-solve guard on/off
    int fd_iso;             // density gradient: isotropic stencil (nonzero) or central differences
    // relaxation and preconditioning constants
    double gamma;
    double w3, w4, w5, w6, w7, w8;
    // wall velocity of each side (west, east, south, north); zero for
    // stationary walls and periodic sides; the peak speed of a west inlet
    double side_u[4][2];
    // open sides of a channel (Sec. 6, square cylinder): west parabolic
    // velocity inlet, east convective outlet.  The outlet keeps a ghost column
    // at x = nx, [5][ny] in the kernel's compute type: the ghost velocity
    // (u_g, v_g) and the populations 3, 6, 7 that enter the domain; a launch
    // reads ghost_in (the source state's) and writes ghost_out.
    int inlet, outlet;
    const void *ghost_in;
    void *ghost_out;
    double Fx, Fy;           // uniform force
    const float *force;      // optional per-cell force: [2][ny][pitch] (fx, fy)
    // optional mask [ny][pitch], 1 = solid, followed in the same allocation by
    // its row table [ny][ceil(nx / 32)]: nonzero when a solid cell lies within
    // rows y - 1 .. y + 1 and the columns of 32-column blocks b - 1 .. b + 1
    // (plus two columns each way); a work item whose rows meet none takes the
    // paths of a domain without a mask (item_meets_solid)
    const uint8_t *solid;
    unsigned long long *guard_count;  // device counter, may be null
    int *error;              // device flag: set when a bounded wait expires
    unsigned int *work;      // device work counters {next item, warps done}, zero between launches
    // work decomposition: items = warp strips x segments, each segment Ly rows
    int Ly, nstrips, nitems;
    // item order of the single-domain kernel: segments are handed out in nwave
    // phases (phase q: segments q, q + nwave, ...; nseg_phase of them per strip)
    // so that a segment starts when the one above it ends and re-reads their
    // shared boundary rows while they are still in L2; nwave = 1: segment-major
    int nseg, nwave, nseg_phase;
    // 16-bit storage: round the stored deviations stochastically (nonzero) or
    // to nearest; the random bits are a hash of (step, cell, direction)
    int sround;
    unsigned int step;       // step index of this launch (low 32 bits), single-domain kernel
    Consts<float> cf;
    Consts<double> cd;
    Consts2 c2;
};

// One domain of a batch, in device memory (TMA descriptors need 64-byte alignment).
struct alignas(128) DomainDesc {
    CUtensorMap tload[2];   // load descriptors of f[0], f[1]
    CUtensorMap tstore[2];  // store descriptors of f[0], f[1]
    StepParams p;           // the domain's parameters (work/error pointers unused)
    const void *f[2];       // population buffers
    int forced;             // nonzero: a body force acts (uniform Fx, Fy)
    double *acc;            // velocity sums for the check-window average ([2][nx*ny]), or null
};

// Active set of a batch, read by the kernel each launch (so a captured graph
// stays valid while domains join and retire).
struct BatchState {
    int n_active;     // active domains
    int total_items;  // prefix[n_active]
    int split_items;  // items of the unforced domains, which come first in the active list
};

struct BatchArgs {
    const DomainDesc *domains;  // all slots
    const int *active;          // active slot ids, n_active of them
    const int *prefix;          // item prefix sums over the active slots (n_active + 1)
    const BatchState *state;
    unsigned int *work;         // work counters {next item, warps done}
    int *error;
    int parity;                 // source buffer of this step (all domains step together)
    const unsigned int *step0;  // per active index: the domain's step count at the start of the tick
    int forced;                 // this launch covers the forced domains (items split .. total) or the others
    int k;                      // launch index within the tick (domain step = step0 + k)
    unsigned int *ctl;          // persistent kernel: {items of even steps, of odd steps, arrivals, generation}
};

// The launchers below are defined per storage type (one translation unit each).
// tin: TMA descriptor of fin for loads (box: one row of all planes of a warp
// strip plus halo); tout: descriptor of fout for stores (box: one strip row).
cudaError_t launch_step_f32(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_f16(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_bf16(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_step_f64(const StepParams &p, const CUtensorMap &tin, const CUtensorMap &tout, const void *fin, void *fout, int grid, cudaStream_t s);
cudaError_t launch_batch_step(int storage, int gi_mode, bool forced, const BatchArgs &a, int grid, cudaStream_t s);
int batch_blocks_per_sm(int storage, int gi_mode, bool forced);
// The persistent batch kernel (FP32/FP16/BF16 storage, full GI kernel, one force
// variant): steps k0 .. k0 + nsteps - 1 of the tick (parity a.parity + k) in one
// cooperative launch of `grid` blocks (at most the resident count) with a
// bounded grid barrier between steps.
bool batch_persistent_supported(int storage, int gi_mode);
cudaError_t launch_batch_persistent(int storage, bool forced, const BatchArgs &a, int k0, int nsteps, int grid,
                                    cudaStream_t s);
int batch_persistent_blocks_per_sm(int storage, bool forced);
int blocks_per_sm_f32(int gi_mode, bool forced);
int blocks_per_sm_f16(int gi_mode, bool forced);
int blocks_per_sm_bf16(int gi_mode, bool forced);
int blocks_per_sm_f64(int gi_mode, bool forced);
// Encode the TMA descriptors of a population buffer: load box {W + 2 PAD, 1, 9}
// with W the strip width of the storage type, and store box {WS, 1, 9}.
cudaError_t make_tensor_maps(CUtensorMap *load, CUtensorMap *store, int storage, void *base, int nx, int ny,
                             int pitch, long long plane);

// Auxiliary kernels (aux_kernels.cu)
cudaError_t launch_init_eq(const StepParams &p, int storage, const double *rho, const double *ux,
                           const double *uy, void *f, cudaStream_t s);
cudaError_t launch_fields(const StepParams &p, int storage, const void *f, double *rho, double *ux,
                          double *uy, cudaStream_t s);
// acc (optional, [2][nx*ny]): the velocity entering the residual is acc *
// inv_count (a window average) instead of the current one; acc is zeroed.
cudaError_t launch_residual(const StepParams &p, int storage, const void *f, double *snap_ux,
                            double *snap_uy, double *partials, int nblocks, double *result,
                            cudaStream_t s, double *acc = nullptr, double inv_count = 0.0);
// Add the current velocity of every active domain of a batch to its window sums
// (DomainDesc::acc), reading the population buffer `a.parity`.
cudaError_t launch_batch_accumulate(int storage, const BatchArgs &a, int grid, cudaStream_t s);
int residual_blocks(const StepParams &p);
cudaError_t launch_bounded_wait_selftest(int *error, unsigned long long *waited_ns, cudaStream_t s);
// Outlet ghost column from the last column of f (velocity and incoming populations).
cudaError_t launch_outlet_seed(const StepParams &p, int storage, const void *f, void *ghost, cudaStream_t s);
// Momentum-exchange force on the solid cells: two FP64 sums into result[0..1]
// (partials: nblocks rows of 2 doubles).
cudaError_t launch_drag(const StepParams &p, int storage, const void *f, double *partials, int nblocks,
                        double *result, cudaStream_t s);
cudaError_t launch_convert(const StepParams &p, int from_storage, const void *fin, int to_storage,
                           void *fout, cudaStream_t s);
cudaError_t launch_pops_to_f64(const StepParams &p, int storage, const void *f, double *out,
                               cudaStream_t s);
cudaError_t launch_pops_from_f64(const StepParams &p, int storage, const double *in, void *f,
                                 cudaStream_t s);

size_t storage_bytes(int storage);

// Host: the row table of a mask (see StepParams::solid) from a host mask
// [ny][nx] (sides periodic in x / y wrap).
std::vector<uint8_t> make_solid_rows(const uint8_t *mask, int nx, int ny, bool perx, bool pery);
// Host: the device layout of StepParams::solid from a host mask [ny][nx]: the
// mask as 0/1 bytes [ny][pitch], then its row table.
std::vector<uint8_t> mask_with_row_table(const uint8_t *mask, int nx, int ny, int pitch, bool perx, bool pery);

// Record a message for lbm_last_error() on this thread and return the status.
lbm_status set_error(lbm_status s, const std::string &msg);

}  // namespace lbm

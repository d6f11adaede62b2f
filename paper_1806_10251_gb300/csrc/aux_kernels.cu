// Auxiliary kernels: equilibrium initialisation, observed fields, the FP64
// convergence residual, the outlet ghost column, the momentum-exchange force,
// and population format conversions.
#include <math.h>

#include <type_traits>

#include "d2q9_collide.cuh"
#include "open_bc.cuh"

namespace lbm {

size_t storage_bytes(int storage)
{
    switch (storage) {
    case LBM_STORAGE_F16:
    case LBM_STORAGE_BF16: return 2;
    case LBM_STORAGE_F64: return 8;
    default: return 4;
    }
}

// Element access in FP64 by storage type (compile time for the per-step
// kernels, run time for the one-off format conversions).
template <typename ST> __device__ __forceinline__ double ld64(const ST *f, size_t i);
template <> __device__ __forceinline__ double ld64<float>(const float *f, size_t i) { return (double)f[i]; }
template <> __device__ __forceinline__ double ld64<double>(const double *f, size_t i) { return f[i]; }
template <> __device__ __forceinline__ double ld64<__half>(const __half *f, size_t i)
{
    return (double)__half2float(f[i]) * (double)F16_INV_SCALE;
}
template <> __device__ __forceinline__ double ld64<__nv_bfloat16>(const __nv_bfloat16 *f, size_t i)
{
    return (double)__bfloat162float(f[i]);
}
template <typename ST> __device__ __forceinline__ void st64(ST *f, size_t i, double v);
template <> __device__ __forceinline__ void st64<float>(float *f, size_t i, double v) { f[i] = (float)v; }
template <> __device__ __forceinline__ void st64<double>(double *f, size_t i, double v) { f[i] = v; }
template <> __device__ __forceinline__ void st64<__half>(__half *f, size_t i, double v)
{
    f[i] = __double2half(v * (double)F16_SCALE);
}
template <> __device__ __forceinline__ void st64<__nv_bfloat16>(__nv_bfloat16 *f, size_t i, double v)
{
    f[i] = __double2bfloat16(v);
}

__device__ __forceinline__ double load_any(const void *f, int storage, size_t i)
{
    switch (storage) {
    case LBM_STORAGE_F16: return ld64(static_cast<const __half *>(f), i);
    case LBM_STORAGE_BF16: return ld64(static_cast<const __nv_bfloat16 *>(f), i);
    case LBM_STORAGE_F64: return ld64(static_cast<const double *>(f), i);
    default: return ld64(static_cast<const float *>(f), i);
    }
}

__device__ __forceinline__ void store_any(void *f, int storage, size_t i, double v)
{
    switch (storage) {
    case LBM_STORAGE_F16: st64(static_cast<__half *>(f), i, v); break;
    case LBM_STORAGE_BF16: st64(static_cast<__nv_bfloat16 *>(f), i, v); break;
    case LBM_STORAGE_F64: st64(static_cast<double *>(f), i, v); break;
    default: st64(static_cast<float *>(f), i, v); break;
    }
}

// Call fn(ST *) with the population pointer cast to the storage type.
template <typename F>
void with_storage(int storage, const void *f, F &&fn)
{
    switch (storage) {
    case LBM_STORAGE_F16: fn(static_cast<const __half *>(f)); break;
    case LBM_STORAGE_BF16: fn(static_cast<const __nv_bfloat16 *>(f)); break;
    case LBM_STORAGE_F64: fn(static_cast<const double *>(f)); break;
    default: fn(static_cast<const float *>(f)); break;
    }
}

__device__ __forceinline__ bool solid_at(const StepParams &p, int x, int y)
{
    return p.solid != nullptr && p.solid[(size_t)y * p.pitch + x] != 0;
}

__device__ __forceinline__ void force_at(const StepParams &p, int x, int y, double &Fx, double &Fy)
{
    if (p.force) {
        const size_t i = (size_t)y * p.pitch + x;
        Fx = p.force[i];
        Fy = p.force[(size_t)p.plane + i];
    } else {
        Fx = p.Fx;
        Fy = p.Fy;
    }
}

// Compute precision of the per-cell auxiliary work: FP32 for the 32- and
// 16-bit formats (their stored values carry no more), FP64 for FP64 storage.
template <typename ST> struct AuxReal { using R = float; };
template <> struct AuxReal<double> { using R = double; };

// Inverse of the Eq. 5 map for the moment order
// (k0, kx, ky, kxx, kyy, kxy, kxxy, kxyy, kxxyy), in precision R.
template <typename R>
__device__ __forceinline__ void pops_from_raw_r(const R (&k)[9], R (&f)[9])
{
    f[0] = k[0] - k[3] - k[4] + k[8];
    f[1] = R(0.5) * (k[1] + k[3] - k[7] - k[8]);
    f[3] = R(0.5) * (-k[1] + k[3] + k[7] - k[8]);
    f[2] = R(0.5) * (k[2] + k[4] - k[6] - k[8]);
    f[4] = R(0.5) * (-k[2] + k[4] + k[6] - k[8]);
    f[5] = R(0.25) * (k[5] + k[6] + k[7] + k[8]);
    f[6] = R(0.25) * (-k[5] + k[6] - k[7] + k[8]);
    f[7] = R(0.25) * (k[5] - k[6] - k[7] + k[8]);
    f[8] = R(0.25) * (-k[5] - k[6] + k[7] + k[8]);
}

// f~0 = f_eq(rho, u) - S/2 stored as deviations g = f - w (rho0 = 1).  The
// raw equilibria of Eq. 15 (gamma^2 cubic terms; fourth moment such that the
// central fourth moment is rho/9) are written minus the rest-state moments
// (1, 0, 0, 1/3, 1/3, 0, 0, 0, 1/9), so the inverse map yields g directly and
// no O(1) weight is subtracted in finite precision.  ig = 1/gamma, ig2 = 1/gamma^2.
template <typename ST>
__global__ void init_eq_kernel(const StepParams p, const double *rho_in, const double *ux_in, const double *uy_in,
                               ST *f, double ig_d, double ig2_d)
{
    using R = typename AuxReal<ST>::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t ic = (size_t)y * p.nx + x;
    const R dr = rho_in ? R(rho_in[ic] - 1.0) : R(0);
    const R r = R(1) + dr;
    const R u = ux_in ? R(ux_in[ic]) : R(0);
    const R v = uy_in ? R(uy_in[ic]) : R(0);
    const R ig = R(ig_d), ig2 = R(ig2_d), third = R(1.0 / 3.0);
    R k[9] = {dr,
              r * u,
              r * v,
              dr * third + r * u * u * ig,
              dr * third + r * v * v * ig,
              r * u * v * ig,
              r * v * third + r * u * u * v * ig2,
              r * u * third + r * u * v * v * ig2,
              dr * R(1.0 / 9.0) + r * (u * u + v * v) * third +
                  r * u * u * v * v * (R(3) - R(6) * ig + R(4) * ig2)};
    R geq[9], S[9];
    pops_from_raw_r(k, geq);
    double Fxd, Fyd;
    force_at(p, x, y, Fxd, Fyd);
    const R Fx = R(Fxd), Fy = R(Fyd);
    R sm[9] = {R(0),
               Fx * ig,
               Fy * ig,
               R(2) * Fx * u * ig2,
               R(2) * Fy * v * ig2,
               (Fx * v + Fy * u) * ig2,
               Fy * u * u + R(2) * Fx * u * v,
               Fx * v * v + R(2) * Fy * v * u,
               R(2) * (Fx * u * v * v + Fy * v * u * u)};
    pops_from_raw_r(sm, S);
    const size_t i = (size_t)y * p.pitch + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) st64(f, (size_t)a * p.plane + i, (double)(geq[a] - R(0.5) * S[a]));
}

cudaError_t launch_init_eq(const StepParams &p, int storage, const double *rho, const double *ux,
                           const double *uy, void *f, cudaStream_t s)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    const double ig = 1.0 / p.gamma, ig2 = ig * ig;
    with_storage(storage, f, [&](auto *fp) {
        using ST = std::remove_const_t<std::remove_pointer_t<decltype(fp)>>;
        init_eq_kernel<ST><<<grid, 128, 0, s>>>(p, rho, ux, uy, const_cast<ST *>(fp), ig, ig2);
    });
    return cudaGetLastError();
}

// Observed fields: rho = 1 + sum g~, rho u = sum g~ e - F/(2 gamma); NaN in solids.
template <typename ST> __device__ __forceinline__ typename AuxReal<ST>::R ldr(const ST *f, size_t i)
{
    return (typename AuxReal<ST>::R)ld64(f, i);
}
__device__ __forceinline__ float recip_aux(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip_aux(double v) { return __drcp_rn(v); }

// Observed fields of one cell in the compute precision of the storage type,
// returned in FP64.
template <typename ST>
__device__ __forceinline__ void local_fields(const StepParams &p, const ST *f, int x, int y, double half_ig, double &rho,
                                             double &ux, double &uy)
{
    using R = typename AuxReal<ST>::R;
    const size_t i = (size_t)y * p.pitch + x;
    R g[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = ldr(f, (size_t)a * p.plane + i);
    const R s = g[0] + (g[1] + g[3]) + (g[2] + g[4]) + ((g[5] + g[6]) + (g[7] + g[8]));
    const R jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    const R jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
    double Fx, Fy;
    force_at(p, x, y, Fx, Fy);
    const R r = R(1) + s;
    const R ir = recip_aux(r);
    rho = (double)r;
    ux = (double)((jx - R(Fx * half_ig)) * ir);
    uy = (double)((jy - R(Fy * half_ig)) * ir);
}

template <typename ST>
__global__ void fields_kernel(const StepParams p, const ST *f, double half_ig, double *rho, double *ux, double *uy)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t o = (size_t)y * p.nx + x;
    double r, u, v;
    if (solid_at(p, x, y)) {
        r = u = v = nan("");
    } else {
        local_fields(p, f, x, y, half_ig, r, u, v);
    }
    if (rho) rho[o] = r;
    if (ux) ux[o] = u;
    if (uy) uy[o] = v;
}

cudaError_t launch_fields(const StepParams &p, int storage, const void *f, double *rho, double *ux,
                          double *uy, cudaStream_t s)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    const double half_ig = 0.5 / p.gamma;
    with_storage(storage, f, [&](auto *fp) {
        using ST = std::remove_const_t<std::remove_pointer_t<decltype(fp)>>;
        fields_kernel<ST><<<grid, 128, 0, s>>>(p, fp, half_ig, rho, ux, uy);
    });
    return cudaGetLastError();
}

// ---- FP64 convergence residual ------------------------------------------------
// Pass 1: each block accumulates {sum|du|^2, sum|u|^2, sum rho, sum rho ux,
// sum rho uy} over whole rows of fluid cells (rows blockIdx.x, + gridDim.x,
// ...), reduces in FP64 with warp shuffles and writes one row of `partials`;
// the velocity snapshot is replaced.  Pass 2: one block reduces the rows in a
// fixed order (deterministic).
constexpr int RES_THREADS = 256;
constexpr int RES_CELLS = 4;  // cells of a row per thread and iteration

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int NT>
__device__ __forceinline__ void block_sum5(double (&v)[5], double *out)
{
    __shared__ double sh[NT / 32][5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
        for (int k = 0; k < 5; ++k) sh[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double t = lane < NT / 32 ? sh[lane][k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) out[k] = t;
        }
    }
}

template <typename ST>
__global__ void residual_pass1(const StepParams p, const ST *__restrict__ f, double half_ig,
                               double *__restrict__ snap_ux, double *__restrict__ snap_uy, double *partials,
                               double *__restrict__ win, double inv_count)
{
    // Per cell in the storage's compute precision R; each thread's sums over
    // the cells it meets in one row (at most nx / blockDim.x of them) are kept
    // in R and added into the FP64 accumulators row by row.  The density sum
    // is formed as (fluid cells) + sum(rho - 1), the momentum directly as
    // rho u = sum g e - F/(2 gamma).  A thread takes RES_CELLS cells of a row
    // at a time and issues all their loads before any store (memory-level
    // parallelism: the kernel is bound by DRAM latency otherwise).
    using R = typename AuxReal<ST>::R;
    const R hig = (R)half_ig, Fx0 = (R)p.Fx, Fy0 = (R)p.Fy;
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int y = blockIdx.x; y < p.ny; y += gridDim.x) {
        R du2 = 0, u2 = 0, sdr = 0, sjx = 0, sjy = 0;
        int cnt = 0;
        for (int x0 = threadIdx.x; x0 < p.nx; x0 += RES_CELLS * blockDim.x) {
            R g[RES_CELLS][9], sx[RES_CELLS], sy[RES_CELLS], fx[RES_CELLS], fy[RES_CELLS];
            bool ok[RES_CELLS];
#pragma unroll
            for (int j = 0; j < RES_CELLS; ++j) {
                const int x = x0 + j * blockDim.x;
                ok[j] = x < p.nx && !solid_at(p, x, y);
                const size_t i = (size_t)y * p.pitch + (ok[j] ? x : 0);
                const size_t c = (size_t)y * p.nx + (ok[j] ? x : 0);
#pragma unroll
                for (int a = 0; a < 9; ++a) g[j][a] = ldr(f, (size_t)a * p.plane + i);
                sx[j] = (R)snap_ux[c];
                sy[j] = (R)snap_uy[c];
                fx[j] = p.force ? (R)p.force[i] : Fx0;
                fy[j] = p.force ? (R)p.force[(size_t)p.plane + i] : Fy0;
            }
#pragma unroll
            for (int j = 0; j < RES_CELLS; ++j) {
                if (!ok[j]) continue;
                const R *q = g[j];
                const R dr = q[0] + (q[1] + q[3]) + (q[2] + q[4]) + ((q[5] + q[6]) + (q[7] + q[8]));
                const R jx = (q[1] - q[3]) + (q[5] - q[6]) + (q[8] - q[7]);
                const R jy = (q[2] - q[4]) + (q[5] + q[6]) - (q[7] + q[8]);
                const R mx = jx - fx[j] * hig, my = jy - fy[j] * hig;
                const R ir = recip_aux(R(1) + dr);
                R u = mx * ir, v = my * ir;
                const size_t c = (size_t)y * p.nx + x0 + j * blockDim.x;
                if (win) {
                    // the window average in place of the current velocity
                    const size_t N = (size_t)p.nx * p.ny;
                    u = (R)(win[c] * inv_count);
                    v = (R)(win[N + c] * inv_count);
                    win[c] = 0.0;
                    win[N + c] = 0.0;
                }
                const R du = u - sx[j], dv = v - sy[j];
                du2 += du * du + dv * dv;
                u2 += u * u + v * v;
                sdr += dr;
                sjx += mx;
                sjy += my;
                ++cnt;
                snap_ux[c] = (double)u;
                snap_uy[c] = (double)v;
            }
        }
        acc[0] += (double)du2;
        acc[1] += (double)u2;
        acc[2] += (double)cnt + (double)sdr;
        acc[3] += (double)sjx;
        acc[4] += (double)sjy;
    }
    block_sum5<RES_THREADS>(acc, partials + (size_t)blockIdx.x * 5);
}

__global__ void residual_pass2(const double *partials, int nrows, double *result)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int r = threadIdx.x; r < nrows; r += blockDim.x)
        for (int k = 0; k < 5; ++k) acc[k] += partials[(size_t)r * 5 + k];
    block_sum5<RES_THREADS>(acc, result);
}

int residual_blocks(const StepParams &p)
{
    // one block per row (each block walks rows with a stride), at most 1024
    return p.ny < 1024 ? (p.ny < 1 ? 1 : p.ny) : 1024;
}

cudaError_t launch_residual(const StepParams &p, int storage, const void *f, double *snap_ux,
                            double *snap_uy, double *partials, int nblocks, double *result,
                            cudaStream_t s, double *acc, double inv_count)
{
    const double half_ig = 0.5 / p.gamma;
    with_storage(storage, f, [&](auto *fp) {
        using ST = std::remove_const_t<std::remove_pointer_t<decltype(fp)>>;
        residual_pass1<ST><<<nblocks, RES_THREADS, 0, s>>>(p, fp, half_ig, snap_ux, snap_uy, partials, acc,
                                                          inv_count);
    });
    residual_pass2<<<1, RES_THREADS, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

// ---- batch: window sums of the velocity (reduced-precision averaging) --------
// The work items of the batch step kernels (a strip of W columns x Ly rows of
// one active domain), distributed over the grid's warps; each lane takes
// columns lane, lane + 32, ... of its strip.  rho u = sum g e - F/(2 gamma).
template <typename ST>
__global__ void batch_accumulate_kernel(const BatchArgs a, int W)
{
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int n_active = a.state->n_active, total = a.state->total_items;
    for (int item = warp; item < total; item += nwarps) {
        int lo = 0, hi = n_active;  // prefix[lo] <= item < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.prefix[mid] <= item) lo = mid;
            else hi = mid;
        }
        const DomainDesc &D = a.domains[a.active[lo]];
        if (!D.acc) continue;
        const StepParams &p = D.p;
        const int local = item - a.prefix[lo];
        const int x0 = (local % p.nstrips) * W, y0 = (local / p.nstrips) * p.Ly;
        const int y1 = min(y0 + p.Ly, p.ny);
        const ST *f = static_cast<const ST *>(D.f[a.parity]);
        const size_t N = (size_t)p.nx * p.ny;
        const double hig = 0.5 / p.gamma;
        for (int y = y0; y < y1; ++y)
            for (int x = x0 + lane; x < min(x0 + W, p.nx); x += 32) {
                if (solid_at(p, x, y)) continue;
                const size_t i = (size_t)y * p.pitch + x;
                double g[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) g[k] = ld64(f, (size_t)k * p.plane + i);
                const double rho = 1.0 + (g[0] + (g[1] + g[3]) + (g[2] + g[4]) + ((g[5] + g[6]) + (g[7] + g[8])));
                const double jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]) - p.Fx * hig;
                const double jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]) - p.Fy * hig;
                const size_t c = (size_t)y * p.nx + x;
                D.acc[c] += jx / rho;
                D.acc[N + c] += jy / rho;
            }
    }
}

cudaError_t launch_batch_accumulate(int storage, const BatchArgs &a, int grid, cudaStream_t s)
{
    const int W = strip_width(storage);
    switch (storage) {
    case LBM_STORAGE_F16: batch_accumulate_kernel<__half><<<grid, 128, 0, s>>>(a, W); break;
    case LBM_STORAGE_BF16: batch_accumulate_kernel<__nv_bfloat16><<<grid, 128, 0, s>>>(a, W); break;
    case LBM_STORAGE_F64: batch_accumulate_kernel<double><<<grid, 128, 0, s>>>(a, W); break;
    default: batch_accumulate_kernel<float><<<grid, 128, 0, s>>>(a, W); break;
    }
    return cudaGetLastError();
}

// ---- convective outlet: ghost column from the last column --------------------
template <typename R, typename ST>
__global__ void outlet_seed_kernel(const StepParams p, const Consts<R> c, const ST *__restrict__ f, R *ghost)
{
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= p.ny) return;
    const int x = p.nx - 1;
    const size_t i = (size_t)y * p.pitch + x;
    R g[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = (R)ld64(f, (size_t)a * p.plane + i);
    R Fx = (R)p.Fx, Fy = (R)p.Fy;
    if (p.force) {
        Fx = (R)p.force[i];
        Fy = (R)p.force[(size_t)p.plane + i];
    }
    R drho, ux, uy;
    cell_state(c, g, Fx, Fy, drho, ux, uy);
    outlet_row(c, p.ny, y, g, drho, ux, uy, ux, uy, ghost);
}

cudaError_t launch_outlet_seed(const StepParams &p, int storage, const void *f, void *ghost, cudaStream_t s)
{
    const int grid = (p.ny + 127) / 128;
    with_storage(storage, f, [&](auto *fp) {
        using ST = std::remove_const_t<std::remove_pointer_t<decltype(fp)>>;
        if constexpr (std::is_same_v<ST, double>)
            outlet_seed_kernel<double, ST><<<grid, 128, 0, s>>>(p, p.cd, fp, static_cast<double *>(ghost));
        else
            outlet_seed_kernel<float, ST><<<grid, 128, 0, s>>>(p, p.cf, fp, static_cast<float *>(ghost));
    });
    return cudaGetLastError();
}

// ---- momentum-exchange force on the solid cells (Sec. 6, square cylinder) ------
// A post-collision population f~_a(x) of a fluid cell heading into a solid cell
// x + e_a returns in the opposite direction at the next streaming (half-way
// bounce-back, stationary solid) and hands the solid 2 e_a f~_a(x); summed in
// FP64 over every such link, one block per row (rows with a stride).
template <typename ST>
__global__ void drag_pass1(const StepParams p, const ST *__restrict__ f, double *partials)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int y = blockIdx.x; y < p.ny; y += gridDim.x)
        for (int x = threadIdx.x; x < p.nx; x += blockDim.x) {
            if (solid_at(p, x, y)) continue;
            const size_t i = (size_t)y * p.pitch + x;
            for (int a = 1; a < 9; ++a) {
                int tx = x + cx(a), ty = y + cy(a);
                if (p.perx) tx = tx < 0 ? tx + p.nx : (tx >= p.nx ? tx - p.nx : tx);
                if (p.pery) ty = ty < 0 ? ty + p.ny : (ty >= p.ny ? ty - p.ny : ty);
                if (tx < 0 || tx >= p.nx || ty < 0 || ty >= p.ny || !solid_at(p, tx, ty)) continue;
                const double fa = weight(a) + ld64(f, (size_t)a * p.plane + i);
                acc[0] += 2.0 * cx(a) * fa;
                acc[1] += 2.0 * cy(a) * fa;
            }
        }
    block_sum5<RES_THREADS>(acc, partials + (size_t)blockIdx.x * 5);
}

cudaError_t launch_drag(const StepParams &p, int storage, const void *f, double *partials, int nblocks,
                        double *result, cudaStream_t s)
{
    with_storage(storage, f, [&](auto *fp) {
        using ST = std::remove_const_t<std::remove_pointer_t<decltype(fp)>>;
        drag_pass1<ST><<<nblocks, RES_THREADS, 0, s>>>(p, fp, partials);
    });
    residual_pass2<<<1, RES_THREADS, 0, s>>>(partials, nblocks, result);
    return cudaGetLastError();
}

// ---- format conversions ------------------------------------------------------
__global__ void convert_kernel(const StepParams p, int from, const void *fin, int to, void *fout)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t i = (size_t)y * p.pitch + x;
    for (int a = 0; a < 9; ++a)
        store_any(fout, to, (size_t)a * p.plane + i, load_any(fin, from, (size_t)a * p.plane + i));
}

cudaError_t launch_convert(const StepParams &p, int from_storage, const void *fin, int to_storage,
                           void *fout, cudaStream_t s)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    convert_kernel<<<grid, 128, 0, s>>>(p, from_storage, fin, to_storage, fout);
    return cudaGetLastError();
}

__global__ void to_f64_kernel(const StepParams p, int storage, const void *f, double *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t i = (size_t)y * p.pitch + x;
    const size_t N = (size_t)p.nx * p.ny, o = (size_t)y * p.nx + x;
    for (int a = 0; a < 9; ++a) out[(size_t)a * N + o] = load_any(f, storage, (size_t)a * p.plane + i) + weight(a);
}

__global__ void from_f64_kernel(const StepParams p, int storage, const double *in, void *f)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const size_t i = (size_t)y * p.pitch + x;
    const size_t N = (size_t)p.nx * p.ny, o = (size_t)y * p.nx + x;
    for (int a = 0; a < 9; ++a) store_any(f, storage, (size_t)a * p.plane + i, in[(size_t)a * N + o] - weight(a));
}

cudaError_t launch_pops_to_f64(const StepParams &p, int storage, const void *f, double *out, cudaStream_t s)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    to_f64_kernel<<<grid, 128, 0, s>>>(p, storage, f, out);
    return cudaGetLastError();
}

cudaError_t launch_pops_from_f64(const StepParams &p, int storage, const double *in, void *f, cudaStream_t s)
{
    dim3 grid((p.nx + 127) / 128, p.ny);
    from_f64_kernel<<<grid, 128, 0, s>>>(p, storage, in, f);
    return cudaGetLastError();
}

}  // namespace lbm

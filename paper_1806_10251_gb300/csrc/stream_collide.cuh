// Fused pull-streaming + GI preconditioned cascaded collision (one time step).
//
// Decomposition: a block of BW threads owns a strip of BW columns and marches
// up a segment of Ly rows (a persistent grid walks the strip x segment items).
// For each row it pulls the nine populations of its cells once (Eq. 2b, with
// half-way bounce-back), keeps them in registers, and writes the cells'
// post-streaming density into a 4-row ring in shared memory.  The collision of
// row y runs after row y+1's densities are in the ring, so the central
// differences of the density (x and y neighbours, same time level) come from
// shared memory: only the two x-halo cells of each row and the two y-halo rows
// of each segment are pulled twice.  One __syncthreads per row.
//
// Shared-memory ring entries hold rho > 0 for fluid cells and -1 for positions
// outside a wall side or inside a solid; the finite difference replaces such a
// neighbour by the cell's own density (one-sided half difference).
#pragma once

#include "d2q9_collide.cuh"

namespace lbm {

template <typename ST>
struct Pull {
    using R = typename StorageTraits<ST>::R;

    const ST *__restrict__ f;
    const StepParams &p;

    __device__ __forceinline__ R ld(int a, int x, int y) const
    {
        return StorageTraits<ST>::load(f + (size_t)a * (size_t)p.plane + (size_t)y * p.pitch + x);
    }

    __device__ __forceinline__ bool is_solid(int x, int y) const
    {
        return p.solid != nullptr && __ldg(p.solid + (size_t)y * p.pitch + x) != 0;
    }

    // Gather gbar_alpha(x, y) = g~_alpha(x - e_alpha, y - e_alpha).  CHECK = false
    // is only used when every source lies inside the domain and no mask exists.
    template <bool CHECK>
    __device__ __forceinline__ void cell(int x, int y, R (&g)[9]) const
    {
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            int sx = x - cx(a), sy = y - cy(a);
            if (!CHECK) {
                g[a] = ld(a, sx, sy);
                continue;
            }
            if (p.perx) sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
            if (p.pery) sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
            const bool outx = sx < 0 || sx >= p.nx;
            const bool outy = sy < 0 || sy >= p.ny;
            if (!outx && !outy && !is_solid(sx, sy)) {
                g[a] = ld(a, sx, sy);
            } else {
                // half-way bounce-back, moving wall: + 6 w_a rho0 (e_a . u_w)
                double uw = 0.0, vw = 0.0;
                if (outx != outy) {
                    const int side = outx ? (sx < 0 ? 0 : 1) : (sy < 0 ? 2 : 3);
                    uw = p.side_u[side][0];
                    vw = p.side_u[side][1];
                }
                g[a] = ld(opposite(a), x, y) + R(6.0 * weight(a) * (cx(a) * uw + cy(a) * vw));
            }
        }
    }
};

// FP32 collision fits four resident blocks per SM in registers; the FP64 one two.
template <typename ST> struct MinBlocks { static constexpr int value = 4; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };

template <typename ST, int MODE>
__global__ void __launch_bounds__(BW, MinBlocks<ST>::value)
stream_collide_kernel(const StepParams p, const ST *__restrict__ fin, ST *__restrict__ fout)
{
    using R = typename StorageTraits<ST>::R;
    __shared__ R ring[4][BW + 2];

    Consts<R> c;
    c.init(p);
    const Pull<ST> pull{fin, p};
    const int tid = threadIdx.x;
    const bool has_force_field = p.force != nullptr;
    const bool uniform_forced = p.Fx != 0.0 || p.Fy != 0.0;

    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
        const int strip = item % p.nstrips;
        const int seg = item / p.nstrips;
        const int x0 = strip * BW;
        const int y0 = seg * p.Ly;
        const int y1 = min(y0 + p.Ly, p.ny);
        const int x = x0 + tid;
        // rows whose every pull stays inside the domain (no wrap, no wall, no mask)
        const bool x_interior = (x0 - 1 >= 1) && (x0 + BW <= p.nx - 2) && p.solid == nullptr;

        // Pull row yr: keep the thread's own populations in g (when own_valid),
        // and publish the density of ring columns 0..BW+1 into ring slot.
        auto produce = [&](int yr, R (&g)[9], bool &own_valid) {
            const int slot = (yr - y0 + 1) & 3;
            int ys = yr;
            if (p.pery) ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
            const bool row_in = ys >= 0 && ys < p.ny;
            const bool fast = x_interior && ys >= 1 && ys <= p.ny - 2;
            // own column (ring column tid + 1 <-> position x)
            own_valid = false;
            R rho_own = R(-1);
            if (row_in) {
                int xs = x;
                if (p.perx && xs == p.nx) xs = 0;
                if (xs < p.nx && !pull.is_solid(xs, ys)) {
                    if (fast) pull.template cell<false>(xs, ys, g);
                    else pull.template cell<true>(xs, ys, g);
                    R s = g[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a) s += g[a];
                    rho_own = R(1) + s;
                    own_valid = (xs == x);
                }
            }
            ring[slot][tid + 1] = rho_own;
            // halo columns: 0 <-> x0 - 1 (thread 0), BW + 1 <-> x0 + BW (thread BW - 1)
            if (tid == 0 || tid == BW - 1) {
                int xh = tid == 0 ? x0 - 1 : x0 + BW;
                R rho_h = R(-1);
                if (p.perx) xh = xh < 0 ? xh + p.nx : (xh >= p.nx ? xh - p.nx : xh);
                if (row_in && xh >= 0 && xh < p.nx && !(tid == BW - 1 && x0 + BW > p.nx) &&
                    !pull.is_solid(xh, ys)) {
                    R gh[9];
                    if (fast) pull.template cell<false>(xh, ys, gh);
                    else pull.template cell<true>(xh, ys, gh);
                    R s = gh[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a) s += gh[a];
                    rho_h = R(1) + s;
                }
                ring[slot][tid == 0 ? 0 : BW + 1] = rho_h;
            }
        };

        __syncthreads();  // previous item's readers are done with the ring
        R cur[9], nxt[9];
        bool cur_valid, nxt_valid, dummy;
        produce(y0 - 1, nxt, dummy);
        produce(y0, cur, cur_valid);

        for (int y = y0; y < y1; ++y) {
            produce(y + 1, nxt, nxt_valid);
            __syncthreads();
            if (cur_valid) {
                const int sm = (y - y0) & 3, s0 = (y - y0 + 1) & 3, sp = (y - y0 + 2) & 3;
                const R rc = ring[s0][tid + 1];
                R drx = 0, dry = 0;
                if (MODE == LBM_GI_FULL) {
                    R re = ring[s0][tid + 2], rw = ring[s0][tid];
                    R rn = ring[sp][tid + 1], rs = ring[sm][tid + 1];
                    re = re < R(0) ? rc : re;
                    rw = rw < R(0) ? rc : rw;
                    rn = rn < R(0) ? rc : rn;
                    rs = rs < R(0) ? rc : rs;
                    drx = R(0.5) * (re - rw);
                    dry = R(0.5) * (rn - rs);
                }
                R Fx = R(p.Fx), Fy = R(p.Fy);
                bool forced = uniform_forced;
                if (has_force_field) {
                    const size_t i = (size_t)y * p.pitch + x;
                    Fx = R(__ldg(p.force + i));
                    Fy = R(__ldg(p.force + (size_t)p.plane + i));
                    forced = true;
                }
                collide_cell<R, MODE>(cur, drx, dry, Fx, Fy, forced, c, p.guard != 0, p.guard_count);
                ST *o = fout + (size_t)y * p.pitch + x;
#pragma unroll
                for (int a = 0; a < 9; ++a) StorageTraits<ST>::store(o + (size_t)a * (size_t)p.plane, cur[a]);
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) cur[a] = nxt[a];
            cur_valid = nxt_valid;
        }
    }
}

template <typename ST>
cudaError_t launch_step_t(const StepParams &p, const void *fin, void *fout, int grid, cudaStream_t s)
{
    const ST *in = static_cast<const ST *>(fin);
    ST *out = static_cast<ST *>(fout);
    switch (p.gi_mode) {
    case LBM_GI_UNCORRECTED:
        stream_collide_kernel<ST, LBM_GI_UNCORRECTED><<<grid, BW, 0, s>>>(p, in, out);
        break;
    case LBM_GI_CUBIC_ONLY:
        stream_collide_kernel<ST, LBM_GI_CUBIC_ONLY><<<grid, BW, 0, s>>>(p, in, out);
        break;
    default:
        stream_collide_kernel<ST, LBM_GI_FULL><<<grid, BW, 0, s>>>(p, in, out);
        break;
    }
    return cudaGetLastError();
}

template <typename ST>
int blocks_per_sm_t(int gi_mode)
{
    int n = 0;
    cudaError_t e;
    switch (gi_mode) {
    case LBM_GI_UNCORRECTED:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_collide_kernel<ST, LBM_GI_UNCORRECTED>, BW, 0);
        break;
    case LBM_GI_CUBIC_ONLY:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_collide_kernel<ST, LBM_GI_CUBIC_ONLY>, BW, 0);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stream_collide_kernel<ST, LBM_GI_FULL>, BW, 0);
        break;
    }
    return e == cudaSuccess && n > 0 ? n : 1;
}

}  // namespace lbm

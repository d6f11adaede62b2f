// Fused pull-streaming + GI preconditioned cascaded collision (one time step),
// with TMA-staged source rows.
//
// Decomposition: a block of BW threads owns a strip of BW columns and marches
// up a segment of rows; a persistent grid walks the strip x segment items.
// Source data is staged row by row: one TMA copy (cp.async.bulk.tensor.3d,
// box {BW + 2 PAD, 1, 9}) brings one row of all nine population planes, PAD
// columns of halo on each side, into a ring of NSLOT shared-memory slots
// completed on per-slot mbarriers.  Every source element is therefore fetched
// from HBM once per step, several rows stay in flight per block, and the pulls
// of Eq. 2b become shared-memory loads.  Cell row y is collided once source row
// y + 2 has landed: the same-step density of rows y - 1, y, y + 1 (central
// differences) sits in a 4-row density ring.  One __syncthreads per row.
//
// Periodic sides: source rows wrap when the copy is issued (y); the two halo
// columns beyond a periodic x edge are patched from global memory when the row
// lands.  Walls and solids use half-way bounce-back with the moving-wall term.
// Density-ring entries hold rho > 0 for fluid cells and -1 for positions
// outside a wall side or inside a solid; the finite difference replaces such a
// neighbour by the cell's own density (one-sided half difference).
//
// Every mbarrier wait is bounded in time; on expiry the block records an error
// in p.error, waits (bounded) for its own copies in flight and returns.
#pragma once

#include <cuda.h>

#include "d2q9_collide.cuh"

namespace lbm {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait

template <typename ST>
struct Tile {
    static constexpr int ES = (int)sizeof(ST);
    static constexpr int PAD = 16 / ES;                  // TMA: x * ES multiple of 16
    static constexpr int BWX = BW + 2 * PAD;             // box width (columns)
    static constexpr int ROW_BYTES = 9 * BWX * ES;       // one source row, nine planes
    static constexpr int SLOT_BYTES = (ROW_BYTES + 127) / 128 * 128;
    static constexpr int NSLOT = ES == 8 ? 8 : 10;
    static constexpr int RING_BYTES = NSLOT * SLOT_BYTES;
    using R = typename StorageTraits<ST>::R;
    static constexpr int RHO_BYTES = 4 * (BW + 2) * (int)sizeof(R);
    static constexpr int SMEM_BYTES = RING_BYTES + RHO_BYTES + NSLOT * 8;
};

// FP32 collision fits four resident blocks per SM; the FP64 one two.
template <typename ST> struct MinBlocks { static constexpr int value = 4; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };

// ---- PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete; false after the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > WAIT_LIMIT_NS) return false;
    return true;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <typename ST, int MODE>
__global__ void __launch_bounds__(BW, MinBlocks<ST>::value)
stream_collide_kernel(const StepParams p, const __grid_constant__ CUtensorMap tin, const ST *__restrict__ fin,
                      ST *__restrict__ fout)
{
    using T = Tile<ST>;
    using R = typename T::R;
    extern __shared__ __align__(1024) unsigned char smem[];
    R(*rho)[BW + 2] = reinterpret_cast<R(*)[BW + 2]>(smem + T::RING_BYTES);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + T::RING_BYTES + T::RHO_BYTES);
    const uint32_t ring_u32 = smem_u32(smem);
    const uint32_t bars_u32 = smem_u32(bars);

    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < T::NSLOT; ++k) mbar_init(bars_u32 + 8 * k, 1);
        fence_mbar_init();
    }
    __syncthreads();

    Consts<R> c;
    c.init(p);
    const bool has_force_field = p.force != nullptr;
    const bool uniform_forced = p.Fx != 0.0 || p.Fy != 0.0;
    const bool has_solid = p.solid != nullptr;
    uint32_t q_base = 0;  // sequence number (over items) of the current item's first source row

    for (int item = blockIdx.x; item < p.nitems; item += gridDim.x) {
        const int strip = item % p.nstrips;
        const int seg = item / p.nstrips;
        const int x0 = strip * BW;
        const int y0 = seg * p.Ly;
        const int y1 = min(y0 + p.Ly, p.ny);
        const int s_first = y0 - 2;
        const int nsrc = (y1 + 1) - s_first + 1;  // source rows y0-2 .. y1+1
        const int x = x0 + tid;
        const int col = tid + T::PAD;             // smem column of this thread's cell
        const bool fix_left = p.perx && x0 == 0;
        // the box reaches column nx (right halo x0 + BW pulls from x0 + BW + 1)
        const bool fix_right = p.perx && x0 + BW + 1 >= p.nx;
        const bool fast_x = !has_solid && (p.perx || (x0 >= 2 && x0 + BW + 2 <= p.nx));

        auto slot_of = [&](int k) -> int { return (int)((q_base + (uint32_t)k) % T::NSLOT); };
        auto row_ptr = [&](int s) -> const ST * {  // source row s (absolute) in the ring
            return reinterpret_cast<const ST *>(smem + slot_of(s - s_first) * T::SLOT_BYTES);
        };
        // Thread 0: start the copy of item row k (source row s_first + k).
        auto issue = [&](int k) {
            const int slot = slot_of(k);
            const uint32_t bar = bars_u32 + 8 * slot;
            int s = s_first + k;
            if (p.pery) s = wrap(s, p.ny);
            if (s < 0 || s >= p.ny) {
                mbar_arrive(bar);  // row outside a wall side: never read
            } else {
                mbar_expect_tx(bar, (uint32_t)T::ROW_BYTES);
                tma_load_3d(ring_u32 + slot * T::SLOT_BYTES, &tin, x0 - T::PAD, s, 0, bar);
            }
        };
        // All threads: wait for item row k, then patch periodic x halo columns.
        auto land = [&](int k, bool &timed_out) {
            const int slot = slot_of(k);
            const uint32_t parity = ((q_base + (uint32_t)k) / T::NSLOT) & 1u;
            if (!mbar_wait_bounded(bars_u32 + 8 * slot, parity)) {
                timed_out = true;
                return;
            }
            int s = s_first + k;
            if (p.pery) s = wrap(s, p.ny);
            if ((fix_left || fix_right) && s >= 0 && s < p.ny && tid < 36) {
                const int side = tid / 18, r = tid % 18, a = r % 9, j = r / 9;
                const bool doit = side == 0 ? fix_left : fix_right;
                if (doit) {
                    // left: columns -2, -1 <- nx-2, nx-1; right: nx, nx+1 <- 0, 1
                    const int xd = side == 0 ? j - 2 : p.nx + j;
                    const int xs = side == 0 ? p.nx - 2 + j : j;
                    const int cd = xd - x0 + T::PAD;
                    if (cd >= 0 && cd < T::BWX) {
                        ST *dst = reinterpret_cast<ST *>(smem + slot * T::SLOT_BYTES);
                        dst[a * T::BWX + cd] = fin[(size_t)a * (size_t)p.plane + (size_t)s * p.pitch + xs];
                    }
                }
            }
        };

        // Gather gbar(xc, r) from the ring; xc is a column of the strip or its
        // halo, r a row of the item (sources r - 1 .. r + 1 have landed).
        auto pull = [&](int xc, int r, bool fast, R(&g)[9]) {
            const ST *rows[3] = {row_ptr(r - 1), row_ptr(r), row_ptr(r + 1)};
            const int cc = xc - x0 + T::PAD;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const int ex = cx(a), ey = cy(a);
                if (fast) {
                    g[a] = StorageTraits<ST>::cvt(rows[1 - ey][a * T::BWX + cc - ex]);
                    continue;
                }
                const int sx = xc - ex, sy = r - ey;
                const bool outx = !p.perx && (sx < 0 || sx >= p.nx);
                const bool outy = !p.pery && (sy < 0 || sy >= p.ny);
                bool inside = !outx && !outy;
                if (inside && has_solid) {
                    const int wx = p.perx ? wrap(sx, p.nx) : sx, wy = p.pery ? wrap(sy, p.ny) : sy;
                    inside = __ldg(p.solid + (size_t)wy * p.pitch + wx) == 0;
                }
                if (inside) {
                    g[a] = StorageTraits<ST>::cvt(rows[1 - ey][a * T::BWX + cc - ex]);
                } else {
                    // half-way bounce-back, moving wall: + 6 w_a rho0 (e_a . u_w)
                    double uw = 0.0, vw = 0.0;
                    if (outx != outy) {
                        const int side = outx ? (sx < 0 ? 0 : 1) : (sy < 0 ? 2 : 3);
                        uw = p.side_u[side][0];
                        vw = p.side_u[side][1];
                    }
                    g[a] = StorageTraits<ST>::cvt(rows[1][opposite(a) * T::BWX + cc]) +
                           R(6.0 * weight(a) * (ex * uw + ey * vw));
                }
            }
        };

        // Density of cell row r into the density ring: own column, and the
        // halo columns (thread 0: x0 - 1, thread BW - 1: x0 + BW).
        auto produce = [&](int r, R(&g)[9], bool &own_valid) {
            const int rslot = (r - y0 + 1) & 3;
            const bool row_in = p.pery || (r >= 0 && r < p.ny);
            const int rw = p.pery ? wrap(r, p.ny) : r;
            const bool fast = fast_x && (p.pery || (r >= 1 && r <= p.ny - 2));
            own_valid = false;
            R rho_own = R(-1);
            if (row_in && (x < p.nx || (p.perx && x == p.nx))) {
                const int xw = x < p.nx ? x : 0;
                if (!has_solid || __ldg(p.solid + (size_t)rw * p.pitch + xw) == 0) {
                    pull(x, r, fast, g);
                    R s = g[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a) s += g[a];
                    rho_own = R(1) + s;
                    own_valid = x < p.nx;
                }
            }
            rho[rslot][tid + 1] = rho_own;
            if (tid == 0 || tid == BW - 1) {
                const int xh = tid == 0 ? x0 - 1 : x0 + BW;
                const bool need = tid == 0 ? (x0 >= 1 || p.perx) : (xh < p.nx || (p.perx && xh == p.nx));
                R rho_h = R(-1);
                if (row_in && need) {
                    const int xw = wrap(xh, p.nx);
                    if (!has_solid || __ldg(p.solid + (size_t)rw * p.pitch + xw) == 0) {
                        R gh[9];
                        pull(xh, r, fast, gh);
                        R s = gh[0];
#pragma unroll
                        for (int a = 1; a < 9; ++a) s += gh[a];
                        rho_h = R(1) + s;
                    }
                }
                rho[rslot][tid == 0 ? 0 : BW + 1] = rho_h;
            }
        };

        __syncthreads();  // the previous item's readers are done with the ring
        if (tid == 0) {
            fence_proxy_async();
            for (int k = 0; k < min(T::NSLOT, nsrc); ++k) issue(k);
        }
        int issued = min(T::NSLOT, nsrc);  // meaningful in thread 0 only
        bool timed_out = false;
        for (int k = 0; k < 5; ++k) land(k, timed_out);
        bool abort = __syncthreads_or(timed_out);

        R cur[9], nxt[9];
        bool cur_valid = false, nxt_valid = false, dummy;
        int landed = 5;
        if (!abort) {
            produce(y0 - 1, nxt, dummy);
            produce(y0, cur, cur_valid);
            for (int y = y0; y < y1; ++y) {
                const int kl = y - y0 + 5;  // source row y + 3
                if (kl < nsrc) {
                    land(kl, timed_out);
                    landed = kl + 1;
                }
                produce(y + 1, nxt, nxt_valid);
                if (__syncthreads_or(timed_out)) {
                    abort = true;
                    break;
                }
                if (tid == 0) {
                    // rows up to y - 2 are free: refill their slots
                    const int kmax = min(nsrc - 1, y - y0 + T::NSLOT);
                    if (issued <= kmax) fence_proxy_async();
                    while (issued <= kmax) issue(issued++);
                }
                if (cur_valid) {
                    const int sm = (y - y0) & 3, s0 = (y - y0 + 1) & 3, sp = (y - y0 + 2) & 3;
                    const R rc = rho[s0][tid + 1];
                    R drx = 0, dry = 0;
                    if (MODE == LBM_GI_FULL) {
                        R re = rho[s0][tid + 2], rw = rho[s0][tid];
                        R rn = rho[sp][tid + 1], rs = rho[sm][tid + 1];
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
        if (abort) {
            // record the failure, let this block's copies in flight finish, return
            if (tid == 0) {
                atomicExch(p.error, 1);
                for (int k = 0; k < issued; ++k) {
                    const uint32_t parity = ((q_base + (uint32_t)k) / T::NSLOT) & 1u;
                    if (!mbar_wait_bounded(bars_u32 + 8 * slot_of(k), parity)) break;
                }
            }
            return;
        }
        (void)landed;
        q_base += (uint32_t)nsrc;
    }
}

template <typename ST>
cudaError_t launch_step_t(const StepParams &p, const CUtensorMap &tin, const void *fin, void *fout, int grid,
                          cudaStream_t s)
{
    using T = Tile<ST>;
    const ST *in = static_cast<const ST *>(fin);
    ST *out = static_cast<ST *>(fout);
    switch (p.gi_mode) {
    case LBM_GI_UNCORRECTED:
        stream_collide_kernel<ST, LBM_GI_UNCORRECTED><<<grid, BW, T::SMEM_BYTES, s>>>(p, tin, in, out);
        break;
    case LBM_GI_CUBIC_ONLY:
        stream_collide_kernel<ST, LBM_GI_CUBIC_ONLY><<<grid, BW, T::SMEM_BYTES, s>>>(p, tin, in, out);
        break;
    default:
        stream_collide_kernel<ST, LBM_GI_FULL><<<grid, BW, T::SMEM_BYTES, s>>>(p, tin, in, out);
        break;
    }
    return cudaGetLastError();
}

template <typename ST, int MODE>
int blocks_per_sm_mode()
{
    using T = Tile<ST>;
    auto fn = stream_collide_kernel<ST, MODE>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, BW, T::SMEM_BYTES) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <typename ST>
int blocks_per_sm_t(int gi_mode)
{
    switch (gi_mode) {
    case LBM_GI_UNCORRECTED: return blocks_per_sm_mode<ST, LBM_GI_UNCORRECTED>();
    case LBM_GI_CUBIC_ONLY: return blocks_per_sm_mode<ST, LBM_GI_CUBIC_ONLY>();
    default: return blocks_per_sm_mode<ST, LBM_GI_FULL>();
    }
}

}  // namespace lbm

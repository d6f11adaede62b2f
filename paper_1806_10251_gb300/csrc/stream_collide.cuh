// Fused pull-streaming + GI preconditioned cascaded collision (one time step).
//
// Decomposition: every warp works on its own strip of WS = 32 columns (one
// cell per lane) and marches up a segment of rows; warps walk the (strip,
// segment) items of the domain independently (no block-wide barrier anywhere
// in the step).
//
// Loads: one TMA copy (cp.async.bulk.tensor.3d, box {WS + 2 PAD, 1, 9}) brings
// one source row of all nine population planes, with PAD halo columns on each
// side, into the warp's ring of NSLOT shared-memory slots, completed on one
// mbarrier per slot.  Each source element crosses HBM once per step and several
// rows are in flight per warp; the pulls of Eq. 2b are shared-memory loads.
//
// Density gradient (same time level, central differences, or the isotropic
// stencil 3 sum_a w_a e_a rho(x + e_a) as a variant): each lane keeps the
// post-streaming density of its column for rows y - 1, y, y + 1 in registers;
// the x neighbours come from the adjacent lanes by shuffles, and the halo
// columns x0 - 1 and x0 + WS from a lane-parallel pull.  Density entries are -1 for
// positions outside a wall side or inside a solid; the difference then uses
// the cell's own density for that neighbour (one-sided half difference).
//
// Stores: each lane writes its nine post-collision values into the warp's
// stage buffer; one TMA bulk-tensor store per row writes them to HBM.
//
// Rows whose pulls meet no wall, solid or ragged edge take a path without any
// boundary logic (and the strip's halo densities come from one shared-memory
// load per lane and a 16-lane shuffle sum); the general path handles the rest.
//
// Periodic sides: source rows wrap when the copy is issued (y); the two halo
// columns beyond a periodic x edge are patched from global memory when a row
// lands.  Walls and solids use half-way bounce-back with the moving-wall term.
//
// Work items (strip, row segment) are handed out through a device counter, so
// the load balances dynamically; the last warp of a launch resets it.
//
// Every mbarrier wait is bounded in time; on expiry the warp records an error
// in p.error, waits (bounded) for its own copies in flight and returns.
#pragma once

#include <cuda.h>

#include "d2q9_collide.cuh"
#include "open_bc.cuh"

namespace lbm {

constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s per wait

template <typename ST>
struct Tile {
    static constexpr int ES = (int)sizeof(ST);
    static constexpr int PAD = 16 / ES;               // TMA: x * ES multiple of 16
    static constexpr int BWX = WS + 2 * PAD;          // load box width (columns)
    static constexpr int ROW_BYTES = 9 * BWX * ES;    // one source row, nine planes
    static constexpr int SLOT_BYTES = (ROW_BYTES + 127) / 128 * 128;
    static constexpr int NSLOT = ES == 8 ? 6 : 8;     // ring depth (3 rows are read at a time)
    static constexpr int STAGE_BYTES = (9 * WS * ES + 127) / 128 * 128;
    static constexpr int STAGE_OFF = NSLOT * SLOT_BYTES;
    static constexpr int BAR_OFF = STAGE_OFF + STAGE_BYTES;
    static constexpr int WARP_BYTES = (BAR_OFF + NSLOT * 8 + 127) / 128 * 128;
    static constexpr int SMEM_BYTES = WARPS * WARP_BYTES;
};

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
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
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

// Whether the work item of columns x0 .. x0 + w - 1 (w = 32 or 64) and rows
// y0 .. y1 - 1 can meet a solid cell: in the pulls, halo columns and density
// stencils of the rows it produces (y0 - 1 .. y1), which the mask's row table
// (after the mask, StepParams::solid) answers per row and 32-column block.
// Warp-uniform (lane k looks at rows y0 - 1 + k, y0 + 31 + k, ...).  An item
// that meets none takes the paths of a domain without a mask.
__device__ __forceinline__ bool item_meets_solid(const StepParams &p, int x0, int y0, int y1, int lane, int w = 64)
{
    if (!p.solid) return false;
    const uint8_t *table = p.solid + (size_t)p.ny * p.pitch;
    const int nb = (p.nx + 31) >> 5;
    const int b0 = x0 >> 5, b1 = min(b0 + (w >> 5) - 1, nb - 1);
    bool any = false;
    for (int r0 = y0 - 1; r0 <= y1; r0 += 32) {
        int r = r0 + lane;
        bool f = false;
        if (r <= y1) {
            if (p.pery) r = wrap(r, p.ny);
            if (r >= 0 && r < p.ny) {
                const uint8_t *row = table + (size_t)r * nb;
                for (int b = b0; b <= b1; ++b) f = f || row[b] != 0;
            }
        }
        any = any || __any_sync(0xffffffffu, f);
    }
    return any;
}

template <typename R> __device__ __forceinline__ const Consts<R> &consts(const StepParams &p);
template <> __device__ __forceinline__ const Consts<float> &consts<float>(const StepParams &p) { return p.cf; }
template <> __device__ __forceinline__ const Consts<double> &consts<double>(const StepParams &p) { return p.cd; }

// Resident blocks per SM the register budget is sized for (shared memory allows
// 4 blocks of the FP32 layout, more of the 16-bit ones, 2 of the FP64 one).
template <typename ST> struct MinBlocks { static constexpr int value = sizeof(ST) == 8 ? 2 : 4; };

// Packed lattice velocities for runtime direction indices: bits 2a..2a+1 hold e + 1.
constexpr uint32_t EX_PACK = (1u << 0) | (2u << 2) | (1u << 4) | (0u << 6) | (1u << 8) | (2u << 10) | (0u << 12) |
                             (0u << 14) | (2u << 16);
constexpr uint32_t EY_PACK = (1u << 0) | (1u << 2) | (2u << 4) | (1u << 6) | (0u << 8) | (2u << 10) | (2u << 12) |
                             (0u << 14) | (0u << 16);
// opposite directions, 4 bits each: 0 3 4 1 2 7 8 5 6
constexpr uint64_t OPP_PACK = 0ull | (3ull << 4) | (4ull << 8) | (1ull << 12) | (2ull << 16) | (7ull << 20) |
                              (8ull << 24) | (5ull << 28) | (6ull << 32);

template <bool V> struct Flag { static constexpr bool value = V; };

// Per-warp state that lives across work items.
struct WarpCtx {
    int lane;
    unsigned char *ws;            // this warp's ring, stage and barriers
    uint32_t ring_u32, stage_u32, bars_u32;
    uint32_t q_base;              // sequence number of the current item's first source row
    int issued;                   // item rows issued so far (lane 0)
    int h_side, h_a, h_ex, h_ey;  // lane-parallel halo: side and direction of this lane
};

template <typename ST>
__device__ __forceinline__ void warp_begin(WarpCtx &w, unsigned char *smem)
{
    using T = Tile<ST>;
    w.lane = threadIdx.x & 31;
    w.ws = smem + (threadIdx.x >> 5) * T::WARP_BYTES;
    w.ring_u32 = smem_u32(w.ws);
    w.stage_u32 = w.ring_u32 + T::STAGE_OFF;
    w.bars_u32 = w.ring_u32 + T::BAR_OFF;
    w.q_base = 0;
    w.issued = 0;
    // lane-parallel halo density: lane l < 9 handles direction l of the left
    // halo cell (x0 - 1), lane 16 + l of the right one (x0 + WS)
    w.h_side = w.lane >> 4;
    w.h_a = w.lane & 15;
    w.h_ex = w.h_a < 9 ? (int)((EX_PACK >> (2 * w.h_a)) & 3u) - 1 : 0;
    w.h_ey = w.h_a < 9 ? (int)((EY_PACK >> (2 * w.h_a)) & 3u) - 1 : 0;
    if (w.lane == 0) {
        for (int k = 0; k < T::NSLOT; ++k) mbar_init(w.bars_u32 + 8 * k, 1);
        fence_mbar_init();
    }
    __syncwarp();
}

// One work item: rows [seg*Ly, ...) of the 32-column strip `strip` of the
// domain described by p, reading fin through tin and writing through tout.
// Returns false when a bounded wait expired (the caller then stops).
template <typename ST, int MODE, bool FORCED, bool ISO = false>
__device__ __forceinline__ bool run_item(WarpCtx &w, const StepParams &p, const CUtensorMap *tin,
                                         const CUtensorMap *tout, const ST *__restrict__ fin, int strip, int seg,
                                         uint32_t step)
{
    using T = Tile<ST>;
    using R = typename StorageTraits<ST>::R;
    const unsigned FULL = 0xffffffffu;
    const int lane = w.lane;
    unsigned char *ws = w.ws;
    const uint32_t ring_u32 = w.ring_u32, stage_u32 = w.stage_u32, bars_u32 = w.bars_u32;
    ST *stage = reinterpret_cast<ST *>(ws + T::STAGE_OFF);
    const uint32_t q_base = w.q_base;
    int &issued = w.issued;
    const int h_side = w.h_side, h_a = w.h_a, h_ex = w.h_ex, h_ey = w.h_ey;
    const Consts<R> &c = consts<R>(p);
    const bool sround = StorageTraits<ST>::kReduced && p.sround;
    const uint32_t seed = sround ? mix32(step) : 0u;
    bool abort = false;
    {
        const int x0 = strip * WS;
        const int y0 = seg * p.Ly;
        const int y1 = min(y0 + p.Ly, p.ny);
        // an item that meets no solid takes the paths of a domain without a mask
        const bool has_solid = item_meets_solid(p, x0, y0, y1, lane, WS);
        const int s_first = y0 - 2;
        const int nsrc = (y1 + 1) - s_first + 1;  // source rows y0-2 .. y1+1
        const int x = x0 + lane;                  // this lane's cell
        const bool fix_left = p.perx && x0 == 0;
        const bool fix_right = p.perx && x0 + WS + 1 >= p.nx;
        // full strip whose pulls (columns x0-2 .. x0+WS+1) never meet a wall or solid
        const bool strip_fast = !has_solid && x0 + WS <= p.nx && (p.perx || (x0 >= 2 && x0 + WS + 2 <= p.nx));

        auto slot_of = [&](int k) -> int { return (int)((q_base + (uint32_t)k) % T::NSLOT); };
        auto row_ptr = [&](int s) -> const ST * {
            return reinterpret_cast<const ST *>(ws + slot_of(s - s_first) * T::SLOT_BYTES);
        };
        // lane 0: start the copy of item row k (source row s_first + k)
        auto issue = [&](int k) {
            const int slot = slot_of(k);
            const uint32_t bar = bars_u32 + 8 * slot;
            int s = s_first + k;
            if (p.pery) s = wrap(s, p.ny);
            if (s < 0 || s >= p.ny) {
                mbar_arrive(bar);  // beyond a wall side: never read
            } else {
                mbar_expect_tx(bar, (uint32_t)T::ROW_BYTES);
                tma_load_3d(ring_u32 + slot * T::SLOT_BYTES, tin, x0 - T::PAD, s, 0, bar);
            }
        };
        // all lanes: wait for item row k, patch periodic x halo columns
        auto land = [&](int k) -> bool {
            const int slot = slot_of(k);
            const uint32_t parity = ((q_base + (uint32_t)k) / T::NSLOT) & 1u;
            const bool ok = mbar_wait_bounded(bars_u32 + 8 * slot, parity);
            if (__any_sync(FULL, !ok)) return false;
            if (fix_left || fix_right) {
                int s = s_first + k;
                if (p.pery) s = wrap(s, p.ny);
                if (s >= 0 && s < p.ny) {
                    ST *dst = reinterpret_cast<ST *>(ws + slot * T::SLOT_BYTES);
                    for (int t = lane; t < 36; t += 32) {
                        const int side = t / 18, r = t % 18, a = r % 9, j = r / 9;
                        if (side == 0 ? !fix_left : !fix_right) continue;
                        // left: columns -2, -1 <- nx-2, nx-1; right: nx, nx+1 <- 0, 1
                        const int xd = side == 0 ? j - 2 : p.nx + j;
                        const int xs = side == 0 ? p.nx - 2 + j : j;
                        const int cd = xd - x0 + T::PAD;
                        const long long fi = (long long)a * p.plane + (long long)s * p.pitch + xs;
                        if (cd >= 0 && cd < T::BWX && LBM_IN_BOUNDS(fi, 9 * p.plane, p.error))
                            dst[a * T::BWX + cd] = fin[fi];
                    }
                }
                __syncwarp();
            }
            return true;
        };
        // General pull of gbar(xc, r) with walls, solids and bounce-back.
        auto pull_general = [&](int xc, int r, R(&g)[9]) {
            const ST *rm = row_ptr(r - 1), *r0 = row_ptr(r), *rp = row_ptr(r + 1);
            const int cc = xc - x0 + T::PAD;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const int ex = cx(a), ey = cy(a);
                const ST *src = ey > 0 ? rm : (ey < 0 ? rp : r0);
                const int sx = xc - ex, sy = r - ey;
                const bool outx = !p.perx && (sx < 0 || sx >= p.nx);
                const bool outy = !p.pery && (sy < 0 || sy >= p.ny);
                bool inside = !outx && !outy;
                if (inside && has_solid) {
                    const int wx = p.perx ? wrap(sx, p.nx) : sx, wy = p.pery ? wrap(sy, p.ny) : sy;
                    const long long si = (long long)wy * p.pitch + wx;
                    inside = LBM_IN_BOUNDS(si, p.plane, p.error) && __ldg(p.solid + si) == 0;
                }
                if (inside && !LBM_IN_BOUNDS(cc - ex, T::BWX, p.error)) inside = false;
                if (inside) {
                    g[a] = StorageTraits<ST>::cvt(src[a * T::BWX + cc - ex]);
                } else if (outx || outy) {
                    g[a] = boundary_value<R>(p, c, a, ex, ey, sx, sy, outx, outy,
                                             StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + cc]));
                } else {
                    // a solid neighbour: half-way bounce-back from a stationary solid
                    g[a] = StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + cc]);
                }
            }
        };
        // One cell of a general row: populations and density (-1 if none).  xc
        // may be a halo column (-1 or nx on a periodic side): the mask is read
        // at the wrapped column, the ring at the unwrapped one.
        auto produce_cell = [&](int xc, int r, bool row_in, int rw, R(&g)[9], bool &valid, R &rho) {
            valid = false;
            rho = R(-1);
#pragma unroll
            for (int a = 0; a < 9; ++a) g[a] = R(0);  // cells without a lattice site collide the rest state
            const bool in_x = (xc >= 0 && xc < p.nx) || (p.perx && (xc == -1 || xc == p.nx));
            if (row_in && in_x) {
                const int xw = wrap(xc, p.nx);
                const long long si = (long long)rw * p.pitch + xw;
                if (!has_solid || (LBM_IN_BOUNDS(si, p.plane, p.error) && __ldg(p.solid + si) == 0)) {
                    pull_general(xc, r, g);
                    R s = g[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a) s += g[a];
                    rho = R(1) + s;
                    valid = xc >= 0 && xc < p.nx;
                }
            }
        };
        // Row r (sources r - 1 .. r + 1 landed) for the lane's cell and the halo
        // columns.  FAST rows have no boundary logic at all; other rows of
        // items that meet no solid load like FAST rows and let only the lanes
        // on a wall cell (and the halo lanes) replace the populations whose
        // source lies beyond the wall; items that meet a solid take the
        // general path.
        auto produce = [&](auto fast_tag, int r, R(&g)[9], bool &valid, R &rho, R &rho_l, R &rho_r) {
            constexpr bool FAST = decltype(fast_tag)::value;
            if (FAST || !has_solid) {
                const bool row_in = FAST || p.pery || (r >= 0 && r < p.ny);
                if (!row_in) {
#pragma unroll
                    for (int a = 0; a < 9; ++a) g[a] = R(0);
                    valid = false;
                    rho = rho_l = rho_r = R(-1);
                    return;
                }
                const ST *rm = row_ptr(r - 1), *r0 = row_ptr(r), *rp = row_ptr(r + 1);
                const int cc = lane + T::PAD;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const ST *src = cy(a) > 0 ? rm : (cy(a) < 0 ? rp : r0);
                    g[a] = StorageTraits<ST>::cvt(src[a * T::BWX + cc - cx(a)]);
                }
                bool own = true;
                if (!FAST) {
                    own = x < p.nx || (p.perx && x == p.nx);
                    const bool near = own && ((!p.perx && (x == 0 || x == p.nx - 1)) ||
                                              (!p.pery && (r == 0 || r == p.ny - 1)));
                    if (near) {
#pragma unroll
                        for (int a = 1; a < 9; ++a) {
                            const int ex = cx(a), ey = cy(a), sx = x - ex, sy = r - ey;
                            const bool outx = !p.perx && (sx < 0 || sx >= p.nx);
                            const bool outy = !p.pery && (sy < 0 || sy >= p.ny);
                            if (outx || outy)
                                g[a] = boundary_value<R>(p, c, a, ex, ey, sx, sy, outx, outy,
                                                         StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + cc]));
                        }
                    }
                }
                if (own) {
                    R s = g[0];
#pragma unroll
                    for (int a = 1; a < 9; ++a) s += g[a];
                    rho = R(1) + s;
                    valid = FAST || x < p.nx;
                } else {
#pragma unroll
                    for (int a = 0; a < 9; ++a) g[a] = R(0);  // no lattice site: collide the rest state
                    rho = R(-1);
                    valid = false;
                }
                // halo densities: one population per lane, then a 16-lane sum
                const bool need_l = FAST || x0 >= 1 || p.perx;
                const bool need_r = FAST || x0 + WS < p.nx || (p.perx && x0 + WS == p.nx);
                R v = R(0);
                if (h_a < 9 && (h_side ? need_r : need_l)) {
                    const int xh = h_side ? x0 + WS : x0 - 1;
                    const int ch = xh - x0 + T::PAD;
                    const ST *src = h_ey > 0 ? rm : (h_ey < 0 ? rp : r0);
                    bool out = false;
                    if (!FAST) {
                        const int sx = xh - h_ex, sy = r - h_ey;
                        const bool outx = !p.perx && (sx < 0 || sx >= p.nx);
                        const bool outy = !p.pery && (sy < 0 || sy >= p.ny);
                        if (outx || outy) {
                            out = true;
                            const int oa = (int)((OPP_PACK >> (4 * h_a)) & 15u);
                            v = boundary_value<R>(p, c, h_a, h_ex, h_ey, sx, sy, outx, outy,
                                                  StorageTraits<ST>::cvt(r0[oa * T::BWX + ch]));
                        }
                    }
                    if (!out) v = StorageTraits<ST>::cvt(src[h_a * T::BWX + ch - h_ex]);
                }
                v += __shfl_xor_sync(FULL, v, 8);
                v += __shfl_xor_sync(FULL, v, 4);
                v += __shfl_xor_sync(FULL, v, 2);
                v += __shfl_xor_sync(FULL, v, 1);
                const R sl = __shfl_sync(FULL, v, 0), sr = __shfl_sync(FULL, v, 16);
                rho_l = need_l ? R(1) + sl : R(-1);
                rho_r = need_r ? R(1) + sr : R(-1);
                return;
            }
            const bool row_in = p.pery || (r >= 0 && r < p.ny);
            const int rw = p.pery ? wrap(r, p.ny) : r;
            produce_cell(x, r, row_in, rw, g, valid, rho);
            R rho_h = R(-1);
            if (lane < 2) {
                R gh[9];
                bool vh;
                produce_cell(lane == 0 ? x0 - 1 : x0 + WS, r, row_in, rw, gh, vh, rho_h);
            }
            rho_l = __shfl_sync(FULL, rho_h, 0);
            rho_r = __shfl_sync(FULL, rho_h, 1);
        };

        if (lane == 0) {
            fence_proxy_async();  // earlier generic-proxy reads of the ring before new copies
            for (int k = 0; k < min(T::NSLOT, nsrc); ++k) issue(k);
            issued = min(T::NSLOT, nsrc);
        }
        const bool ok = land(0) && land(1) && land(2) && land(3);
        if (!ok) return false;
        // cur = populations of row y, nxt = row y + 1; densities of rows y-1, y, y+1
        R cur[9], nxt[9];
        bool cur_valid, nxt_valid;
        R rm, r0, rp, hl0, hr0, hlp, hrp, d0, d1;
        auto produce_any = [&](int r, R(&g)[9], bool &valid, R &rho, R &rho_l, R &rho_r) {
            if (strip_fast && (p.pery || (r >= 1 && r <= p.ny - 2)))
                produce(Flag<true>(), r, g, valid, rho, rho_l, rho_r);
            else
                produce(Flag<false>(), r, g, valid, rho, rho_l, rho_r);
        };
        produce_any(y0 - 1, nxt, nxt_valid, rm, d0, d1);
        produce_any(y0, cur, cur_valid, r0, hl0, hr0);
        R hlm = d0, hrm = d1;  // halo densities of row y - 1 (isotropic gradient only)
        __syncwarp();
        if (lane == 0) {
            // source row y0 - 2 is no longer read: refill its slot
            const int kmax = min(nsrc - 1, T::NSLOT);
            if (issued <= kmax) fence_proxy_async();
            while (issued <= kmax) issue(issued++);
        }

        // One time-step row: land source y + 2, produce row y + 1, collide row y.
        auto iter = [&](auto fast_tag, int y) -> bool {
            constexpr bool FAST = decltype(fast_tag)::value;
            const int kl = y - y0 + 4;  // source row y + 2
            if (kl < nsrc && !land(kl)) return false;
            produce(fast_tag, y + 1, nxt, nxt_valid, rp, hlp, hrp);
            __syncwarp();
            if (lane == 0) {
                // source rows up to y are no longer read: refill their slots
                const int kmax = min(nsrc - 1, y - y0 + 2 + T::NSLOT);
                if (issued <= kmax) fence_proxy_async();
                while (issued <= kmax) issue(issued++);
            }
            // density gradient (x neighbours by shuffles; the isotropic stencil
            // takes the diagonal neighbours from rows y - 1 and y + 1 the same way)
            R re = __shfl_down_sync(FULL, r0, 1), rw = __shfl_up_sync(FULL, r0, 1);
            if (lane == 31) re = hr0;
            if (lane == 0) rw = hl0;
            R rn = rp, rs = rm;
            R rne = rp, rnw = rp, rse = rm, rsw = rm;
            if constexpr (ISO) {
                rne = __shfl_down_sync(FULL, rp, 1);
                rnw = __shfl_up_sync(FULL, rp, 1);
                rse = __shfl_down_sync(FULL, rm, 1);
                rsw = __shfl_up_sync(FULL, rm, 1);
                if (lane == 31) {
                    rne = hrp;
                    rse = hrm;
                }
                if (lane == 0) {
                    rnw = hlp;
                    rsw = hlm;
                }
            }
            if (!FAST) {
                // a missing neighbour (wall side, solid) takes the cell's own density
                re = re < R(0) ? r0 : re;
                rw = rw < R(0) ? r0 : rw;
                rn = rn < R(0) ? r0 : rn;
                rs = rs < R(0) ? r0 : rs;
                if constexpr (ISO) {
                    rne = rne < R(0) ? r0 : rne;
                    rnw = rnw < R(0) ? r0 : rnw;
                    rse = rse < R(0) ? r0 : rse;
                    rsw = rsw < R(0) ? r0 : rsw;
                }
            }
            R drx, dry;
            if constexpr (ISO) {
                // d_i rho = 3 sum_a w_a e_ai rho(x + e_a): a third of the axis
                // differences plus a twelfth of the diagonal ones
                drx = (re - rw) / R(3) + ((rne + rse) - (rnw + rsw)) / R(12);
                dry = (rn - rs) / R(3) + ((rne + rnw) - (rse + rsw)) / R(12);
            } else {
                drx = R(0.5) * (re - rw);
                dry = R(0.5) * (rn - rs);
            }
            R Fx = R(0), Fy = R(0);
            if (FORCED) {
                Fx = c.Fx;
                Fy = c.Fy;
                if (p.force) {
                    const size_t i = (size_t)y * p.pitch + min(x, p.nx - 1);
                    if (LBM_IN_BOUNDS(i, p.plane, p.error)) {
                        Fx = R(__ldg(p.force + i));
                        Fy = R(__ldg(p.force + (size_t)p.plane + i));
                    }
                }
            }
            R out[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) out[a] = cur[a];
            collide_cell<R, MODE, FORCED>(out, drx, dry, Fx, Fy, c, p.guard != 0, p.guard_count);
            if (!FAST && p.outlet && x == p.nx - 1 && cur_valid) outlet_update<R>(p, c, y, out, Fx, Fy);
            // stage the row (the previous row's store must have read the buffer)
            if (lane == 0) bulk_wait_read_0();
            __syncwarp();
            if (sround) {
                const uint32_t h = mix32(seed ^ (uint32_t)(y * p.nx + x));
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    StorageTraits<ST>::store_sr(stage + a * WS + lane, (FAST || cur_valid) ? out[a] : R(0),
                                                sr_bits(h, a));
            } else {
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    StorageTraits<ST>::store(stage + a * WS + lane, (FAST || cur_valid) ? out[a] : R(0));
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                tma_store_3d(tout, x0, y, 0, stage_u32);
                bulk_commit();
            }
#pragma unroll
            for (int a = 0; a < 9; ++a) cur[a] = nxt[a];
            cur_valid = nxt_valid;
            rm = r0;
            r0 = rp;
            if constexpr (ISO) {
                hlm = hl0;
                hrm = hr0;
            }
            hl0 = hlp;
            hr0 = hrp;
            return true;
        };
        // rows whose iteration is boundary-free: y and y + 1 both fast rows
        int yf0 = y1, yf1 = y1;
        if (strip_fast) {
            yf0 = p.pery ? y0 : max(y0, 1);
            yf1 = p.pery ? y1 : min(y1, p.ny - 2);
            if (yf1 < yf0) yf0 = yf1 = y1;
        }
        for (int y = y0; y < yf0 && !abort; ++y) abort = !iter(Flag<false>(), y);
        for (int y = yf0; y < yf1 && !abort; ++y) abort = !iter(Flag<true>(), y);
        for (int y = max(yf1, yf0); y < y1 && !abort; ++y) abort = !iter(Flag<false>(), y);
        if (abort) return false;
        w.q_base += (uint32_t)nsrc;
    }
    return true;
}

// End of a warp's work: on failure record it and let the warp's copies in
// flight finish; wait for the stores; sign off on the work counter (the last
// warp of the launch resets the counters for the next launch).
template <typename ST>
__device__ __forceinline__ void warp_end(WarpCtx &w, bool abort, int *error, unsigned int *work)
{
    using T = Tile<ST>;
    if (abort && w.lane == 0) {
        atomicExch(error, 1);
        for (int k = max(0, w.issued - T::NSLOT); k < w.issued; ++k) {
            const uint32_t q = w.q_base + (uint32_t)k;
            if (!mbar_wait_bounded(w.bars_u32 + 8 * (q % T::NSLOT), (q / T::NSLOT) & 1u)) break;
        }
    }
    if (w.lane == 0) {
        bulk_wait_all();  // stores done before the stage memory goes away
        __threadfence();
        const unsigned total = gridDim.x * WARPS;
        if (atomicAdd(work + 1, 1u) == total - 1) {
            atomicExch(work, 0u);
            atomicExch(work + 1, 0u);
        }
    }
    __syncwarp();
}

// Items are handed out dynamically (one atomic per item), so warps that finish
// early take more work and the slowest warp bounds the tail.
__device__ __forceinline__ int next_item(const WarpCtx &w, unsigned int *work)
{
    int it = 0;
    if (w.lane == 0) it = (int)atomicAdd(work, 1u);
    return __shfl_sync(0xffffffffu, it, 0);
}

// One time step of one domain (ISO: the variant with the isotropic
// density-gradient stencil).
template <typename ST, int MODE, bool FORCED, bool ISO = false>
__global__ void __launch_bounds__(THREADS, MinBlocks<ST>::value)
stream_collide_kernel(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap tin,
                      const __grid_constant__ CUtensorMap tout, const ST *__restrict__ fin)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    WarpCtx w;
    warp_begin<ST>(w, smem);
    bool abort = false;
    for (int item = next_item(w, p.work); item < p.nitems; item = next_item(w, p.work)) {
        if (!run_item<ST, MODE, FORCED, ISO>(w, p, &tin, &tout, fin, item % p.nstrips, item / p.nstrips, p.step)) {
            abort = true;
            break;
        }
    }
    warp_end<ST>(w, abort, p.error, p.work);
}

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(m) : "memory");
}

// One time step of every active domain of a batch that has (FORCED) or has no
// body force (see stream_collide_x2_batch_kernel).
template <typename ST, int MODE, bool FORCED>
__global__ void __launch_bounds__(THREADS, MinBlocks<ST>::value)
stream_collide_batch_kernel(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    WarpCtx w;
    warp_begin<ST>(w, smem);
    bool abort = false;
    const int first = FORCED ? a.state->split_items : 0;
    const int end = FORCED ? a.state->total_items : a.state->split_items;
    const int n_active = a.state->n_active;
    int last_slot = -1;
    for (int item = first + next_item(w, a.work); item < end; item = first + next_item(w, a.work)) {
        int lo = 0, hi = n_active;  // prefix[lo] <= item < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.prefix + mid) <= item) lo = mid;
            else hi = mid;
        }
        const int slot = __ldg(a.active + lo);
        const DomainDesc &D = a.domains[slot];
        if (slot != last_slot) {
            tensormap_acquire(&D.tload[a.parity]);
            tensormap_acquire(&D.tstore[a.parity ^ 1]);
            last_slot = slot;
        }
        const int local = item - __ldg(a.prefix + lo);
        const StepParams &p = D.p;
        const ST *fin = static_cast<const ST *>(D.f[a.parity]);
        const uint32_t step = __ldg(a.step0 + lo) + (uint32_t)a.k;
        if (!run_item<ST, MODE, FORCED>(w, p, &D.tload[a.parity], &D.tstore[a.parity ^ 1], fin, local % p.nstrips,
                                        local / p.nstrips, step)) {
            abort = true;
            break;
        }
    }
    warp_end<ST>(w, abort, a.error, a.work);
}

}  // namespace lbm

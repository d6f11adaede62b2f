// Fused stream-collide step with two cells per lane (FP32, FP16 and BF16 storage).
//
// Same method and memory scheme as stream_collide.cuh (pull streaming, Eq. 2b,
// with half-way bounce-back; density gradient by central differences; the
// collision of Sec. 5), with these differences:
//   * a warp owns a strip of 64 columns and lane l the two neighbouring cells
//     x0 + 2l and x0 + 2l + 1 of each row;
//   * the collision runs on packed FP32 pairs (collide_x2.cuh): one
//     instruction updates both cells;
//   * source rows arrive by TMA (one cp.async.bulk.tensor.3d per row, box
//     {64 + 2 PAD, 1, 9}) in a per-warp ring, as in the one-cell kernel;
//     unshifted directions are read from the ring as aligned pairs;
//   * results are written straight from registers with one 2-wide store per
//     direction (coalesced: a warp writes 64 consecutive values of a plane).
// FP64 storage keeps the one-cell kernel.
#pragma once

#include "collide_x2.cuh"
#include "stream_collide.cuh"

namespace lbm {

constexpr int SW = 2 * WS;  // strip width: columns per warp

template <typename ST>
struct Tile2 {
    static constexpr int ES = (int)sizeof(ST);
    static constexpr int PAD = 16 / ES;           // TMA: x * ES multiple of 16; keeps pairs aligned
    static constexpr int BWX = SW + 2 * PAD;      // load box width (columns)
    static constexpr int ROW_BYTES = 9 * BWX * ES;
    static constexpr int SLOT_BYTES = (ROW_BYTES + 127) / 128 * 128;
    // ring depth (3 rows are read at a time; a power of two keeps the slot
    // arithmetic to a mask)
    static constexpr int NSLOT = ES == 4 ? 4 : 8;
    static constexpr int BAR_OFF = NSLOT * SLOT_BYTES;
    static constexpr int WARP_BYTES = (BAR_OFF + NSLOT * 8 + 127) / 128 * 128;
    static constexpr int SMEM_BYTES = WARPS * WARP_BYTES;
};

// Resident blocks per SM the register budget is sized for: four (16 warps) for
// the unforced kernels; three for the forced ones (the source terms).  The
// batch kernels read a domain's parameters from a per-warp copy in shared
// memory (see copy_params): through global memory they held about 40 more
// registers and forced three blocks per SM.
constexpr int MIN_BLOCKS_X2 = 4;
constexpr int MIN_BLOCKS_BATCH_X2 = 3;

// Copy a domain's parameters into the warp's shared-memory slot (when the
// warp's item moves to another domain), so that the step reads them like the
// single-domain kernel reads its launch parameters.
__device__ __forceinline__ void copy_params(StepParams &dst, const StepParams &src, int lane)
{
    static_assert(sizeof(StepParams) % 4 == 0, "word copy");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int i = lane; i < (int)(sizeof(StepParams) / 4); i += 32) d[i] = s[i];
    __syncwarp();
}

// Pairs of stored values <-> F2 (storage scale and rounding as StorageTraits).
template <typename ST> struct PairIO;
template <> struct PairIO<float> {
    __device__ static __forceinline__ F2 lds2(const float *p)
    {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        return F2{v.x, v.y};
    }
    __device__ static __forceinline__ F2 join(float a, float b) { return F2{a, b}; }
    __device__ static __forceinline__ void stg2(float *p, F2 v)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(v.x, v.y);
    }
    __device__ static __forceinline__ void stg2_sr(float *p, F2 v, uint32_t) { stg2(p, v); }
    static constexpr uint32_t HALF_ULP = 0u;
};
// 16-bit pairs are rounded by the hardware's stochastic conversion
// (cvt.rs.{f16x2,bf16x2}.f32 d, hi, lo, rbits): the low half of d (the even
// cell) adds rbits[12:0] (FP16) or rbits[15:0] (BF16) to the mantissa bits it
// drops, the high half (the odd cell) rbits[28:16] or rbits[31:16], and both
// truncate -- unbiased, in the FP16 subnormal range as well.  From 32 random
// bits r the pair takes rbits = r ^ (r >> 16), so that the even cell's field
// depends on the high bits of r too.
__device__ __forceinline__ uint32_t sr_fold(uint32_t r) { return r ^ (r >> 16); }

template <> struct PairIO<__half> {  // holds F16_SCALE * g
    // one mixed-precision FMA per value: the conversion and the inverse scale
    __device__ static __forceinline__ float from_h(__half h) { return f16_unscaled(h); }
    __device__ static __forceinline__ F2 lds2(const __half *p)
    {
        const __half2 h = *reinterpret_cast<const __half2 *>(p);
        return F2{from_h(__low2half(h)), from_h(__high2half(h))};
    }
    __device__ static __forceinline__ F2 join(__half a, __half b) { return F2{from_h(a), from_h(b)}; }
    __device__ static __forceinline__ void stg2(__half *p, F2 v)
    {
        const F2 s = v * f2(F16_SCALE);
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(s.x, s.y);
    }
    // HALF_ULP in place of random bits folds to rbits = 0x10001000: half of the
    // dropped range in both cells, i.e. rounding to nearest, ties away from zero.
    static constexpr uint32_t HALF_ULP = 0x10000000u;
    __device__ static __forceinline__ void stg2_sr(__half *p, F2 v, uint32_t r)
    {
        const F2 s = v * f2(F16_SCALE);
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(s.y), "f"(s.x), "r"(sr_fold(r)));
        *reinterpret_cast<uint32_t *>(p) = d;
    }
};
template <> struct PairIO<__nv_bfloat16> {
    __device__ static __forceinline__ F2 from_b2(__nv_bfloat162 h)
    {
        const float2 f = __bfloat1622float2(h);
        return F2{f.x, f.y};
    }
    __device__ static __forceinline__ F2 lds2(const __nv_bfloat16 *p)
    {
        return from_b2(*reinterpret_cast<const __nv_bfloat162 *>(p));
    }
    __device__ static __forceinline__ F2 join(__nv_bfloat16 a, __nv_bfloat16 b)
    {
        return from_b2(__halves2bfloat162(a, b));
    }
    __device__ static __forceinline__ void stg2(__nv_bfloat16 *p, F2 v)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
    // HALF_ULP folds to rbits = 0x80008000: rounding to nearest, ties away from zero.
    static constexpr uint32_t HALF_ULP = 0x80000000u;
    __device__ static __forceinline__ void stg2_sr(__nv_bfloat16 *p, F2 v, uint32_t r)
    {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(sr_fold(r)));
        *reinterpret_cast<uint32_t *>(p) = d;
    }
};

__device__ __forceinline__ float &comp(F2 &v, int c) { return c ? v.y : v.x; }
__device__ __forceinline__ float comp(const F2 &v, int c) { return c ? v.y : v.x; }

template <typename ST>
__device__ __forceinline__ void warp_begin_x2(WarpCtx &w, unsigned char *smem)
{
    using T = Tile2<ST>;
    w.lane = threadIdx.x & 31;
    w.ws = smem + (threadIdx.x >> 5) * T::WARP_BYTES;
    w.ring_u32 = smem_u32(w.ws);
    w.stage_u32 = 0;
    w.bars_u32 = w.ring_u32 + T::BAR_OFF;
    w.q_base = 0;
    w.issued = 0;
    // lane-parallel halo density: lane l < 9 handles direction l of the left
    // halo cell (x0 - 1), lane 16 + l of the right one (x0 + SW)
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

// End of a warp's work: on failure record it and let the warp's copies in
// flight finish; make the stores visible; sign off on the work counter (the
// last warp of the launch resets the counters for the next launch).
template <typename ST>
__device__ __forceinline__ void warp_end_x2(WarpCtx &w, bool abort, int *error, unsigned int *work)
{
    using T = Tile2<ST>;
    if (abort && w.lane == 0) {
        atomicExch(error, 1);
        for (int k = max(0, w.issued - T::NSLOT); k < w.issued; ++k) {
            const uint32_t q = w.q_base + (uint32_t)k;
            if (!mbar_wait_bounded(w.bars_u32 + 8 * (q % T::NSLOT), (q / T::NSLOT) & 1u)) break;
        }
    }
    __syncwarp();
    if (w.lane == 0) {
        __threadfence();
        const unsigned total = gridDim.x * WARPS;
        if (atomicAdd(work + 1, 1u) == total - 1) {
            atomicExch(work, 0u);
            atomicExch(work + 1, 0u);
        }
    }
    __syncwarp();
}

// One work item: rows [seg*Ly, ...) of the 64-column strip `strip` of the
// domain described by p, reading fin through tin (wide load box) and writing
// fout directly.  Returns false when a bounded wait expired.
template <typename ST, int MODE, bool FORCED, bool GUARD = false, bool ISO = false>
__device__ __forceinline__ bool run_item_x2(WarpCtx &w, const StepParams &p, const CUtensorMap *tin,
                                            const ST *__restrict__ fin, ST *__restrict__ fout, int strip, int seg,
                                            uint32_t step)
{
    using T = Tile2<ST>;
    using IO = PairIO<ST>;
    using R = float;
    const unsigned FULL = 0xffffffffu;
    const int lane = w.lane;
    unsigned char *ws = w.ws;
    const uint32_t ring_u32 = w.ring_u32, bars_u32 = w.bars_u32;
    const uint32_t q_base = w.q_base;
    int &issued = w.issued;
    const int h_side = w.h_side, h_a = w.h_a, h_ex = w.h_ex, h_ey = w.h_ey;
    const Consts<float> &c = p.cf;
    const bool sround = StorageTraits<ST>::kReduced && p.sround;
    const uint32_t seed = sround ? mix32(step) : 0u;

    const int x0 = strip * SW;
    const int y0 = seg * p.Ly;
    const int y1 = min(y0 + p.Ly, p.ny);
    // an item that meets no solid takes the paths of a domain without a mask
    const bool has_solid = item_meets_solid(p, x0, y0, y1, lane);
    const int s_first = y0 - 2;
    const int nsrc = (y1 + 1) - s_first + 1;  // source rows y0-2 .. y1+1
    const int xe = x0 + 2 * lane;             // this lane's even cell; the odd one is xe + 1
    const int cc = 2 * lane + T::PAD;         // its ring column
    const bool fix_left = p.perx && x0 == 0;
    const bool fix_right = p.perx && x0 + SW + 1 >= p.nx;
    // full strip whose pulls (columns x0-2 .. x0+SW+1) never meet a wall or solid
    const bool strip_fast = !has_solid && x0 + SW <= p.nx && (p.perx || (x0 >= 2 && x0 + SW + 2 <= p.nx));

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
    // all lanes: wait for item row k, patch periodic x halo columns (FIX: the
    // item is an end strip of a periodic domain; a compile-time flag keeps the
    // patch code out of the other items' row loop)
    auto land = [&](auto fix_tag, int k) -> bool {
        constexpr bool FIX = decltype(fix_tag)::value;
        const int slot = slot_of(k);
        const uint32_t parity = ((q_base + (uint32_t)k) / T::NSLOT) & 1u;
        const bool ok = mbar_wait_bounded(bars_u32 + 8 * slot, parity);
        if (__any_sync(FULL, !ok)) return false;
        if (FIX) {
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
    // General pull of gbar(xc, r) (one cell) with walls, solids and bounce-back.
    auto pull_general = [&](int xc, int r, R(&g)[9]) {
        const ST *rm = row_ptr(r - 1), *r0 = row_ptr(r), *rp = row_ptr(r + 1);
        const int ck = xc - x0 + T::PAD;
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
            if (inside && !LBM_IN_BOUNDS(ck - ex, T::BWX, p.error)) inside = false;
            if (inside) g[a] = StorageTraits<ST>::cvt(src[a * T::BWX + ck - ex]);
            else if (outx || outy)
                g[a] = boundary_value<R>(p, c, a, ex, ey, sx, sy, outx, outy,
                                         StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + ck]));
            else g[a] = StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + ck]);  // solid neighbour
        }
    };
    // One cell of a general row: populations and density (-1 if none).  xc
    // may be a halo column (-1 or nx on a periodic side): the mask is read at
    // the wrapped column, the ring at the unwrapped one.
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
    // Row r (sources r - 1 .. r + 1 landed) for the lane's two cells and the
    // halo columns.  FAST rows have no boundary logic at all; other rows of
    // items that meet no solid load like FAST rows and let only the cells on
    // a wall (and the halo lanes) replace the populations whose source lies
    // beyond the wall; items that meet a solid take the general path per cell.
    // valid: bit c set when cell xe + c is a lattice site of the domain.
    auto produce = [&](auto fast_tag, int r, F2(&g)[9], int &valid, F2 &rho, R &rho_l, R &rho_r) {
        constexpr bool FAST = decltype(fast_tag)::value;
        if (FAST || !has_solid) {
            const bool row_in = FAST || p.pery || (r >= 0 && r < p.ny);
            if (!row_in) {
#pragma unroll
                for (int a = 0; a < 9; ++a) g[a] = f2(0.f);
                valid = 0;
                rho = f2(-1.f);
                rho_l = rho_r = R(-1);
                return;
            }
            const ST *rm = row_ptr(r - 1), *r0 = row_ptr(r), *rp = row_ptr(r + 1);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const ST *src = (cy(a) > 0 ? rm : (cy(a) < 0 ? rp : r0)) + a * T::BWX + cc;
                if (cx(a) == 0) g[a] = IO::lds2(src);
                else g[a] = IO::join(src[-cx(a)], src[1 - cx(a)]);
            }
            int own = 3;
            if (!FAST) {
                own = 0;
                valid = 0;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int x = xe + k;
                    const bool ownk = x < p.nx || (p.perx && x == p.nx);
                    own |= ownk ? 1 << k : 0;
                    valid |= x < p.nx ? 1 << k : 0;
                    const bool near = ownk && ((!p.perx && (x == 0 || x == p.nx - 1)) ||
                                               (!p.pery && (r == 0 || r == p.ny - 1)));
                    if (near) {
#pragma unroll
                        for (int a = 1; a < 9; ++a) {
                            const int ex = cx(a), ey = cy(a), sx = x - ex, sy = r - ey;
                            const bool outx = !p.perx && (sx < 0 || sx >= p.nx);
                            const bool outy = !p.pery && (sy < 0 || sy >= p.ny);
                            if (outx || outy)
                                comp(g[a], k) = boundary_value<R>(
                                    p, c, a, ex, ey, sx, sy, outx, outy,
                                    StorageTraits<ST>::cvt(r0[opposite(a) * T::BWX + cc + k]));
                        }
                    }
                }
            } else {
                valid = 3;
            }
            F2 s = (g[0] + g[1]) + (g[2] + g[3]);
            s = s + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
            rho = f2(1.f) + s;
            if (!FAST && own != 3) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (!(own >> k & 1)) {
#pragma unroll
                        for (int a = 0; a < 9; ++a) comp(g[a], k) = 0.f;  // no lattice site: rest state
                        comp(rho, k) = -1.f;
                    }
            }
            // halo densities: one population per lane, then a 16-lane sum
            const bool need_l = FAST || x0 >= 1 || p.perx;
            const bool need_r = FAST || x0 + SW < p.nx || (p.perx && x0 + SW == p.nx);
            R v = R(0);
            if (h_a < 9 && (h_side ? need_r : need_l)) {
                const int xh = h_side ? x0 + SW : x0 - 1;
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
        // general path (solids): per cell
        const bool row_in = p.pery || (r >= 0 && r < p.ny);
        const int rw = p.pery ? wrap(r, p.ny) : r;
        valid = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            R gk[9], rk;
            bool vk;
            produce_cell(xe + k, r, row_in, rw, gk, vk, rk);
#pragma unroll
            for (int a = 0; a < 9; ++a) comp(g[a], k) = gk[a];
            comp(rho, k) = rk;
            valid |= vk ? 1 << k : 0;
        }
        R rho_h = R(-1);
        if (lane < 2) {
            R gh[9];
            bool vh;
            produce_cell(lane == 0 ? x0 - 1 : x0 + SW, r, row_in, rw, gh, vh, rho_h);
        }
        rho_l = __shfl_sync(FULL, rho_h, 0);
        rho_r = __shfl_sync(FULL, rho_h, 1);
    };

    if (lane == 0) {
        fence_proxy_async();  // earlier generic-proxy reads of the ring before new copies
        for (int k = 0; k < min(T::NSLOT, nsrc); ++k) issue(k);
        issued = min(T::NSLOT, nsrc);
    }
    const bool fix = fix_left || fix_right;
    if (fix ? !(land(Flag<true>(), 0) && land(Flag<true>(), 1)) : !(land(Flag<false>(), 0) && land(Flag<false>(), 1)))
        return false;
    // cur = populations of row y, nxt = row y + 1; densities of rows y-1, y, y+1
    // (filled by the two warm-up passes of the row loop, y = y0-2 and y0-1)
    F2 cur[9], nxt[9];
    int cur_valid = 0, nxt_valid = 0;
    F2 rm = f2(-1.f), r0 = f2(-1.f), rp;
    R hl0 = R(-1), hr0 = R(-1), hlp, hrp;
    R hlm = R(-1), hrm = R(-1);  // halo densities of row y - 1 (isotropic gradient only)
#pragma unroll
    for (int a = 0; a < 9; ++a) cur[a] = f2(0.f);
    const size_t plane = (size_t)p.plane;

    // One pass: land source y + 2, produce row y + 1, collide row y (rows
    // y >= y0; the passes y0-2 and y0-1 only produce, so the item needs no
    // separate prologue code).
    auto iter = [&](auto fast_tag, auto fix_tag, int y) -> bool {
        constexpr bool FAST = decltype(fast_tag)::value;
        const int kl = y - y0 + 4;  // source row y + 2
        if (kl < nsrc && !land(fix_tag, kl)) return false;
        produce(fast_tag, y + 1, nxt, nxt_valid, rp, hlp, hrp);
        __syncwarp();
        if (lane == 0) {
            // source rows up to y are no longer read: refill their slots
            const int kmax = min(nsrc - 1, y - y0 + 2 + T::NSLOT);
            if (issued <= kmax) fence_proxy_async();
            while (issued <= kmax) issue(issued++);
        }
        if (y >= y0) {  // the warm-up passes only produce
            // density gradient: x neighbours of the pair by shuffles (odd cell of
            // the lane to the left, even cell of the one to the right), halo
            // densities at the strip ends; the isotropic stencil takes the
            // diagonal neighbours from rows y - 1 and y + 1 the same way
            R wl = __shfl_up_sync(FULL, r0.y, 1), er = __shfl_down_sync(FULL, r0.x, 1);
            if (lane == 0) wl = hl0;
            if (lane == 31) er = hr0;
            F2 re = f2(r0.y, er), rw = f2(wl, r0.x);
            F2 rn = rp, rs = rm;
            F2 rne = rp, rnw = rp, rse = rm, rsw = rm;
            if constexpr (ISO) {
                R wlp = __shfl_up_sync(FULL, rp.y, 1), erp = __shfl_down_sync(FULL, rp.x, 1);
                R wlm = __shfl_up_sync(FULL, rm.y, 1), erm = __shfl_down_sync(FULL, rm.x, 1);
                if (lane == 0) {
                    wlp = hlp;
                    wlm = hlm;
                }
                if (lane == 31) {
                    erp = hrp;
                    erm = hrm;
                }
                rne = f2(rp.y, erp);
                rnw = f2(wlp, rp.x);
                rse = f2(rm.y, erm);
                rsw = f2(wlm, rm.x);
            }
            if (!FAST) {
                // a missing neighbour (wall side, solid) takes the cell's own density
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const R own = comp(r0, k);
                    if (comp(re, k) < R(0)) comp(re, k) = own;
                    if (comp(rw, k) < R(0)) comp(rw, k) = own;
                    if (comp(rn, k) < R(0)) comp(rn, k) = own;
                    if (comp(rs, k) < R(0)) comp(rs, k) = own;
                    if constexpr (ISO) {
                        if (comp(rne, k) < R(0)) comp(rne, k) = own;
                        if (comp(rnw, k) < R(0)) comp(rnw, k) = own;
                        if (comp(rse, k) < R(0)) comp(rse, k) = own;
                        if (comp(rsw, k) < R(0)) comp(rsw, k) = own;
                    }
                }
            }
            F2 Fx = f2(0.f), Fy = f2(0.f);
            if (FORCED) {
                Fx = ld(p.c2.Fx);
                Fy = ld(p.c2.Fy);
                if (p.force) {
                    const size_t i = (size_t)y * p.pitch + xe;
                    if (LBM_IN_BOUNDS(i + 1, plane, p.error)) {
                        const float2 fx2 = __ldg(reinterpret_cast<const float2 *>(p.force + i));
                        const float2 fy2 = __ldg(reinterpret_cast<const float2 *>(p.force + plane + i));
                        Fx = f2(fx2.x, fx2.y);
                        Fy = f2(fy2.x, fy2.y);
                    }
                }
            }
            F2 out[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) out[a] = cur[a];
            F2 drx, dry;
            if constexpr (ISO) {
                // d_i rho = 3 sum_a w_a e_ai rho(x + e_a): a third of the axis
                // differences plus a twelfth of the diagonal ones
                const F2 third = ld(p.c2.third), twelfth = f2(1.f / 12.f);
                drx = fma2(twelfth, (rne + rse) - (rnw + rsw), third * (re - rw));
                dry = fma2(twelfth, (rne + rnw) - (rse + rsw), third * (rn - rs));
            } else {
                const F2 half = ld(p.c2.half);
                drx = half * (re - rw);
                dry = half * (rn - rs);
            }
            collide_x2<MODE, FORCED, GUARD>(out, drx, dry, Fx, Fy, p.c2, p.guard != 0, p.guard_count);
            if (!FAST && p.outlet) {
                // convective outlet: the lane holding the last column advances its ghost row
                const int k = p.nx - 1 - xe;
                if ((k == 0 || k == 1) && (cur_valid >> k & 1)) {
                    R gk[9];
#pragma unroll
                    for (int a = 0; a < 9; ++a) gk[a] = comp(out[a], k);
                    outlet_update<R>(p, c, y, gk, comp(Fx, k), comp(Fy, k));
                }
            }
            if (!FAST && cur_valid != 3) {
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    if (!(cur_valid >> k & 1)) {
#pragma unroll
                        for (int a = 0; a < 9; ++a) comp(out[a], k) = 0.f;
                    }
            }
            // 2-wide stores of the row (x0 + SW <= pitch: the odd cell past nx, if
            // any, lands in the row padding)
            ST *fo = fout + (size_t)y * p.pitch + xe;
            if (!LBM_IN_BOUNDS((long long)y * p.pitch + xe + 1, p.plane, p.error)) {
                // debug build: a row index outside the buffer skips the stores
            } else if constexpr (StorageTraits<ST>::kReduced) {
                // one store path for both rounding modes (no cold alternative in the loop)
                const uint32_t h = mix32(seed ^ (uint32_t)(y * p.nx + xe));  // one hash per pair of cells
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    IO::stg2_sr(fo + a * plane, out[a], sround ? sr_bits(h, a) : IO::HALF_ULP);
            } else {
#pragma unroll
                for (int a = 0; a < 9; ++a) IO::stg2(fo + a * plane, out[a]);
            }
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
    // passes without boundary logic: rows y and y + 1 both fast rows
    int yf0 = y1, yf1 = y1;
    if (strip_fast) {
        yf0 = p.pery ? y0 - 2 : max(y0 - 2, 1);
        yf1 = p.pery ? y1 : min(y1, p.ny - 2);
        if (yf1 < yf0) yf0 = yf1 = y1;
    }
    bool abort = false;
    auto rows = [&](auto fix_tag) {
        for (int y = y0 - 2; y < yf0 && !abort; ++y) abort = !iter(Flag<false>(), fix_tag, y);
        for (int y = yf0; y < yf1 && !abort; ++y) abort = !iter(Flag<true>(), fix_tag, y);
        for (int y = max(yf1, yf0); y < y1 && !abort; ++y) abort = !iter(Flag<false>(), fix_tag, y);
    };
    if (fix) rows(Flag<true>());
    else rows(Flag<false>());
    if (abort) return false;
    w.q_base += (uint32_t)nsrc;
    return true;
}

// One time step of one domain (GUARD: the variant with the strain-solve guard,
// launched only when a context turns the guard on; ISO: the variant with the
// isotropic density-gradient stencil, which carries the guard as well and
// leaves it to the context's flag).
template <typename ST, int MODE, bool FORCED, bool GUARD = false, bool ISO = false>
__global__ void __launch_bounds__(THREADS, FORCED ? MIN_BLOCKS_BATCH_X2 : MIN_BLOCKS_X2)
stream_collide_x2_kernel(const __grid_constant__ StepParams p, const __grid_constant__ CUtensorMap tin,
                         const ST *__restrict__ fin, ST *__restrict__ fout)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    WarpCtx w;
    warp_begin_x2<ST>(w, smem);
    bool abort = false;
    for (int item = next_item(w, p.work); item < p.nitems; item = next_item(w, p.work)) {
        // phase-ordered items (see StepParams::nwave); items past the last
        // segment of a phase are empty
        const int per = p.nstrips * p.nseg_phase;
        const int phase = item / per, r = item - phase * per;
        const int strip = r % p.nstrips, seg = phase + (r / p.nstrips) * p.nwave;
        if (seg >= p.nseg) continue;
        if (!run_item_x2<ST, MODE, FORCED, GUARD, ISO>(w, p, &tin, fin, fout, strip, seg, p.step)) {
            abort = true;
            break;
        }
    }
    warp_end_x2<ST>(w, abort, p.error, p.work);
}

// One time step of every active domain of a batch that has (FORCED) or has no
// body force: the items of one launch run over those domains' (strip, segment)
// lists back to back, and a warp finds its item's domain by binary search in
// the prefix sums.  A domain's arithmetic does not depend on which other
// domains share the launch.
template <typename ST, int MODE, bool FORCED>
__global__ void __launch_bounds__(THREADS, FORCED ? MIN_BLOCKS_BATCH_X2 : MIN_BLOCKS_X2)
stream_collide_x2_batch_kernel(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ StepParams sp[WARPS];
    StepParams &p = sp[threadIdx.x >> 5];
    WarpCtx w;
    warp_begin_x2<ST>(w, smem);
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
            // the descriptor was written by a host copy into global memory:
            // acquire it for the tensor-map proxy before the first TMA use
            tensormap_acquire(&D.tload[a.parity]);
            copy_params(p, D.p, w.lane);
            last_slot = slot;
        }
        const int local = item - __ldg(a.prefix + lo);
        const ST *fin = static_cast<const ST *>(D.f[a.parity]);
        ST *fout = static_cast<ST *>(const_cast<void *>(D.f[a.parity ^ 1]));
        const uint32_t step = __ldg(a.step0 + lo) + (uint32_t)a.k;
        if (!run_item_x2<ST, MODE, FORCED>(w, p, &D.tload[a.parity], fin, fout, local % p.nstrips,
                                           local / p.nstrips, step)) {
            abort = true;
            break;
        }
    }
    warp_end_x2<ST>(w, abort, a.error, a.work);
}

// Grid-wide barrier of a cooperative launch, with bounded waits.  Thread 0 of
// every block arrives once, after all warps of the block are done; the last
// arrival resets the arrival count and *reset (an item counter that the next
// step but one uses), then releases the others by advancing the generation.
// A wait longer than twice the bounded TMA wait raises the error flag and
// gives up.  Returns false when the launch must stop (a wait gave up here, or
// any warp raised the flag before arriving).  ctl[2] = arrivals, ctl[3] =
// generation.
__device__ __forceinline__ bool grid_barrier_bounded(unsigned int *ctl, unsigned int *reset, int *error)
{
    __shared__ int go;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // this block's stores before its arrival
        const unsigned int g = *reinterpret_cast<volatile unsigned int *>(ctl + 3);
        int ok = 1;
        if (atomicAdd(ctl + 2, 1u) == gridDim.x - 1) {
            atomicExch(ctl + 2, 0u);
            atomicExch(reset, 0u);
            __threadfence();
            atomicAdd(ctl + 3, 1u);
        } else {
            const unsigned long long t0 = globaltimer();
            while (*reinterpret_cast<volatile unsigned int *>(ctl + 3) == g)
                if (globaltimer() - t0 > 2 * WAIT_LIMIT_NS) {
                    atomicExch(error, 1);
                    ok = 0;
                    break;
                }
        }
        __threadfence();
        go = ok && *reinterpret_cast<volatile int *>(error) == 0;
    }
    __syncthreads();
    return go != 0;
}

// Persistent form of the batch kernel: steps k0 .. k0 + nsteps - 1 of a tick in
// one cooperative launch (every block resident), a grid barrier between steps.
// Each step hands out the items of the active domains (of one force variant)
// from its own counter, ctl[k & 1]; a domain's arithmetic per step is that of
// stream_collide_x2_batch_kernel, so the results are the same bit for bit.
// After the barrier every thread orders the generic-proxy stores of the step
// before the async-proxy (TMA) loads of the next.
template <typename ST, int MODE, bool FORCED>
__global__ void __launch_bounds__(THREADS, FORCED ? MIN_BLOCKS_BATCH_X2 : MIN_BLOCKS_X2)
stream_collide_x2_batch_persistent_kernel(const __grid_constant__ BatchArgs a, int k0, int nsteps)
{
    using T = Tile2<ST>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ StepParams sp[WARPS];
    StepParams &p = sp[threadIdx.x >> 5];
    WarpCtx w;
    warp_begin_x2<ST>(w, smem);
    unsigned int *ctl = a.ctl;
    const int first = FORCED ? a.state->split_items : 0;
    const int end = FORCED ? a.state->total_items : a.state->split_items;
    const int n_active = a.state->n_active;
    bool abort = false;
    for (int k = k0; k < k0 + nsteps; ++k) {
        const int parity = (a.parity + k) & 1;
        unsigned int *work = ctl + (k & 1);
        int last_slot = -1;
        for (int item = abort ? end : first + next_item(w, work); item < end; item = first + next_item(w, work)) {
            int lo = 0, hi = n_active;  // prefix[lo] <= item < prefix[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(a.prefix + mid) <= item) lo = mid;
                else hi = mid;
            }
            const int slot = __ldg(a.active + lo);
            const DomainDesc &D = a.domains[slot];
            if (slot != last_slot) {
                tensormap_acquire(&D.tload[parity]);
                copy_params(p, D.p, w.lane);
                last_slot = slot;
            }
            const int local = item - __ldg(a.prefix + lo);
            const ST *fin = static_cast<const ST *>(D.f[parity]);
            ST *fout = static_cast<ST *>(const_cast<void *>(D.f[parity ^ 1]));
            const uint32_t step = __ldg(a.step0 + lo) + (uint32_t)k;
            if (!run_item_x2<ST, MODE, FORCED>(w, p, &D.tload[parity], fin, fout, local % p.nstrips,
                                               local / p.nstrips, step)) {
                abort = true;
                if (w.lane == 0) atomicExch(a.error, 1);
                break;
            }
        }
        if (!grid_barrier_bounded(ctl, ctl + ((k + 1) & 1), a.error)) {
            abort = true;
            break;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    if (abort && w.lane == 0) {
        // let this warp's copies in flight land before the shared memory goes away
        for (int j = max(0, w.issued - T::NSLOT); j < w.issued; ++j) {
            const uint32_t q = w.q_base + (uint32_t)j;
            if (!mbar_wait_bounded(w.bars_u32 + 8 * (q % T::NSLOT), (q / T::NSLOT) & 1u)) break;
        }
    }
    __syncwarp();
}

template <typename KernelFn>
int occupancy_of(KernelFn fn, int smem)
{
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, THREADS, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

}  // namespace lbm

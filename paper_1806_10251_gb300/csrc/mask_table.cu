// Host code: the row table of a solid mask (the device layout that
// StepParams::solid points to: the mask, then its table).  Plain C++ (no CUDA
// constructs), so that it builds with the host compiler alone as well.
#include <stdint.h>
#include <string.h>

#include <vector>

namespace lbm {
std::vector<uint8_t> make_solid_rows(const uint8_t *mask, int nx, int ny, bool perx, bool pery);
std::vector<uint8_t> mask_with_row_table(const uint8_t *mask, int nx, int ny, int pitch, bool perx, bool pery);
}  // namespace lbm

// The row table of a mask: for each row r and 32-column block b, whether a solid cell lies in
// rows r - 1 .. r + 1 and columns 32 b - 34 .. 32 b + 65 (blocks b - 1 .. b + 1
// with the two columns each way that a strip's halo pulls reach); periodic
// sides wrap, wall sides clip.  Row prefix sums answer each range.
std::vector<uint8_t> lbm::make_solid_rows(const uint8_t *mask, int nx, int ny, bool perx, bool pery)
{
    const int nb = (nx + 31) / 32;
    std::vector<int> pre((size_t)ny * (nx + 1), 0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            pre[(size_t)y * (nx + 1) + x + 1] = pre[(size_t)y * (nx + 1) + x] + (mask[(size_t)y * nx + x] != 0);
    auto count = [&](int y, int a, int b) -> int {  // solids of row y in columns a .. b (a <= b)
        if (perx) {
            if (b - a + 1 >= nx) return pre[(size_t)y * (nx + 1) + nx];
            int aw = ((a % nx) + nx) % nx, bw = ((b % nx) + nx) % nx;
            if (aw <= bw) return pre[(size_t)y * (nx + 1) + bw + 1] - pre[(size_t)y * (nx + 1) + aw];
            return pre[(size_t)y * (nx + 1) + nx] - pre[(size_t)y * (nx + 1) + aw] + pre[(size_t)y * (nx + 1) + bw + 1];
        }
        a = a < 0 ? 0 : a;
        b = b >= nx ? nx - 1 : b;
        return a > b ? 0 : pre[(size_t)y * (nx + 1) + b + 1] - pre[(size_t)y * (nx + 1) + a];
    };
    std::vector<uint8_t> out((size_t)ny * nb, 0);
    for (int y = 0; y < ny; ++y)
        for (int b = 0; b < nb; ++b) {
            int n = 0;
            for (int dy = -1; dy <= 1 && !n; ++dy) {
                int yy = y + dy;
                if (pery) yy = (yy + ny) % ny;
                if (yy < 0 || yy >= ny) continue;
                n += count(yy, 32 * b - 34, 32 * b + 65);
            }
            out[(size_t)y * nb + b] = n ? 1 : 0;
        }
    return out;
}

std::vector<uint8_t> lbm::mask_with_row_table(const uint8_t *mask, int nx, int ny, int pitch, bool perx, bool pery)
{
    const std::vector<uint8_t> rows = make_solid_rows(mask, nx, ny, perx, pery);
    std::vector<uint8_t> h((size_t)pitch * ny + rows.size(), 0);
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) h[(size_t)y * pitch + x] = mask[(size_t)y * nx + x] ? 1 : 0;
    memcpy(h.data() + (size_t)pitch * ny, rows.data(), rows.size());
    return h;
}


// Grid geometry and the packed-gradient word layout (no CUDA runtime dependency, so the
// same definitions compile for host and device code).
#pragma once

#include <stdint.h>

namespace msc {

constexpr uint32_t NONE = 0xFFFFFFFFu;

// Exact unsigned 32-bit division by a divisor fixed at plan time, as a multiply-high and
// shifts (the round-up method of Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> 1)) >> (l - 1) where t = mulhi(n, m); d = 1 is passed through.
struct FastDiv {
    uint32_t d = 1, m = 0, s = 0;
    FastDiv() = default;
    explicit FastDiv(uint32_t div) : d(div) {
        if (div <= 1) return;
        uint32_t l = 0;
        while ((uint64_t(1) << l) < div) ++l;
        m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << l) - div)) / div + 1);
        s = l - 1;
    }
    __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
        if (d == 1) return n;
#ifdef __CUDA_ARCH__
        const uint32_t t = __umulhi(n, m);
#else
        const uint32_t t = uint32_t((uint64_t(n) * m) >> 32);
#endif
        return (t + ((n - t) >> 1)) >> s;
    }
};

// ---- grid geometry ---------------------------------------------------------------------
// Vertex (x,y,z) has index x + nx*(y + ny*z).  Cells live on the refined grid
// (2nx-1)x(2ny-1)x(2nz-1).  Vertex (x,y,z) owns the 8 cells (2x+a, 2y+b, 2z+c).
struct Geom {
    int nx, ny, nz;
    int W;            // 32-bit words per bitmap row: ceil(nx / 32)
    int64_t nverts;
    uint32_t rx, ry;  // refined extents along x and y (for cell ids)
    FastDiv div_nx, div_ny, div_rx, div_ry, div_W;  // divisions by nx, ny, rx, ry, W (index decoding)

    // Fills the derived fields from nx, ny, nz.
    void finish() {
        W = (nx + 31) / 32;
        nverts = int64_t(nx) * ny * nz;
        rx = uint32_t(2 * nx - 1);
        ry = uint32_t(2 * ny - 1);
        div_nx = FastDiv(uint32_t(nx));
        div_ny = FastDiv(uint32_t(ny));
        div_rx = FastDiv(rx);
        div_ry = FastDiv(ry);
        div_W = FastDiv(uint32_t(W));
    }

    __host__ __device__ uint32_t cell_id(int cx, int cy, int cz) const {
        return uint32_t(cx) + rx * (uint32_t(cy) + ry * uint32_t(cz));
    }
    __host__ __device__ int64_t vid(int x, int y, int z) const {
        return int64_t(x) + int64_t(nx) * (int64_t(y) + int64_t(ny) * int64_t(z));
    }
    // Row-bitmap layout used for per-slot bitmaps: [slot][z][y][w]
    __host__ __device__ int64_t slot_word(int s, int z, int y, int w) const {
        return ((int64_t(s) * nz + z) * ny + y) * W + w;
    }
    __host__ __device__ int64_t slot_words() const { return int64_t(8) * nz * ny * W; }
    // 1-cell row layout: word (((z*2 + c)*ny + y)*2 + b)*W + w for the 1-cell
    // (2x+a, 2y+b, 2z+c), a = 1-b-c.
    __host__ __device__ int64_t edge_word(int z, int c, int y, int b, int w) const {
        return (((int64_t(z) * 2 + c) * ny + y) * 2 + b) * W + w;
    }
    __host__ __device__ int64_t edge_words() const { return int64_t(4) * nz * ny * W; }
};

// Decoded 3-bit codes of the packed gradient word (see msc.h).
__host__ __device__ __forceinline__ uint32_t slot_code(uint32_t word, int s) { return (word >> (3 * s)) & 7u; }

}  // namespace msc

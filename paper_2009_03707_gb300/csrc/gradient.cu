// (a1) Lower-star discrete gradient + (a2, first half) critical-cell bitmaps.
//
// Sec. 3 / Sec. 3.5 "Gradient pairs and critical points" of arXiv:2009.03707: every cell is
// paired with a facet or cofacet or left critical.  The rule is the lower-star pairing of
// Robins, Wood and Sheppard (2011, cited in Sec. 1.1): the cells whose maximal vertex is x
// (the lower star L(x)) are paired among themselves, so every vertex is independent work.
//
// GB300 design (not the paper's texture-object kernel):
//  * One CTA owns a 32 x 8 x 8 tile of vertices.  The field tile plus a (-1,+2) halo is
//    staged in shared memory as order-preserving uint32 keys.  The CTA computes the lower
//    stars of the tile plus one layer on the + side (a cell is owned by its lowest corner
//    vertex but decided by its highest one) and ORs 3-bit codes into shared words.
//  * A lower star is handled as 27-bit masks over the offsets d in {-1,0,1}^3: membership
//    (all sub-offsets lower), facets / cofacets (one component cleared / set), classified,
//    and the two priority queues.  Cell keys are rank bitmasks: with the vertices of L(x)
//    ranked, the key of a cell is the OR of its vertices' rank bits, and comparing these
//    integers is exactly the lexicographic comparison of the vertices sorted downwards.
//  * The epilogue writes the packed words with coalesced 128-byte rows, and one warp ballot
//    per slot turns 32 vertices into one 32-bit word of the critical-cell bitmap of that
//    slot -- the input of the ordered compaction (critical.cu).
#include "lower_star.cuh"
#include "msc_internal.cuh"

namespace msc {

namespace {

constexpr int TX = 32, TY = 8, TZ = 8;               // owned tile
constexpr int EX = TX + 1, EY = TY + 1, EZ = TZ + 1;  // lower stars computed (tile + 1 on + side)
constexpr int FX = TX + 3, FY = TY + 3, FZ = TZ + 3;  // field keys staged (x0-1 .. x0+TX+1)
constexpr int THREADS = 256;
constexpr uint32_t OUTSIDE_KEY = 0xFFFFFFFFu;

using star::pdx;
using star::pdy;
using star::pdz;

// Monotone map float -> uint32 (IEEE order; -0 and +0 map to the same key).
__device__ __forceinline__ uint32_t order_key(float f) {
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7fffffffu) == 0) u = 0;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

constexpr int NEXT = EX * EY * EZ;  // vertices whose lower stars a CTA computes

struct Shared {
    uint32_t fkey[FZ][FY][FX];   // order keys of the field tile (OUTSIDE_KEY off-grid)
    uint32_t words[TZ][TY][TX];  // packed codes of the owned tile
    uint32_t vkey[27][THREADS];  // per-thread scratch: keys of the star's vertices
    uint32_t ckey[27][THREADS];  // per-thread scratch: rank-bitmask keys of the star's cells
    uint16_t order[NEXT];        // non-minimal vertices, grouped by lower-star size
    uint8_t size[NEXT];          // |L(x)| - 1 of every vertex (0 for minima and off-grid)
    int bin[28];                 // counting-sort bins by size
};

// The 27 order keys of the star of the vertex at tile-local (lx,ly,lz).
__device__ __forceinline__ void star_keys(const Shared& sh, int lx, int ly, int lz, uint32_t (&k)[27]) {
#pragma unroll
    for (int p = 0; p < 27; ++p) k[p] = sh.fkey[lz + 1 + pdz(p)][ly + 1 + pdy(p)][lx + 1 + pdx(p)];
}

__global__ void __launch_bounds__(THREADS) gradient_kernel(Geom g, const float* __restrict__ field,
                                                           uint32_t* __restrict__ words_out,
                                                           uint32_t* __restrict__ crit_bits,
                                                           uint32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Shared& sh = *reinterpret_cast<Shared*>(smem_raw);
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;

    for (int i = t; i < TX * TY * TZ; i += THREADS) (&sh.words[0][0][0])[i] = 0;
    bool saw_nan = false;
    for (int i = t; i < FX * FY * FZ; i += THREADS) {
        int fx = i % FX, fy = (i / FX) % FY, fz = i / (FX * FY);
        int gx = x0 - 1 + fx, gy = y0 - 1 + fy, gz = z0 - 1 + fz;
        uint32_t key = OUTSIDE_KEY;
        if (gx >= 0 && gy >= 0 && gz >= 0 && gx < g.nx && gy < g.ny && gz < g.nz) {
            float v = __ldg(field + g.vid(gx, gy, gz));
            saw_nan |= isnan(v);
            key = order_key(v);
        }
        sh.fkey[fz][fy][fx] = key;
    }
    if (saw_nan) atomicOr(status, ST_NAN);
    __syncthreads();

    // Lower stars differ widely in size (1..27 cells), and a warp runs as long as its largest
    // one.  So first size every star (cheap mask arithmetic), counting-sort the non-minimal
    // vertices by size, and let consecutive threads take consecutive entries.
    if (t < 28) sh.bin[t] = 0;
    __syncthreads();
    for (int i = t; i < NEXT; i += THREADS) {
        const int lx = i % EX, ly = (i / EX) % EY, lz = i / (EX * EY);
        int m = 0;
        if (x0 + lx < g.nx && y0 + ly < g.ny && z0 + lz < g.nz) {
            uint32_t k[27];
            star_keys(sh, lx, ly, lz, k);
            m = __popc(star::lower_star_mask(star::lower_mask(k))) - 1;
        }
        sh.size[i] = uint8_t(m);
        if (m > 0) atomicAdd(&sh.bin[m], 1);
    }
    __syncthreads();
    if (t == 0) {
        int acc = 0;
        for (int m = 27; m >= 1; --m) {  // largest stars first
            const int c = sh.bin[m];
            sh.bin[m] = acc;
            acc += c;
        }
        sh.bin[0] = acc;  // number of non-minimal vertices
    }
    __syncthreads();
    for (int i = t; i < NEXT; i += THREADS) {
        const int m = sh.size[i];
        if (m > 0) sh.order[atomicAdd(&sh.bin[m], 1)] = uint16_t(i);
    }
    __syncthreads();
    const int n_items = sh.bin[0];

    bool ok = true;
    const star::Scratch sc{&sh.vkey[0][t], &sh.ckey[0][t], THREADS};
    for (int it = t; it < n_items; it += THREADS) {
        const int i = sh.order[it];
        const int lx = i % EX, ly = (i / EX) % EY, lz = i / (EX * EY);
        uint32_t k[27];
        star_keys(sh, lx, ly, lz, k);
        // a cell is owned by its lowest corner vertex: record its code there if that vertex
        // belongs to this CTA's tile
        auto emit = [&](int p, uint32_t code) {
            const int dx = pdx(p), dy = pdy(p), dz = pdz(p);
            const int ox = lx + (dx < 0 ? -1 : 0), oy = ly + (dy < 0 ? -1 : 0), oz = lz + (dz < 0 ? -1 : 0);
            if (ox < 0 || oy < 0 || oz < 0 || ox >= TX || oy >= TY || oz >= TZ) return;
            const int slot = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
            atomicOr(&sh.words[oz][oy][ox], code << (3 * slot));
        };
        ok &= star::process_lower_star(k, sc, emit);
    }
    if (!ok) atomicOr(status, ST_INTERNAL);
    __syncthreads();

    // epilogue: packed words + per-slot critical bitmaps (one ballot per slot and row)
    const int lane = t & 31, warp = t >> 5;
    const int gx = x0 + lane;
    for (int r = warp; r < TY * TZ; r += THREADS / 32) {
        const int ly = r % TY, lz = r / TY;
        const int gy = y0 + ly, gz = z0 + lz;
        if (gy >= g.ny || gz >= g.nz) continue;  // warp-uniform
        const bool valid = gx < g.nx;
        uint32_t w = sh.words[lz][ly][lane];
        // slots beyond the far boundary hold code 7
        for (int s = 0; s < 8; ++s) {
            bool out = ((s & 1) && gx == g.nx - 1) || ((s & 2) && gy == g.ny - 1) || ((s & 4) && gz == g.nz - 1);
            if (out) w |= 7u << (3 * s);
        }
        if (valid) words_out[g.vid(gx, gy, gz)] = w;
        uint32_t mine = 0;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            uint32_t bits = __ballot_sync(0xFFFFFFFFu, valid && slot_code(w, s) == 0);
            if (lane == s) mine = bits;
        }
        if (lane < 8) crit_bits[g.slot_word(lane, gz, gy, x0 >> 5)] = mine;
    }
}

}  // namespace

msc_status run_gradient(Plan* p, const float* d_field, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    if ((st = ensure(p, p->words, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->crit_bits, sizeof(uint32_t) * size_t(g.slot_words())))) return st;
    const size_t smem = sizeof(Shared);
    // set on every call: the attribute is per device, and plans may live on several devices
    if ((st = check_cuda(p, cudaFuncSetAttribute(gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(smem)),
                         "cudaFuncSetAttribute(gradient)")))
        return st;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
    gradient_kernel<<<grid, THREADS, smem, s>>>(g, d_field, static_cast<uint32_t*>(p->words.ptr),
                                                static_cast<uint32_t*>(p->crit_bits.ptr),
                                                static_cast<uint32_t*>(p->status.ptr));
    launched(p);
    return check_cuda(p, cudaGetLastError(), "gradient_kernel launch");
}

// Launch of the same kernel on caller-supplied buffers, with no plan and no allocation (used by
// the no-allocation entry point, static_entry.cu).
cudaError_t launch_gradient_raw(const Geom& g, const float* d_field, uint32_t* words, uint32_t* crit_bits,
                                uint32_t* status, cudaStream_t s) {
    const size_t smem = sizeof(Shared);
    cudaError_t e = cudaFuncSetAttribute(gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + TZ - 1) / TZ);
    gradient_kernel<<<grid, THREADS, smem, s>>>(g, d_field, words, crit_bits, status);
    return cudaGetLastError();
}

}  // namespace msc

// Host harness for tests only: runs the kernel's lower-star core (lower_star.cuh) on the CPU,
// one vertex at a time, and assembles the packed gradient words of a whole grid.
#include <cstdint>
#include <cstring>

#define __host__
#define __device__
#define __forceinline__ inline
#include "../../paper_2009_03707_gb300/csrc/lower_star.cuh"

using namespace msc::star;

static uint32_t order_key(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) == 0) u = 0;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

extern "C" int host_words(const int64_t* d, const float* f, uint32_t* words) {
    const int nx = int(d[0]), ny = int(d[1]), nz = int(d[2]);
    std::memset(words, 0, sizeof(uint32_t) * size_t(nx) * ny * nz);
    Tables T;
    for (int p = 0; p < 27; p++) fill_tables(T, p, 3, 9);
    int bad = 0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                uint32_t k[27];
                for (int p = 0; p < 27; p++) {
                    const int X = x + pdx(p), Y = y + pdy(p), Z = z + pdz(p);
                    const bool out = X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz;
                    k[p] = out ? 0xFFFFFFFFu : order_key(f[X + nx * (Y + ny * Z)]);
                }
                auto emit = [&](int p, uint32_t code) {
                    const int dx = pdx(p), dy = pdy(p), dz = pdz(p);
                    const int ox = x + (dx < 0 ? -1 : 0), oy = y + (dy < 0 ? -1 : 0), oz = z + (dz < 0 ? -1 : 0);
                    const int slot = (dx != 0) | ((dy != 0) << 1) | ((dz != 0) << 2);
                    words[ox + nx * (oy + ny * oz)] |= code << (3 * slot);
                };
                if (!process_lower_star(k, &T, emit)) bad++;
            }
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                for (int s = 0; s < 8; s++) {
                    const bool out = ((s & 1) && x == nx - 1) || ((s & 2) && y == ny - 1) || ((s & 4) && z == nz - 1);
                    if (out) words[x + nx * (y + ny * z)] |= 7u << (3 * s);
                }
    return bad;
}

// The bit-parallel "exactly one unclassified facet" test of the core against its definition (a
// popcount of the cell's facet mask) for every cell position and every one of `n` free-cell sets
// drawn from a fixed 64-bit LCG; returns the number of disagreements.
extern "C" int host_one_free_facet_mismatches(int n) {
    Tables T;
    for (int p = 0; p < 27; p++) fill_tables(T, p, 3, 9);
    uint64_t s = 0x9E3779B97F4A7C15ull;
    int bad = 0;
    for (int i = 0; i < n; i++) {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const uint32_t free = uint32_t(s >> 37) & ALL;
        const uint32_t m = one_free_facet_mask(free);
        for (int q = 0; q < 27; q++) {
            const bool want = __builtin_popcount(T.facet[q] & free) == 1;
            if (bool((m >> q) & 1u) != want) bad++;
        }
    }
    return bad;
}

// The least edge by vertex keys against the general least-cell rule, on random keys (with many
// ties) and random non-empty sets of edges; returns the number of disagreements.
extern "C" int host_edge_min_mismatches(int n) {
    Tables T;
    for (int p = 0; p < 27; p++) fill_tables(T, p, 3, 9);
    uint64_t s = 0x243F6A8885A308D3ull;
    int bad = 0;
    for (int i = 0; i < n; i++) {
        uint32_t k[27];
        for (int p = 0; p < 27; p++) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            k[p] = (i & 1) ? uint32_t(s >> 61) : uint32_t(s >> 32);  // odd rounds: keys 0..7
        }
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        const uint32_t edges = uint32_t(s >> 40) & DIM1;
        if (!edges) continue;
        const Star st{k + CENTER, &T};
        if (pop_min_edge(edges, st) != pop_min(edges, st)) bad++;
    }
    return bad;
}

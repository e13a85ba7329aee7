// Lower-star pairing of one vertex (a1) on 27-bit masks; host+device so the same code can
// be exercised on the CPU.
//
// The star of vertex x is indexed by position p = 9*(dz+1) + 3*(dy+1) + (dx+1) of the offset
// d in {-1,0,1}^3 of the cell 2x+d on the refined grid (p = 13 is x itself).  The vertex at
// offset d has the same position index.  The rule is ProcessLowerStars (Robins, Wood and
// Sheppard 2011, the locally independent gradient the paper cites in Sec. 1.1 and uses in
// Sec. 3): x is paired with its lowest edge; cells of the lower star with exactly one
// unclassified facet wait in queue "one", the others in queue "zero"; "one" is drained first
// (pairing each popped cell with its free facet), then the least cell of "zero" becomes
// critical; a popped cell that is already classified is skipped.
//
// Everything is a 27-bit mask: membership in L(x) (a cell is in L(x) iff all its vertices
// other than x are lower, i.e. every sub-offset is lower), facets through x (clear one
// non-zero component), cofacets (set one zero component), a cell's vertex set (its
// sub-offsets), the classified set and both queues.  Two cells are compared by their vertex
// lists sorted downwards, lexicographically: the cell whose vertex set holds the largest vertex
// of the symmetric difference is the larger one (a proper prefix is therefore smaller), so a
// comparison costs one key lookup per vertex in the symmetric difference and no ranking.
#pragma once

#include <stdint.h>

#ifdef __CUDA_ARCH__
#define MSC_FFS(x) __ffs(x)
#define MSC_POPC(x) __popc(x)
#else
#define MSC_FFS(x) __builtin_ffs(int(x))
#define MSC_POPC(x) __builtin_popcount(x)
#endif

namespace msc {
namespace star {

constexpr int CENTER = 13;
constexpr uint32_t ALL = 0x7FFFFFFu;
// positions with dx = -1 / 0 / +1, dy = -1 / 0 / +1, dz = -1 / 0 / +1
constexpr uint32_t XN = 0x1249249u, XZ = XN << 1, XP = XN << 2;
constexpr uint32_t YN = 0x1C0E07u, YZ = YN << 3, YP = YN << 6;
constexpr uint32_t ZN = 0x1FFu, ZZ = ZN << 9, ZP = ZN << 18;
constexpr uint32_t DIM1 = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
constexpr uint32_t DIM3 =
    (1u << 0) | (1u << 2) | (1u << 6) | (1u << 8) | (1u << 18) | (1u << 20) | (1u << 24) | (1u << 26);
constexpr uint32_t DIM2 = ALL & ~DIM1 & ~DIM3 & ~(1u << CENTER);

__host__ __device__ constexpr int pdx(int p) { return p % 3 - 1; }
__host__ __device__ constexpr int pdy(int p) { return (p / 3) % 3 - 1; }
__host__ __device__ constexpr int pdz(int p) { return p / 9 - 1; }

__host__ __device__ constexpr uint32_t facet_mask(int p) {
    return (pdx(p) ? 1u << (p - pdx(p)) : 0u) | (pdy(p) ? 1u << (p - 3 * pdy(p)) : 0u) |
           (pdz(p) ? 1u << (p - 9 * pdz(p)) : 0u);
}
__host__ __device__ constexpr uint32_t cofacet_mask(int p) {
    return (pdx(p) ? 0u : (1u << (p - 1)) | (1u << (p + 1))) | (pdy(p) ? 0u : (1u << (p - 3)) | (1u << (p + 3))) |
           (pdz(p) ? 0u : (1u << (p - 9)) | (1u << (p + 9)));
}

// 3-bit direction code of the partner at position q seen from the cell at position p:
// q - p = -1, +1, -3, +3, -9, +9 gives 1..6 (axis x, y, z; - side first).
__host__ __device__ inline uint32_t dir_code(int p, int q) {
    const int d = q - p;
    const int ad = d < 0 ? -d : d;
    return 1u + 2u * (uint32_t(ad > 1) + uint32_t(ad > 3)) + uint32_t(d > 0);
}

// Cells of the star in L(x): AND of the "lower" mask over every projection of the offset.
__host__ __device__ inline uint32_t lower_star_mask(uint32_t lower_with_center) {
    uint32_t m = lower_with_center;
    m &= ((m >> 1) & XN) | ((m << 1) & XP) | XZ;
    m &= ((m >> 3) & YN) | ((m << 3) & YP) | YZ;
    m &= ((m >> 9) & ZN) | ((m << 9) & ZP) | ZZ;
    return m & ALL;
}

// The vertices of the cell at position p (other than x): the positions q whose every
// component is 0 or equal to p's.
__host__ __device__ inline uint32_t cell_vertices(int p) {
    const uint32_t xs = XZ | (XN & (0u - ((XN >> p) & 1u))) | (XP & (0u - ((XP >> p) & 1u)));
    const uint32_t ys = YZ | (YN & (0u - ((YN >> p) & 1u))) | (YP & (0u - ((YP >> p) & 1u)));
    const uint32_t zs = ZZ | (ZN & (0u - ((ZN >> p) & 1u))) | (ZP & (0u - ((ZP >> p) & 1u)));
    return xs & ys & zs & ~(1u << CENTER);
}

// Per-position masks, tabulated once per CTA (shared memory on the device): a 27-entry table of
// 32-bit words sits in 27 distinct banks, so divergent lanes read it without conflicts.  off[p]
// is where the key of the vertex at position p sits relative to the key of x in the caller's
// key array (on the device: the CTA's staged field tile).
struct Tables {
    uint32_t cellv[27];
    uint32_t facet[27];
    uint32_t cofacet[27];
    int off[27];
};

__host__ __device__ inline void fill_tables(Tables& T, int p, int row, int plane) {
    T.cellv[p] = cell_vertices(p);
    T.facet[p] = facet_mask(p);
    T.cofacet[p] = cofacet_mask(p);
    T.off[p] = pdx(p) + row * pdy(p) + plane * pdz(p);
}

// One lower star: the key of x and the tables; key(p) is the order key of the vertex at p.
struct Star {
    const uint32_t* center;
    const Tables* T;
    __host__ __device__ uint32_t key(int p) const { return center[T->off[p]]; }
};

// True if the cell at position a is smaller than the one at b (a != b): the larger one owns
// the largest vertex (key, then position) of the symmetric difference of their vertex sets.
__host__ __device__ __forceinline__ bool cell_less(int a, int b, const Star& st) {
    const uint32_t vb = st.T->cellv[b];
    uint32_t d = st.T->cellv[a] ^ vb;
    int w = MSC_FFS(d) - 1;
    uint32_t kw = st.key(w);
    d &= d - 1;
    while (d) {  // ascending positions: on equal keys the later position wins
        const int q = MSC_FFS(d) - 1;
        d &= d - 1;
        const uint32_t kq = st.key(q);
        if (kq >= kw) {
            kw = kq;
            w = q;
        }
    }
    return (vb >> w) & 1u;
}

__host__ __device__ __forceinline__ int pop_min(uint32_t mask, const Star& st) {
    int best = MSC_FFS(mask) - 1;
    mask &= mask - 1;
    while (mask) {
        const int p = MSC_FFS(mask) - 1;
        mask &= mask - 1;
        if (cell_less(p, best, st)) best = p;
    }
    return best;
}

// The least edge of a non-empty set of edges (positions with one non-zero component): an edge's
// only vertex other than x is the one at its own position, so edges compare as their vertices do
// (key, then position).
__host__ __device__ __forceinline__ int pop_min_edge(uint32_t mask, const Star& st) {
    int best = MSC_FFS(mask) - 1;
    uint32_t kb = st.key(best);
    mask &= mask - 1;
    while (mask) {  // ascending positions: a later position wins only with a smaller key
        const int p = MSC_FFS(mask) - 1;
        mask &= mask - 1;
        const uint32_t kp = st.key(p);
        if (kp < kb) {
            kb = kp;
            best = p;
        }
    }
    return best;
}

// The positions whose cell has exactly one facet (through x) in `free`, for all 27 at once: a
// cell's facet along an axis on which its offset is d = +-1 sits one step back towards 0 on that
// axis (position p - d, p - 3d, p - 9d), so a shift of `free` by 1, 3 or 9 brings each facet's bit
// to its cofacet's position; the result is "exactly one of the three".
__host__ __device__ __forceinline__ uint32_t one_free_facet_mask(uint32_t free) {
    const uint32_t fx = ((free << 1) & XP) | ((free >> 1) & XN);
    const uint32_t fy = ((free << 3) & YP) | ((free >> 3) & YN);
    const uint32_t fz = ((free << 9) & ZP) | ((free >> 9) & ZN);
    return (fx ^ fy ^ fz) & ~((fx & fy) | (fz & (fx | fy)));
}

// Bit p set iff the vertex at position p is lower than x (value, then index; the index order
// of the star's vertices is the order of their positions).  Bit 13 (x itself) is set too.
__host__ __device__ inline uint32_t lower_mask(const uint32_t* k) {
    const uint32_t kc = k[CENTER];
    uint32_t lower = 1u << CENTER;
#pragma unroll
    for (int p = 0; p < 27; ++p) {
        if (p == CENTER) continue;
        const bool lo = (k[p] < kc) || (k[p] == kc && p < CENTER);
        lower |= uint32_t(lo) << p;
    }
    return lower;
}

// Pairs the cells of L(x) given inL (the lower-star mask, with more than x in it); st.key(p)
// must be valid for every p in inL.  Vertices with equal keys are ordered by position, which
// is their index order.  emit(p, code) is called for every non-critical cell with its
// direction code.  Returns false if the procedure did not classify every cell (an internal
// error).
template <class Emit>
__host__ __device__ __forceinline__ bool pair_lower_star(const uint32_t inL, const Star& st, Emit&& emit) {
    const Tables* T = st.T;
    const int delta = pop_min_edge(inL & DIM1, st);
    uint32_t cls = (1u << CENTER) | (1u << delta);
    emit(CENTER, dir_code(CENTER, delta));
    emit(delta, dir_code(delta, CENTER));
    uint32_t pq0 = inL & DIM1 & ~(1u << delta);
    // cofacets (in L(x), unclassified) of a newly classified cell with one unclassified facet
    uint32_t pq1 = T->cofacet[delta] & inL & ~cls & one_free_facet_mask(inL & ~cls);
    for (int guard = 0; guard < 64; ++guard) {
        while (pq1) {
            int a = pop_min(pq1, st);
            pq1 &= ~(1u << a);
            if (cls & (1u << a)) continue;
            uint32_t uf = T->facet[a] & inL & ~cls;
            if (uf == 0) {
                pq0 |= 1u << a;
                continue;
            }
            int pf = MSC_FFS(uf) - 1;  // the only unclassified facet
            cls |= (1u << pf) | (1u << a);
            pq0 &= ~(1u << pf);
            emit(pf, dir_code(pf, a));
            emit(a, dir_code(a, pf));
            pq1 |= (T->cofacet[a] | T->cofacet[pf]) & inL & ~cls & one_free_facet_mask(inL & ~cls);
        }
        if (!pq0) return cls == inL;
        int c0 = pop_min(pq0, st);
        pq0 &= ~(1u << c0);
        if (cls & (1u << c0)) continue;
        cls |= 1u << c0;  // critical
        pq1 |= T->cofacet[c0] & inL & ~cls & one_free_facet_mask(inL & ~cls);
    }
    return false;
}

// Pairs the cells of L(x) given the 27 vertex order keys k[] (k[13] = x; an off-grid vertex
// has key 0xFFFFFFFF) and tables filled with row = 3, plane = 9.  See pair_lower_star.
template <class Emit>
__host__ __device__ bool process_lower_star(const uint32_t* k, const Tables* T, Emit&& emit) {
    const uint32_t inL = lower_star_mask(lower_mask(k));
    if (inL == (1u << CENTER)) return true;  // a minimum: every code stays 0
    return pair_lower_star(inL, Star{k + CENTER, T}, emit);
}

}  // namespace star
}  // namespace msc

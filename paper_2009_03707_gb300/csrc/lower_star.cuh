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
// The queues are not kept.  A cell enters "one" when one of its facets is classified and it
// is left with exactly one unclassified facet, and the number of unclassified facets only
// falls; a popped cell whose count has reached zero moves to "zero"; and edges sit in "zero"
// from the start.  So whenever "one" is drained, "zero" holds exactly the unclassified cells
// with no unclassified facet, and the live part of "one" is exactly the unclassified cells with
// one.  The procedure is therefore: pair the least unclassified cell that has exactly one
// unclassified facet with that facet; if there is none, declare the least unclassified cell
// with no unclassified facet critical; repeat.  The counts are kept as two bit planes (a 2-bit
// counter per position), so each step is a few mask operations and one "least cell of a set".
//
// Everything is a 27-bit mask: membership in L(x) (a cell is in L(x) iff all its vertices
// other than x are lower, i.e. every sub-offset is lower), facets through x (clear one
// non-zero component), cofacets (set one zero component), a cell's vertex set (its
// sub-offsets) and the unclassified set.  Two cells are compared by their vertex lists sorted
// downwards, lexicographically.  Two ways of finding the least cell of a set give the same
// answer:
//  * small stars compare two cells directly: the cell whose vertex set holds the largest vertex
//    of the symmetric difference is the larger one (a proper prefix is therefore smaller);
//  * large stars first rank the vertices of L(x) once (a sorting network over the packed
//    keys), give every cell the integer key "OR of 1 << rank over its vertices" -- comparing
//    those integers is exactly the lexicographic order above -- and take minima of integers.
// The vertices of L(x) other than x correspond one to one to its cells other than x (the cell
// at position p is in L(x) iff the vertex at p and every sub-offset of p are lower), so a
// star with m cells besides x has m vertices to rank.
#pragma once

#include <stdint.h>

#ifdef __CUDA_ARCH__
#define MSC_FFS(x) __ffs(x)
#define MSC_POPC(x) __popc(x)
#define MSC_UMIN(a, b) min(a, b)
#else
#define MSC_FFS(x) __builtin_ffs(int(x))
#define MSC_POPC(x) __builtin_popcount(x)
#define MSC_UMIN(a, b) ((a) < (b) ? (a) : (b))
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

// Emits the pair (p, q) of neighbouring positions: each cell gets the 3-bit direction code of
// the other, 1..6 for the partner at -1, +1, -3, +3, -9, +9 positions away (axis x, y, z; - side
// first) -- the same axis for both, opposite signs.
template <class Emit>
__host__ __device__ __forceinline__ void emit_pair(int p, int q, Emit& emit) {
    const int d = q - p;
    const int ad = d < 0 ? -d : d;
    const uint32_t base = 1u + 2u * (uint32_t(ad > 1) + uint32_t(ad > 3));
    emit(p, base + uint32_t(d > 0));
    emit(q, base + uint32_t(d < 0));
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

// The least cell of a non-empty set, by pairwise comparisons.
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

// Number of unclassified facets (through x) of every position, as a 2-bit counter in two bit
// planes: a cube of L(x) starts at 3, a quad at 2, an edge at 0 (its one facet, x, is classified
// first).  dec() takes one off every position of a mask; counts never go below zero because each
// facet is classified once.
struct FacetCount {
    uint32_t c0, c1;
    __host__ __device__ __forceinline__ void dec(uint32_t d) {
        c1 ^= d & ~c0;
        c0 ^= d;
    }
    __host__ __device__ __forceinline__ uint32_t one(uint32_t u) const { return u & c0 & ~c1; }
    __host__ __device__ __forceinline__ uint32_t zero(uint32_t u) const { return u & ~(c0 | c1); }
};

// Classifies the cells of L(x) (inL, with more than x in it) once x's lowest edge delta is known.
// least(S) returns the least cell of a non-empty set S; emit(p, code) is called for every
// non-critical cell with its direction code.  Returns false if a cell was left unclassified (an
// internal error).
//
// One step either pairs or declares a cell critical; both take the least cell of one set (the
// cells with one unclassified facet if there are any, else those with none), so a step runs the
// same instructions whichever it does -- threads of a warp that differ there do not serialise.
template <class Least, class Emit>
__host__ __device__ __forceinline__ bool classify_star(const uint32_t inL, const int delta, const Tables* T,
                                                       Least&& least, Emit&& emit) {
    emit_pair(CENTER, delta, emit);
    uint32_t U = inL & ~((1u << CENTER) | (1u << delta));
    FacetCount n{inL & DIM3, inL & (DIM2 | DIM3)};
    n.dec(T->cofacet[delta] & U);
    for (int guard = 0; guard < 27 && U; ++guard) {
        const uint32_t one = n.one(U);
        const uint32_t S = one ? one : n.zero(U);
        if (!S) return false;
        const int a = least(S);
        // pairing: a's only unclassified facet; otherwise a is critical and its code stays 0
        const uint32_t fb = one ? (T->facet[a] & U) : 0u;
        U &= ~((1u << a) | fb);
        uint32_t cof = T->cofacet[a];
        if (fb) {
            const int f = MSC_FFS(fb) - 1;
            emit_pair(f, a, emit);
            // a cell with both a and f as facets would have two dimensions: the sets are disjoint
            cof |= T->cofacet[f];
        }
        n.dec(cof & U);
    }
    return U == 0;
}

// ---- the ranked path for large stars -------------------------------------------------------

// Batcher's odd-even merge sort for n inputs (Knuth, TAOCP vol. 3, 5.3.4), enumerated at compile
// time: oem_comparator(c) is the c-th comparator (lower index * 256 + upper index), or -1 past
// the last one.  A comparator leaves the smaller value at its lower index.
template <int N>
__host__ __device__ constexpr int oem_comparator(int c) {
    int n = 0;
    for (int p = 1; p < N; p <<= 1)
        for (int k = p; k >= 1; k >>= 1)
            for (int j = k % p; j + k < N; j += 2 * k)
                for (int i = 0; i < k && i < N - j - k; ++i)
                    if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                        if (n == c) return (i + j) * 256 + (i + j + k);
                        ++n;
                    }
    return -1;
}

template <int C>
__host__ __device__ __forceinline__ void sort26_from(uint32_t* v) {
    constexpr int ab = oem_comparator<26>(C);
    if constexpr (ab >= 0) {
        constexpr int A = ab >> 8, B = ab & 255;
        const uint32_t x = v[A], y = v[B];
        v[A] = MSC_UMIN(x, y);
        v[B] = x ^ y ^ MSC_UMIN(x, y);
        sort26_from<C + 1>(v);
    }
}

// The 26 positions other than x, in index order: i -> position.
__host__ __device__ constexpr int star_pos(int i) { return i < CENTER ? i : i + 1; }

// Integer keys of the cells of L(x) (inL, at least two cells besides x) for the large-star path.
// center points at x's key; ROW and PLANE are the key array's strides along y and z.
//  1. Each vertex of L(x) gets the 32-bit word (key with its low 5 bits cleared) | position, and
//     each other position a padding word above all of them (spaced 32 apart).  A sorting
//     network orders the 26 words; these words order two vertices exactly as (key, position)
//     does unless both keys agree in all but their low 5 bits -- then two adjacent sorted words
//     agree above bit 4, and the function returns false (the caller uses the pairwise
//     comparisons instead; on smooth float data this is rare).
//  2. The vertex of rank r gets the bit 1 << r; a cell's key is the OR of its vertices' bits,
//     built edge -> quad -> cube from the facets through x.
//  3. K(p) receives (key << 5) | p for every position of L(x) (K(p) is scratch of the caller,
//     one 32-bit word per position; other positions are left with unspecified values).
template <int ROW, int PLANE, class Scratch>
__host__ __device__ __forceinline__ bool rank_cell_keys(const uint32_t inL, const uint32_t* center, Scratch&& K) {
    uint32_t v[26];
#pragma unroll
    for (int i = 0; i < 26; ++i) {
        const int p = star_pos(i);
        const uint32_t k = center[pdx(p) + ROW * pdy(p) + PLANE * pdz(p)];
        v[i] = ((inL >> p) & 1u) ? ((k & ~31u) | uint32_t(p)) : (0xFFFFFFFFu - 32u * uint32_t(i));
    }
    sort26_from<0>(v);
    uint32_t gap = 0xFFFFFFFFu;  // adjacent words with equal high parts differ below bit 5
#pragma unroll
    for (int j = 0; j < 25; ++j) gap = MSC_UMIN(gap, v[j + 1] ^ v[j]);
    if (gap < 32u) return false;
    const int m = MSC_POPC(inL) - 1;
#pragma unroll
    for (int j = 0; j < 26; ++j)
        if (j < m) K(int(v[j] & 31u)) = uint32_t(j);
    uint32_t key[27];
#pragma unroll
    for (int p = 0; p < 27; ++p) {  // dimension order within each position's facets: edges first
        if (p == CENTER) continue;
        key[p] = 1u << (K(p) & 31u);
    }
    // quads then cubes: a cell's vertices are its own position's vertex and its facets' vertices
#pragma unroll
    for (int pass = 2; pass <= 3; ++pass)
#pragma unroll
        for (int p = 0; p < 27; ++p) {
            const int dim = (pdx(p) != 0) + (pdy(p) != 0) + (pdz(p) != 0);
            if (dim != pass) continue;
            uint32_t k = key[p];
            if (pdx(p)) k |= key[p - pdx(p)];
            if (pdy(p)) k |= key[p - 3 * pdy(p)];
            if (pdz(p)) k |= key[p - 9 * pdz(p)];
            key[p] = k;
        }
#pragma unroll
    for (int p = 0; p < 27; ++p) {
        if (p == CENTER) continue;
        K(p) = (key[p] << 5) | uint32_t(p);
    }
    return true;
}

// The least cell of a non-empty set under the integer keys left in K by rank_cell_keys.
template <class Scratch>
__host__ __device__ __forceinline__ int least_by_keys(uint32_t s, Scratch&& K) {
    uint32_t best = K(MSC_FFS(s) - 1);
    s &= s - 1;
    while (s) {
        best = MSC_UMIN(best, K(MSC_FFS(s) - 1));
        s &= s - 1;
    }
    return int(best & 31u);
}

// Stars with at least this many cells besides x take the ranked path.
constexpr int RANKED_MIN_CELLS = 12;

// Pairs the cells of L(x) given inL (the lower-star mask, with more than x in it); st.key(p)
// must be valid for every p in inL, and the key array must have strides ROW and PLANE.
// Vertices with equal keys are ordered by position, which is their index order.  emit(p, code)
// is called for every non-critical cell with its direction code; K is per-star scratch of 27
// words (see rank_cell_keys).  Returns false if the procedure did not classify every cell (an
// internal error).
template <int ROW, int PLANE, class Scratch, class Emit>
__host__ __device__ __forceinline__ bool pair_lower_star(const uint32_t inL, const Star& st, Scratch&& K,
                                                         Emit&& emit) {
    if (MSC_POPC(inL) - 1 >= RANKED_MIN_CELLS && rank_cell_keys<ROW, PLANE>(inL, st.center, K)) {
        const int delta = least_by_keys(inL & DIM1, K);
        return classify_star(inL, delta, st.T, [&](uint32_t s) { return least_by_keys(s, K); }, emit);
    }
    const int delta = pop_min_edge(inL & DIM1, st);
    return classify_star(inL, delta, st.T, [&](uint32_t s) { return pop_min(s, st); }, emit);
}

// Pairs the cells of L(x) given the 27 vertex order keys k[] (k[13] = x; an off-grid vertex
// has key 0xFFFFFFFF) and tables filled with row = 3, plane = 9.  See pair_lower_star.
template <class Emit>
__host__ __device__ bool process_lower_star(const uint32_t* k, const Tables* T, Emit&& emit) {
    const uint32_t inL = lower_star_mask(lower_mask(k));
    if (inL == (1u << CENTER)) return true;  // a minimum: every code stays 0
    uint32_t scratch[27];
    return pair_lower_star<3, 9>(inL, Star{k + CENTER, T}, [&](int p) -> uint32_t& { return scratch[p]; }, emit);
}

}  // namespace star
}  // namespace msc

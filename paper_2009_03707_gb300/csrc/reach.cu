// (a4) Saddle-saddle reachability and (a5, first half) junction nodes.
//
// Sec. 3.2 and Sec. 3.5 "Saddle-Saddle reachability": the 1-cells reachable from the
// 1-saddles in the DAG of 1-2 gradient pairs, level by level; the traversal ends when a level
// adds nothing.  The paper runs a frontier BFS (expand, then stream-compact a 4x candidate
// array).  Here the same level sets are computed by pulling instead of pushing, on the 1-cell
// bitmap itself:
//
//  * A 1-cell e has in-edges only if it is paired with a quad q; they come from the other three
//    facets of q (a facet f of q has the out-edge f -> e because q is a cofacet of f that is not
//    f's own partner).  So with R_k the set reached within k levels,
//        R_{k+1} = R_k  u  { e paired with a quad q : some other facet of q is in R_k },
//    R_0 = the 1-saddles.  That is one data-parallel sweep per level over the bitmap rows:
//    for each 32-cell word, four pairing-direction masks select which neighbouring rows (shifted
//    by one bit where the step is along x) feed it.  Sweep k+1 changes the bitmap iff BFS level
//    k+1 is non-empty, so the level count is the paper's.
//  * Every access is a coalesced word of a row, where a queue frontier scatters a 4-byte access
//    per node over the whole grid.  One loop iteration is two sweeps (A -> B, B -> A, so the
//    set always ends in A) and a one-thread decision kernel; the loop is a conditional WHILE node
//    when the pipeline runs as a graph, so no level needs a host round trip.
//
// Sec. 3.3 / Sec. 3.5 "Gradient path counting": a junction is a reachable 1-cell that is not a
// 1-saddle and has out-degree > 1.  One warp per bitmap word (a lane per 1-cell) evaluates the
// out-edges of each reachable cell, marks junctions, and records each node's successor for the
// path tracer.  Junctions are stream-compacted in cell-id order (scan.cuh), which also gives
// O(1) ranks for the minor's matrix indices.
#include "dag.cuh"
#include "scan.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;

__device__ __forceinline__ int other_axis(int a, int j) { return j == 0 ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2); }

// Word addressing of the bitmaps, per thread: the 1-cell row layout is
//   edge_word(z, c, y, b, w) = z*sz + y*sy + off[axis] + w   (sz = 4 ny W, sy = 2 W),
// and the quad bitmaps hold one row per (even axis k, z, y): quad_word = ((k nz + z) ny + y) W + w.
// Word indices are 32-bit: a plan's bitmaps have fewer than 2^28 words (nverts < 2^29).
struct Rows {
    int w, y, z;  // this thread's word: x = 32w .. 32w+31 of row (y, z)
    int W, ny, nz;
    int sy, sz;   // 1-cell layout strides
    int base;     // z*sz + y*sy + w
    int qbase;    // (z ny + y) W + w
    int qplane;   // nz ny W
    __device__ Rows(const Geom& g, int64_t t) {
        const uint32_t q = g.div_W.div(uint32_t(t));
        w = int(uint32_t(t) - q * uint32_t(g.W));
        const uint32_t q2 = g.div_ny.div(q);
        y = int(q - q2 * uint32_t(g.ny));
        z = int(q2);
        W = g.W;
        ny = g.ny;
        nz = g.nz;
        sy = 2 * W;
        sz = 4 * ny * W;
        base = z * sz + y * sy + w;
        qbase = (z * ny + y) * W + w;
        qplane = nz * ny * W;
    }
    template <int AX>
    __device__ __forceinline__ int edge(int dy, int dz) const {
        return base + (AX == 1 ? W : AX == 2 ? 2 * ny * W : 0) + dy * sy + dz * sz;
    }
    template <int DY, int DZ>
    __device__ __forceinline__ bool in_range() const {
        return (DY >= 0 || y > 0) && (DY <= 0 || y < ny - 1) && (DZ >= 0 || z > 0) && (DZ <= 0 || z < nz - 1);
    }
};

// Bits of a row word at index `at` (the word of x = 32w..), shifted so that bit i refers to x + DX.
template <int DX>
__device__ __forceinline__ uint32_t shifted(const uint32_t* __restrict__ R, int at, const Rows& r) {
    const uint32_t mid = R[at];
    if (DX == 0) return mid;
    if (DX > 0) return __funnelshift_r(mid, r.w + 1 < r.W ? R[at + 1] : 0u, 1);
    return __funnelshift_l(r.w > 0 ? R[at - 1] : 0u, mid, 1);
}

// Reach bits of the AX-cells owned by vertex (x + DX, y + DY, z + DZ); 0 outside the grid.
template <int AX, int DX, int DY, int DZ>
__device__ __forceinline__ uint32_t reach_row(const uint32_t* __restrict__ R, const Rows& r) {
    if (!r.in_range<DY, DZ>()) return 0;
    return shifted<DX>(R, r.edge<AX>(DY, DZ), r);
}

// Cells of axis A whose partner is the quad on side S along axis B (mask m) and that have a
// facet of that quad in R: the quad's other facets are the parallel A-cell one vertex along
// S u_B and the two B-cells at the ends of the A-cell, owned by v (+ u_A) (- u_B if S < 0).
template <int A, int B, int S>
__device__ __forceinline__ uint32_t pull(uint32_t m, const uint32_t* __restrict__ R, const Rows& r) {
    if (!m) return 0;
    constexpr int back = S < 0 ? 1 : 0;
    constexpr int ux = A == 0, uy = A == 1, uz = A == 2, bx = B == 0, by = B == 1, bz = B == 2;
    const uint32_t p = reach_row<A, S * bx, S * by, S * bz>(R, r) |
                       reach_row<B, ux - back * bx, uy - back * by, uz - back * bz>(R, r) |
                       reach_row<B, -back * bx, -back * by, -back * bz>(R, r);
    return m & p;
}

// Per vertex-row word: for each axis the four masks of 1-cells paired with the quad on the - / +
// side along the first / second other axis, R_0 = the 1-saddles, and for each quad orientation (by
// its even axis k) the bitmap of quads that are critical or paired with a facet (the quads that
// give an out-edge to every other facet).  A warp takes `chunk` (4..32, a multiple of RI_WORDS)
// consecutive row words: it builds each word's bitmaps with one ballot apiece (a lane per x),
// RI_WORDS words' loads issued together, keeps word u's bitmaps in lane u, and then writes all of
// them with one store per array.  Large grids take chunks of 32 (the stores fully coalesced), small
// ones smaller chunks so that enough warps share the work.
constexpr int RI_WORDS = 4;
__global__ void __launch_bounds__(THREADS) reach_init(Geom g, const uint32_t* __restrict__ words,
                                                      uint4* __restrict__ masks, uint32_t* __restrict__ R0,
                                                      uint32_t* __restrict__ R1, uint32_t* __restrict__ qdown,
                                                      uint32_t* __restrict__ stamp, int chunk) {
    const int lane = threadIdx.x & 31;
    const int64_t nrw = int64_t(g.nz) * g.ny * g.W;
    const int64_t step = ((int64_t(gridDim.x) * THREADS) >> 5) * chunk;
    for (int64_t t0 = ((int64_t(blockIdx.x) * THREADS + threadIdx.x) >> 5) * chunk; t0 < nrw; t0 += step) {
        uint4 m[3];
        uint32_t crit[3], qd[3];
        for (int u0 = 0; u0 < chunk && t0 + u0 < nrw; u0 += RI_WORDS) {  // warp-uniform
            uint32_t words_of[RI_WORDS];
#pragma unroll
            for (int v = 0; v < RI_WORDS; ++v) {
                const Rows r(g, min(t0 + u0 + v, nrw - 1));
                const int x = r.w * 32 + lane;
                words_of[v] = x < g.nx ? words[vid32(g, x, r.y, r.z)] : 0x00FFFFFFu;  // all codes 7 off-grid
            }
#pragma unroll
            for (int v = 0; v < RI_WORDS; ++v) {
                const bool mine = lane == u0 + v;  // this lane keeps word u0 + v's bitmaps
                const uint32_t word = words_of[v];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const uint32_t code = slot_code(word, 1 << a);
                    const int k = int(code - 1) >> 1;  // axis of the partner (code 1..6)
                    const bool quad = code >= 1 && code <= 6 && k != a;
                    const int sel = quad ? 2 * (k == other_axis(a, 0) ? 0 : 1) + int(!(code & 1u)) : -1;  // odd: - side
                    const uint32_t m0 = __ballot_sync(0xFFFFFFFFu, sel == 0), m1 = __ballot_sync(0xFFFFFFFFu, sel == 1);
                    const uint32_t m2 = __ballot_sync(0xFFFFFFFFu, sel == 2), m3 = __ballot_sync(0xFFFFFFFFu, sel == 3);
                    const uint32_t c0 = __ballot_sync(0xFFFFFFFFu, code == 0);
                    if (mine) {
                        m[a] = make_uint4(m0, m1, m2, m3);
                        crit[a] = c0;
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const uint32_t code = slot_code(word, 7 ^ (1 << k));
                    const bool down = code == 0 || (code <= 6 && (int(code - 1) >> 1) != k);
                    const uint32_t q = __ballot_sync(0xFFFFFFFFu, down);
                    if (mine) qd[k] = q;
                }
            }
        }
        const int64_t t = t0 + lane;
        if (lane < chunk && t < nrw) {
            const Rows r(g, t);
            const int e0 = r.edge<0>(0, 0), e1 = r.edge<1>(0, 0), e2 = r.edge<2>(0, 0);
            masks[e0] = m[0];
            masks[e1] = m[1];
            masks[e2] = m[2];
            R0[e0] = crit[0];
            R0[e1] = crit[1];
            R0[e2] = crit[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) qdown[k * r.qplane + r.qbase] = qd[k];
            if (r.w == 0) stamp[r.z * r.ny + r.y] = 1;  // every row is new at the start
            // the unused slot of the 1-cell layout stays empty in both buffers
            masks[e2 + r.W] = make_uint4(0, 0, 0, 0);
            R0[e2 + r.W] = 0;
            R1[e2 + r.W] = 0;
        }
    }
}

template <int A>
__device__ __forceinline__ bool sweep_word(const Rows& r, const uint4* __restrict__ masks,
                                           const uint32_t* __restrict__ Rin, uint32_t* __restrict__ Rout) {
    constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
    const int i = r.edge<A>(0, 0);
    const uint32_t cur = Rin[i];
    const uint4 m = masks[i];
    uint32_t add = 0;
    if ((m.x | m.y | m.z | m.w) & ~cur)
        add = pull<A, B1, -1>(m.x & ~cur, Rin, r) | pull<A, B1, 1>(m.y & ~cur, Rin, r) |
              pull<A, B2, -1>(m.z & ~cur, Rin, r) | pull<A, B2, 1>(m.w & ~cur, Rin, r);
    Rout[i] = cur | add;
    return add != 0;
}

// One level: Rout = Rin | cells whose partner quad has another facet in Rin.  A thread takes one
// vertex-row word at a time for all three axes (one neighbourhood check, three independent chains
// of loads).  Sets *changed if any word grew.
// Rows (y, z) are stamped with 1 + the last sweep that changed them (1: the start).  A cell's
// predecessors lie within one step in y and z, so a row none of whose 3 x 3 neighbour rows changed
// in the previous sweep cannot change now; it is skipped, Rout included: that buffer already
// holds the row's value from two sweeps ago, which is still its value.  Fronts that move slowly
// through a large grid (many levels) then cost only the rows near the front.
__global__ void __launch_bounds__(THREADS, 4) reach_sweep(Geom g, const uint4* __restrict__ masks,
                                                       const uint32_t* __restrict__ Rin, uint32_t* __restrict__ Rout,
                                                       uint32_t* __restrict__ stamp, const Summary* __restrict__ sum,
                                                       int parity, uint32_t* __restrict__ changed) {
    const int64_t nrw = int64_t(g.nz) * g.ny * g.W;
    const uint32_t k = 2u * uint32_t(sum->sweep_iters) + 1u + uint32_t(parity);  // this sweep
    bool grew = false;
    // grid-stride over the row words (a few tiles of THREADS words per CTA): a sweep in which few
    // rows are near a front then costs fewer CTA launches for the rest
    for (int64_t t = int64_t(blockIdx.x) * THREADS + threadIdx.x; t < nrw; t += int64_t(gridDim.x) * THREADS) {
        const Rows r(g, t);
        uint32_t recent = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = r.y + dy, z = r.z + dz;
                if (y >= 0 && y < g.ny && z >= 0 && z < g.nz) recent = max(recent, stamp[int64_t(z) * g.ny + y]);
            }
        if (recent >= k) {
            const bool g0 = sweep_word<0>(r, masks, Rin, Rout);
            const bool g1 = sweep_word<1>(r, masks, Rin, Rout);
            const bool g2 = sweep_word<2>(r, masks, Rin, Rout);
            if (g0 || g1 || g2) {
                stamp[int64_t(r.z) * g.ny + r.y] = k + 1;
                grew = true;
            }
        }
    }
    if (__syncthreads_or(grew) && threadIdx.x == 0) *changed = 1u;
}

// Level 0: the 1-saddles, if there are any.
__global__ void reach_start(Summary* sum) { sum->levels = sum->counts[1] > 0 ? 1 : 0; }

// End of one loop iteration (two sweeps): the non-empty levels found, and the continue decision
// (while the second sweep still grew the set, up to the iteration cap).
__global__ void reach_decide(Summary* sum, int64_t max_iter, cudaGraphConditionalHandle h, int use_handle) {
    const uint32_t c0 = sum->loop_flag[0], c1 = sum->loop_flag[1];
    sum->loop_flag[0] = 0;
    sum->loop_flag[1] = 0;
    ++sum->sweep_iters;
    sum->levels += (c0 ? 1 : 0) + (c1 ? 1 : 0);
    bool more = c1 != 0;
    if (more && int64_t(sum->levels) >= max_iter) {
        atomicOr(&sum->status, uint32_t(ST_ITER));
        more = false;
    }
    sum->loop_flag[3] = more ? 1u : 0u;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Down-quad bits of the quads with even axis K owned by vertex (x + DX, y + DY, z + DZ).
template <int K, int DX, int DY, int DZ>
__device__ __forceinline__ uint32_t quad_row(const uint32_t* __restrict__ qdown, const Rows& r) {
    if (!r.in_range<DY, DZ>()) return 0;
    return shifted<DX>(qdown, K * r.qplane + r.qbase + DY * r.W + DZ * r.ny * r.W, r);
}

// The bitmap words one axis of a vertex-row word needs: reached and critical bits, the four
// partner masks, and the down-quad rows of the quads on the - / + side along the first / second
// other axis (the order of the masks).
struct AxisIn {
    uint32_t vis, crit;
    uint4 m;
    uint32_t q[4];
};

template <int A>
__device__ __forceinline__ AxisIn load_axis(const Geom& g, const Rows& r, const uint32_t* __restrict__ visited,
                                            const uint4* __restrict__ masks, const uint32_t* __restrict__ qdown,
                                            const uint32_t* __restrict__ crit_bits) {
    constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
    constexpr int K1 = 3 - A - B1, K2 = 3 - A - B2;  // even axes of the quads along B1, B2
    AxisIn in;
    in.vis = visited[r.edge<A>(0, 0)];
    in.crit = crit_bits[g.slot_word(1 << A, r.z, r.y, r.w)];
    in.m = masks[r.edge<A>(0, 0)];
    in.q[0] = quad_row<K1, -(B1 == 0), -(B1 == 1), -(B1 == 2)>(qdown, r);
    in.q[1] = quad_row<K1, 0, 0, 0>(qdown, r);
    in.q[2] = quad_row<K2, -(B2 == 0), -(B2 == 1), -(B2 == 2)>(qdown, r);
    in.q[3] = quad_row<K2, 0, 0, 0>(qdown, r);
    return in;
}

// Gradient word of the vertex one step down axis B from v (0 off the grid), loaded for a whole
// row of lanes at once.
template <int B>
__device__ __forceinline__ uint32_t minus_word(const Geom& g, const uint32_t* __restrict__ words, const Rows& r, int x,
                                               uint32_t v) {
    if (x >= g.nx) return 0u;
    if (B == 0) return x > 0 ? words[v - 1] : 0u;
    if (B == 1) return r.y > 0 ? words[v - uint32_t(g.nx)] : 0u;
    return r.z > 0 ? words[v - uint32_t(g.nx) * uint32_t(g.ny)] : 0u;
}

// The A-cells of one vertex-row word (a lane per cell).  The out-edges of a 1-cell e go through
// its cofacet quads other than its partner that are critical or paired with a facet, so with the
// down-quad rows the out-degree is a popcount.  Reachable cells that are not 1-saddles get their
// info record; a single successor is decoded from the one quad it goes through, whose owner is v
// itself (+ side) or v one step down the quad's other axis (- side, gradient word w_b1 / w_b2).
template <int A>
__device__ __forceinline__ void classify_axis(const Geom& g, const Rows& r, int lane, int x, uint32_t v,
                                              const AxisIn& in, uint32_t w_self, uint32_t w_b1, uint32_t w_b2,
                                              uint32_t* __restrict__ info, uint32_t* __restrict__ junc,
                                              unsigned long long& cnt) {
    constexpr int B1 = A == 0 ? 1 : 0, B2 = A == 2 ? 1 : 2;
    // every record of the row is written (whole sectors: no read-modify-write in L2); cells
    // that are not reached, or are 1-saddles, get a dead-end record that nothing reads
    if (lane == 0) cnt += __popc(in.vis);
    const uint32_t partner = ((in.m.x >> lane) & 1u) | (((in.m.y >> lane) & 1u) << 1) |
                             (((in.m.z >> lane) & 1u) << 2) | (((in.m.w >> lane) & 1u) << 3);
    const uint32_t out = (((in.q[0] >> lane) & 1u) | (((in.q[1] >> lane) & 1u) << 1) |
                          (((in.q[2] >> lane) & 1u) << 2) | (((in.q[3] >> lane) & 1u) << 3)) &
                         ~partner;
    const int n = __popc(out);
    const bool mine = ((in.vis & ~in.crit) >> lane) & 1u;
    uint32_t rec = INFO_DEAD;
    if (mine) {
        rec = n == 0 ? INFO_DEAD : INFO_BRANCH;
        if (n == 1) {
            const int sel = __ffs(out) - 1;
            const int b = sel < 2 ? B1 : B2;
            const int k = 3 - A - b;  // the quad's even axis
            const bool plus = sel & 1;
            uint32_t ov = v, ow = w_self;
            if (!plus) {
                ov -= b == 0 ? 1u : b == 1 ? uint32_t(g.nx) : uint32_t(g.nx) * uint32_t(g.ny);
                ow = sel < 2 ? w_b1 : w_b2;
            }
            const uint32_t qc = slot_code(ow, 7 ^ (1 << k));
            if (qc == 0) {
                rec = 0x80000000u | (ov << 2) | uint32_t(k);  // a 2-saddle
            } else {                                           // the facet the quad is paired with
                const int kk = int(qc - 1) >> 1;
                if (!(qc & 1u)) ov += kk == 0 ? 1u : kk == 1 ? uint32_t(g.nx) : uint32_t(g.nx) * uint32_t(g.ny);
                rec = edge_handle(ov, kk == A ? b : A);
            }
        }
    }
    if (x < g.nx) info[info_index(g, edge_handle(v, A))] = rec;
    const uint32_t jw = __ballot_sync(0xFFFFFFFFu, mine && n > 1);
    if (lane == 0) junc[r.edge<A>(0, 0)] = jw;
}

// One warp per vertex-row word, all three axes: every load of the word (the bitmaps of the three
// axes and the gradient words of v and of its three down neighbours, coalesced rows) is issued
// before any result is computed, so a warp has them all in flight at once.
__global__ void __launch_bounds__(THREADS, 4) classify_reached(Geom g, const uint32_t* __restrict__ words,
                                                            const uint32_t* __restrict__ visited,
                                                            const uint4* __restrict__ masks,
                                                            const uint32_t* __restrict__ qdown,
                                                            const uint32_t* __restrict__ crit_bits,
                                                            uint32_t* __restrict__ info, uint32_t* __restrict__ junc,
                                                            unsigned long long* __restrict__ n_reached) {
    const int lane = threadIdx.x & 31;
    const int64_t nrw = int64_t(g.nz) * g.ny * g.W;
    unsigned long long cnt = 0;
    for (int64_t t = (int64_t(blockIdx.x) * THREADS + threadIdx.x) >> 5; t < nrw;
         t += (int64_t(gridDim.x) * THREADS) >> 5) {  // warp-uniform
        const Rows r(g, t);
        const int x = r.w * 32 + lane;
        const uint32_t v = vid32(g, x, r.y, r.z);
        const AxisIn i0 = load_axis<0>(g, r, visited, masks, qdown, crit_bits);
        const AxisIn i1 = load_axis<1>(g, r, visited, masks, qdown, crit_bits);
        const AxisIn i2 = load_axis<2>(g, r, visited, masks, qdown, crit_bits);
        const uint32_t w0 = x < g.nx ? words[v] : 0u;
        const uint32_t wx = minus_word<0>(g, words, r, x, v), wy = minus_word<1>(g, words, r, x, v),
                       wz = minus_word<2>(g, words, r, x, v);
        classify_axis<0>(g, r, lane, x, v, i0, w0, wy, wz, info, junc, cnt);
        classify_axis<1>(g, r, lane, x, v, i1, w0, wx, wz, info, junc, cnt);
        classify_axis<2>(g, r, lane, x, v, i2, w0, wx, wy, info, junc, cnt);
        if (lane == 0) junc[g.edge_word(r.z, 1, r.y, 1, r.w)] = 0;  // the unused slot of the 1-cell layout
    }
    __shared__ unsigned long long part[THREADS / 32];
    if (lane == 0) part[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int k = 0; k < THREADS / 32; ++k) s += part[k];
        if (s) atomicAdd(n_reached, s);
    }
}

int grid_for(const Plan* p, int64_t threads) {
    const int64_t want = (threads + THREADS - 1) / THREADS;
    const int64_t cap = int64_t(p->num_sms > 0 ? p->num_sms : 148) * 8;
    return int(std::max<int64_t>(1, std::min(want, cap)));
}

struct SweepCtx {
    dim3 grid;
    const uint4* masks;
    uint32_t* a;
    uint32_t* b;
    uint32_t* stamp;
};

void sweep_body(Plan* p, cudaStream_t s, cudaGraphConditionalHandle h, void* ctx) {
    const SweepCtx& c = *static_cast<SweepCtx*>(ctx);
    reach_sweep<<<c.grid, THREADS, 0, s>>>(p->g, c.masks, c.a, c.b, c.stamp, p->dsum(), 0, &p->dsum()->loop_flag[0]);
    reach_sweep<<<c.grid, THREADS, 0, s>>>(p->g, c.masks, c.b, c.a, c.stamp, p->dsum(), 1, &p->dsum()->loop_flag[1]);
    reach_decide<<<1, 1, 0, s>>>(p->dsum(), p->opts.max_iterations, h, h != 0);
}

}  // namespace

msc_status run_reachability(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t nw = g.edge_words();
    const int64_t nrw = int64_t(g.nz) * g.ny * g.W;  // vertex-row words
    if ((st = ensure(p, p->visited, sizeof(uint32_t) * size_t(nw)))) return st;
    if ((st = ensure(p, p->reach_tmp, sizeof(uint32_t) * size_t(nw)))) return st;
    if ((st = ensure(p, p->reach_masks, sizeof(uint4) * size_t(nw)))) return st;
    if ((st = ensure(p, p->reach_qdown, sizeof(uint32_t) * 3 * size_t(nrw)))) return st;
    if ((st = ensure(p, p->reach_stamp, sizeof(uint32_t) * size_t(g.nz) * size_t(g.ny)))) return st;
    auto* masks = static_cast<uint4*>(p->reach_masks.ptr);
    auto* stamp = static_cast<uint32_t*>(p->reach_stamp.ptr);
    uint32_t* A = static_cast<uint32_t*>(p->visited.ptr);
    uint32_t* B = static_cast<uint32_t*>(p->reach_tmp.ptr);
    // row words per warp: 32 when every SM still gets 32 warps' worth, else fewer (at least 4)
    int chunk = 32;
    while (chunk > RI_WORDS && nrw < int64_t(chunk) * 32 * std::max(1, p->num_sms)) chunk >>= 1;
    reach_init<<<grid_for(p, (nrw + chunk - 1) / chunk * 32), THREADS, 0, s>>>(
        g, static_cast<const uint32_t*>(p->words.ptr), masks, A, B, static_cast<uint32_t*>(p->reach_qdown.ptr), stamp,
        chunk);
    reach_start<<<1, 1, 0, s>>>(p->dsum());
    launched(p, 2);
    if ((st = check_cuda(p, cudaGetLastError(), "reach_init launch"))) return st;
    // sweep grid: at most 4 tiles per CTA and at least one resident wave (4 CTAs per SM).  Fewer,
    // longer CTAs would cost little alone but leave long tails when other passes share the device.
    const int64_t tiles = (nrw + THREADS - 1) / THREADS;
    const int64_t sweep_ctas = std::min<int64_t>(tiles, std::max<int64_t>(int64_t(std::max(1, p->num_sms)) * 4, (tiles + 3) / 4));
    SweepCtx ctx{dim3(unsigned(std::max<int64_t>(1, sweep_ctas)), 1), masks, A, B, stamp};
    return run_loop(p, s, 1, 3, sweep_body, &ctx);
}

msc_status run_junctions(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t nw = g.edge_words();
    if ((st = ensure(p, p->junc_bits, sizeof(uint32_t) * size_t(nw)))) return st;
    if ((st = ensure(p, p->junc_prefix, sizeof(uint32_t) * size_t(nw)))) return st;
    if ((st = ensure(p, p->node_info, sizeof(uint32_t) * 3 * size_t(g.nverts)))) return st;
    const int64_t nrw = int64_t(g.nz) * g.ny * g.W;
    classify_reached<<<grid_for(p, nrw * 32), THREADS, 0, s>>>(
        g, static_cast<const uint32_t*>(p->words.ptr), static_cast<const uint32_t*>(p->visited.ptr),
        static_cast<const uint4*>(p->reach_masks.ptr), static_cast<const uint32_t*>(p->reach_qdown.ptr),
        static_cast<const uint32_t*>(p->crit_bits.ptr), static_cast<uint32_t*>(p->node_info.ptr),
        static_cast<uint32_t*>(p->junc_bits.ptr), &p->dsum()->reached);
    launched(p);
    if ((st = check_cuda(p, cudaGetLastError(), "classify_reached launch"))) return st;
    EdgeSource src{};
    src.g = g;
    src.bits = static_cast<const uint32_t*>(p->junc_bits.ptr);
    src.prefix = static_cast<uint32_t*>(p->junc_prefix.ptr);
    src.status = p->status_word();
    if ((st = compaction_sums(p, s, src, 1, &p->dsum()->n_junctions))) return st;
    int64_t cap = p->caps.nj;
    if (!p->capturing) {  // size the list exactly
        if ((st = read_summary(p, s))) return st;
        cap = int64_t(p->hsum->n_junctions);
        p->n_junctions = cap;
    }
    if ((st = ensure(p, p->junc_cells, sizeof(uint32_t) * size_t(cap ? cap : 1)))) return st;
    src.out = static_cast<uint32_t*>(p->junc_cells.ptr);
    src.cap = uint64_t(cap);
    return compaction_emit(p, s, src, 1);
}

}  // namespace msc

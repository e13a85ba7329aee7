// (a3) Saddle-extremum arcs and the destination extremum of every vertex and cube.
//
// Sec. 3.4 and Sec. 3.5 "Saddle-Extrema arcs": gradient paths that end at extrema only merge
// or only split, so following them is root finding in a forest, done by pointer jumping.
//  * Vertex forest: a vertex paired with edge (v,w) points to w; a minimum points to itself.
//  * Cube forest: a cube paired with quad q points to the other cube of q; a maximum points
//    to itself; a cube whose quad lies on the domain boundary points to NONE (the path leaves
//    the domain).
// Labels are vertex indices while jumping (every cube is named by its owner vertex); each
// jump round also writes the outputs, as cell ids, from the labels it reached.  The links are first resolved inside tiles of 16 x 8 x 8
// vertices, in shared memory: each CTA computes its vertices' and cubes' links from the gradient
// words, and each thread follows its own two paths through the tile until they reach a root
// inside it or the first vertex outside it.  The global rounds then only hop from tile to tile.  Each global round lets every
// thread follow up to JUMPS links, updating its own entry in place; the paper's ping-pong
// buffers are not needed because any value a thread reads is an ancestor of the one it
// replaces.  Rounds repeat until no entry changes: a device flag decides, so the loop runs
// without the host when it is part of a captured pipeline (a conditional WHILE node), and is
// capped by the plan's iteration limit.
#include "msc_internal.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;
constexpr int JUMPS = 64;
constexpr uint32_t NO_LINK = 0xFFFFFFFFu;

// Links resolved per tile.  A CTA owns TLX x TLY x TLZ vertices, one per thread.  In shared
// memory a link is a local index (a vertex of the tile; a root points to itself), or
// OUTSIDE | global index of the first vertex outside the tile, or NO_LINK.  Each thread then
// walks its vertex's and its cube's paths through the tile (read-only, so no barriers: the
// forests are acyclic, and a path within the tile has at most TL_THREADS links); the global
// labels are the root's or the exit's global index.
constexpr int TLX = 16, TLY = 8, TLZ = 8, TL_THREADS = TLX * TLY * TLZ;
constexpr uint32_t OUTSIDE = 0x80000000u;

__global__ void __launch_bounds__(TL_THREADS) tile_links(Geom g, const uint32_t* __restrict__ words,
                                                         uint32_t* __restrict__ lab_v, uint32_t* __restrict__ lab_c,
                                                         uint32_t* __restrict__ status) {
    __shared__ uint32_t lv[TL_THREADS], lc[TL_THREADS];
    const int t = threadIdx.x;
    const int tx = t % TLX, ty = (t / TLX) % TLY, tz = t / (TLX * TLY);
    const int x0 = blockIdx.x * TLX, y0 = blockIdx.y * TLY, z0 = blockIdx.z * TLZ;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool valid = x < g.nx && y < g.ny && z < g.nz;
    const uint32_t v = valid ? uint32_t(g.vid(x, y, z)) : 0u;
    // the link of a neighbour (x,y,z) + d along `axis`: local if it lies in the tile
    auto link_to = [&](int axis, int sign) -> uint32_t {
        const int ox = x + (axis == 0 ? sign : 0), oy = y + (axis == 1 ? sign : 0), oz = z + (axis == 2 ? sign : 0);
        const int lx = ox - x0, ly = oy - y0, lz = oz - z0;
        if (lx >= 0 && lx < TLX && ly >= 0 && ly < TLY && lz >= 0 && lz < TLZ) return uint32_t((lz * TLY + ly) * TLX + lx);
        return OUTSIDE | uint32_t(g.vid(ox, oy, oz));
    };
    uint32_t a = NO_LINK, c = NO_LINK;
    if (valid) {
        const uint32_t w = words[v];
        const uint32_t cv = slot_code(w, 0);  // the vertex
        a = uint32_t(t);
        if (cv >= 1 && cv <= 6) {
            const int axis = int(cv - 1) >> 1, sign = (cv & 1) ? -1 : 1;
            const int o = (axis == 0 ? x : axis == 1 ? y : z) + sign, n = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
            if (o >= 0 && o < n) a = link_to(axis, sign);
            else atomicOr(status, ST_INTERNAL);  // a vertex paired with an edge that leaves the grid
        }
        const uint32_t cc = slot_code(w, 7);  // the cube v owns
        if (cc == 0) {
            c = uint32_t(t);
        } else if (cc <= 6) {
            const int axis = int(cc - 1) >> 1, sign = (cc & 1) ? -1 : 1;
            const int o = (axis == 0 ? x : axis == 1 ? y : z) + sign, n = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
            if (o >= 0 && o <= n - 2) c = link_to(axis, sign);
        }
    }
    lv[t] = a;
    lc[t] = c;
    __syncthreads();
    if (!valid) return;
    // local links have the OUTSIDE bit clear (NO_LINK has it set); each thread leaves its end point
    // in its own entry, a shortcut for the threads that reach it later (any value read is still an
    // ancestor)
    for (int hop = 0; hop < TL_THREADS && !(a & OUTSIDE); ++hop) {
        const uint32_t b = lv[a];
        if (b == a) break;  // a root
        a = b;
    }
    lv[t] = a;
    for (int hop = 0; hop < TL_THREADS && !(c & OUTSIDE); ++hop) {
        const uint32_t b = lc[c];
        if (b == c) break;
        c = b;
    }
    lc[t] = c;
    auto global_of = [&](uint32_t l) -> uint32_t {
        if (l == NO_LINK) return NO_LINK;
        if (l & OUTSIDE) return l & ~OUTSIDE;
        const int lx = int(l) % TLX, ly = (int(l) / TLX) % TLY, lz = int(l) / (TLX * TLY);
        return uint32_t(g.vid(x0 + lx, y0 + ly, z0 + lz));
    };
    lab_v[v] = global_of(a);
    lab_c[v] = global_of(c);
}

// Cell id of the extremum a label names: a vertex (minimum) or the cube a vertex owns (maximum).
__device__ __forceinline__ uint32_t label_cell(const Geom& g, uint32_t u, int off) {
    const uint32_t q = g.div_nx.div(u);
    const int x = int(u - q * uint32_t(g.nx));
    const int z = int(g.div_ny.div(q));
    const int y = int(q - uint32_t(z) * uint32_t(g.ny));
    return g.cell_id(2 * x + off, 2 * y + off, 2 * z + off);
}

// One round of in-place pointer jumping over both forests (labels are vertex indices); every
// round also writes each vertex's and cube's extremum as a cell id (NONE for a path that leaves
// the domain) -- the last round's values are the results.
__global__ void __launch_bounds__(THREADS) jump_round(Geom g, uint32_t* __restrict__ lab_v,
                                                      uint32_t* __restrict__ lab_c, uint32_t* __restrict__ out_v,
                                                      uint32_t* __restrict__ out_c, uint32_t* __restrict__ changed) {
    const int64_t v = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (v >= g.nverts) return;
    bool open = false;
    {
        uint32_t p = lab_v[v], start = p;
        for (int j = 0; j < JUMPS; ++j) {
            uint32_t q = lab_v[p];
            if (q == p) break;
            p = q;
        }
        if (p != start) lab_v[v] = p;
        open |= lab_v[p] != p;
        out_v[v] = label_cell(g, p, 0);
    }
    {
        uint32_t p = lab_c[v], start = p;
        if (p != NO_LINK) {
            for (int j = 0; j < JUMPS; ++j) {
                uint32_t q = lab_c[p];
                if (q == p || q == NO_LINK) {
                    p = q == NO_LINK ? NO_LINK : p;
                    break;
                }
                p = q;
            }
            if (p != start) lab_c[v] = p;
            open |= p != NO_LINK && lab_c[p] != p;
        }
        out_c[v] = p == NO_LINK ? NONE : label_cell(g, p, 1);
    }
    if (open) *changed = 1;
}

// End of one round: the continue decision (more rounds while some chain is still open, up to the
// iteration cap), the round count, and the graph condition when the loop runs in a graph.
__global__ void jump_decide(Summary* sum, int64_t max_iter, cudaGraphConditionalHandle h, int use_handle) {
    const bool open = sum->jump_flag[0] != 0;
    sum->jump_flag[0] = 0;
    const unsigned long long r = ++sum->jump_rounds;
    bool more = open;
    if (more && int64_t(r) >= max_iter) {
        atomicOr(&sum->status, uint32_t(ST_ITER));
        more = false;
    }
    sum->jump_flag[1] = more ? 1u : 0u;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

struct CellCoord {
    int x, y, z;
};

__device__ __forceinline__ CellCoord decode_cell(const Geom& g, uint32_t id) {
    CellCoord c;
    const uint32_t q = g.div_rx.div(id);
    c.x = int(id - q * g.rx);
    c.z = int(g.div_ry.div(q));
    c.y = int(q - uint32_t(c.z) * g.ry);
    return c;
}

// 1-saddle arcs: the minima of the edge's lower-coordinate and upper-coordinate vertices.
// Count of a list produced earlier in the pass; 0 (nothing to do) when the pass is to be rerun.
__device__ __forceinline__ int64_t clamp_count(const unsigned long long* n_dev, int64_t cap, uint32_t* status) {
    const unsigned long long n = *n_dev;
    if (pass_retrying(status) || !count_fits(status, n, cap)) return 0;
    return int64_t(n);
}

__global__ void __launch_bounds__(THREADS) min_arcs_kernel(Geom g, const uint32_t* __restrict__ s1,
                                                           const unsigned long long* n_dev, int64_t cap,
                                                           const uint32_t* __restrict__ vmin, uint32_t* __restrict__ out,
                                                           uint32_t* __restrict__ status) {
    const int64_t n1 = clamp_count(n_dev, cap, status);
    for (int64_t i = int64_t(blockIdx.x) * THREADS + threadIdx.x; i < n1; i += int64_t(gridDim.x) * THREADS) {
    CellCoord c = decode_cell(g, s1[i]);
    int lo[3] = {c.x >> 1, c.y >> 1, c.z >> 1};
    int hi[3] = {(c.x + 1) >> 1, (c.y + 1) >> 1, (c.z + 1) >> 1};
    out[2 * i] = vmin[g.vid(lo[0], lo[1], lo[2])];
    out[2 * i + 1] = vmin[g.vid(hi[0], hi[1], hi[2])];
    }
}

// 2-saddle arcs: the maxima of the quad's cofacet cubes on the - and + side of its even axis.
__global__ void __launch_bounds__(THREADS) max_arcs_kernel(Geom g, const uint32_t* __restrict__ s2,
                                                           const unsigned long long* n_dev, int64_t cap,
                                                           const uint32_t* __restrict__ cmax, uint32_t* __restrict__ out,
                                                           uint32_t* __restrict__ status) {
    const int64_t n2 = clamp_count(n_dev, cap, status);
    for (int64_t i = int64_t(blockIdx.x) * THREADS + threadIdx.x; i < n2; i += int64_t(gridDim.x) * THREADS) {
    CellCoord c = decode_cell(g, s2[i]);
    int cc[3] = {c.x, c.y, c.z};
    const int axis = !(cc[0] & 1) ? 0 : !(cc[1] & 1) ? 1 : 2;
    const int extent[3] = {2 * g.nx - 1, 2 * g.ny - 1, 2 * g.nz - 1};
    for (int side = 0; side < 2; ++side) {
        int d[3] = {cc[0], cc[1], cc[2]};
        d[axis] += side ? 1 : -1;
        uint32_t lab = NONE;
        if (d[axis] >= 0 && d[axis] < extent[axis]) lab = cmax[g.vid(d[0] >> 1, d[1] >> 1, d[2] >> 1)];
        out[2 * i + side] = lab;
    }
    }
}

int blocks(int64_t n) { return int((n + THREADS - 1) / THREADS); }

struct JumpCtx {
    int64_t n;
    uint32_t* lab_v;
    uint32_t* lab_c;
    uint32_t* vmin;
    uint32_t* cmax;
};

void jump_body(Plan* p, cudaStream_t s, cudaGraphConditionalHandle h, void* ctx) {
    const JumpCtx& c = *static_cast<JumpCtx*>(ctx);
    jump_round<<<blocks(c.n), THREADS, 0, s>>>(p->g, c.lab_v, c.lab_c, c.vmin, c.cmax, &p->dsum()->jump_flag[0]);
    jump_decide<<<1, 1, 0, s>>>(p->dsum(), p->opts.max_iterations, h, h != 0);
}

}  // namespace

msc_status run_extremum(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t cap1 = p->capturing ? p->caps.cells[1] : p->counts[1];
    const int64_t cap2 = p->capturing ? p->caps.cells[2] : p->counts[2];
    if ((st = ensure(p, p->vmin, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->cmax, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->min_arcs, sizeof(uint32_t) * size_t(2 * cap1 + 1)))) return st;
    if ((st = ensure(p, p->max_arcs, sizeof(uint32_t) * size_t(2 * cap2 + 1)))) return st;
    // labels (vertex indices) while jumping; the outputs are written as cell ids by every round
    if ((st = ensure(p, p->ext_lab_v, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->ext_lab_c, sizeof(uint32_t) * size_t(g.nverts)))) return st;
    auto* vmin = static_cast<uint32_t*>(p->vmin.ptr);
    auto* cmax = static_cast<uint32_t*>(p->cmax.ptr);
    auto* lab_v = static_cast<uint32_t*>(p->ext_lab_v.ptr);
    auto* lab_c = static_cast<uint32_t*>(p->ext_lab_c.ptr);
    const dim3 tiles(unsigned((g.nx + TLX - 1) / TLX), unsigned((g.ny + TLY - 1) / TLY), unsigned((g.nz + TLZ - 1) / TLZ));
    tile_links<<<tiles, TL_THREADS, 0, s>>>(g, static_cast<const uint32_t*>(p->words.ptr), lab_v, lab_c,
                                            p->status_word());
    launched(p);
    JumpCtx ctx{g.nverts, lab_v, lab_c, vmin, cmax};
    if ((st = run_loop(p, s, 0, 2, jump_body, &ctx))) return st;
    if (cap1) {
        min_arcs_kernel<<<grid_cap(p, cap1, THREADS), THREADS, 0, s>>>(
            g, static_cast<const uint32_t*>(p->cells[1].ptr), &p->dsum()->counts[1], cap1, vmin,
            static_cast<uint32_t*>(p->min_arcs.ptr), p->status_word());
        launched(p);
    }
    if (cap2) {
        max_arcs_kernel<<<grid_cap(p, cap2, THREADS), THREADS, 0, s>>>(
            g, static_cast<const uint32_t*>(p->cells[2].ptr), &p->dsum()->counts[2], cap2, cmax,
            static_cast<uint32_t*>(p->max_arcs.ptr), p->status_word());
        launched(p);
    }
    return check_cuda(p, cudaGetLastError(), "extremum launch");
}

}  // namespace msc

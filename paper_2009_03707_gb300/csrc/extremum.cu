// (a3) Saddle-extremum arcs and the destination extremum of every vertex and cube.
//
// Sec. 3.4 and Sec. 3.5 "Saddle-Extrema arcs": gradient paths that end at extrema only merge
// or only split, so following them is root finding in a forest, done by pointer jumping.
//  * Vertex forest: a vertex paired with edge (v,w) points to w; a minimum points to itself.
//  * Cube forest: a cube paired with quad q points to the other cube of q; a maximum points
//    to itself; a cube whose quad lies on the domain boundary points to NONE (the path leaves
//    the domain).
// Labels are vertex indices while jumping (every cube is named by its owner vertex), and
// become cell ids at the end.  Each jump round lets every thread follow up to JUMPS links,
// updating its own entry in place; the paper's ping-pong buffers are not needed because any
// value a thread reads is an ancestor of the one it replaces.  Rounds repeat until no entry
// changes: a device flag decides, so the loop runs without the host when it is part of a
// captured pipeline (a conditional WHILE node), and is capped by the plan's iteration limit.
#include "msc_internal.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;
constexpr int JUMPS = 64;
constexpr uint32_t NO_LINK = 0xFFFFFFFFu;

// Initial links.  lab_v[v] = the vertex across v's paired edge, or v for a minimum.
// lab_c[v] = owner of the cube across the quad paired with v's cube, v for a maximum,
// NO_LINK if that quad is on the boundary or v owns no cube.
__global__ void __launch_bounds__(THREADS) init_links(Geom g, const uint32_t* __restrict__ words,
                                                      uint32_t* __restrict__ lab_v, uint32_t* __restrict__ lab_c,
                                                      uint32_t* __restrict__ status) {
    const int64_t v = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (v >= g.nverts) return;
    const uint32_t w = words[v];
    const uint32_t qv = g.div_nx.div(uint32_t(v));
    const int x = int(uint32_t(v) - qv * uint32_t(g.nx));
    const int z = int(g.div_ny.div(qv));
    const int y = int(qv - uint32_t(z) * uint32_t(g.ny));
    // vertex slot 0
    const uint32_t cv = slot_code(w, 0);
    int64_t pv = v;
    if (cv >= 1 && cv <= 6) {
        const int axis = (cv - 1) >> 1, sign = (cv & 1) ? -1 : 1;
        int o[3] = {x, y, z};
        const int n[3] = {g.nx, g.ny, g.nz};
        o[axis] += sign;
        if (o[axis] >= 0 && o[axis] < n[axis]) pv = g.vid(o[0], o[1], o[2]);
        else atomicOr(status, ST_INTERNAL);  // a vertex paired with an edge that leaves the grid
    }
    lab_v[v] = uint32_t(pv);
    // cube slot 7
    const uint32_t cc = slot_code(w, 7);
    uint32_t pc = NO_LINK;
    if (cc == 0) {
        pc = uint32_t(v);
    } else if (cc <= 6) {
        const int axis = (cc - 1) >> 1, sign = (cc & 1) ? -1 : 1;
        int o[3] = {x, y, z};
        const int n[3] = {g.nx, g.ny, g.nz};
        o[axis] += sign;
        if (o[axis] >= 0 && o[axis] <= n[axis] - 2) pc = uint32_t(g.vid(o[0], o[1], o[2]));
    }
    lab_c[v] = pc;
}

// One round of in-place pointer jumping over both forests.
__global__ void __launch_bounds__(THREADS) jump_round(int64_t n, uint32_t* __restrict__ lab_v,
                                                      uint32_t* __restrict__ lab_c, uint32_t* __restrict__ changed) {
    const int64_t v = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (v >= n) return;
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
    }
    if (open) *changed = 1;
}

// End of one round: the continue decision (more rounds while some chain is still open, up to the
// iteration cap), the round count, and the graph condition when the loop runs in a graph.
__global__ void jump_decide(Summary* sum, int64_t max_iter, cudaGraphConditionalHandle h, int use_handle) {
    const bool open = sum->loop_flag[0] != 0;
    sum->loop_flag[0] = 0;
    const unsigned long long r = ++sum->jump_rounds;
    bool more = open;
    if (more && int64_t(r) >= max_iter) {
        sum->status |= ST_ITER;
        more = false;
    }
    sum->loop_flag[3] = more ? 1u : 0u;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Vertex indices -> cell ids of the extremum (in place).
__global__ void __launch_bounds__(THREADS) finish_labels(Geom g, uint32_t* __restrict__ lab_v,
                                                         uint32_t* __restrict__ lab_c) {
    const int64_t v = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (v >= g.nverts) return;
    auto cell_of = [&](uint32_t u, int off) {
        const uint32_t q = g.div_nx.div(u);
        const int x = int(u - q * uint32_t(g.nx));
        const int z = int(g.div_ny.div(q));
        const int y = int(q - uint32_t(z) * uint32_t(g.ny));
        return g.cell_id(2 * x + off, 2 * y + off, 2 * z + off);
    };
    lab_v[v] = cell_of(lab_v[v], 0);
    const uint32_t c = lab_c[v];
    lab_c[v] = c == NO_LINK ? NONE : cell_of(c, 1);
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
    uint32_t* vmin;
    uint32_t* cmax;
};

void jump_body(Plan* p, cudaStream_t s, cudaGraphConditionalHandle h, void* ctx) {
    const JumpCtx& c = *static_cast<JumpCtx*>(ctx);
    jump_round<<<blocks(c.n), THREADS, 0, s>>>(c.n, c.vmin, c.cmax, &p->dsum()->loop_flag[0]);
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
    auto* vmin = static_cast<uint32_t*>(p->vmin.ptr);
    auto* cmax = static_cast<uint32_t*>(p->cmax.ptr);
    init_links<<<blocks(g.nverts), THREADS, 0, s>>>(g, static_cast<const uint32_t*>(p->words.ptr), vmin, cmax,
                                                     p->status_word());
    launched(p);
    JumpCtx ctx{g.nverts, vmin, cmax};
    if ((st = run_loop(p, s, 0, 2, jump_body, &ctx))) return st;
    finish_labels<<<blocks(g.nverts), THREADS, 0, s>>>(g, vmin, cmax);
    launched(p);
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

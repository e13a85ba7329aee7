// (a4) Saddle-saddle reachability and (a5, first half) junction nodes.
//
// Sec. 3.2 and Sec. 3.5 "Saddle-Saddle reachability": a BFS over the DAG of 1-2 gradient
// pairs from all 1-saddles at once.  The frontier starts as the 1-saddles; each level
// expands every frontier node along its <= 4 out-edges, marks newly reached 1-cells in a
// visited bitmap and appends them to the next frontier; the traversal ends when a level
// adds nothing.  Where the paper stream-compacts a 4x-sized candidate array after each
// level, here the first thread that sets a visited bit (atomicOr) owns the node and appends
// it with one warp-aggregated atomic per warp, so the next frontier is already compact.
//
// Sec. 3.3 / Sec. 3.5 "Gradient path counting": a junction is a reachable 1-cell that is
// not a 1-saddle and has out-degree > 1.  Junctions are marked in a bitmap with the same
// row layout as the visited set and stream-compacted in cell-id order (scan.cuh), which
// also gives O(1) ranks for the minor's matrix indices.
#include "dag.cuh"
#include "scan.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;

int blocks(int64_t n) { return int((n + THREADS - 1) / THREADS); }

struct CellXYZ {
    int x, y, z;
};
__device__ __forceinline__ CellXYZ decode(const Geom& g, uint32_t id) {
    CellXYZ c;
    const uint32_t q = g.div_rx.div(id);
    c.x = int(id - q * g.rx);
    c.z = int(g.div_ry.div(q));
    c.y = int(q - uint32_t(c.z) * g.ry);
    return c;
}

// Frontier 0: every 1-saddle (cell id -> handle), marked visited.
__global__ void __launch_bounds__(THREADS) bfs_seed(Geom g, const uint32_t* __restrict__ s1, int64_t n1,
                                                    uint32_t* __restrict__ visited, uint32_t* __restrict__ front) {
    const int64_t i = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (i >= n1) return;
    CellXYZ c = decode(g, s1[i]);
    const int axis = (c.x & 1) ? 0 : (c.y & 1) ? 1 : 2;
    const int x = c.x >> 1, y = c.y >> 1, z = c.z >> 1;
    atomicOr(&visited[edge_bitmap_word(g, x, y, z, axis)], 1u << (x & 31));
    front[i] = edge_handle(vid32(g, x, y, z), axis);
}

// One BFS level.  All lanes of a warp reach the aggregated append.
__global__ void __launch_bounds__(THREADS) bfs_expand(Geom g, const uint32_t* __restrict__ words,
                                                      const uint32_t* __restrict__ cur, int64_t ncur,
                                                      uint32_t* __restrict__ visited, uint32_t* __restrict__ info,
                                                      uint32_t* __restrict__ next,
                                                      unsigned long long* __restrict__ next_count, uint64_t cap,
                                                      uint32_t* __restrict__ status) {
    const int64_t i = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    uint32_t found[4];
    int nf = 0;
    if (i < ncur) {
        const uint32_t h = cur[i];
        const Vtx v = vtx_of(g, h >> 2);
        DagTarget t[4];
        const int n = dag_out(g, words, v.x, v.y, v.z, int(h & 3), t);
        info[h] = node_info(n, t);  // read later by the junction marking and the path tracer
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (t[k].kind != 1) continue;
            const uint32_t bit = 1u << (t[k].x & 31);
            const uint32_t old = atomicOr(&visited[edge_bitmap_word(g, t[k].x, t[k].y, t[k].z, t[k].sub)], bit);
            if (!(old & bit)) found[nf++] = edge_handle(t[k].v, t[k].sub);
        }
    }
    // warp-aggregated append of the newly reached nodes
    const int lane = threadIdx.x & 31;
    int incl = nf;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(next_count, (unsigned long long)total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    uint64_t pos = base + uint64_t(incl - nf);
    for (int k = 0; k < nf; ++k, ++pos) {
        if (pos < cap) next[pos] = found[k];
        else atomicOr(status, ST_CAPACITY);
    }
}

// Junction bitmap: one thread per visited word; a set bit whose 1-cell is not critical and
// has more than one out-edge is a junction.
__global__ void __launch_bounds__(THREADS) mark_junctions(Geom g, const uint32_t* __restrict__ words,
                                                          const uint32_t* __restrict__ visited,
                                                          const uint32_t* __restrict__ info,
                                                          uint32_t* __restrict__ junc) {
    const int64_t i = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (i >= g.edge_words()) return;
    uint32_t vis = visited[i];
    uint32_t out = 0;
    if (vis) {
        RowCoord r = decode_row(g, i);
        const int axis = r.c ? 2 : (r.b ? 1 : 0);
        while (vis) {
            const int bit = __ffs(vis) - 1;
            vis &= vis - 1;
            const int x = r.w * 32 + bit;
            const uint32_t v = vid32(g, x, r.y, r.z);
            if (slot_code(words[v], edge_slot(axis)) == 0) continue;  // a 1-saddle
            if (info[edge_handle(v, axis)] == INFO_BRANCH) out |= 1u << bit;
        }
    }
    junc[i] = out;
}

}  // namespace

msc_status run_reachability(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t n1 = p->counts[1];
    const int64_t n_edges = int64_t(g.nx - 1) * g.ny * g.nz + int64_t(g.nx) * (g.ny - 1) * g.nz +
                            int64_t(g.nx) * g.ny * (g.nz - 1);
    if ((st = ensure(p, p->visited, sizeof(uint32_t) * size_t(g.edge_words())))) return st;
    if ((st = ensure(p, p->qcount, sizeof(unsigned long long) * 2))) return st;
    if ((st = ensure(p, p->node_info, sizeof(uint32_t) * 4 * size_t(g.nverts)))) return st;
    if ((st = ensure(p, p->frontier[0], sizeof(uint32_t) * size_t(n1 ? n1 : 1)))) return st;
    auto* visited = static_cast<uint32_t*>(p->visited.ptr);
    auto* qcount = static_cast<unsigned long long*>(p->qcount.ptr);
    if ((st = check_cuda(p, cudaMemsetAsync(visited, 0, sizeof(uint32_t) * size_t(g.edge_words()), s),
                         "memset visited")))
        return st;
    int cur = 0;
    if (n1) {
        bfs_seed<<<blocks(n1), THREADS, 0, s>>>(g, static_cast<const uint32_t*>(p->cells[1].ptr), n1, visited,
                                                static_cast<uint32_t*>(p->frontier[0].ptr));
        launched(p);
    }
    int64_t ncur = n1, levels = 0, reached = n1;
    while (ncur > 0) {
        if (levels >= p->opts.max_iterations) return fail(p, MSC_ERR_ITER_LIMIT, "BFS exceeded the iteration cap");
        ++levels;
        const int64_t cap = std::min<int64_t>(4 * ncur, n_edges);
        if ((st = ensure(p, p->frontier[cur ^ 1], sizeof(uint32_t) * size_t(cap)))) return st;
        if ((st = check_cuda(p, cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), s), "memset qcount")))
            return st;
        bfs_expand<<<blocks(ncur), THREADS, 0, s>>>(g, static_cast<const uint32_t*>(p->words.ptr),
                                                    static_cast<const uint32_t*>(p->frontier[cur].ptr), ncur, visited,
                                                    static_cast<uint32_t*>(p->node_info.ptr),
                                                    static_cast<uint32_t*>(p->frontier[cur ^ 1].ptr), qcount,
                                                    uint64_t(cap), static_cast<uint32_t*>(p->status.ptr));
        launched(p);
        unsigned long long nn = 0;
        if ((st = check_cuda(p, cudaMemcpyAsync(&nn, qcount, sizeof(nn), cudaMemcpyDeviceToHost, s), "qcount copy")))
            return st;
        if ((st = check_cuda(p, cudaStreamSynchronize(s), "bfs sync"))) return st;
        if (int64_t(nn) > cap) return fail(p, MSC_ERR_CUDA, "internal: BFS frontier overflow");
        cur ^= 1;
        ncur = int64_t(nn);
        reached += ncur;
    }
    p->stats.n_bfs_levels = levels;
    p->stats.n_reachable = reached;
    return check_cuda(p, cudaGetLastError(), "bfs launch");
}

msc_status run_junctions(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t nw = g.edge_words();
    if ((st = ensure(p, p->junc_bits, sizeof(uint32_t) * size_t(nw)))) return st;
    if ((st = ensure(p, p->junc_prefix, sizeof(uint32_t) * size_t(nw)))) return st;
    mark_junctions<<<blocks(nw), THREADS, 0, s>>>(g, static_cast<const uint32_t*>(p->words.ptr),
                                                  static_cast<const uint32_t*>(p->visited.ptr),
                                                  static_cast<const uint32_t*>(p->node_info.ptr),
                                                  static_cast<uint32_t*>(p->junc_bits.ptr));
    launched(p);
    if ((st = check_cuda(p, cudaGetLastError(), "mark_junctions launch"))) return st;
    EdgeSource src{};
    src.g = g;
    src.bits = static_cast<const uint32_t*>(p->junc_bits.ptr);
    src.prefix = static_cast<uint32_t*>(p->junc_prefix.ptr);
    src.status = static_cast<uint32_t*>(p->status.ptr);
    unsigned long long tot = 0;
    if ((st = compaction_count(p, s, src, 1, &tot))) return st;
    p->n_junctions = int64_t(tot);
    p->stats.n_junctions = int64_t(tot);
    if ((st = ensure(p, p->junc_cells, sizeof(uint32_t) * size_t(tot ? tot : 1)))) return st;
    src.out = static_cast<uint32_t*>(p->junc_cells.ptr);
    src.cap = tot;
    return compaction_emit(p, s, src, 1);
}

}  // namespace msc

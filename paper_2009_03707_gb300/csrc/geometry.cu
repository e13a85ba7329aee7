// The cells along every saddle-extremum arc, on request (Sec. 3.4 and Sec. 3.5 "Data structure":
// the complex keeps its arcs' geometry beside their end points).  An arc is the V-path (Sec. 2.2)
// that leaves its saddle: descending from a 1-saddle through vertex-edge pairs to a minimum,
// ascending from a 2-saddle through cube-quad pairs to a maximum, or out of the domain through a
// boundary quad.  The pass's labels give each arc's end point; the geometry needs the path itself,
// so one thread walks one arc in the packed gradient words: once to count its cells, then, after a
// scan of the counts into offsets, again to write them.  The walks are independent and read only
// the words; an arc that took more steps than the grid has vertices would be a cycle, which the
// gradient cannot have, and raises ST_INTERNAL.
#include "rowscan.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;

struct Coord {
    int x, y, z;
};

__device__ __forceinline__ Coord decode(const Geom& g, uint32_t id) {
    Coord c;
    const uint32_t q = g.div_rx.div(id);
    c.x = int(id - q * g.rx);
    c.z = int(g.div_ry.div(q));
    c.y = int(q - uint32_t(c.z) * g.ry);
    return c;
}

// Appends a cell: counted always, written when out is given.
struct Emit {
    uint32_t* out;
    uint32_t n;
    __device__ __forceinline__ void operator()(uint32_t cell) {
        if (out) out[n] = cell;
        ++n;
    }
};

// Walks arc a (a < 2*n1: the 1-saddle a/2, its lower-coordinate vertex for even a; otherwise the
// 2-saddle (a - 2*n1)/2, its cofacet cube on the - side for even a - 2*n1) and emits its cells.
__device__ void walk_arc(const Geom& g, const uint32_t* __restrict__ words, int64_t a, int64_t n1,
                         const uint32_t* __restrict__ s1, const uint32_t* __restrict__ s2, Emit& emit,
                         uint32_t* status) {
    const int64_t limit = g.nverts;  // every step reaches a new vertex (or cube)
    if (a < 2 * n1) {
        const uint32_t e = s1[a >> 1];
        const Coord c = decode(g, e);
        const int up = int(a & 1);
        int v[3] = {(c.x + up) >> 1, (c.y + up) >> 1, (c.z + up) >> 1};
        emit(e);
        emit(g.cell_id(2 * v[0], 2 * v[1], 2 * v[2]));
        for (int64_t steps = 0;; ++steps) {
            const uint32_t code = slot_code(words[g.vid(v[0], v[1], v[2])], 0);
            if (code == 0) return;  // a minimum
            if (code > 6 || steps > limit) {
                atomicOr(status, ST_INTERNAL);
                return;
            }
            const int axis = int(code - 1) >> 1, sign = (code & 1) ? -1 : 1;
            int ed[3] = {2 * v[0], 2 * v[1], 2 * v[2]};
            ed[axis] += sign;  // the edge v is paired with
            emit(g.cell_id(ed[0], ed[1], ed[2]));
            v[axis] += sign;  // its other vertex
            emit(g.cell_id(2 * v[0], 2 * v[1], 2 * v[2]));
        }
    }
    const int64_t b = a - 2 * n1;
    const uint32_t q = s2[b >> 1];
    const Coord qc = decode(g, q);
    int d[3] = {qc.x, qc.y, qc.z};
    const int axis = !(d[0] & 1) ? 0 : !(d[1] & 1) ? 1 : 2;
    const int ext[3] = {2 * g.nx - 1, 2 * g.ny - 1, 2 * g.nz - 1};
    const int n[3] = {g.nx, g.ny, g.nz};
    emit(q);
    d[axis] += (b & 1) ? 1 : -1;
    if (d[axis] < 0 || d[axis] >= ext[axis]) return;  // no cube on that side
    int o[3] = {d[0] >> 1, d[1] >> 1, d[2] >> 1};  // the cube's owner vertex
    emit(g.cell_id(d[0], d[1], d[2]));
    for (int64_t steps = 0;; ++steps) {
        const uint32_t code = slot_code(words[g.vid(o[0], o[1], o[2])], 7);
        if (code == 0) return;  // a maximum
        if (code > 6 || steps > limit) {
            atomicOr(status, ST_INTERNAL);
            return;
        }
        const int ax = int(code - 1) >> 1, sign = (code & 1) ? -1 : 1;
        int cq[3] = {2 * o[0] + 1, 2 * o[1] + 1, 2 * o[2] + 1};
        cq[ax] += sign;  // the quad the cube is paired with
        emit(g.cell_id(cq[0], cq[1], cq[2]));
        o[ax] += sign;  // the cube across it, if the grid has one
        if (o[ax] < 0 || o[ax] > n[ax] - 2) return;  // the path leaves the domain
        emit(g.cell_id(2 * o[0] + 1, 2 * o[1] + 1, 2 * o[2] + 1));
    }
}

__global__ void __launch_bounds__(THREADS) arc_lengths(Geom g, const uint32_t* __restrict__ words, int64_t n1,
                                                       int64_t n_arcs, const uint32_t* __restrict__ s1,
                                                       const uint32_t* __restrict__ s2, uint32_t* __restrict__ len,
                                                       uint32_t* status) {
    for (int64_t a = int64_t(blockIdx.x) * THREADS + threadIdx.x; a < n_arcs; a += int64_t(gridDim.x) * THREADS) {
        Emit e{nullptr, 0};
        walk_arc(g, words, a, n1, s1, s2, e, status);
        len[a] = e.n;
    }
}

__global__ void __launch_bounds__(THREADS) arc_cells(Geom g, const uint32_t* __restrict__ words, int64_t n1,
                                                     int64_t n_arcs, const uint32_t* __restrict__ s1,
                                                     const uint32_t* __restrict__ s2, const int64_t* __restrict__ off,
                                                     uint32_t* __restrict__ cells, uint32_t* status) {
    for (int64_t a = int64_t(blockIdx.x) * THREADS + threadIdx.x; a < n_arcs; a += int64_t(gridDim.x) * THREADS) {
        Emit e{cells + off[a], 0};
        walk_arc(g, words, a, n1, s1, s2, e, status);
    }
}

}  // namespace

// Builds the arcs' offsets and cells into the plan (host-synchronised: the total sizes the cells).
msc_status build_arc_geometry(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    const int64_t n1 = p->counts[1], n_arcs = 2 * (p->counts[1] + p->counts[2]);
    msc_status st;
    if ((st = ensure(p, p->geo_len, sizeof(uint32_t) * size_t(n_arcs + 1)))) return st;
    if ((st = ensure(p, p->geo_off, sizeof(int64_t) * size_t(n_arcs + 1)))) return st;
    if ((st = ensure(p, p->geo_scan, row_scan_scratch_bytes(n_arcs)))) return st;
    const auto* words = static_cast<const uint32_t*>(p->words.ptr);
    const auto* s1 = static_cast<const uint32_t*>(p->cells[1].ptr);
    const auto* s2 = static_cast<const uint32_t*>(p->cells[2].ptr);
    auto* len = static_cast<uint32_t*>(p->geo_len.ptr);
    auto* off = static_cast<int64_t*>(p->geo_off.ptr);
    if (n_arcs) {
        arc_lengths<<<grid_cap(p, n_arcs, THREADS), THREADS, 0, s>>>(g, words, n1, n_arcs, s1, s2, len,
                                                                     p->status_word());
        launched(p);
    }
    if ((st = check_cuda(p, row_scan(p, len, nullptr, n_arcs, off,
                                     static_cast<unsigned long long*>(p->geo_scan.ptr), s),
                         "arc geometry scan")))
        return st;
    int64_t total = 0;
    if ((st = check_cuda(p, cudaMemcpyAsync(&total, off + n_arcs, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                         "arc geometry total")))
        return st;
    if ((st = check_status_word(p, s))) return st;  // synchronises
    if ((st = ensure(p, p->geo_cells, sizeof(uint32_t) * size_t(total + 1)))) return st;
    if (n_arcs) {
        arc_cells<<<grid_cap(p, n_arcs, THREADS), THREADS, 0, s>>>(g, words, n1, n_arcs, s1, s2, off,
                                                                   static_cast<uint32_t*>(p->geo_cells.ptr),
                                                                   p->status_word());
        launched(p);
    }
    p->geo_cells_n = total;
    return check_cuda(p, cudaGetLastError(), "arc geometry launch");
}

}  // namespace msc

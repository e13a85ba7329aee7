// The cells along every saddle-extremum arc, on request (Sec. 3.4 and Sec. 3.5 "Data structure":
// the complex keeps its arcs' geometry beside their end points).  An arc is the V-path (Sec. 2.2)
// that leaves its saddle: descending from a 1-saddle through vertex-edge pairs to a minimum,
// ascending from a 2-saddle through cube-quad pairs to a maximum, or out of the domain through a
// boundary quad.  The pass's labels give each arc's end point; the geometry needs the path itself,
// so one thread walks one arc in the packed gradient words: once to count its cells, then, after a
// scan of the counts into offsets, again to write them.  The walks are independent and read only
// the words; an arc that took more steps than the grid has vertices would be a cycle, which the
// gradient cannot have, and raises ST_INTERNAL.  The saddle-saddle arcs of multiplicity 1 follow
// (their own comment below).
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

// ---- saddle-saddle arcs of multiplicity 1 ---------------------------------------------------
// A D* entry (s, t) of count 1 is one V-path (Sec. 2.2) from the 2-saddle t down to the 1-saddle
// s; walked from s against the gradient it is s, then (quad, 1-cell) per step, then t.  The minor
// says which way it goes: at a source (s, or a junction the path reaches) exactly one traced slot
// leads on to t -- a slot whose destination is t itself, or a junction whose row of J (the path
// counts from junctions to 2-saddles, junction_dp.cu) holds t.  Along the slot the path is the
// simple path the trace followed: a quad, the 1-cell it is paired with, that 1-cell's one cofacet
// quad (other than its partner) that is critical or paired with a 1-cell, ... up to the slot's
// junction or to t.  A thread per D* entry walks it, once to count and once to write.

struct SsArgs {
    Geom g;
    const uint32_t* words;
    const uint32_t* s1;
    const uint32_t* s2;
    const uint32_t* junc_cells;
    const uint32_t* tgt;    // 4 destination ranks per source (1-saddles, then junctions)
    const uint32_t* kinds;  // per source, byte k: kind of slot k (1 junction, 2 2-saddle, 0 none)
    const unsigned long long* j_off;  // J row of each junction: offset and length in the pool
    const uint32_t* j_len;
    const uint32_t* j_col;  // pool columns (2-saddle ranks), ascending within a row
    const int64_t* rowptr;  // D* CSR over 1-saddle ranks
    const uint32_t* erow;   // the row of every D* entry
    const uint32_t* col;
    const unsigned long long* cnt;
    int64_t n1, nnz;
    uint32_t* status;
};

struct C3 {
    int c[3];
};

__device__ __forceinline__ C3 coords(const Geom& g, uint32_t id) {
    const Coord k = decode(g, id);
    return C3{{k.x, k.y, k.z}};
}

__device__ __forceinline__ uint32_t id_of(const Geom& g, const C3& c) { return g.cell_id(c.c[0], c.c[1], c.c[2]); }

// The 3-bit code of cell c in its owner's word.
__device__ __forceinline__ uint32_t code_of(const Geom& g, const uint32_t* words, const C3& c) {
    const int slot = (c.c[0] & 1) | ((c.c[1] & 1) << 1) | ((c.c[2] & 1) << 2);
    return slot_code(words[g.vid(c.c[0] >> 1, c.c[1] >> 1, c.c[2] >> 1)], slot);
}

// Cofacet quad k of edge e in the trace's slot order: along the axis after e's odd axis (k = 0, 1:
// - then + side), then the axis before it (k = 2, 3); false outside the grid.
__device__ __forceinline__ bool cofacet_quad(const Geom& g, const C3& e, int k, C3& q) {
    const int a = (e.c[0] & 1) ? 0 : (e.c[1] & 1) ? 1 : 2;
    const int b = k < 2 ? (a == 2 ? 0 : a + 1) : (a == 0 ? 2 : a - 1);
    const int ext = 2 * (b == 0 ? g.nx : b == 1 ? g.ny : g.nz) - 1;
    q = e;
    q.c[b] += (k & 1) ? 1 : -1;
    return q.c[b] >= 0 && q.c[b] < ext;
}

// True if quad q (code qc, 1..6) is paired with a 1-cell: its partner lies along one of its odd axes.
__device__ __forceinline__ bool paired_down(const C3& q, uint32_t qc) {
    return qc >= 1 && qc <= 6 && (q.c[int(qc - 1) >> 1] & 1);
}

__device__ __forceinline__ C3 partner(C3 c, uint32_t code) {
    c.c[int(code - 1) >> 1] += (code & 1) ? -1 : 1;
    return c;
}

// True if row j of J holds column t (binary search).
__device__ __forceinline__ bool j_has(const SsArgs& a, uint32_t j, uint32_t t) {
    const uint32_t* r = a.j_col + a.j_off[j];
    uint32_t lo = 0, hi = a.j_len[j];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (r[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    return lo < a.j_len[j] && r[lo] == t;
}

// Walks the path of entry (row, t); false (and ST_INTERNAL) if the minor and the gradient disagree.
__device__ bool walk_ss(const SsArgs& a, int64_t row, uint32_t t, Emit& emit) {
    const Geom& g = a.g;
    const uint32_t tcell = a.s2[t];
    uint32_t src = uint32_t(row);  // source index in the trace
    C3 e = coords(g, a.s1[row]);
    emit(a.s1[row]);
    const int64_t limit = 3 * g.nverts;  // cells the walk may emit before it must have repeated one
    for (;;) {
        const uint32_t kw = a.kinds[src];
        int slot = -1, hits = 0;
        for (int k = 0; k < 4; ++k) {
            const uint32_t kind = trace_kind(kw, k), d = a.tgt[4 * int64_t(src) + k];
            if ((kind == 2 && d == t) || (kind == 1 && j_has(a, d, t))) {
                slot = k;
                ++hits;
            }
        }
        if (hits != 1) return false;
        const uint32_t kind = trace_kind(kw, slot), dest = a.tgt[4 * int64_t(src) + slot];
        const uint32_t jcell = kind == 1 ? a.junc_cells[dest] : 0xFFFFFFFFu;
        C3 q;
        if (!cofacet_quad(g, e, slot, q)) return false;
        for (;;) {
            emit(id_of(g, q));
            const uint32_t qc = code_of(g, a.words, q);
            if (qc == 0) return kind == 2 && id_of(g, q) == tcell;  // reached a 2-saddle
            if (!paired_down(q, qc) || int64_t(emit.n) > limit) return false;
            e = partner(q, qc);
            const uint32_t eid = id_of(g, e);
            emit(eid);
            if (eid == jcell) {  // the slot's junction: the next source
                src = uint32_t(a.n1) + dest;
                break;
            }
            // e's one successor: a cofacet quad other than q, critical or paired with a 1-cell
            int found = 0;
            C3 nq = q;
            for (int k = 0; k < 4; ++k) {
                C3 c;
                if (!cofacet_quad(g, e, k, c) || id_of(g, c) == id_of(g, q)) continue;
                const uint32_t cc = code_of(g, a.words, c);
                if (cc == 0 || paired_down(c, cc)) {
                    nq = c;
                    ++found;
                }
            }
            if (found != 1) return false;
            q = nq;
        }
    }
}

// The row of every D* entry, a thread per row.
__global__ void __launch_bounds__(THREADS) ss_entry_rows(const int64_t* __restrict__ rowptr, int64_t n1,
                                                         uint32_t* __restrict__ erow) {
    for (int64_t r = int64_t(blockIdx.x) * THREADS + threadIdx.x; r < n1; r += int64_t(gridDim.x) * THREADS)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) erow[k] = uint32_t(r);
}

__global__ void __launch_bounds__(THREADS) ss_lengths(SsArgs a, uint32_t* __restrict__ len) {
    for (int64_t k = int64_t(blockIdx.x) * THREADS + threadIdx.x; k < a.nnz; k += int64_t(gridDim.x) * THREADS) {
        Emit e{nullptr, 0};
        if (a.cnt[k] == 1 && !walk_ss(a, a.erow[k], a.col[k], e)) atomicOr(a.status, ST_INTERNAL);
        len[k] = a.cnt[k] == 1 ? e.n : 0u;
    }
}

__global__ void __launch_bounds__(THREADS) ss_cells(SsArgs a, const int64_t* __restrict__ off,
                                                    uint32_t* __restrict__ cells) {
    for (int64_t k = int64_t(blockIdx.x) * THREADS + threadIdx.x; k < a.nnz; k += int64_t(gridDim.x) * THREADS) {
        if (a.cnt[k] != 1) continue;
        Emit e{cells + off[k], 0};
        if (!walk_ss(a, a.erow[k], a.col[k], e)) atomicOr(a.status, ST_INTERNAL);
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

// Builds the saddle-saddle arcs' offsets (one per D* entry, in CSR order) and cells into the plan.
// Needs the pass's D* and the rows of J (the caller makes sure both are current); host-synchronised.
msc_status build_ss_geometry(Plan* p, cudaStream_t s) {
    const int64_t nnz = p->dstar_nnz;
    msc_status st;
    if ((st = ensure(p, p->ss_len, sizeof(uint32_t) * size_t(nnz + 1)))) return st;
    if ((st = ensure(p, p->ss_off, sizeof(int64_t) * size_t(nnz + 1)))) return st;
    if ((st = ensure(p, p->ss_scan, row_scan_scratch_bytes(nnz)))) return st;
    if ((st = ensure(p, p->ss_row, sizeof(uint32_t) * size_t(nnz + 1)))) return st;
    SsArgs a{};
    a.g = p->g;
    a.words = static_cast<const uint32_t*>(p->words.ptr);
    a.s1 = static_cast<const uint32_t*>(p->cells[1].ptr);
    a.s2 = static_cast<const uint32_t*>(p->cells[2].ptr);
    a.junc_cells = static_cast<const uint32_t*>(p->junc_cells.ptr);
    a.tgt = static_cast<const uint32_t*>(p->trace.ptr);
    a.kinds = static_cast<const uint32_t*>(p->trace_kinds.ptr);
    a.j_off = static_cast<const unsigned long long*>(p->dp_j_off.ptr);
    a.j_len = static_cast<const uint32_t*>(p->dp_j_len.ptr);
    a.j_col = static_cast<const uint32_t*>(p->dp_pool_col.ptr);
    a.rowptr = static_cast<const int64_t*>(p->dstar_rowptr.ptr);
    a.erow = static_cast<const uint32_t*>(p->ss_row.ptr);
    a.col = static_cast<const uint32_t*>(p->dstar_col.ptr);
    a.cnt = static_cast<const unsigned long long*>(p->dstar_count.ptr);
    a.n1 = p->counts[1];
    a.nnz = nnz;
    a.status = p->status_word();
    auto* len = static_cast<uint32_t*>(p->ss_len.ptr);
    auto* off = static_cast<int64_t*>(p->ss_off.ptr);
    if (nnz) {
        ss_entry_rows<<<grid_cap(p, a.n1, THREADS), THREADS, 0, s>>>(a.rowptr, a.n1, static_cast<uint32_t*>(p->ss_row.ptr));
        ss_lengths<<<grid_cap(p, nnz, THREADS), THREADS, 0, s>>>(a, len);
        launched(p, 2);
    }
    if ((st = check_cuda(p, row_scan(p, len, nullptr, nnz, off, static_cast<unsigned long long*>(p->ss_scan.ptr), s),
                         "saddle-saddle geometry scan")))
        return st;
    int64_t total = 0;
    if ((st = check_cuda(p, cudaMemcpyAsync(&total, off + nnz, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                         "saddle-saddle geometry total")))
        return st;
    if ((st = check_status_word(p, s))) return st;  // synchronises
    if ((st = ensure(p, p->ss_cells, sizeof(uint32_t) * size_t(total + 1)))) return st;
    if (nnz) {
        ss_cells<<<grid_cap(p, nnz, THREADS), THREADS, 0, s>>>(a, off, static_cast<uint32_t*>(p->ss_cells.ptr));
        launched(p);
    }
    p->ss_cells_n = total;
    return check_cuda(p, cudaGetLastError(), "saddle-saddle geometry launch");
}

}  // namespace msc

// (a5) DAG minor: simple-path tracing and the adjacency matrices A, B, B*, D.
//
// Sec. 3.3 "DAG minor construction" and Sec. 3.5 "Gradient path counting": every maximal
// simple path of the reachable DAG is contracted to one edge.  From each out-edge of every
// 1-saddle and junction the path follows the unique successor until it reaches a junction
// or a 2-saddle; a path that runs into a node without successors is dropped.  Each traced
// path is one unit of multiplicity of its (source, destination) entry in
// A (1-saddle -> junction), B (junction -> junction), B* (junction -> 2-saddle) or
// D (1-saddle -> 2-saddle).
//
// The paper traces all paths in lock step with a stream compaction per step and builds the
// matrices through adjacency lists and cuSPARSE.  Here one thread traces its source's <= 4
// paths to the end (no global step barrier), and the destinations -- ranked in O(1) from
// the junction and critical-cell bitmaps -- are stored as a fixed 4-slot trace per source.
// The path-count stage reads that trace directly as the minor's adjacency; CSR matrices are
// built from it (count, scan, fill) for the ABI and the statistics.
#include "dag.cuh"
#include "rowscan.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;
int blocks(int64_t n) { return int((n + THREADS - 1) / THREADS); }

__device__ __forceinline__ uint32_t bit_rank(const uint32_t* bits, const uint32_t* prefix, int64_t wi, int bit) {
    return prefix[wi] + __popc(bits[wi] & ((1u << bit) - 1u));
}

struct TraceArgs {
    Geom g;
    const uint32_t* words;
    const uint32_t* s1;
    const uint32_t* junc_cells;
    const uint32_t* junc_bits;
    const uint32_t* junc_prefix;
    const uint32_t* crit_bits;
    const uint32_t* crit_prefix;
    const uint32_t* info;  // per reachable 1-cell (info_index): dead end, branch point, or its one successor
    uint32_t* tgt;    // 4 per source: destination rank
    uint8_t* kinds;   // 4 per source: 0 none / 1 junction / 2 2-saddle (read as one word per source)
    uint32_t* cnt[4];  // distinct destinations per row of A, B, B*, D
    const unsigned long long* n1_dev;  // 1-saddles and junctions, counted earlier in the pass
    const unsigned long long* nj_dev;
    int64_t cap1, capj;                // the capacities the buffers were sized for
    unsigned long long* nnz;           // distinct entries of A, B, B*, D (summed here)
    int64_t max_steps;
    uint32_t* status;
};

// Distinct destinations of one source among slots of kind `want`, sorted, with multiplicity.
__device__ __forceinline__ int distinct_targets(const uint32_t* tgt, uint32_t kinds, uint32_t want, uint32_t col[4],
                                                uint32_t mult[4]) {
    uint32_t v[4];
    int n = 0;
    for (int k = 0; k < 4; ++k)
        if (trace_kind(kinds, k) == want) v[n++] = tgt[k];
    for (int i = 1; i < n; ++i)  // insertion sort of <= 4 values
        for (int j = i; j > 0 && v[j - 1] > v[j]; --j) {
            uint32_t tmp = v[j];
            v[j] = v[j - 1];
            v[j - 1] = tmp;
        }
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (m > 0 && col[m - 1] == v[i]) {
            mult[m - 1] += 1;
        } else {
            col[m] = v[i];
            mult[m] = 1;
            ++m;
        }
    }
    return m;
}

// One thread per source (1-saddle or junction): its <= 4 out-edges are found once, then the
// simple paths are followed in an interleaved loop (one independent record load per live path
// per step), and the destinations are ranked and counted per matrix row.  Grid-stride over the
// sources, whose numbers are read on the device.
__global__ void __launch_bounds__(THREADS) trace_kernel(TraceArgs a) {
    const unsigned long long n1 = *a.n1_dev, nj = *a.nj_dev;
    if (pass_retrying(a.status) || !count_fits(a.status, n1, a.cap1) || !count_fits(a.status, nj, a.capj)) return;
    const int64_t N1 = int64_t(n1), NJ = int64_t(nj);
    unsigned long long nnz[4] = {0, 0, 0, 0};
    for (int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x; u < N1 + NJ;
         u += int64_t(gridDim.x) * THREADS) {
    const Geom& g = a.g;
    const uint32_t id = u < N1 ? a.s1[u] : a.junc_cells[u - N1];
    const uint32_t q1 = g.div_rx.div(id);
    const int cx = int(id - q1 * g.rx);
    const int cz = int(g.div_ry.div(q1));
    const int cy = int(q1 - uint32_t(cz) * g.ry);
    const int axis = (cx & 1) ? 0 : (cy & 1) ? 1 : 2;
    DagTarget out[4];
    dag_out(g, a.words, cx >> 1, cy >> 1, cz >> 1, axis, out);
    // per path: the current 1-cell handle while live; at the end the terminal (a junction's
    // handle, or a 2-saddle as bit 31 | owner << 2 | even axis)
    uint32_t h[4], kind[4];
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kind[k] = out[k].kind;
        if (out[k].kind == 1) {
            h[k] = edge_handle(out[k].v, out[k].sub);
            live |= 1u << k;
        } else {
            const uint32_t even = (out[k].sub & 1u) == 0 ? 0u : (out[k].sub & 2u) == 0 ? 1u : 2u;
            h[k] = 0x80000000u | (out[k].v << 2) | even;
        }
    }
    for (int64_t step = 0; live; ++step) {
        if (step > a.max_steps) {
            atomicOr(a.status, ST_ITER);
            break;
        }
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = (live >> k) & 1u ? a.info[info_index(g, h[k])] : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!((live >> k) & 1u)) continue;
            if (w[k] == INFO_DEAD) {  // a dead path: dropped
                kind[k] = 0;
                live &= ~(1u << k);
            } else if (w[k] == INFO_BRANCH) {  // ends at the junction h[k]
                live &= ~(1u << k);
            } else if (w[k] & 0x80000000u) {  // ends at a 2-saddle
                kind[k] = 2;
                h[k] = w[k];
                live &= ~(1u << k);
            } else {
                h[k] = w[k];
            }
        }
    }
    uint32_t rank[4], kinds = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rank[k] = 0;
        if (kind[k] == 1) {
            const Vtx q = vtx_of(g, h[k] >> 2);
            const int64_t wi = edge_bitmap_word(g, q.x, q.y, q.z, int(h[k] & 3));
            if (!((a.junc_bits[wi] >> (q.x & 31)) & 1u)) atomicOr(a.status, ST_INTERNAL);
            rank[k] = bit_rank(a.junc_bits, a.junc_prefix, wi, q.x & 31);
        } else if (kind[k] == 2) {
            const Vtx q = vtx_of(g, (h[k] & 0x7FFFFFFFu) >> 2);
            const int slot = 7 ^ (1 << (h[k] & 3u));
            rank[k] = bit_rank(a.crit_bits, a.crit_prefix, g.slot_word(slot, q.z, q.y, q.x >> 5), q.x & 31);
        }
        kinds |= kind[k] << (8 * k);
    }
    reinterpret_cast<uint4*>(a.tgt)[u] = make_uint4(rank[0], rank[1], rank[2], rank[3]);
    reinterpret_cast<uint32_t*>(a.kinds)[u] = kinds;
    uint32_t col[4], mult[4];
    const bool saddle = u < N1;
    const int64_t row = saddle ? u : u - N1;
    const uint32_t mj = uint32_t(distinct_targets(rank, kinds, 1, col, mult));
    const uint32_t m2 = uint32_t(distinct_targets(rank, kinds, 2, col, mult));
    a.cnt[saddle ? 0 : 1][row] = mj;
    a.cnt[saddle ? 3 : 2][row] = m2;
    nnz[saddle ? 0 : 1] += mj;
    nnz[saddle ? 3 : 2] += m2;
    }
    __shared__ unsigned long long part[4][THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long v = nnz[k];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) part[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long t = 0;
        for (int w = 0; w < THREADS / 32; ++w) t += part[threadIdx.x][w];
        if (t) atomicAdd(&a.nnz[threadIdx.x], t);
    }
}

// which: 0 A, 1 B, 2 B*, 3 D.  Sources 0..n1-1 are 1-saddles (rows of A and D), n1.. are
// junctions (rows of B and B*).
struct CsrArgs {
    int64_t n1, nj;
    const uint32_t* tgt;
    const uint32_t* kinds;
    uint32_t* cnt[4];
    const int64_t* rowptr[4];
    uint32_t* col[4];
    uint32_t* mult[4];
};

__global__ void __launch_bounds__(THREADS) csr_fill(CsrArgs a) {
    const int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (u >= a.n1 + a.nj) return;
    uint32_t col[4], mult[4];
    const bool saddle = u < a.n1;
    const int64_t row = saddle ? u : u - a.n1;
    for (int want = 1; want <= 2; ++want) {
        const int which = saddle ? (want == 1 ? 0 : 3) : (want == 1 ? 1 : 2);
        const int m = distinct_targets(a.tgt + 4 * u, a.kinds[u], uint32_t(want), col, mult);
        const int64_t base = a.rowptr[which][row];
        for (int i = 0; i < m; ++i) {
            a.col[which][base + i] = col[i];
            a.mult[which][base + i] = mult[i];
        }
    }
}

}  // namespace

msc_status run_trace(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t cap1 = p->capturing ? p->caps.cells[1] : p->counts[1];
    const int64_t capj = p->capturing ? p->caps.nj : p->n_junctions;
    const int64_t nsrc = cap1 + capj;
    if ((st = ensure(p, p->trace, sizeof(uint32_t) * 4 * size_t(nsrc ? nsrc : 1)))) return st;
    if ((st = ensure(p, p->trace_kinds, sizeof(uint32_t) * size_t(nsrc ? nsrc : 1)))) return st;
    // per-row counts of A (cap1 rows), B, B* (capj), D (cap1), in that order
    if ((st = ensure(p, p->minor_rowcnt, sizeof(uint32_t) * size_t(2 * nsrc ? 2 * nsrc : 1)))) return st;
    const int64_t rows[4] = {cap1, capj, capj, cap1};
    TraceArgs ta{};
    ta.g = g;
    ta.words = static_cast<const uint32_t*>(p->words.ptr);
    ta.s1 = static_cast<const uint32_t*>(p->cells[1].ptr);
    ta.junc_cells = static_cast<const uint32_t*>(p->junc_cells.ptr);
    ta.junc_bits = static_cast<const uint32_t*>(p->junc_bits.ptr);
    ta.junc_prefix = static_cast<const uint32_t*>(p->junc_prefix.ptr);
    ta.crit_bits = static_cast<const uint32_t*>(p->crit_bits.ptr);
    ta.crit_prefix = static_cast<const uint32_t*>(p->crit_prefix.ptr);
    ta.info = static_cast<const uint32_t*>(p->node_info.ptr);
    ta.tgt = static_cast<uint32_t*>(p->trace.ptr);
    ta.kinds = static_cast<uint8_t*>(p->trace_kinds.ptr);
    size_t off = 0;
    for (int w = 0; w < 4; ++w) {
        p->minor_cnt_off[w] = int64_t(off);
        ta.cnt[w] = static_cast<uint32_t*>(p->minor_rowcnt.ptr) + off;
        off += size_t(rows[w]);
    }
    ta.n1_dev = &p->dsum()->counts[1];
    ta.nj_dev = &p->dsum()->n_junctions;
    ta.cap1 = cap1;
    ta.capj = capj;
    ta.nnz = p->dsum()->minor_nnz;
    ta.max_steps = p->opts.max_iterations;
    ta.status = p->status_word();
    record_event(p, p->tev0, s);
    if (nsrc) {
        trace_kernel<<<grid_cap(p, nsrc, THREADS, 6), THREADS, 0, s>>>(ta);
        launched(p);
    }
    record_event(p, p->tev1, s);
    return check_cuda(p, cudaGetLastError(), "trace launch");
}

// CSR of A, B, B*, D from the trace and its per-row counts (host synchronised; called when the
// matrices are asked for -- the path count reads the trace directly).
msc_status build_minor_csr(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = read_summary(p, s))) return st;
    const int64_t n1 = int64_t(p->hsum->counts[1]), nj = int64_t(p->hsum->n_junctions);
    const int64_t rows[4] = {n1, nj, nj, n1};
    size_t scratch_total = 0;
    size_t scratch_off[4];
    for (int w = 0; w < 4; ++w) {
        scratch_off[w] = scratch_total;
        scratch_total += (row_scan_scratch_bytes(rows[w]) + 255) / 256 * 256;
    }
    if ((st = ensure(p, p->minor_scan, scratch_total ? scratch_total : 1))) return st;
    CsrArgs ca{};
    ca.n1 = n1;
    ca.nj = nj;
    ca.tgt = static_cast<const uint32_t*>(p->trace.ptr);
    ca.kinds = static_cast<const uint32_t*>(p->trace_kinds.ptr);
    for (int w = 0; w < 4; ++w) {
        ca.cnt[w] = static_cast<uint32_t*>(p->minor_rowcnt.ptr) + p->minor_cnt_off[w];
        if ((st = ensure(p, p->minor_rowptr[w], sizeof(int64_t) * size_t(rows[w] + 1)))) return st;
        ca.rowptr[w] = static_cast<const int64_t*>(p->minor_rowptr[w].ptr);
        p->minor_rows[w] = rows[w];
        auto* scratch = reinterpret_cast<unsigned long long*>(static_cast<char*>(p->minor_scan.ptr) + scratch_off[w]);
        if ((st = check_cuda(p,
                             row_scan(p, ca.cnt[w], nullptr, rows[w], static_cast<int64_t*>(p->minor_rowptr[w].ptr),
                                      scratch, s),
                             "minor row scan")))
            return st;
    }
    for (int w = 0; w < 4; ++w) {
        const int64_t nnz = int64_t(p->hsum->minor_nnz[w]);
        p->minor_nnz[w] = nnz;
        if ((st = ensure(p, p->minor_col[w], sizeof(uint32_t) * size_t(nnz ? nnz : 1)))) return st;
        if ((st = ensure(p, p->minor_mult[w], sizeof(uint32_t) * size_t(nnz ? nnz : 1)))) return st;
        ca.col[w] = static_cast<uint32_t*>(p->minor_col[w].ptr);
        ca.mult[w] = static_cast<uint32_t*>(p->minor_mult[w].ptr);
    }
    if (n1 + nj) {
        csr_fill<<<blocks(n1 + nj), THREADS, 0, s>>>(ca);
        launched(p);
    }
    return check_cuda(p, cudaGetLastError(), "csr launch");
}

}  // namespace msc

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

// Distinct destinations of kind `want` among a source's four slots (a slot counts if no earlier
// slot holds the same destination); static indexing keeps everything in registers.
__device__ __forceinline__ uint32_t distinct_count(const uint32_t rank[4], const uint32_t kind[4], uint32_t want) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bool first = kind[k] == want;
#pragma unroll
        for (int j = 0; j < k; ++j) first = first && !(kind[j] == want && rank[j] == rank[k]);
        m += first ? 1u : 0u;
    }
    return m;
}

// One thread per source (1-saddle or junction): its <= 4 out-edges are found once, then the
// simple paths are followed in an interleaved loop (one independent record load per live path
// per step), and the destinations are ranked in O(1) from the junction and critical-cell
// bitmaps.  Grid-stride over the sources, whose numbers are read on the device.  The out-edges
// and the ranks are computed without branches on the slot (selects and predicated loads), and
// all index arithmetic is 32-bit (a plan's bitmap words and vertex ids fit in 32 bits).
__global__ void __launch_bounds__(THREADS, 6) trace_kernel(TraceArgs a) {
    const unsigned long long n1 = *a.n1_dev, nj = *a.nj_dev;
    if (pass_retrying(a.status) || !count_fits(a.status, n1, a.cap1) || !count_fits(a.status, nj, a.capj)) return;
    const Geom& g = a.g;
    const uint32_t nx = uint32_t(g.nx), ny = uint32_t(g.ny), nz = uint32_t(g.nz), W = uint32_t(g.W);
    const uint32_t N1 = uint32_t(n1), NS = uint32_t(n1 + nj);
    unsigned long long nnz_a = 0, nnz_b = 0, nnz_bs = 0, nnz_d = 0;
    // Both source lists are in cell-id order.  The grid is split between them in proportion
    // (whole warps), so every grid-stride step covers the same slab of the volume in both lists
    // and the records of that slab are read from DRAM once rather than once per list.
    const uint32_t G = gridDim.x * THREADS, t = blockIdx.x * THREADS + threadIdx.x;
    uint32_t G1 = NS ? uint32_t((uint64_t(G) * N1 + NS / 2) / NS + 16) / 32 * 32 : 0;
    if (N1 && G1 < 32) G1 = 32;
    if (NS > N1 && G1 > G - 32) G1 = G - 32;
    if (NS == N1) G1 = G;
    const bool sad_thread = t < G1;
    const uint32_t stride = sad_thread ? G1 : G - G1, lim = sad_thread ? N1 : NS - N1;
    for (uint32_t i = sad_thread ? t : t - G1; i < lim; i += stride) {
        const uint32_t u = sad_thread ? i : N1 + i;
        const uint32_t id = sad_thread ? a.s1[i] : a.junc_cells[i];
        const uint32_t q1 = g.div_rx.div(id);
        const uint32_t cx = id - q1 * g.rx;
        const uint32_t cz = g.div_ry.div(q1);
        const uint32_t cy = q1 - cz * g.ry;
        const int axis = (cx & 1u) ? 0 : (cy & 1u) ? 1 : 2;
        const uint32_t x = cx >> 1, y = cy >> 1, z = cz >> 1;
        const uint32_t v = x + nx * (y + ny * z);
        // the cofacet quads lie along the two other axes (slots 0,1: axis+1, slots 2,3: axis+2,
        // - then + side); a quad on the + side shares e's owner, one on the - side is owned by the
        // vertex one step back
        const int bA = axis == 2 ? 0 : axis + 1, bB = axis == 0 ? 2 : axis - 1;
        const uint32_t cA = pick3(bA, x, y, z), cB = pick3(bB, x, y, z);
        const uint32_t nA = pick3(bA, nx, ny, nz), nB = pick3(bB, nx, ny, nz);
        const uint32_t sA = pick3(bA, 1u, nx, nx * ny), sB = pick3(bB, 1u, nx, nx * ny);
        const uint32_t w_own = a.words[v];
        const uint32_t w_A = cA > 0 ? a.words[v - sA] : 0u;
        const uint32_t w_B = cB > 0 ? a.words[v - sB] : 0u;
        const uint32_t own = slot_code(w_own, 1 << axis);
        // per path: the current 1-cell handle while live; at the end the terminal (a junction's
        // handle, or a 2-saddle as bit 31 | owner << 2 | even axis)
        uint32_t h[4], kind[4];
        uint32_t live = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int b = i < 2 ? bA : bB;
            const bool plus = i & 1;
            const uint32_t cb = i < 2 ? cA : cB, sb = i < 2 ? sA : sB, nb = i < 2 ? nA : nB;
            const bool exists = plus ? cb + 1 < nb : cb > 0;
            const bool partner = own == uint32_t(1 + 2 * b + (plus ? 1 : 0));
            const uint32_t ow = plus ? w_own : (i < 2 ? w_A : w_B);
            const uint32_t ov = plus ? v : v - sb;
            const int other = 3 - axis - b;  // the quad's even axis
            const uint32_t qc = slot_code(ow, (1 << axis) | (1 << b));
            const int k = int(qc - 1) >> 1;  // the axis of the quad's partner (when paired)
            const uint32_t tv = (qc & 1u) ? ov : ov + (k == 0 ? 1u : k == 1 ? nx : nx * ny);
            kind[i] = 0;
            h[i] = 0;
            if (exists && !partner) {
                if (qc == 0) {
                    kind[i] = 2;
                    h[i] = 0x80000000u | (ov << 2) | uint32_t(other);
                } else if (k != other) {  // paired with a facet: edge to that facet
                    kind[i] = 1;
                    h[i] = edge_handle(tv, k == axis ? b : axis);
                    live |= 1u << i;
                }
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
        // ranks: a junction's in the junction bitmap (1-cell row layout), a 2-saddle's in the
        // critical bitmap of its slot
        uint32_t rank[4], kinds = 0;
        bool missing = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool isj = kind[k] == 1;
            const uint32_t t = h[k] & 3u;
            const uint32_t tv = (h[k] & 0x7FFFFFFFu) >> 2;
            const uint32_t q = g.div_nx.div(tv);
            const uint32_t tx = tv - q * nx;
            const uint32_t tz = g.div_ny.div(q);
            const uint32_t ty = q - tz * ny;
            const uint32_t wi = isj ? (((tz * 2 + (t == 2)) * ny + ty) * 2 + (t == 1)) * W + (tx >> 5)
                                    : (((7u ^ (1u << t)) * nz + tz) * ny + ty) * W + (tx >> 5);
            const uint32_t* bits = isj ? a.junc_bits : a.crit_bits;
            const uint32_t* pre = isj ? a.junc_prefix : a.crit_prefix;
            rank[k] = 0;
            if (kind[k]) {
                const uint32_t bw = bits[wi];
                rank[k] = pre[wi] + __popc(bw & ((1u << (tx & 31u)) - 1u));
                missing |= isj && !((bw >> (tx & 31u)) & 1u);
            }
            kinds |= kind[k] << (8 * k);
        }
        if (missing) atomicOr(a.status, ST_INTERNAL);
        reinterpret_cast<uint4*>(a.tgt)[u] = make_uint4(rank[0], rank[1], rank[2], rank[3]);
        reinterpret_cast<uint32_t*>(a.kinds)[u] = kinds;
        const bool saddle = u < N1;
        const uint32_t mj = distinct_count(rank, kind, 1), m2 = distinct_count(rank, kind, 2);
        nnz_a += saddle ? mj : 0u;
        nnz_b += saddle ? 0u : mj;
        nnz_bs += saddle ? 0u : m2;
        nnz_d += saddle ? m2 : 0u;
    }
    __shared__ unsigned long long part[4][THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long nnz[4] = {nnz_a, nnz_b, nnz_bs, nnz_d};
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

__global__ void __launch_bounds__(THREADS) csr_count(CsrArgs a) {
    const int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x;
    if (u >= a.n1 + a.nj) return;
    const uint4 t = reinterpret_cast<const uint4*>(a.tgt)[u];
    const uint32_t kw = a.kinds[u];
    const uint32_t rank[4] = {t.x, t.y, t.z, t.w};
    const uint32_t kind[4] = {trace_kind(kw, 0), trace_kind(kw, 1), trace_kind(kw, 2), trace_kind(kw, 3)};
    const bool saddle = u < a.n1;
    const int64_t row = saddle ? u : u - a.n1;
    a.cnt[saddle ? 0 : 1][row] = distinct_count(rank, kind, 1);
    a.cnt[saddle ? 3 : 2][row] = distinct_count(rank, kind, 2);
}

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
    // per-row counts of A (n1 rows), B, B* (nj), D (n1), in that order
    if ((st = ensure(p, p->minor_rowcnt, sizeof(uint32_t) * size_t(2 * (n1 + nj) ? 2 * (n1 + nj) : 1)))) return st;
    CsrArgs ca{};
    ca.n1 = n1;
    ca.nj = nj;
    ca.tgt = static_cast<const uint32_t*>(p->trace.ptr);
    ca.kinds = static_cast<const uint32_t*>(p->trace_kinds.ptr);
    for (int64_t w = 0, off = 0; w < 4; ++w) {
        ca.cnt[w] = static_cast<uint32_t*>(p->minor_rowcnt.ptr) + off;
        off += rows[w];
    }
    if (n1 + nj) {
        csr_count<<<blocks(n1 + nj), THREADS, 0, s>>>(ca);
        launched(p);
    }
    for (int w = 0; w < 4; ++w) {
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

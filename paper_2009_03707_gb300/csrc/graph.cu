// The 1-skeleton as one adjacency over all critical cells, built on the device and copied to
// the host.
//
// Sec. 3.5 "Data structure": the complex is kept as its critical points with, for each, the arcs
// incident on it in both directions (every arc stored twice), filled on the CPU in the paper.
// Here the same structure is a CSR over nodes = critical cells, numbered minima, 1-saddles,
// 2-saddles, maxima (each group in its critical-list order), built from the arc outputs:
//   * a minimum's row: the 1-saddles with an arc to it (the min arcs regrouped by minimum);
//   * a 1-saddle's row: its minima, then its 2-saddles (the row of D*);
//   * a 2-saddle's row: its 1-saddles (the column of D*, transpose.cu), then its maxima;
//   * a maximum's row: the 2-saddles with an arc to it (the max arcs regrouped by maximum).
// Node ids grow along every row.  The multiplicity of an entry is the number of arcs between
// the two nodes: a D* entry's path count, and 1 or 2 for a saddle-extremum pair (a saddle whose
// two arcs reach the same extremum).  Arcs that leave the domain (NONE) are left out.
#include "radix.cuh"

namespace msc {

namespace {

constexpr uint32_t NONE_CELL = 0xFFFFFFFFu;

// Rank of a vertex cell (minimum) or cube cell (maximum) in its critical list, from the
// per-slot critical bitmaps and their prefixes (slot 0 for vertices, slot 7 for cubes).
__device__ __forceinline__ uint32_t extremum_rank(const Geom& g, const uint32_t* bits, const uint32_t* prefix,
                                                  uint32_t cell, int slot) {
    const uint32_t q = g.div_rx.div(cell);
    const uint32_t cx = cell - q * g.rx;
    const uint32_t cz = g.div_ry.div(q);
    const uint32_t cy = q - cz * g.ry;
    const uint32_t x = cx >> 1, y = cy >> 1, z = cz >> 1;
    const int64_t wi = g.slot_word(slot, int(z), int(y), int(x >> 5));
    return prefix[wi] + __popc(bits[wi] & ((1u << (x & 31u)) - 1u));
}

// Extremum ranks of the saddle arcs: arcs[2i], arcs[2i+1] of saddle i -> key (extremum rank, or
// `none_key` for an arc that leaves the domain, counted in *n_none), value = saddle index.
__global__ void __launch_bounds__(256) arc_pairs(Geom g, const uint32_t* __restrict__ arcs, int64_t nsad, int slot,
                                                 const uint32_t* __restrict__ bits,
                                                 const uint32_t* __restrict__ prefix, uint32_t none_key,
                                                 uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                                                 unsigned long long* __restrict__ n_none) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < 2 * nsad;
         i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t c = arcs[i];
        if (c == NONE_CELL) atomicAdd(n_none, 1ull);
        key[i] = c == NONE_CELL ? none_key : extremum_rank(g, bits, prefix, c, slot);
        val[i] = uint32_t(i >> 1);
    }
}

// The two extremum ranks of saddle i (keys in arc order), sorted, merged, those >= none_key
// (arcs that leave the domain) dropped: returns how many distinct extrema (0..2) and writes them
// with their multiplicities.
__device__ __forceinline__ int saddle_extrema(const uint32_t* key, int64_t i, uint32_t none_key, uint32_t e[2],
                                              uint32_t m[2]) {
    uint32_t a = key[2 * i], b = key[2 * i + 1];
    if (a > b) {
        const uint32_t t = a;
        a = b;
        b = t;
    }
    int n = 0;
    if (a < none_key) {
        e[n] = a;
        m[n] = 1;
        ++n;
    }
    if (b < none_key) {
        if (n && e[n - 1] == b) {
            ++m[n - 1];
        } else {
            e[n] = b;
            m[n] = 1;
            ++n;
        }
    }
    return n;
}

struct GraphArgs {
    int64_t c0, c1, c2, c3;
    const uint32_t* min_key;   // per 1-saddle arc (arc order): minimum rank
    const uint32_t* max_key;   // per 2-saddle arc: maximum rank, or c3 for an arc that leaves the domain
    const uint32_t* smin_key;  // min arcs sorted by minimum: keys, saddle values
    const uint32_t* smin_val;
    const uint32_t* smax_key;  // max arcs sorted by maximum
    const uint32_t* smax_val;
    int64_t nmax_arcs;         // max arcs with a maximum (those that leave the domain sort last)
    const int64_t* rowptr;     // D* CSR
    const uint32_t* col;
    const unsigned long long* cnt;
    const int64_t* colptr;     // D* CSC
    const uint32_t* row;
    const unsigned long long* ccnt;
    uint32_t* len;             // per node
    const int64_t* nodeptr;
    uint32_t* adj;
    unsigned long long* mult;
};

// Heads of runs of equal (key, value) in a sorted pair list: the first entry of each run.
__device__ __forceinline__ bool run_head(const uint32_t* k, const uint32_t* v, int64_t i) {
    return i == 0 || k[i] != k[i - 1] || v[i] != v[i - 1];
}

// Row lengths of every node.
__global__ void __launch_bounds__(256) graph_lengths(GraphArgs a) {
    const int64_t nodes = a.c0 + a.c1 + a.c2 + a.c3;
    for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < nodes; u += int64_t(gridDim.x) * blockDim.x) {
        if (u >= a.c0 && u < a.c0 + a.c1) {
            const int64_t s = u - a.c0;
            uint32_t e[2], m[2];
            a.len[u] = uint32_t(saddle_extrema(a.min_key, s, uint32_t(a.c0), e, m) + (a.rowptr[s + 1] - a.rowptr[s]));
        } else if (u >= a.c0 + a.c1 && u < a.c0 + a.c1 + a.c2) {
            const int64_t t = u - a.c0 - a.c1;
            uint32_t e[2], m[2];
            a.len[u] = uint32_t((a.colptr[t + 1] - a.colptr[t]) + saddle_extrema(a.max_key, t, uint32_t(a.c3), e, m));
        } else {
            a.len[u] = 0;  // extrema: counted from the sorted arc lists
        }
    }
}

// Extremum rows: one count per run head of the sorted arc lists.
__global__ void __launch_bounds__(256) graph_extremum_lengths(GraphArgs a) {
    const int64_t nmin = 2 * a.c1;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nmin + a.nmax_arcs;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (i < nmin) {
            const uint32_t k = a.smin_key[i];
            if (k < a.c0 && run_head(a.smin_key, a.smin_val, i)) atomicAdd(&a.len[k], 1u);
        } else {
            const int64_t j = i - nmin;
            const uint32_t k = a.smax_key[j];
            if (k < a.c3 && run_head(a.smax_key, a.smax_val, j)) atomicAdd(&a.len[a.c0 + a.c1 + a.c2 + k], 1u);
        }
    }
}

// Saddle rows: extrema and D* row (1-saddles) or D* column and extrema (2-saddles).
__global__ void __launch_bounds__(256) graph_fill_saddles(GraphArgs a) {
    const uint32_t base1 = uint32_t(a.c0), base2 = uint32_t(a.c0 + a.c1), base3 = uint32_t(a.c0 + a.c1 + a.c2);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < a.c1 + a.c2;
         i += int64_t(gridDim.x) * blockDim.x) {
        uint32_t e[2], m[2];
        if (i < a.c1) {
            int64_t at = a.nodeptr[base1 + i];
            const int n = saddle_extrema(a.min_key, i, uint32_t(a.c0), e, m);
            for (int k = 0; k < n; ++k, ++at) {
                a.adj[at] = e[k];
                a.mult[at] = m[k];
            }
            for (int64_t q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q, ++at) {
                a.adj[at] = base2 + a.col[q];
                a.mult[at] = a.cnt[q];
            }
        } else {
            const int64_t t = i - a.c1;
            int64_t at = a.nodeptr[base2 + t];
            for (int64_t q = a.colptr[t]; q < a.colptr[t + 1]; ++q, ++at) {
                a.adj[at] = base1 + a.row[q];
                a.mult[at] = a.ccnt[q];
            }
            const int n = saddle_extrema(a.max_key, t, uint32_t(a.c3), e, m);
            for (int k = 0; k < n; ++k, ++at) {
                a.adj[at] = base3 + e[k];
                a.mult[at] = m[k];
            }
        }
    }
}

// Extremum rows from the sorted arc lists: a run head's place is its row start plus the run
// heads of the same extremum before it, i.e. head_rank - the head rank of the row's first entry.
__global__ void __launch_bounds__(256) graph_fill_extrema(GraphArgs a, const int64_t* __restrict__ head_min,
                                                          const int64_t* __restrict__ head_max) {
    const int64_t nmin = 2 * a.c1;
    const uint32_t base1 = uint32_t(a.c0), base2 = uint32_t(a.c0 + a.c1), base3 = uint32_t(a.c0 + a.c1 + a.c2);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nmin + a.nmax_arcs;
         i += int64_t(gridDim.x) * blockDim.x) {
        const bool is_min = i < nmin;
        const int64_t j = is_min ? i : i - nmin;
        const uint32_t* k = is_min ? a.smin_key : a.smax_key;
        const uint32_t* v = is_min ? a.smin_val : a.smax_val;
        const int64_t n = is_min ? nmin : a.nmax_arcs;
        if (k[j] >= uint32_t(is_min ? a.c0 : a.c3) || !run_head(k, v, j)) continue;
        const unsigned long long m = (j + 1 < n && k[j + 1] == k[j] && v[j + 1] == v[j]) ? 2ull : 1ull;
        // minima rows start at 0 and hold exactly the min-arc run heads in order; maxima rows
        // likewise from the first maximum's row
        const int64_t at = is_min ? head_min[j] : a.nodeptr[base3] + head_max[j];
        a.adj[at] = (is_min ? base1 : base2) + v[j];
        a.mult[at] = m;
    }
}

// 1 for the run heads whose key is an extremum rank (below `limit`), else 0.
__global__ void __launch_bounds__(256) head_flags(const uint32_t* __restrict__ k, const uint32_t* __restrict__ v,
                                                  int64_t n, uint32_t limit, uint32_t* __restrict__ flag) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        flag[i] = k[i] < limit && run_head(k, v, i) ? 1u : 0u;
}

int grid_of(const Plan* p, int64_t n) {
    const int64_t want = (n + 255) / 256;
    return int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(1, p->num_sms)) * 16)));
}

}  // namespace

msc_status build_complex_graph(Plan* p, cudaStream_t s) {
    msc_status st;
    const Geom& g = p->g;
    const int64_t c0 = p->counts[0], c1 = p->counts[1], c2 = p->counts[2], c3 = p->counts[3];
    const int64_t nodes = c0 + c1 + c2 + c3;
    if (nodes >= (int64_t(1) << 32)) return fail(p, MSC_ERR_TOO_LARGE, "2^32 or more critical cells");
    const int64_t na = 2 * std::max(c1, c2);  // arcs of either kind
    // work space: arc keys/values (two buffer pairs), run-head flags and their scan, node lengths
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_mk = carve(sizeof(uint32_t) * size_t(2 * c1)), o_xk = carve(sizeof(uint32_t) * size_t(2 * c2));
    const size_t o_k0 = carve(sizeof(uint32_t) * size_t(na)), o_k1 = carve(sizeof(uint32_t) * size_t(na));
    const size_t o_v0 = carve(sizeof(uint32_t) * size_t(na)), o_v1 = carve(sizeof(uint32_t) * size_t(na));
    const size_t o_smk = carve(sizeof(uint32_t) * size_t(2 * c1)), o_smv = carve(sizeof(uint32_t) * size_t(2 * c1));
    const size_t o_sxk = carve(sizeof(uint32_t) * size_t(2 * c2)), o_sxv = carve(sizeof(uint32_t) * size_t(2 * c2));
    const size_t o_flag = carve(sizeof(uint32_t) * size_t(na));
    const size_t o_hmin = carve(sizeof(int64_t) * size_t(2 * c1 + 1)), o_hmax = carve(sizeof(int64_t) * size_t(2 * c2 + 1));
    const size_t o_len = carve(sizeof(uint32_t) * size_t(nodes));
    const int64_t scan_n = std::max<int64_t>({nodes, na, int64_t(radix_hist_count(na))});
    const size_t o_hist = carve(sizeof(uint32_t) * radix_hist_count(na));
    const size_t o_offs = carve(sizeof(int64_t) * (radix_hist_count(na) + 1));
    const size_t o_scr = carve(row_scan_scratch_bytes(scan_n));
    if ((st = ensure(p, p->graph_work, off))) return st;
    char* w = static_cast<char*>(p->graph_work.ptr);
    auto at = [&](size_t o) { return reinterpret_cast<uint32_t*>(w + o); };
    uint32_t* keys[2] = {at(o_k0), at(o_k1)};
    uint32_t* vals[2] = {at(o_v0), at(o_v1)};
    const RadixSpace ws{at(o_hist), reinterpret_cast<int64_t*>(w + o_offs),
                        reinterpret_cast<unsigned long long*>(w + o_scr)};
    auto* head_min = reinterpret_cast<int64_t*>(w + o_hmin);
    auto* head_max = reinterpret_cast<int64_t*>(w + o_hmax);
    const auto* bits = static_cast<const uint32_t*>(p->crit_bits.ptr);
    const auto* prefix = static_cast<const uint32_t*>(p->crit_prefix.ptr);
    GraphArgs a{};
    a.c0 = c0;
    a.c1 = c1;
    a.c2 = c2;
    a.c3 = c3;
    // arc ends as extremum ranks, then each kind sorted by extremum (stable: saddles ascend); an
    // arc that leaves the domain gets the key one past the last maximum, so it sorts last
    if ((st = ensure(p, p->graph_none, sizeof(unsigned long long)))) return st;
    auto* n_none = static_cast<unsigned long long*>(p->graph_none.ptr);
    if ((st = check_cuda(p, cudaMemsetAsync(n_none, 0, sizeof(unsigned long long), s), "memset"))) return st;
    for (int kind = 0; kind < 2; ++kind) {
        const int64_t nsad = kind == 0 ? c1 : c2;
        uint32_t* key_out = at(kind == 0 ? o_mk : o_xk);
        uint32_t* sk = at(kind == 0 ? o_smk : o_sxk);
        uint32_t* sv = at(kind == 0 ? o_smv : o_sxv);
        if (nsad == 0) continue;
        const auto* arcs = static_cast<const uint32_t*>(kind == 0 ? p->min_arcs.ptr : p->max_arcs.ptr);
        const uint32_t none_key = uint32_t(kind == 0 ? c0 : c3);
        arc_pairs<<<grid_of(p, 2 * nsad), 256, 0, s>>>(g, arcs, nsad, kind == 0 ? 0 : 7, bits, prefix, none_key,
                                                       keys[0], vals[0], n_none);
        launched(p);
        if ((st = check_cuda(p, cudaMemcpyAsync(key_out, keys[0], sizeof(uint32_t) * size_t(2 * nsad),
                                                cudaMemcpyDeviceToDevice, s), "copy")))
            return st;
        int cur = 0;
        if ((st = check_cuda(p, radix_sort_pairs(p, keys, vals, &cur, 2 * nsad, none_key, ws, s), "arc sort")))
            return st;
        if ((st = check_cuda(p, cudaMemcpyAsync(sk, keys[cur], sizeof(uint32_t) * size_t(2 * nsad),
                                                cudaMemcpyDeviceToDevice, s), "copy")) ||
            (st = check_cuda(p, cudaMemcpyAsync(sv, vals[cur], sizeof(uint32_t) * size_t(2 * nsad),
                                                cudaMemcpyDeviceToDevice, s), "copy")))
            return st;
    }
    // max arcs that reach a maximum (every min arc reaches a minimum)
    unsigned long long none_arcs = 0;
    if ((st = check_cuda(p, cudaMemcpyAsync(&none_arcs, n_none, sizeof(none_arcs), cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (st = check_cuda(p, cudaStreamSynchronize(s), "sync")))
        return st;
    const int64_t nmax_arcs = 2 * c2 - int64_t(none_arcs);
    a.min_key = at(o_mk);
    a.max_key = at(o_xk);
    a.smin_key = at(o_smk);
    a.smin_val = at(o_smv);
    a.smax_key = at(o_sxk);
    a.smax_val = at(o_sxv);
    a.nmax_arcs = nmax_arcs;
    a.rowptr = static_cast<const int64_t*>(p->dstar_rowptr.ptr);
    a.col = static_cast<const uint32_t*>(p->dstar_col.ptr);
    a.cnt = static_cast<const unsigned long long*>(p->dstar_count.ptr);
    a.colptr = static_cast<const int64_t*>(p->csc_colptr.ptr);
    a.row = static_cast<const uint32_t*>(p->csc_row.ptr);
    a.ccnt = static_cast<const unsigned long long*>(p->csc_count.ptr);
    a.len = at(o_len);
    // row lengths and the node pointers
    if ((st = ensure(p, p->graph_nodeptr, sizeof(int64_t) * size_t(nodes + 1)))) return st;
    auto* nodeptr = static_cast<int64_t*>(p->graph_nodeptr.ptr);
    a.nodeptr = nodeptr;
    auto* scratch = reinterpret_cast<unsigned long long*>(w + o_scr);
    if (nodes) {
        graph_lengths<<<grid_of(p, nodes), 256, 0, s>>>(a);
        launched(p);
    }
    if (2 * c1 + nmax_arcs) {
        graph_extremum_lengths<<<grid_of(p, 2 * c1 + nmax_arcs), 256, 0, s>>>(a);
        launched(p);
    }
    if ((st = check_cuda(p, row_scan(p, a.len, nullptr, nodes, nodeptr, scratch, s), "node scan"))) return st;
    // run-head ranks of the sorted arc lists (their places in the extremum rows)
    for (int kind = 0; kind < 2; ++kind) {
        const int64_t n = kind == 0 ? 2 * c1 : nmax_arcs;
        int64_t* head = kind == 0 ? head_min : head_max;
        uint32_t* flag = at(o_flag);
        if (n) {
            head_flags<<<grid_of(p, n), 256, 0, s>>>(kind == 0 ? a.smin_key : a.smax_key,
                                                     kind == 0 ? a.smin_val : a.smax_val, n,
                                                     uint32_t(kind == 0 ? c0 : c3), flag);
            launched(p);
        }
        if ((st = check_cuda(p, row_scan(p, flag, nullptr, n, head, scratch, s), "head scan"))) return st;
    }
    int64_t nadj = 0;
    if ((st = check_cuda(p, cudaMemcpyAsync(&nadj, nodeptr + nodes, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                         "copy")) ||
        (st = check_cuda(p, cudaStreamSynchronize(s), "sync")))
        return st;
    if ((st = ensure(p, p->graph_adj, sizeof(uint32_t) * size_t(nadj ? nadj : 1)))) return st;
    if ((st = ensure(p, p->graph_mult, sizeof(unsigned long long) * size_t(nadj ? nadj : 1)))) return st;
    a.adj = static_cast<uint32_t*>(p->graph_adj.ptr);
    a.mult = static_cast<unsigned long long*>(p->graph_mult.ptr);
    if (c1 + c2) {
        graph_fill_saddles<<<grid_of(p, c1 + c2), 256, 0, s>>>(a);
        launched(p);
    }
    if (2 * c1 + nmax_arcs) {
        graph_fill_extrema<<<grid_of(p, 2 * c1 + nmax_arcs), 256, 0, s>>>(a, head_min, head_max);
        launched(p);
    }
    p->graph_nodes = nodes;
    p->graph_nadj = nadj;
    return check_cuda(p, cudaGetLastError(), "graph launch");
}

}  // namespace msc

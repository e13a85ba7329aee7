// Simplification of the 1-skeleton by cancellation of critical-point pairs (Sec. 4), on request.
//
// The paper cancels, in order of persistence, pairs of critical points of consecutive index that
// are joined by exactly one arc (several arcs: a strangulation); a cancellation reroutes the upper
// point's descending arcs to the end points of the lower point's ascending arcs and deletes the
// two points.  It runs the cancellations serially inside subgrids on the CPU and reports that a
// data-parallel form -- an independent set of arcs under the 3-link neighbourhood, cancelled
// together -- is the generic alternative.  Here that form runs on the GPU, in rounds:
//   * keys: (persistence = |value(upper) - value(lower)|, cell id of the upper point, cell id of
//     the lower point), where a critical cell's value is that of its highest vertex;
//   * a round cancels every valid arc (both ends alive, consecutive index, multiplicity 1,
//     persistence <= threshold) whose key is the least among the valid arcs with an end within
//     two links of one of its ends -- so the arcs of one round are more than two links apart and
//     the nodes each cancellation touches (its ends and their neighbours) are disjoint, and the
//     globally least valid arc is always among them;
//   * rounds repeat until no valid arc is left.
// State: the complex as a CSR over nodes = critical cells (numbered as msc_complex_graph), each arc
// in both rows, rows sorted, with exact uint64 multiplicities.  A round is
//   least key of the valid arcs at each node -> least within one link -> within two links ->
//   selection by the upper node -> footprint marking (every touched node learns the one
//   cancellation that touches it) -> per-row merge of the surviving old entries with the sorted
//   list of new neighbours that cancellation gives it (count, scan, fill).
// No global sort is needed: a node's new neighbours all come from one cancellation, in the order
// of the other node's row.
#include "rowscan.cuh"

namespace msc {

namespace {

constexpr int THREADS = 256;
constexpr uint32_t NO_NODE = 0xFFFFFFFFu;

struct Key {
    unsigned long long hi, lo;  // persistence (bits of a non-negative double), upper cell << 32 | lower cell
};
__device__ __forceinline__ bool key_less(const Key& a, const Key& b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ Key key_min(const Key& a, const Key& b) { return key_less(b, a) ? b : a; }
__device__ __forceinline__ Key no_key() { return Key{~0ull, ~0ull}; }

struct SimpArgs {
    int64_t n;            // nodes
    int64_t base[4];      // first node of each index (minima, 1-saddles, 2-saddles, maxima)
    double threshold;
    const uint32_t* cell;  // node -> cell id
    const double* value;   // node -> value of the cell's highest vertex
    const int64_t* ptr;    // current CSR
    const uint32_t* nbr;
    const unsigned long long* mult;
    const uint8_t* alive;
    uint8_t* alive_next;
    Key* m0;
    Key* m1;
    Key* m2;
    uint32_t* sel;      // upper node -> selected lower node, or NO_NODE
    uint32_t* owner;    // touched node -> upper node of the cancellation that touches it, or NO_NODE
    uint8_t* role;      // 1: descending neighbour of the upper node, 2: ascending neighbour of the lower,
                        // 3: another neighbour of either (loses its arc only), 0: untouched
    unsigned long long* factor;  // multiplicity of the touched node's arc to the cancelled node
    uint32_t* flags;    // 1 per selected upper node (for the log positions)
    uint32_t* status;
    unsigned int* any_valid;
};

__device__ __forceinline__ int node_index(const SimpArgs& a, int64_t u) {
    return int(u >= a.base[1]) + int(u >= a.base[2]) + int(u >= a.base[3]);
}

// The key of the arc (u, v) if it is valid, else no_key().
__device__ __forceinline__ Key arc_key(const SimpArgs& a, int64_t u, int64_t v, unsigned long long m) {
    if (m != 1 || !a.alive[u] || !a.alive[v]) return no_key();
    const int iu = node_index(a, u), iv = node_index(a, v);
    if (iu - iv != 1 && iv - iu != 1) return no_key();
    const double pers = fabs(a.value[u] - a.value[v]);
    if (!(pers <= a.threshold)) return no_key();
    const int64_t up = iu > iv ? u : v, lo = iu > iv ? v : u;
    return Key{(unsigned long long)__double_as_longlong(pers),
               ((unsigned long long)a.cell[up] << 32) | (unsigned long long)a.cell[lo]};
}

__global__ void __launch_bounds__(THREADS) simp_values(Geom g, const float* __restrict__ f, int64_t n,
                                                       const uint32_t* __restrict__ cell, double* __restrict__ value) {
    for (int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x; u < n; u += int64_t(gridDim.x) * THREADS) {
        const uint32_t c = cell[u];
        const uint32_t q = g.div_rx.div(c);
        const int cx = int(c - q * g.rx), cz = int(g.div_ry.div(q)), cy = int(q - uint32_t(cz) * g.ry);
        float best = -INFINITY;
        for (int dz = 0; dz <= (cz & 1); ++dz)
            for (int dy = 0; dy <= (cy & 1); ++dy)
                for (int dx = 0; dx <= (cx & 1); ++dx)
                    best = fmaxf(best, f[g.vid((cx >> 1) + dx, (cy >> 1) + dy, (cz >> 1) + dz)]);
        value[u] = double(best);
    }
}

// Least key of the valid arcs at each node; resets the per-round marks.  A live node the previous
// round left untouched (role 0: same row, no neighbour died) keeps its key from that round.
__global__ void __launch_bounds__(THREADS) simp_min0(SimpArgs a, int first) {
    for (int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x; u < a.n; u += int64_t(gridDim.x) * THREADS) {
        Key k = no_key();
        const uint8_t role = first ? 1 : a.role[u];
        const bool keep = a.alive[u] && role == 0;
        if (keep) {
            k = a.m0[u];
        } else {
            if (a.alive[u])
                for (int64_t e = a.ptr[u]; e < a.ptr[u + 1]; ++e) k = key_min(k, arc_key(a, u, a.nbr[e], a.mult[e]));
            a.m0[u] = k;
        }
        // the marks of the previous round (everything in the first): only what was set is cleared
        if (role != 0) {
            a.owner[u] = NO_NODE;
            a.role[u] = 0;
        }
        if (first || a.sel[u] != NO_NODE) {
            a.sel[u] = NO_NODE;
            a.flags[u] = 0;
        }
        a.alive_next[u] = a.alive[u];
        if (k.hi != ~0ull) atomicOr(a.any_valid, 1u);
    }
}

// Least over the closed neighbourhood: out[u] = min(in[u], in[v] for v in row(u)).  With only_valid,
// just at the nodes that have a valid arc (selection reads the second spread only there).
__global__ void __launch_bounds__(THREADS) simp_spread(SimpArgs a, const Key* __restrict__ in, Key* __restrict__ out,
                                                       int only_valid) {
    for (int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x; u < a.n; u += int64_t(gridDim.x) * THREADS) {
        if (only_valid && a.m0[u].hi == ~0ull) continue;
        Key k = in[u];
        for (int64_t e = a.ptr[u]; e < a.ptr[u + 1]; ++e) k = key_min(k, in[a.nbr[e]]);
        out[u] = k;
    }
}

// Selection by the upper node: its valid arc whose key is the least within two links of both ends
// (at most one per node: two valid arcs at one node are within each other's neighbourhood).  Such an
// arc's key k satisfies m0[p] <= k = min(m2[p], m2[q]) <= m2[p] <= m0[p], so it is p's own least key
// and p's least key is the least within two links; only such nodes look at their rows, for that arc.
__global__ void __launch_bounds__(THREADS) simp_select(SimpArgs a) {
    for (int64_t p = int64_t(blockIdx.x) * THREADS + threadIdx.x; p < a.n; p += int64_t(gridDim.x) * THREADS) {
        const Key k0 = a.m0[p];
        if (!a.alive[p] || k0.hi == ~0ull) continue;
        const Key k2 = a.m2[p];
        if (k2.hi != k0.hi || k2.lo != k0.lo) continue;
        const int ip = node_index(a, p);
        for (int64_t e = a.ptr[p]; e < a.ptr[p + 1]; ++e) {
            const uint32_t q = a.nbr[e];
            if (node_index(a, q) != ip - 1) continue;
            const Key k = arc_key(a, p, q, a.mult[e]);
            if (k.hi != k0.hi || k.lo != k0.lo) continue;
            const Key z = a.m2[q];
            if (k.hi == z.hi && k.lo == z.lo) {
                a.sel[p] = q;
                a.flags[p] = 1;
            }
            break;  // keys are distinct: no other arc of p has this one
        }
    }
}

// Footprints of the selected arcs: each descending neighbour of p (other than q) and each ascending
// neighbour of q (other than p) learns its cancellation (role 1, 2); the other neighbours of p and q
// only lose their arc (role 3); p and q die; the log gets (p, q, round).  Every other live node keeps
// its row as it is (role 0).
__global__ void __launch_bounds__(THREADS) simp_mark(SimpArgs a, const int64_t* __restrict__ log_pos, uint32_t* log,
                                                     uint32_t round) {
    for (int64_t p = int64_t(blockIdx.x) * THREADS + threadIdx.x; p < a.n; p += int64_t(gridDim.x) * THREADS) {
        const uint32_t q = a.sel[p];
        if (q == NO_NODE) continue;
        const int iq = node_index(a, q);
        for (int64_t e = a.ptr[p]; e < a.ptr[p + 1]; ++e) {
            const uint32_t x = a.nbr[e];
            if (x == q) continue;
            if (node_index(a, x) != iq) {
                a.role[x] = 3;
                continue;
            }
            a.owner[x] = uint32_t(p);
            a.role[x] = 1;
            a.factor[x] = a.mult[e];
        }
        for (int64_t e = a.ptr[q]; e < a.ptr[q + 1]; ++e) {
            const uint32_t x = a.nbr[e];
            if (x == uint32_t(p)) continue;
            if (node_index(a, x) != iq + 1) {
                a.role[x] = 3;
                continue;
            }
            a.owner[x] = uint32_t(p);
            a.role[x] = 2;
            a.factor[x] = a.mult[e];
        }
        a.alive_next[p] = 0;
        a.alive_next[q] = 0;
        const int64_t at = log_pos[p];
        log[3 * at] = uint32_t(p);
        log[3 * at + 1] = q;
        log[3 * at + 2] = round;
    }
}

// The extra (new) neighbours of node u: the row to walk and the node to skip and the index kept.
struct Extra {
    int64_t from, to;  // range in the current CSR
    uint32_t skip;
    int keep_index;
};

__device__ __forceinline__ Extra extra_of(const SimpArgs& a, int64_t u) {
    Extra x{0, 0, NO_NODE, -1};
    if (a.role[u] != 1 && a.role[u] != 2) return x;
    const uint32_t p = a.owner[u], q = a.sel[p];
    if (a.role[u] == 1) {  // u is a descending neighbour of p: gains q's ascending neighbours
        x.from = a.ptr[q];
        x.to = a.ptr[q + 1];
        x.skip = p;
        x.keep_index = node_index(a, p);
    } else {  // u is an ascending neighbour of q: gains p's descending neighbours
        x.from = a.ptr[p];
        x.to = a.ptr[p + 1];
        x.skip = q;
        x.keep_index = node_index(a, q);
    }
    return x;
}

// Merges row u (entries to surviving nodes) with its extra neighbours; with out_nbr null only
// counts.  Multiplicities: old + factor * (the extra row's multiplicity), overflow -> ST_OVERFLOW.
__device__ int64_t merge_row(const SimpArgs& a, int64_t u, uint32_t* out_nbr, unsigned long long* out_mult) {
    if (!a.alive_next[u]) return 0;
    const uint8_t role = a.role[u];
    if (role == 0) {  // no neighbour dies and none is added: the row as it is
        const int64_t b = a.ptr[u], len = a.ptr[u + 1] - b;
        if (out_nbr)
            for (int64_t k = 0; k < len; ++k) {
                out_nbr[k] = a.nbr[b + k];
                out_mult[k] = a.mult[b + k];
            }
        return len;
    }
    const Extra x = extra_of(a, u);
    int64_t i = a.ptr[u], ie = a.ptr[u + 1], j = x.from, n = 0;
    const unsigned long long fu = (role == 1 || role == 2) ? a.factor[u] : 0ull;
    while (true) {
        while (i < ie && !a.alive_next[a.nbr[i]]) ++i;
        while (j < x.to && (a.nbr[j] == x.skip || node_index(a, a.nbr[j]) != x.keep_index)) ++j;
        const bool hi = i < ie, hj = j < x.to;
        if (!hi && !hj) break;
        const uint32_t vi = hi ? a.nbr[i] : NO_NODE, vj = hj ? a.nbr[j] : NO_NODE;
        const uint32_t v = vi < vj ? vi : vj;
        unsigned long long m = 0;
        if (vi == v) m = a.mult[i++];
        if (vj == v) {
            const unsigned long long mj = a.mult[j++];
            const unsigned long long prod = fu * mj;
            if (mj != 0 && (__umul64hi(fu, mj) != 0)) atomicOr(a.status, ST_OVERFLOW);
            if (m + prod < m) atomicOr(a.status, ST_OVERFLOW);
            m += prod;
        }
        if (out_nbr) {
            out_nbr[n] = v;
            out_mult[n] = m;
        }
        ++n;
    }
    return n;
}

__global__ void __launch_bounds__(THREADS) simp_count(SimpArgs a, uint32_t* __restrict__ len) {
    for (int64_t u = int64_t(blockIdx.x) * THREADS + threadIdx.x; u < a.n; u += int64_t(gridDim.x) * THREADS)
        len[u] = uint32_t(merge_row(a, u, nullptr, nullptr));
}

// A thread per row -- except that when none of a warp's 32 consecutive nodes changes (each either
// untouched or already without arcs), their rows are one contiguous block in both CSRs and the warp
// copies it lane by lane.
__global__ void __launch_bounds__(THREADS) simp_fill(SimpArgs a, const int64_t* __restrict__ ptr_next,
                                                     uint32_t* __restrict__ nbr_next,
                                                     unsigned long long* __restrict__ mult_next) {
    const int lane = threadIdx.x & 31;
    const int64_t step = int64_t(gridDim.x) * THREADS;
    for (int64_t base = int64_t(blockIdx.x) * THREADS + (threadIdx.x & ~31); base < a.n; base += step) {
        const int64_t u = base + lane;
        const bool same = u >= a.n || (a.alive_next[u] ? a.role[u] == 0 : a.ptr[u + 1] == a.ptr[u]);
        if (__all_sync(0xFFFFFFFFu, same) && base + 32 <= a.n) {
            const int64_t b = a.ptr[base], len = a.ptr[base + 32] - b, o = ptr_next[base];
            for (int64_t k = lane; k < len; k += 32) {
                nbr_next[o + k] = a.nbr[b + k];
                mult_next[o + k] = a.mult[b + k];
            }
        } else if (u < a.n) {
            merge_row(a, u, nbr_next + ptr_next[u], mult_next + ptr_next[u]);
        }
    }
}

__global__ void simp_copy_alive(int64_t n, const uint8_t* __restrict__ from, uint8_t* __restrict__ to) {
    for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < n; u += int64_t(gridDim.x) * blockDim.x)
        to[u] = from[u];
}

__global__ void simp_init(int64_t n, const int64_t* __restrict__ base4, const uint32_t* __restrict__ c0,
                          const uint32_t* __restrict__ c1, const uint32_t* __restrict__ c2,
                          const uint32_t* __restrict__ c3, uint32_t* __restrict__ cell, uint8_t* __restrict__ alive) {
    for (int64_t u = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; u < n; u += int64_t(gridDim.x) * blockDim.x) {
        const int k = int(u >= base4[1]) + int(u >= base4[2]) + int(u >= base4[3]);
        const uint32_t* src = k == 0 ? c0 : k == 1 ? c1 : k == 2 ? c2 : c3;
        cell[u] = src[u - base4[k]];
        alive[u] = 1;
    }
}

}  // namespace

// Simplifies the plan's 1-skeleton (built by build_complex_graph) up to `threshold`; d_field is the
// field of the plan's last pass (for the critical cells' values).  Host-synchronised once per round.
msc_status run_simplify(Plan* p, const float* d_field, double threshold, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    const int64_t n = p->graph_nodes, nnz0 = p->graph_nadj;
    int64_t base[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) base[k + 1] = base[k] + p->counts[k];
    const size_t nn = size_t(n ? n : 1);
    if ((st = ensure(p, p->simp_cell, sizeof(uint32_t) * nn))) return st;
    if ((st = ensure(p, p->simp_value, sizeof(double) * nn))) return st;
    if ((st = ensure(p, p->simp_alive, 2 * nn))) return st;
    if ((st = ensure(p, p->simp_keys, 3 * sizeof(Key) * nn))) return st;
    if ((st = ensure(p, p->simp_node, sizeof(unsigned long long) * nn + 3 * sizeof(uint32_t) * nn + nn + 64)))
        return st;
    if ((st = ensure(p, p->simp_len, sizeof(uint32_t) * (nn + 1)))) return st;
    if ((st = ensure(p, p->simp_pos, sizeof(int64_t) * (nn + 1)))) return st;
    if ((st = ensure(p, p->simp_scan, row_scan_scratch_bytes(int64_t(nn)) + 64))) return st;
    if ((st = ensure(p, p->simp_ptr[0], sizeof(int64_t) * (nn + 1)))) return st;
    if ((st = ensure(p, p->simp_ptr[1], sizeof(int64_t) * (nn + 1)))) return st;
    if ((st = ensure(p, p->simp_log, sizeof(uint32_t) * 3 * (nn / 2 + 1)))) return st;
    int64_t cap = nnz0 ? nnz0 : 1;
    for (int b = 0; b < 2; ++b) {
        if ((st = ensure(p, p->simp_nbr[b], sizeof(uint32_t) * size_t(cap)))) return st;
        if ((st = ensure(p, p->simp_mult[b], sizeof(unsigned long long) * size_t(cap)))) return st;
    }
    auto* cell = static_cast<uint32_t*>(p->simp_cell.ptr);
    auto* value = static_cast<double*>(p->simp_value.ptr);
    auto* alive = static_cast<uint8_t*>(p->simp_alive.ptr);
    auto* keys = static_cast<Key*>(p->simp_keys.ptr);
    // per-node scratch: factor (8 B), sel, owner, flags (4 B each), role (1 B), then the 4 bases
    auto* factor = static_cast<unsigned long long*>(p->simp_node.ptr);
    auto* sel = reinterpret_cast<uint32_t*>(factor + nn);
    auto* owner = sel + nn;
    auto* flags = owner + nn;
    auto* role = reinterpret_cast<uint8_t*>(flags + nn);
    auto* base4 = reinterpret_cast<int64_t*>((reinterpret_cast<uintptr_t>(role + nn) + 15) & ~uintptr_t(15));
    auto* len = static_cast<uint32_t*>(p->simp_len.ptr);
    auto* pos = static_cast<int64_t*>(p->simp_pos.ptr);
    auto* scan = static_cast<unsigned long long*>(p->simp_scan.ptr);
    // the initial complex: a copy of the exported graph
    if ((st = check_cuda(p, cudaMemcpyAsync(base4, base, sizeof(int64_t) * 4, cudaMemcpyHostToDevice, s), "simplify init")))
        return st;
    if (n) {
        simp_init<<<grid_cap(p, n, THREADS), THREADS, 0, s>>>(
            n, base4, static_cast<const uint32_t*>(p->cells[0].ptr), static_cast<const uint32_t*>(p->cells[1].ptr),
            static_cast<const uint32_t*>(p->cells[2].ptr), static_cast<const uint32_t*>(p->cells[3].ptr), cell, alive);
        simp_values<<<grid_cap(p, n, THREADS), THREADS, 0, s>>>(g, d_field, n, cell, value);
        launched(p, 2);
    }
    if ((st = check_cuda(p, cudaMemcpyAsync(p->simp_ptr[0].ptr, p->graph_nodeptr.ptr, sizeof(int64_t) * size_t(n + 1),
                                            cudaMemcpyDeviceToDevice, s), "simplify copy")))
        return st;
    if (nnz0 && ((st = check_cuda(p, cudaMemcpyAsync(p->simp_nbr[0].ptr, p->graph_adj.ptr, sizeof(uint32_t) * size_t(nnz0),
                                                     cudaMemcpyDeviceToDevice, s), "simplify copy")) ||
                 (st = check_cuda(p, cudaMemcpyAsync(p->simp_mult[0].ptr, p->graph_mult.ptr,
                                                     sizeof(unsigned long long) * size_t(nnz0),
                                                     cudaMemcpyDeviceToDevice, s), "simplify copy"))))
        return st;
    // per-round results read by the host: any valid arc, selected count, next nnz
    struct RoundOut {
        unsigned int any_valid;
        unsigned int pad;
        unsigned long long selected;
        unsigned long long nnz;
    };
    if ((st = ensure(p, p->simp_round, sizeof(RoundOut)))) return st;
    auto* rout = static_cast<RoundOut*>(p->simp_round.ptr);
    int cur = 0;
    int64_t nnz = nnz0, cancelled = 0, rounds = 0;
    const int64_t max_rounds = p->opts.max_iterations > 0 ? p->opts.max_iterations : (int64_t(1) << 20);
    while (n > 0) {
        if (rounds >= max_rounds) return fail(p, MSC_ERR_ITER_LIMIT, "simplification reached the iteration cap");
        SimpArgs a;
        a.n = n;
        for (int k = 0; k < 4; ++k) a.base[k] = base[k];
        a.threshold = threshold;
        a.cell = cell;
        a.value = value;
        a.ptr = static_cast<const int64_t*>(p->simp_ptr[cur].ptr);
        a.nbr = static_cast<const uint32_t*>(p->simp_nbr[cur].ptr);
        a.mult = static_cast<const unsigned long long*>(p->simp_mult[cur].ptr);
        a.alive = alive + size_t(cur) * nn;
        a.alive_next = alive + size_t(1 - cur) * nn;
        a.m0 = keys;
        a.m1 = keys + nn;
        a.m2 = keys + 2 * nn;
        a.sel = sel;
        a.owner = owner;
        a.role = role;
        a.factor = factor;
        a.flags = flags;
        a.status = p->status_word();
        a.any_valid = &rout->any_valid;
        if ((st = check_cuda(p, cudaMemsetAsync(rout, 0, sizeof(RoundOut), s), "simplify round"))) return st;
        const int grid = grid_cap(p, n, THREADS);
        simp_min0<<<grid, THREADS, 0, s>>>(a, rounds == 0 ? 1 : 0);
        simp_spread<<<grid, THREADS, 0, s>>>(a, a.m0, a.m1, 0);
        simp_spread<<<grid, THREADS, 0, s>>>(a, a.m1, a.m2, 1);
        simp_select<<<grid, THREADS, 0, s>>>(a);
        launched(p, 4);
        // log positions of the selected upper nodes (node order), then the footprints
        if ((st = check_cuda(p, row_scan(p, flags, nullptr, n, pos, scan, s, &rout->selected), "simplify scan")))
            return st;
        auto* log = static_cast<uint32_t*>(p->simp_log.ptr) + 3 * cancelled;
        simp_mark<<<grid, THREADS, 0, s>>>(a, pos, log, uint32_t(rounds));
        simp_count<<<grid, THREADS, 0, s>>>(a, len);
        launched(p, 2);
        auto* ptr_next = static_cast<int64_t*>(p->simp_ptr[1 - cur].ptr);
        if ((st = check_cuda(p, row_scan(p, len, nullptr, n, ptr_next, scan, s, &rout->nnz), "simplify scan")))
            return st;
        RoundOut h{};
        if ((st = check_cuda(p, cudaMemcpyAsync(&h, rout, sizeof(RoundOut), cudaMemcpyDeviceToHost, s), "simplify read")))
            return st;
        if ((st = check_status_word(p, s))) return st;  // synchronises
        if (!h.any_valid) break;
        const int64_t next_nnz = int64_t(h.nnz);
        if (next_nnz > cap) {  // grow the next buffers (the current ones are still read by the fill)
            cap = next_nnz + next_nnz / 4;
            if ((st = ensure(p, p->simp_nbr[1 - cur], sizeof(uint32_t) * size_t(cap)))) return st;
            if ((st = ensure(p, p->simp_mult[1 - cur], sizeof(unsigned long long) * size_t(cap)))) return st;
        }
        simp_fill<<<grid, THREADS, 0, s>>>(a, ptr_next, static_cast<uint32_t*>(p->simp_nbr[1 - cur].ptr),
                                           static_cast<unsigned long long*>(p->simp_mult[1 - cur].ptr));
        launched(p);
        if ((st = check_cuda(p, cudaGetLastError(), "simplify launch"))) return st;
        cur = 1 - cur;
        nnz = next_nnz;
        cancelled += int64_t(h.selected);
        ++rounds;
    }
    if ((st = check_status_word(p, s))) return st;
    p->simp_cur = cur;
    p->simp_nnz = nnz;
    p->simp_rounds = rounds;
    p->simp_cancelled = cancelled;
    return MSC_OK;
}

}  // namespace msc

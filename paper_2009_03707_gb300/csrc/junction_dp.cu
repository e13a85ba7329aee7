// (a6) Saddle-saddle path counts, D* = D + sum_{k>=0} A B^k B* (Sec. 3.3 "Path counting via
// matrix operations"), evaluated right to left.
//
// The paper iterates A <- A B (SpGEMM) and accumulates A* B* + D: every 1-saddle row walks the
// whole sub-DAG below it, so a junction reached from many 1-saddles, at many depths, is expanded
// again for every one of them -- on a field with long V-path networks (the paper's noisy volumes,
// the 512^3 blob field here: 197 iterations, 1e9 frontier entries, path counts near 1.6e10)
// that repetition is most of the work.  The same matrix identity read from the right,
//     J = sum_k B^k B*  (paths from each junction to the 2-saddles),  J = B* + B J,
//     D* = D + A J,
// needs every junction's row once, in topological order of the minor (a DAG): a junction's row
// is ready as soon as the rows of the junctions it points to are.  So:
//   1. the reverse adjacency of B (junction -> the junctions pointing at it) and, per junction,
//      the number of its out-slots that point at junctions;
//   2. waves: wave 0 is the junctions with no junction successor; a junction's J row is the
//      merge of its 4 trace slots -- a 2-saddle slot is one path to that 2-saddle, a junction
//      slot adds that junction's J row -- and finishing it decrements the pending counts of its
//      predecessors; the one that takes a count to 0 stamps it with the next wave's number and
//      flags its chunk of 32 junctions in that wave's chunk bitmap.  A wave reads the bitmap and
//      scans only the flagged chunks' pending words for its own stamp (no shared queue, whose
//      single append counter would serialise millions of atomics; no pass over every junction
//      for a wave with few), and a junction released during a wave waits for the next one, when
//      the rows it reads are complete.  The waves run as a
//      device loop (a conditional WHILE node in a graph); the non-empty ones number the paper's
//      iteration count, 1 + the longest chain of junctions;
//   3. D* row s = the same merge over 1-saddle s's slots, written to staging and gathered into
//      CSR (pathcount.cu's staging, row scan and gather).
// Rows are merged sorted by column with exact uint64 sums (an add that wraps raises the overflow
// flag).  J rows live in one pool, allocated with a warp-aggregated bump pointer.  A merge is a
// chain of dependent loads, one step per output entry, so a wave lasts as long as its longest
// merge: junctions whose inputs hold more than LONG_ROW entries are handed to a second kernel of
// the same wave, where a warp splits the key range over its 32 lanes (pivots from the longest
// input row, a binary search per lane and input) and each lane merges its slice.
#include <cooperative_groups.h>

#include <cstddef>

#include "rowscan.cuh"

namespace cg = cooperative_groups;

namespace msc {

namespace {

constexpr int THREADS = 256;
constexpr uint32_t READY = 0x80000000u;  // pend[j] = READY | wave: j's row is computed in that wave
constexpr uint32_t DONE = 0xFFFFFFFFu;
constexpr int SCAN_BATCH = 8;  // pending words a thread reads at once in a wave
constexpr uint32_t LONG_ROW = 12;  // merges with more input entries go to the warp kernel
typedef unsigned long long u64;

struct DpArgs {
    const uint32_t* tgt;                 // 4 destination ranks per source (1-saddles, then junctions)
    const uint32_t* kinds;               // per source: byte k = kind of slot k
    const unsigned long long* n1_dev;    // 1-saddles and junctions, counted earlier in the pass
    const unsigned long long* nj_dev;
    int64_t cap1, capj;                  // the capacities the buffers were sized for
    uint32_t* pend;                      // per junction: junction slots whose rows are not ready, or
                                         // READY | wave once they all are, or DONE
    uint32_t* chunk_map;                 // two bitmaps (waves of even / odd number): bit c of word w
                                         // flags chunk 32 w + c, junctions 32 (32 w + c) ..
    int64_t map_words;                   // words per bitmap
    uint32_t* in_cnt;                    // per junction: slots of other junctions pointing at it
    int64_t* in_ptr;                     // CSR of those predecessors
    uint32_t* in_fill;
    uint32_t* in_idx;
    uint32_t* long_list;                 // this wave's junctions with long merges (dp_long)
    u64* j_off;                          // per junction: its J row in the pool
    uint32_t* j_len;
    uint32_t* pool_col;                  // J rows: 2-saddle ranks increasing, uint64 counts
    u64* pool_cnt;
    u64 pool_cap;
    uint32_t* out_col;                   // D* rows (staging) and their place
    u64* out_cnt;
    u64 out_cap;
    int64_t* row_start;
    uint32_t* row_len;
    Summary* sum;
    uint32_t* status;
};

// The pass's counts; false (do nothing) when the pass is to be rerun.
__device__ __forceinline__ bool counts_of(const DpArgs& a, int64_t& n1, int64_t& nj) {
    const u64 x = *a.n1_dev, y = *a.nj_dev;
    if (pass_retrying(a.status) || !count_fits(a.status, x, a.cap1) || !count_fits(a.status, y, a.capj)) return false;
    n1 = int64_t(x);
    nj = int64_t(y);
    return true;
}

// Place for n items in a shared array: one atomic per group of active threads.
__device__ __forceinline__ u64 bump(u64* counter, u64 n) {
    cg::coalesced_group g = cg::coalesced_threads();
    u64 incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = g.shfl_up(incl, o);
        if (int(g.thread_rank()) >= o) incl += y;
    }
    const u64 total = g.shfl(incl, g.size() - 1);
    u64 base = 0;
    if (g.thread_rank() == g.size() - 1) base = atomicAdd(counter, total);
    base = g.shfl(base, g.size() - 1);
    return base + incl - n;
}

// Merge of one source's 4 slots: a 2-saddle slot is one path to that 2-saddle, a junction slot
// contributes that junction's J row.  Inputs are sorted by column; the output is sorted with
// equal columns summed.  Returns the output length; *bound gets the sum of the input lengths.
struct Inputs {
    const uint32_t* col[4];
    const u64* cnt[4];
    uint32_t len[4];
    uint32_t single[4];  // the 2-saddle of a 2-saddle slot
    uint32_t kind[4];
};

__device__ __forceinline__ Inputs inputs_of(const DpArgs& a, int64_t src, int64_t n1, uint32_t* bound) {
    Inputs in;
    const uint4 q = *reinterpret_cast<const uint4*>(a.tgt + 4 * src);
    const uint32_t kinds = a.kinds[src];
    const uint32_t t[4] = {q.x, q.y, q.z, q.w};
    uint32_t b = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        in.kind[k] = trace_kind(kinds, k);
        in.single[k] = t[k];
        in.len[k] = 0;
        in.col[k] = nullptr;
        in.cnt[k] = nullptr;
        if (in.kind[k] == 2) {
            in.len[k] = 1;
        } else if (in.kind[k] == 1) {
            in.len[k] = a.j_len[t[k]];
            in.col[k] = a.pool_col + a.j_off[t[k]];
            in.cnt[k] = a.pool_cnt + a.j_off[t[k]];
        }
        b += in.len[k];
    }
    (void)n1;
    *bound = b;
    return in;
}

__device__ __forceinline__ uint32_t merge_into(const Inputs& in, uint32_t* out_col, u64* out_cnt, uint64_t room,
                                               u64* max_seen, uint32_t* status) {
    uint32_t pos[4] = {0, 0, 0, 0};
    uint32_t n = 0;
    bool wrapped = false;
    for (;;) {
        uint32_t c = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (pos[k] < in.len[k]) c = min(c, in.kind[k] == 2 ? in.single[k] : in.col[k][pos[k]]);
        if (c == 0xFFFFFFFFu) break;
        u64 s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (pos[k] >= in.len[k]) continue;
            const uint32_t ck = in.kind[k] == 2 ? in.single[k] : in.col[k][pos[k]];
            if (ck != c) continue;
            const u64 v = in.kind[k] == 2 ? 1ull : in.cnt[k][pos[k]];
            wrapped |= s + v < s;
            s += v;
            ++pos[k];
        }
        if (n < room) {
            out_col[n] = c;
            out_cnt[n] = s;
        }
        *max_seen = max(*max_seen, s);
        ++n;
    }
    if (wrapped) atomicOr(status, ST_OVERFLOW);
    return n;
}

// Per junction: its pending junction slots (wave 0 if none) and the reverse-adjacency counts.
__global__ void __launch_bounds__(THREADS) dp_init(DpArgs a) {
    int64_t n1, nj;
    if (!counts_of(a, n1, nj)) return;
    for (int64_t j = int64_t(blockIdx.x) * THREADS + threadIdx.x; j < nj; j += int64_t(gridDim.x) * THREADS) {
        const uint4 q = *reinterpret_cast<const uint4*>(a.tgt + 4 * (n1 + j));
        const uint32_t kinds = a.kinds[n1 + j];
        const uint32_t t[4] = {q.x, q.y, q.z, q.w};
        uint32_t pending = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (trace_kind(kinds, k) == 1) {
                ++pending;
                atomicAdd(&a.in_cnt[t[k]], 1u);
            }
        a.pend[j] = pending ? pending : READY;
        if (!pending) atomicOr(&a.chunk_map[j >> 10], 1u << ((j >> 5) & 31));  // wave 0
    }
}

// The reverse adjacency: predecessors of every junction, one entry per slot.
__global__ void __launch_bounds__(THREADS) dp_fill(DpArgs a) {
    int64_t n1, nj;
    if (!counts_of(a, n1, nj)) return;
    for (int64_t j = int64_t(blockIdx.x) * THREADS + threadIdx.x; j < nj; j += int64_t(gridDim.x) * THREADS) {
        const uint4 q = *reinterpret_cast<const uint4*>(a.tgt + 4 * (n1 + j));
        const uint32_t kinds = a.kinds[n1 + j];
        const uint32_t t[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (trace_kind(kinds, k) == 1) a.in_idx[a.in_ptr[t[k]] + atomicAdd(&a.in_fill[t[k]], 1u)] = uint32_t(j);
    }
}

// One wave: the J rows of the junctions stamped with this wave, then the predecessors they
// release (stamped with the next wave).
__global__ void __launch_bounds__(THREADS) dp_wave(DpArgs a) {
    int64_t n1, nj;
    if (!counts_of(a, n1, nj)) return;
    const uint32_t wave = a.sum->dp_wave;
    const uint32_t mine = READY | wave, next = READY | (wave + 1);
    uint32_t* const map_cur = a.chunk_map + (wave & 1u) * a.map_words;
    uint32_t* const map_next = a.chunk_map + ((wave + 1) & 1u) * a.map_words;
    unsigned done = 0;
    u64 mx = 0;
    // a lane per chunk of 32 junctions, a warp per bitmap word; a flagged chunk's pending words
    // are read SCAN_BATCH at a time, all in flight together
    const int lane = threadIdx.x & 31;
    const int64_t nchunks = (nj + 31) / 32;
    const int64_t stride = int64_t(gridDim.x) * THREADS;  // a multiple of 32: warps stay on whole words
    for (int64_t cbase = int64_t(blockIdx.x) * THREADS + (threadIdx.x & ~31); cbase < nchunks; cbase += stride) {
        const uint32_t flags = map_cur[cbase >> 5];
        __syncwarp();
        if (lane == 0 && flags) map_cur[cbase >> 5] = 0;  // consumed: the next even/odd wave starts clean
        const int64_t c = cbase + lane;
        if (c >= nchunks || !((flags >> lane) & 1u)) continue;
        uint32_t hit = 0;
#pragma unroll
        for (int b = 0; b < 32; b += SCAN_BATCH) {
#pragma unroll
            for (int k = 0; k < SCAN_BATCH; ++k) {
                const int64_t j = c * 32 + b + k;
                hit |= uint32_t(j < nj && a.pend[j] == mine) << (b + k);
            }
        }
#pragma unroll 1
        for (; hit; hit &= hit - 1) {
            const int64_t j = c * 32 + (__ffs(hit) - 1);
            uint32_t bound;
            const Inputs in = inputs_of(a, n1 + j, n1, &bound);
            if (bound > LONG_ROW) {  // merged by dp_long in this wave, which also releases its predecessors
                a.long_list[atomicAdd(&a.sum->dp_long_n, 1ull)] = uint32_t(j);
                continue;
            }
            const u64 off = bump(&a.sum->dp_pool_used, bound);
            uint32_t len = 0;
            if (off + bound <= a.pool_cap) {
                len = merge_into(in, a.pool_col + off, a.pool_cnt + off, bound, &mx, a.status);
            } else {
                atomicOr(a.status, ST_RETRY);  // the pool is too small: the host grows it and reruns
            }
            a.j_off[j] = off;
            a.j_len[j] = len;
            a.pend[j] = DONE;
            ++done;
            for (int64_t e = a.in_ptr[j]; e < a.in_ptr[j + 1]; ++e) {
                const uint32_t p = a.in_idx[e];
                if (atomicSub(&a.pend[p], 1u) == 1u) {
                    a.pend[p] = next;
                    atomicOr(&map_next[p >> 10], 1u << ((p >> 5) & 31));
                }
            }
        }
    }
    for (int o = 16; o; o >>= 1) done += __shfl_xor_sync(0xFFFFFFFFu, done, o);
    if ((threadIdx.x & 31) == 0 && done) atomicAdd(&a.sum->dp_wave_done, (u64)done);
}

// First position in col[0..len) whose column is >= key.
__device__ __forceinline__ uint32_t lower_bound(const uint32_t* col, uint32_t len, uint32_t key) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (col[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One lane's slice of a merge: the columns in [lo, hi) (hi_open: no upper end) of every input,
// merged with equal columns summed; counts them, and writes them from out_col / out_cnt when
// `write` is set.
__device__ __forceinline__ uint32_t slice_merge(const Inputs& in, const uint32_t s[4], const uint32_t e[4],
                                                uint32_t lo, uint32_t hi, bool hi_open, bool write, uint32_t* out_col,
                                                u64* out_cnt, bool* wrapped) {
    uint32_t pos[4], end[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        pos[k] = s[k];
        end[k] = e[k];
        if (in.kind[k] == 2) {  // a 2-saddle slot: its one column, if it falls in the slice
            const bool mine = in.single[k] >= lo && (hi_open || in.single[k] < hi);
            pos[k] = 0;
            end[k] = mine ? 1 : 0;
        }
    }
    uint32_t n = 0;
    for (;;) {
        uint32_t c = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (pos[k] < end[k]) c = min(c, in.kind[k] == 2 ? in.single[k] : in.col[k][pos[k]]);
        if (c == 0xFFFFFFFFu) break;
        u64 sum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (pos[k] >= end[k]) continue;
            const uint32_t ck = in.kind[k] == 2 ? in.single[k] : in.col[k][pos[k]];
            if (ck != c) continue;
            const u64 v = in.kind[k] == 2 ? 1ull : in.cnt[k][pos[k]];
            *wrapped |= sum + v < sum;
            sum += v;
            ++pos[k];
        }
        if (write) {
            out_col[n] = c;
            out_cnt[n] = sum;
        }
        ++n;
    }
    return n;
}

// The long merges of this wave, a warp each: the longest input row gives 32 pivot columns, lane l
// merges the columns in [pivot l, pivot l+1) of every input (binary searches for its slice), twice
// -- to count, then, after a warp prefix of the counts, to write -- and the warp releases the
// junction's predecessors.
__global__ void __launch_bounds__(THREADS) dp_long(DpArgs a) {
    int64_t n1, nj;
    if (!counts_of(a, n1, nj)) return;
    const uint32_t next = READY | (a.sum->dp_wave + 1);
    uint32_t* const map_next = a.chunk_map + ((a.sum->dp_wave + 1) & 1u) * a.map_words;
    const u64 n = a.sum->dp_long_n;
    const int lane = threadIdx.x & 31;
    const u64 nwarps = (u64(gridDim.x) * THREADS) >> 5;
    unsigned done = 0;
    bool wrapped = false;
    for (u64 i = (u64(blockIdx.x) * THREADS + threadIdx.x) >> 5; i < n; i += nwarps) {  // warp-uniform
        const uint32_t j = a.long_list[i];
        uint32_t bound;
        const Inputs in = inputs_of(a, n1 + j, n1, &bound);
        uint32_t L = 0;  // the longest input row
        const uint32_t* P = nullptr;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (in.kind[k] == 1 && in.len[k] > L) {
                L = in.len[k];
                P = in.col[k];
            }
        const uint32_t lo = (lane == 0 || L == 0) ? 0u : P[uint32_t((u64(lane) * L) >> 5)];
        const uint32_t hi = __shfl_down_sync(0xFFFFFFFFu, lo, 1);
        const bool hi_open = lane == 31;
        uint32_t s[4], e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            s[k] = e[k] = 0;
            if (in.kind[k] == 1) {
                s[k] = lane == 0 ? 0u : lower_bound(in.col[k], in.len[k], lo);
                e[k] = hi_open ? in.len[k] : lower_bound(in.col[k], in.len[k], hi);
            }
        }
        u64 off = 0;
        if (lane == 0) off = atomicAdd(&a.sum->dp_pool_used, u64(bound));
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        const bool fits = off + bound <= a.pool_cap;  // uniform
        uint32_t len = 0;
        if (fits) {
            const uint32_t cnt = slice_merge(in, s, e, lo, hi, hi_open, false, nullptr, nullptr, &wrapped);
            uint32_t incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            slice_merge(in, s, e, lo, hi, hi_open, true, a.pool_col + off + (incl - cnt),
                        a.pool_cnt + off + (incl - cnt), &wrapped);
            len = __shfl_sync(0xFFFFFFFFu, incl, 31);
        } else if (lane == 0) {
            atomicOr(a.status, ST_RETRY);  // the pool is too small: the host grows it and reruns
        }
        if (lane == 0) {
            a.j_off[j] = off;
            a.j_len[j] = len;
            a.pend[j] = DONE;
            ++done;
        }
        for (int64_t q = a.in_ptr[j] + lane; q < a.in_ptr[j + 1]; q += 32) {
            const uint32_t pr = a.in_idx[q];
            if (atomicSub(&a.pend[pr], 1u) == 1u) {
                a.pend[pr] = next;
                atomicOr(&map_next[pr >> 10], 1u << ((pr >> 5) & 31));
            }
        }
    }
    if (wrapped) atomicOr(a.status, ST_OVERFLOW);
    for (int o = 16; o; o >>= 1) done += __shfl_xor_sync(0xFFFFFFFFu, done, o);
    if (lane == 0 && done) atomicAdd(&a.sum->dp_wave_done, (u64)done);
}

// End of a wave: count it, and go on while it found junctions to do (the loop ends after the
// first empty wave).
__global__ void dp_decide(Summary* sum, int64_t max_iter, cudaGraphConditionalHandle h, int use_handle) {
    const u64 done = sum->dp_wave_done;
    sum->dp_wave_done = 0;
    sum->dp_long_n = 0;
    ++sum->dp_iters;
    bool more = done != 0;
    if (more) {
        ++sum->pc[PC_ITER];
        sum->dp_junctions_done += done;
        ++sum->dp_wave;
        if (int64_t(sum->pc[PC_ITER]) >= max_iter) {
            atomicOr(&sum->status, uint32_t(ST_ITER));
            more = false;
        }
    }
    sum->loop_flag[3] = more ? 1u : 0u;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// D* rows: the merge of each 1-saddle's slots, into staging.  Also checks that every junction
// was reached by the waves (the minor is a DAG, so it must be).
__global__ void __launch_bounds__(THREADS) dp_rows(DpArgs a) {
    int64_t n1, nj;
    if (!counts_of(a, n1, nj)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.sum->dp_junctions_done != u64(nj)) atomicOr(a.status, ST_INTERNAL);
    u64 mx = 0;
    for (int64_t s = int64_t(blockIdx.x) * THREADS + threadIdx.x; s < n1; s += int64_t(gridDim.x) * THREADS) {
        uint32_t bound;
        const Inputs in = inputs_of(a, s, n1, &bound);
        const u64 off = bump(&a.sum->pc[PC_CURSOR], bound);
        uint32_t len = 0;
        if (off + bound <= a.out_cap) {
            len = merge_into(in, a.out_col + off, a.out_cnt + off, bound, &mx, a.status);
        } else {
            atomicOr(a.status, ST_RETRY);  // staging too small: the host grows it and reruns
        }
        a.row_start[s] = int64_t(off);
        a.row_len[s] = len;
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, (u64)__shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(&a.sum->pc[PC_MAX], mx);
}

struct WaveCtx {
    int grid;
    int long_grid;  // the long merges of a wave are few: a smaller grid of warps
    DpArgs a;
};

void wave_body(Plan* p, cudaStream_t s, cudaGraphConditionalHandle h, void* ctx) {
    const WaveCtx& c = *static_cast<WaveCtx*>(ctx);
    dp_wave<<<c.grid, THREADS, 0, s>>>(c.a);
    dp_long<<<c.long_grid, THREADS, 0, s>>>(c.a);
    dp_decide<<<1, 1, 0, s>>>(p->dsum(), p->opts.max_iterations, h, h != 0);
}

}  // namespace

// Enqueues the junction DP and the D* rows into staging (the caller scans and gathers them).
// pool_cap / out_cap: capacities of the J-row pool and of the staging.
msc_status run_junction_dp(Plan* p, cudaStream_t s, uint64_t pool_cap, uint64_t out_cap) {
    msc_status st;
    const int64_t cap1 = p->capturing ? p->caps.cells[1] : p->counts[1];
    const int64_t capj = p->capturing ? p->caps.nj : p->n_junctions;
    const size_t njc = size_t(capj ? capj : 1);
    if ((st = ensure(p, p->dp_pend, sizeof(uint32_t) * njc))) return st;
    const int64_t map_words = int64_t((njc + 1023) / 1024);
    if ((st = ensure(p, p->dp_chunks, sizeof(uint32_t) * 2 * size_t(map_words)))) return st;
    if ((st = ensure(p, p->dp_long, sizeof(uint32_t) * njc))) return st;
    if ((st = ensure(p, p->dp_in_cnt, sizeof(uint32_t) * 2 * njc))) return st;  // counts, then fill cursors
    if ((st = ensure(p, p->dp_in_ptr, sizeof(int64_t) * (njc + 1)))) return st;
    if ((st = ensure(p, p->dp_in_idx, sizeof(uint32_t) * 4 * njc))) return st;
    if ((st = ensure(p, p->dp_j_off, sizeof(u64) * njc))) return st;
    if ((st = ensure(p, p->dp_j_len, sizeof(uint32_t) * njc))) return st;
    if ((st = ensure(p, p->dp_pool_col, sizeof(uint32_t) * size_t(pool_cap ? pool_cap : 1)))) return st;
    if ((st = ensure(p, p->dp_pool_cnt, sizeof(u64) * size_t(pool_cap ? pool_cap : 1)))) return st;
    if ((st = ensure(p, p->minor_scan, std::max(row_scan_scratch_bytes(capj), row_scan_scratch_bytes(cap1))))) return st;
    DpArgs a{};
    a.tgt = static_cast<const uint32_t*>(p->trace.ptr);
    a.kinds = static_cast<const uint32_t*>(p->trace_kinds.ptr);
    a.n1_dev = &p->dsum()->counts[1];
    a.nj_dev = &p->dsum()->n_junctions;
    a.cap1 = cap1;
    a.capj = capj;
    a.pend = static_cast<uint32_t*>(p->dp_pend.ptr);
    a.chunk_map = static_cast<uint32_t*>(p->dp_chunks.ptr);
    a.map_words = map_words;
    a.long_list = static_cast<uint32_t*>(p->dp_long.ptr);
    a.in_cnt = static_cast<uint32_t*>(p->dp_in_cnt.ptr);
    a.in_fill = a.in_cnt + njc;
    a.in_ptr = static_cast<int64_t*>(p->dp_in_ptr.ptr);
    a.in_idx = static_cast<uint32_t*>(p->dp_in_idx.ptr);
    a.j_off = static_cast<u64*>(p->dp_j_off.ptr);
    a.j_len = static_cast<uint32_t*>(p->dp_j_len.ptr);
    a.pool_col = static_cast<uint32_t*>(p->dp_pool_col.ptr);
    a.pool_cnt = static_cast<u64*>(p->dp_pool_cnt.ptr);
    a.pool_cap = pool_cap;
    a.out_col = static_cast<uint32_t*>(p->pc_col.ptr);
    a.out_cnt = static_cast<u64*>(p->pc_cnt.ptr);
    a.out_cap = out_cap;
    a.row_start = static_cast<int64_t*>(p->pc_rowstart.ptr);
    a.row_len = static_cast<uint32_t*>(p->pc_rowlen.ptr);
    a.sum = p->dsum();
    a.status = p->status_word();
    if ((st = check_cuda(p, cudaMemsetAsync(a.in_cnt, 0, sizeof(uint32_t) * 2 * njc, s), "memset"))) return st;
    if ((st = check_cuda(p, cudaMemsetAsync(a.chunk_map, 0, sizeof(uint32_t) * 2 * size_t(map_words), s), "memset")))
        return st;
    // the wave state of the summary (a rerun of the stage starts it afresh)
    if ((st = check_cuda(p, cudaMemsetAsync(&p->dsum()->dp_wave_done, 0,
                                            offsetof(Summary, loop_flag) - offsetof(Summary, dp_wave_done), s),
                         "memset")))
        return st;
    const int gj = grid_cap(p, capj, THREADS, 8);
    dp_init<<<gj, THREADS, 0, s>>>(a);
    launched(p);
    if ((st = check_cuda(p, row_scan(p, a.in_cnt, a.nj_dev, capj, a.in_ptr, static_cast<u64*>(p->minor_scan.ptr), s),
                         "predecessor scan")))
        return st;
    dp_fill<<<gj, THREADS, 0, s>>>(a);
    launched(p);
    if ((st = check_cuda(p, cudaGetLastError(), "junction dp launch"))) return st;
    record_event(p, p->kev0, s);
    WaveCtx ctx{grid_cap(p, capj, THREADS, 8), std::max(1, p->num_sms) * 4, a};
    if ((st = run_loop(p, s, 2, 3, wave_body, &ctx))) return st;
    dp_rows<<<grid_cap(p, cap1, THREADS, 8), THREADS, 0, s>>>(a);
    record_event(p, p->kev1, s);
    launched(p);
    return check_cuda(p, cudaGetLastError(), "junction dp launch");
}

}  // namespace msc

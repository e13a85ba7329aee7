// (a6) Saddle-saddle path counting: D* = D + sum_{k>=0} A B^k B* (Sec. 3.3 "Path counting
// via matrix operations").
//
// The paper iterates A <- A B over the whole matrix (cuSPARSE SpGEMM), accumulating A* until
// the product is zero, then forms A* B* + D.  Row s of every product depends only on row s of
// A, so here the same iteration runs row by row (Gustavson's row-wise product): the worker that
// owns 1-saddle s keeps the frontier A_k[s,:] keyed by junction rank and the accumulator
// D*[s,:] keyed by 2-saddle rank, and repeats "for each (j, c) in A_k[s,:]: every traced path
// j -> j' adds c to A_{k+1}[s,j'], every traced path j -> t adds c to D*[s,t]" until the
// frontier is empty.  The minor's adjacency is the 4-slot trace of each junction (minor.cu); a
// repeated destination is a repeated path, i.e. the multiplicity.  Counts are exact uint64 and
// an add that wraps sets the overflow flag (the paper reports multiplicities near 1e10).
//
// Rows are latency-bound chains of dependent gathers, so the work goes to the smallest worker
// that can hold it, to keep as many rows in flight as possible:
//   tier 0  a row per lane, frontier (<= 8) and D* row (<= 16) hash tables in shared memory,
//           32-bit counts; each frontier step is spread over the warp item by item;
//   tier 1  one warp per row, 256-slot hash tables in shared memory;
//   tier 2+ one CTA per row, hash tables in global memory, grown until the row fits.
// A row that overflows its worker is deferred, intact, to the next tier.  Finished rows are
// sorted by column and appended to a staging buffer; a scan of the row lengths and one gather
// give the CSR of D*.
#include "rowscan.cuh"

namespace msc {

namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr int T0_WARPS = 8;
constexpr int T0_THREADS = T0_WARPS * 32;
// tier 0: frontier and D* table slots per row (powers of two); tier 0b: the same kernel with
// larger tables for the few rows that outgrow tier 0 (more shared memory per row, so fewer rows
// in flight -- which only the deferred rows pay for)
constexpr int T0_F = 8, T0_LF = 3, T0_D = 16, T0_LD = 4;
constexpr int T0B_F = 16, T0B_LF = 4, T0B_D = 32, T0B_LD = 5;
constexpr int T0_OUT_CHUNK = 1024;  // staging slots a warp takes at a time
constexpr int T1_WARPS = 4;
constexpr int T1_HASH = 256;  // slots per table (power of two)
constexpr int T1_LIST = T1_HASH / 2;
constexpr int T2_THREADS = 256;

typedef unsigned long long u64;

struct PcArgs {
    int64_t n1;             // 1-saddles (resolved on the device from n1_dev, see resolve)
    const uint32_t* rows;   // the 1-saddle ranks this launch owns (null: 0..nrows-1)
    int64_t nrows;          // rows of this launch (resolved on the device from nrows_dev)
    const unsigned long long* n1_dev;     // counted earlier in the pass
    const unsigned long long* nrows_dev;  // the 1-saddle count, or the previous tier's deferrals
    const unsigned long long* nj_dev;     // junctions: their ranks index the trace
    int64_t n1_cap, nj_cap;               // the capacities the buffers were sized for
    int retry_on_defer;     // a deferral means the pass must be rerun (the last tier of a graph)
    const uint32_t* tgt;    // 4 destination ranks per source (1-saddles, then junctions)
    const uint32_t* kinds;  // per source, byte k = kind of slot k: 1 junction, 2 2-saddle
    uint32_t* out_col;      // staging: columns of finished rows
    u64* out_cnt;
    uint64_t out_cap;
    u64* out_cursor;
    int64_t* row_start;
    uint32_t* row_len;
    uint32_t* deferred;     // rows handed to the next tier
    u64* deferred_count;
    u64* max_count;
    u64* n_iter;
    u64* n_entries;         // sum of frontier sizes of finished rows
    int64_t max_iter;
    uint32_t* status;
};

__device__ __forceinline__ int64_t row_of(const PcArgs& a, int64_t i) { return a.rows ? int64_t(a.rows[i]) : i; }

// The counts a launch works on, read on the device (they are produced earlier in the same pass);
// false (do nothing) when the pass is to be rerun.
__device__ __forceinline__ bool resolve(PcArgs& a) {
    const unsigned long long n1 = *a.n1_dev, nj = *a.nj_dev;
    if (pass_retrying(a.status) || !count_fits(a.status, n1, a.n1_cap) || !count_fits(a.status, nj, a.nj_cap))
        return false;
    a.n1 = int64_t(n1);
    a.nrows = int64_t(min(*a.nrows_dev, n1));
    return true;
}

__device__ __forceinline__ uint4 trace_of(const PcArgs& a, int64_t src) {
    return *reinterpret_cast<const uint4*>(a.tgt + 4 * src);
}

// ---------------------------------------------------------------------------------------
// tier 0: a row per lane, frontier steps item-parallel across the warp
// ---------------------------------------------------------------------------------------
// Each lane owns a row and its tables in shared memory, stored [slot][lane] per warp: two
// frontier hash tables (current and next, T0_F slots) and the D* row (T0_D slots), keys and
// 32-bit counts.  A frontier step is run by the whole warp on the list of all its rows'
// frontier entries (compacted with one ballot per slot): lane i takes entry i, reads the
// junction's trace and adds each traced path to the owning row's next frontier or D* table
// with shared-memory atomics.  So a lane's work does not depend on its own row's size, and
// every per-row loop is a fixed, unrolled one.  A row whose table fills up, or whose counts
// outgrow 32 bits, is deferred intact to the next tier (tier 0b, the same kernel with larger
// tables, then the uint64 warp tier).
//
// Packed tables (PK): a slot is one word, key << 8 | count, for keys below 2^24 - 1 (then a
// packed slot never equals EMPTY) and counts up to 255.  That halves the tables, so more warps fit
// on an SM.  An add whose count would carry into the key defers the row to tier 0b, which keeps
// 32-bit counts (the corrupted slot is never expanded: the row's tables are cleared at the end of
// that round).  The count arrays shrink to one unused slot.
template <int F, int D, bool PK>
struct T0Warp {
    uint32_t fk[2][F][32];
    uint32_t fv[PK ? 1 : 2][PK ? 1 : F][32];
    uint32_t dk[D][32];
    uint32_t dv[PK ? 1 : D][32];
    unsigned long long base[32];  // staging offset of each finishing row
    uint16_t items[32 * (F > D ? F : D)];  // this round's work list: slot << 5 | row
};

// Adds val to key's entry in row r's table (K, V: [slot][32] arrays of 2^lg slots); false if
// the table is full or the count wraps.  Lanes may add to the same row at once: keys are
// claimed with atomicCAS.  Either of a row's tables goes through this one code path.
__device__ __forceinline__ bool t0_add_rt(uint32_t* K, uint32_t* V, int lg, int r, uint32_t key, uint32_t val) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = (key * 2654435761u) >> (32 - lg);
#pragma unroll 1
    for (uint32_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
        uint32_t k = *reinterpret_cast<volatile uint32_t*>(&K[h * 32 + r]);
        if (k == EMPTY) {
            k = atomicCAS(&K[h * 32 + r], EMPTY, key);
            if (k == EMPTY) k = key;
        }
        if (k == key) {
            const uint32_t old = atomicAdd(&V[h * 32 + r], val);
            return old + val >= old;
        }
    }
    return false;
}

// The packed form of t0_add_rt: K holds key << 8 | count; val <= 255.  A new key is claimed with
// its count in one atomicCAS.
__device__ __forceinline__ bool t0_add_pk(uint32_t* K, int lg, int r, uint32_t key, uint32_t val) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h = (key * 2654435761u) >> (32 - lg);
#pragma unroll 1
    for (uint32_t p = 0; p <= mask; ++p, h = (h + 1) & mask) {
        uint32_t k = *reinterpret_cast<volatile uint32_t*>(&K[h * 32 + r]);
        if (k == EMPTY) {
            k = atomicCAS(&K[h * 32 + r], EMPTY, (key << 8) | val);
            if (k == EMPTY) return true;
        }
        if ((k >> 8) == key) {
            const uint32_t old = atomicAdd(&K[h * 32 + r], val);
            return (old & 0xFFu) + val <= 0xFFu;  // a carry would change the key
        }
    }
    return false;
}

// One table add of either form; lg is the table's log2 size.
template <bool PK>
__device__ __forceinline__ bool t0_add(uint32_t* K, uint32_t* V, int lg, int r, uint32_t key, uint32_t val) {
    if constexpr (PK) return t0_add_pk(K, lg, r, key, val);
    else return t0_add_rt(K, V, lg, r, key, val);
}

// Exclusive prefix of n over the warp; *total gets the sum.
__device__ __forceinline__ unsigned warp_prefix(unsigned n, int lane, unsigned* total) {
    unsigned incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    *total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    return incl - n;
}

__device__ __forceinline__ u64 warp_sum(u64 v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ u64 warp_max(u64 v) {
    for (int o = 16; o; o >>= 1) v = max(v, (u64)__shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}
// Warp-wide exclusive offsets of n, with one atomicAdd on `counter` for the whole warp.
__device__ __forceinline__ u64 warp_append(u64* counter, unsigned n) {
    const int lane = threadIdx.x & 31;
    unsigned incl = n;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    u64 base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, (u64)total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + (incl - n);
}

// Persistent: lanes without a row take new ones (one atomic per warp); every round advances all
// of the warp's rows by one frontier step, and finished rows are written out item-parallel,
// each entry at its rank within the row (rows come out sorted by column).
template <int F, int LF, int D, int LD, bool PK>
__global__ void __launch_bounds__(T0_THREADS) rows_thread(PcArgs args, u64* next_row) {
    PcArgs a = args;
    if (!resolve(a)) return;
    extern __shared__ __align__(16) unsigned char t0_raw[];
    T0Warp<F, D, PK>& sh = reinterpret_cast<T0Warp<F, D, PK>*>(t0_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint32_t lane_bit = 1u << lane;
    // a slot's key and count, and clearing a lane's slot, in either table form
    auto fkey = [&](int c2, int j, int r) { return PK ? sh.fk[c2][j][r] >> 8 : sh.fk[c2][j][r]; };
    auto fcnt = [&](int c2, int j, int r) { return PK ? sh.fk[c2][j][r] & 0xFFu : sh.fv[PK ? 0 : c2][PK ? 0 : j][r]; };
    auto fclear = [&](int c2, int j) {
        sh.fk[c2][j][lane] = EMPTY;
        if constexpr (!PK) sh.fv[c2][j][lane] = 0;
    };
    auto dclear = [&](int j) {
        sh.dk[j][lane] = EMPTY;
        if constexpr (!PK) sh.dv[j][lane] = 0;
    };
#pragma unroll
    for (int j = 0; j < F; ++j) {
        fclear(0, j);
        fclear(1, j);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) dclear(j);
    __syncwarp();
    int64_t s = -1;  // the lane's current row (-1: none)
    int c = 0;       // which frontier table is current (warp-uniform)
    u64 iter = 0, entries = 0, it_max = 0, en_sum = 0, mx_all = 0;
    // warp-private pools of row indices and staging slots, refilled in chunks so that the
    // shared counters see one atomic per chunk rather than one per round
    const u64 nwarps = u64(gridDim.x) * T0_WARPS;
    u64 pool_next = 0, pool_end = 0, seen = 0;
    u64 out_next = 0, out_end = 0;
    bool exhausted = false;
    while (true) {
        // lanes without a row take the next ones; a new row starts from A[s,:] and D[s,:]
        const unsigned want = __ballot_sync(0xFFFFFFFFu, s < 0 && !exhausted);
        if (want) {
            const u64 k = u64(__popc(want));
            const u64 rem = pool_end - pool_next;
            u64 fresh = pool_end;  // start of a newly taken chunk (if any)
            if (rem < k) {         // guided chunk size: large while much work is left
                const u64 left = u64(a.nrows) > seen ? u64(a.nrows) - seen : 0;
                const u64 ch = max(u64(32), min(u64(1024), left / (4 * nwarps)));
                if (lane == 0) fresh = atomicAdd(next_row, ch);
                fresh = __shfl_sync(0xFFFFFFFFu, fresh, 0);
                seen = fresh + ch;
                const u64 q = u64(__popc(want & (lane_bit - 1u)));
                const u64 mine = q < rem ? pool_next + q : fresh + (q - rem);
                pool_next = fresh + (k - rem);
                pool_end = fresh + ch;
                if (want & lane_bit) {
                    if (mine < (u64)a.nrows) s = row_of(a, int64_t(mine));
                    else exhausted = true;
                }
            } else {
                const u64 mine = pool_next + u64(__popc(want & (lane_bit - 1u)));
                pool_next += k;
                if (want & lane_bit) {
                    if (mine < (u64)a.nrows) s = row_of(a, int64_t(mine));
                    else exhausted = true;
                }
            }
            if ((want & lane_bit) && s >= 0) {
                iter = entries = 0;
                const uint32_t kinds = a.kinds[s];
                const uint4 t4 = trace_of(a, s);
                const uint32_t tg[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
                for (int k2 = 0; k2 < 4; ++k2) {  // at most 4 entries: these tables cannot fill
                    const uint32_t kind = trace_kind(kinds, k2);
                    if (!kind) continue;
                    const bool junction = kind == 1;
                    t0_add<PK>(junction ? &sh.fk[c][0][0] : &sh.dk[0][0],
                               junction ? &sh.fv[PK ? 0 : c][0][0] : &sh.dv[0][0], junction ? LF : LD, lane, tg[k2], 1);
                }
            }
        }
        if (!__any_sync(0xFFFFFFFFu, s >= 0)) break;
        __syncwarp();
        // one frontier step of every row: the list of (slot, row) frontier entries
        bool expand = false;
#pragma unroll
        for (int j = 0; j < F; ++j) expand |= s >= 0 && sh.fk[c][j][lane] != EMPTY;
        if (expand && int64_t(++iter) > a.max_iter) {
            atomicOr(a.status, ST_ITER);  // the row is cut short; the result is void anyway
            expand = false;
        }
        // the warp's list of (slot, row) frontier entries, then one entry per lane
        unsigned fm = 0;
#pragma unroll
        for (int j = 0; j < F; ++j) fm |= unsigned(expand && sh.fk[c][j][lane] != EMPTY) << j;
        entries += __popc(fm);
        unsigned total = 0;
        unsigned at = warp_prefix(unsigned(__popc(fm)), lane, &total);
#pragma unroll
        for (int j = 0; j < F; ++j)
            if ((fm >> j) & 1u) sh.items[at++] = uint16_t((j << 5) | lane);
        __syncwarp();
        uint32_t bad = 0;
        uint32_t* const nk = &sh.fk[c ^ 1][0][0];
        uint32_t* const nv = &sh.fv[PK ? 0 : c ^ 1][0][0];
        for (unsigned i = lane; i < total; i += 32) {
            const int it = sh.items[i];
            const int j = it >> 5, r = it & 31;
            const uint32_t key = fkey(c, j, r);
            const uint32_t cnt = fcnt(c, j, r);
            const int64_t src = a.n1 + int64_t(key);
            const uint32_t kj = a.kinds[src];
            const uint4 q = trace_of(a, src);
            const uint32_t tq[4] = {q.x, q.y, q.z, q.w};
            bool ok = true;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t kind = trace_kind(kj, k);
                if (!kind) continue;
                const bool junction = kind == 1;
                ok &= t0_add<PK>(junction ? nk : &sh.dk[0][0], junction ? nv : &sh.dv[0][0], junction ? LF : LD, r,
                                 tq[k], cnt);
            }
            if (!ok) bad |= 1u << r;
        }
        bad = __reduce_or_sync(0xFFFFFFFFu, bad);
        __syncwarp();
        // the current tables are spent: clear this lane's and swap
#pragma unroll
        for (int j = 0; j < F; ++j) fclear(c, j);
        c ^= 1;
        bool more = false;
#pragma unroll
        for (int j = 0; j < F; ++j) more |= sh.fk[c][j][lane] != EMPTY;
        const bool defer = s >= 0 && (bad & lane_bit);
        const bool done = s >= 0 && !defer && !more;
        // finished rows: entries of the D* tables, item-parallel, placed by rank within the row
        unsigned dm = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) dm |= unsigned(done && sh.dk[j][lane] != EMPTY) << j;
        const unsigned mine_n = unsigned(__popc(dm));
        unsigned nout = 0;
        const unsigned off = warp_prefix(mine_n, lane, &nout);
        if (nout) {
            // staging slots from the warp's chunk (a new chunk when this round's rows do not fit)
            if (u64(nout) > out_end - out_next) {
                const u64 ch = max(u64(nout), u64(T0_OUT_CHUNK));
                u64 b = 0;
                if (lane == 0) b = atomicAdd(a.out_cursor, ch);
                out_next = __shfl_sync(0xFFFFFFFFu, b, 0);
                out_end = out_next + ch;
            }
            const u64 base = out_next + off;
            out_next += u64(nout);
            sh.base[lane] = base;
            unsigned o = off;
#pragma unroll
            for (int j = 0; j < D; ++j)
                if ((dm >> j) & 1u) sh.items[o++] = uint16_t((j << 5) | lane);
            if (done) {
                a.row_start[s] = int64_t(base);
                a.row_len[s] = mine_n;
            }
            __syncwarp();
            for (unsigned i = lane; i < nout; i += 32) {
                const int it = sh.items[i];
                const int j = it >> 5, r = it & 31;
                const uint32_t slot = sh.dk[j][r];  // packed slots order by key too
                const uint32_t key = PK ? slot >> 8 : slot;
                const uint32_t val = PK ? slot & 0xFFu : sh.dv[PK ? 0 : j][r];
                int rank = 0;
#pragma unroll
                for (int jj = 0; jj < D; ++jj) rank += sh.dk[jj][r] < slot;  // EMPTY sorts last
                const u64 dst = sh.base[r] + u64(rank);
                if (dst < a.out_cap) {
                    a.out_col[dst] = key;
                    a.out_cnt[dst] = val;
                } else {
                    atomicOr(a.status, ST_RETRY);  // staging too small: the host grows it and reruns
                }
                mx_all = max(mx_all, (u64)val);
            }
        } else if (done) {
            a.row_start[s] = 0;
            a.row_len[s] = 0;
        }
        if (done) {
            it_max = max(it_max, iter);
            en_sum += entries;
        }
        __syncwarp();
        const u64 dpos = warp_append(a.deferred_count, defer ? 1u : 0u);
        if (defer) a.deferred[dpos] = uint32_t(s);
        if (done || defer) {  // leave this lane's tables clean for its next row
#pragma unroll
            for (int j = 0; j < D; ++j) dclear(j);
#pragma unroll
            for (int j = 0; j < F; ++j) fclear(c, j);
            s = -1;
        }
        __syncwarp();
    }
    mx_all = warp_max(mx_all);
    it_max = warp_max(it_max);
    en_sum = warp_sum(en_sum);
    if (lane == 0) {
        if (mx_all) atomicMax(a.max_count, mx_all);
        if (it_max) atomicMax(a.n_iter, it_max);
        if (en_sum) atomicAdd(a.n_entries, en_sum);
    }
}

// ---------------------------------------------------------------------------------------
// tiers 1 and 2+: hash tables shared by a group of G threads
// ---------------------------------------------------------------------------------------
struct Tables {
    uint32_t* fk;     // frontier hash keys (junction rank)
    u64* fv;          // frontier hash counts
    uint32_t* focc;   // occupied frontier slots, in claim order
    uint32_t* dk;     // D* row hash keys (2-saddle rank)
    u64* dv;          // D* row hash counts
    uint32_t* docc;   // occupied D* slots
    uint32_t* lk;     // current frontier list / sort buffer keys
    u64* lv;          // current frontier list / sort buffer counts
    int cap;          // hash slots (power of two); lists hold cap/2
    int lg;           // log2(cap)
    int* fsize;       // claimed frontier slots
    int* dsize;       // claimed D* slots
    int* bad;         // a table overflowed in this row
    u64* base;        // staging offset of the finished row
};

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int lg) { return (key * 2654435761u) >> (32 - lg); }

// Adds val to key's entry; false if the table is over its load limit.
__device__ bool table_add(uint32_t* K, u64* V, uint32_t* occ, int cap, int lg, int* size, uint32_t key, u64 val,
                          uint32_t* status) {
    uint32_t h = slot_of(key, lg);
    for (int probe = 0; probe < cap; ++probe) {
        uint32_t k = K[h];
        if (k == EMPTY) {
            k = atomicCAS(&K[h], EMPTY, key);
            if (k == EMPTY) {
                const int idx = atomicAdd(size, 1);
                if (idx >= cap / 2) return false;  // the row is abandoned and the tables scrubbed
                occ[idx] = h;
                k = key;
            }
        }
        if (k == key) {
            const u64 old = atomicAdd(&V[h], val);
            if (old + val < old) atomicOr(status, ST_OVERFLOW);
            return true;
        }
        h = (h + 1) & uint32_t(cap - 1);
    }
    return false;
}

template <int G>
__device__ __forceinline__ void group_sync() {
    if (G == 32) __syncwarp();
    else __syncthreads();
}

// Moves the n occupied entries of a table into the list (in claim order) and clears them.
template <int G>
__device__ void drain(uint32_t* K, u64* V, const uint32_t* occ, int n, const Tables& t, int r) {
    for (int i = r; i < n; i += G) {
        const uint32_t h = occ[i];
        t.lk[i] = K[h];
        t.lv[i] = V[h];
        K[h] = EMPTY;
        V[h] = 0;
    }
}

template <int G>
__device__ void scrub(const Tables& t, int r) {
    for (int i = r; i < t.cap; i += G) {
        t.fk[i] = EMPTY;
        t.fv[i] = 0;
        t.dk[i] = EMPTY;
        t.dv[i] = 0;
    }
}

// Row s of D*, computed by a group of G threads (rank r in the group).  Returns false if a
// table overflowed; the tables are left clean either way.
template <int G>
__device__ bool count_row(const PcArgs& a, const Tables& t, int64_t s, int r) {
    if (r == 0) {
        *t.fsize = 0;
        *t.dsize = 0;
        *t.bad = 0;
    }
    group_sync<G>();
    if (r < 4) {  // row s of A (the frontier A_0) and of D
        const uint32_t kind = trace_kind(a.kinds[s], r);
        const uint32_t dst = a.tgt[s * 4 + r];
        bool ok = true;
        if (kind == 1) ok = table_add(t.fk, t.fv, t.focc, t.cap, t.lg, t.fsize, dst, 1, a.status);
        if (kind == 2) ok = table_add(t.dk, t.dv, t.docc, t.cap, t.lg, t.dsize, dst, 1, a.status);
        if (!ok) *t.bad = 1;
    }
    group_sync<G>();
    u64 iter = 0, entries = 0;
    bool ok = true;
    while (true) {
        const int claimed = *t.fsize;
        const bool bad = *t.bad || claimed > t.cap / 2;
        group_sync<G>();
        if (bad) {
            ok = false;
            break;
        }
        const int n = claimed;
        drain<G>(t.fk, t.fv, t.focc, n, t, r);  // A_k[s,:] -> list; frontier table cleared
        group_sync<G>();
        if (r == 0) *t.fsize = 0;
        group_sync<G>();
        if (n == 0) break;
        if (int64_t(++iter) > a.max_iter) {
            if (r == 0) atomicOr(a.status, ST_ITER);
            break;
        }
        entries += u64(n);
        // A_{k+1}[s,:] += c B[j,:]  and  D*[s,:] += c B*[j,:]: one unit per traced path
        for (int i = r; i < n; i += G) {
            const int64_t j = a.n1 + int64_t(t.lk[i]);
            const u64 c = t.lv[i];
            const uint32_t kinds = a.kinds[j];
            const uint4 q = trace_of(a, j);
            const uint32_t tq[4] = {q.x, q.y, q.z, q.w};
            for (int k = 0; k < 4; ++k) {
                const uint32_t kind = trace_kind(kinds, k);
                if (!kind) continue;
                const bool added = kind == 1 ? table_add(t.fk, t.fv, t.focc, t.cap, t.lg, t.fsize, tq[k], c, a.status)
                                             : table_add(t.dk, t.dv, t.docc, t.cap, t.lg, t.dsize, tq[k], c, a.status);
                if (!added) *t.bad = 1;
            }
        }
        group_sync<G>();
    }
    const int nd = *t.dsize;
    ok = ok && !*t.bad && nd <= t.cap / 2;
    group_sync<G>();
    if (!ok) {
        scrub<G>(t, r);
        group_sync<G>();
        return false;
    }
    if (r == 0 && iter > 0) atomicMax(a.n_iter, iter);
    if (r == 0 && entries > 0) atomicAdd(a.n_entries, entries);
    drain<G>(t.dk, t.dv, t.docc, nd, t, r);  // D*[s,:] -> list
    int P = 1;
    while (P < nd) P <<= 1;
    for (int i = nd + r; i < P; i += G) {
        t.lk[i] = EMPTY;
        t.lv[i] = 0;
    }
    group_sync<G>();
    for (int k = 2; k <= P; k <<= 1)  // bitonic sort of (column, count) by column
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = r; i < P; i += G) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t ki = t.lk[i], kl = t.lk[l];
                    if ((ki > kl) == up) {
                        t.lk[i] = kl;
                        t.lk[l] = ki;
                        const u64 v = t.lv[i];
                        t.lv[i] = t.lv[l];
                        t.lv[l] = v;
                    }
                }
            }
            group_sync<G>();
        }
    if (r == 0) {
        const u64 b = nd ? atomicAdd(a.out_cursor, (u64)nd) : 0ull;
        a.row_start[s] = int64_t(b);
        a.row_len[s] = uint32_t(nd);
        *t.base = b;
    }
    group_sync<G>();
    const u64 base = *t.base;
    u64 mx = 0;
    for (int i = r; i < nd; i += G) {
        if (base + i < a.out_cap) {
            a.out_col[base + i] = t.lk[i];
            a.out_cnt[base + i] = t.lv[i];
        } else {
            atomicOr(a.status, ST_RETRY);  // staging too small: the host grows it and reruns
        }
        mx = max(mx, t.lv[i]);
    }
    if (mx) atomicMax(a.max_count, mx);
    group_sync<G>();
    return true;
}

// Tier 1: warps pull rows from a shared counter.
__global__ void __launch_bounds__(T1_WARPS * 32) rows_warp(PcArgs args, u64* next_row) {
    PcArgs a = args;
    if (!resolve(a)) return;
    __shared__ uint32_t fk[T1_WARPS][T1_HASH], dk[T1_WARPS][T1_HASH];
    __shared__ u64 fv[T1_WARPS][T1_HASH], dv[T1_WARPS][T1_HASH];
    __shared__ uint32_t focc[T1_WARPS][T1_LIST], docc[T1_WARPS][T1_LIST], lk[T1_WARPS][T1_LIST];
    __shared__ u64 lv[T1_WARPS][T1_LIST];
    __shared__ int counters[T1_WARPS][3];
    __shared__ u64 bases[T1_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < T1_HASH; i += 32) {
        fk[w][i] = dk[w][i] = EMPTY;
        fv[w][i] = dv[w][i] = 0;
    }
    __syncwarp();
    const Tables t{fk[w], fv[w], focc[w], dk[w], dv[w], docc[w], lk[w], lv[w], T1_HASH, 8,
                   &counters[w][0], &counters[w][1], &counters[w][2], &bases[w]};
    while (true) {
        u64 i = 0;
        if (lane == 0) i = atomicAdd(next_row, 1ull);
        i = __shfl_sync(0xFFFFFFFFu, i, 0);
        if (i >= (u64)a.nrows) break;
        const int64_t s = row_of(a, int64_t(i));
        if (!count_row<32>(a, t, s, lane) && lane == 0) {
            const u64 pos = atomicAdd(a.deferred_count, 1ull);
            if (a.retry_on_defer) atomicOr(a.status, ST_RETRY);
            a.deferred[pos] = uint32_t(s);
        }
    }
}

// Tiers 2+: one CTA per row, tables in global memory (one set per CTA).
__global__ void __launch_bounds__(T2_THREADS) rows_block(PcArgs args, uint32_t* gk, u64* gv, uint32_t* gocc, int cap,
                                                         int lg) {
    PcArgs a = args;
    if (!resolve(a)) return;
    __shared__ int counters[3];
    __shared__ u64 base;
    const size_t per = size_t(cap);
    uint32_t* k = gk + size_t(blockIdx.x) * 3 * per;
    u64* v = gv + size_t(blockIdx.x) * 3 * per;
    uint32_t* occ = gocc + size_t(blockIdx.x) * per;
    const Tables t{k, v, occ, k + per, v + per, occ + per / 2, k + 2 * per, v + 2 * per, cap, lg,
                   &counters[0], &counters[1], &counters[2], &base};
    for (int64_t i = blockIdx.x; i < a.nrows; i += gridDim.x) {
        const int64_t s = row_of(a, i);
        if (!count_row<T2_THREADS>(a, t, s, threadIdx.x) && threadIdx.x == 0) {
            const u64 pos = atomicAdd(a.deferred_count, 1ull);
            if (a.retry_on_defer) atomicOr(a.status, ST_RETRY);
            a.deferred[pos] = uint32_t(s);
        }
    }
}

__global__ void init_tables(uint32_t* k, u64* v, size_t n) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        k[i] = EMPTY;
        v[i] = 0;
    }
}

// One warp per 32 consecutive rows: their CSR range is contiguous, and the warp copies it one
// output entry per lane (coalesced writes).  A lane finds the row of its entry among the warp's 32
// row starts by a binary search over the lanes (shuffles); an empty row shares its start with the
// next one, and the search takes the last row starting at or before the entry.
__global__ void gather_rows(const unsigned long long* n1_dev, int64_t cap, const int64_t* __restrict__ row_start,
                            const int64_t* __restrict__ rowptr, const uint32_t* __restrict__ in_col,
                            const u64* __restrict__ in_cnt, uint32_t* __restrict__ col, u64* __restrict__ cnt,
                            uint32_t* status) {
    if (pass_retrying(status) || !count_fits(status, *n1_dev, cap)) return;
    const int64_t n1 = int64_t(*n1_dev);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t s0 = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; s0 < n1; s0 += nwarps * 32) {
        const int64_t s = s0 + lane;
        const int64_t end = rowptr[min(s0 + 32, n1)];
        const int64_t start = s < n1 ? rowptr[s] : end;  // past the last row: never at or before an entry
        const int64_t src = s < n1 ? row_start[s] : 0;
        const int64_t begin = __shfl_sync(0xFFFFFFFFu, start, 0);
        for (int64_t base = begin; base < end; base += 32) {  // warp-uniform
            const int64_t o = base + lane;
            int r = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const int64_t v = __shfl_sync(0xFFFFFFFFu, start, r + step);
                if (v <= o) r += step;
            }
            const int64_t rs = __shfl_sync(0xFFFFFFFFu, start, r), rsrc = __shfl_sync(0xFFFFFFFFu, src, r);
            if (o < end) {
                col[o] = in_col[rsrc + (o - rs)];
                cnt[o] = in_cnt[rsrc + (o - rs)];
            }
        }
    }
}

// Counter slots in Summary::pc.
enum { C_CURSOR = PC_CURSOR, C_MAX = PC_MAX, C_ITER = PC_ITER, C_ENTRIES = PC_ENTRIES, C_DEFER0 = PC_DEFER0,
       C_DEFER1 = PC_DEFER1, C_NEXT = PC_NEXT, C_DEFER2 = PC_DEFER2, C_DEFER3 = PC_DEFER3 };

}  // namespace

msc_status run_path_count(Plan* p, cudaStream_t s) {
    msc_status st;
    const bool cap_mode = p->capturing;
    const int64_t n1cap = cap_mode ? p->caps.cells[1] : p->counts[1];
    const int64_t njcap = cap_mode ? p->caps.nj : p->n_junctions;
    const int64_t n2cap = cap_mode ? p->caps.cells[2] : p->counts[2];
    const size_t n1c = size_t(n1cap ? n1cap : 1);
    if ((st = ensure(p, p->dstar_rowptr, sizeof(int64_t) * size_t(n1cap + 1)))) return st;
    if ((st = ensure(p, p->pc_rowstart, sizeof(int64_t) * n1c))) return st;
    if ((st = ensure(p, p->pc_rowlen, sizeof(uint32_t) * n1c))) return st;
    if ((st = ensure(p, p->pc_big, sizeof(uint32_t) * n1c * 2))) return st;
    if ((st = ensure(p, p->minor_scan, row_scan_scratch_bytes(n1cap)))) return st;
    u64* ctr = p->dsum()->pc;
    // method: forced by the options, else chosen after the plan's first run (which uses the
    // junction waves, whose cost does not grow with the depth of the minor)
    const int method = p->opts.path_count_method ? int(p->opts.path_count_method)
                                                 : (p->pc_method_chosen > 0 ? p->pc_method_chosen : 2);
    p->pc_method_used = method;
    if (method == 2) {  // junction waves (junction_dp.cu) into the same staging
        uint64_t cap = cap_mode ? uint64_t(p->caps.staging)
                                : uint64_t(std::max<int64_t>(p->dstar_nnz + p->dstar_nnz / 4, 8 * n1cap + 1024));
        uint64_t pool = cap_mode ? uint64_t(p->caps.dp_pool)
                                 : uint64_t(std::max<int64_t>(p->dp_pool_cap, 4 * njcap + 1024));
        for (int attempt = 0; attempt < 8; ++attempt) {
            if ((st = ensure(p, p->pc_col, sizeof(uint32_t) * cap))) return st;
            if ((st = ensure(p, p->pc_cnt, sizeof(u64) * cap))) return st;
            if ((st = ensure(p, p->dstar_col, sizeof(uint32_t) * cap))) return st;
            if ((st = ensure(p, p->dstar_count, sizeof(u64) * cap))) return st;
            if ((st = check_cuda(p, cudaMemsetAsync(ctr, 0, sizeof(u64) * PC_SLOTS, s), "memset counters"))) return st;
            if ((st = run_junction_dp(p, s, pool, cap))) return st;
            if (!cap_mode) {
                if ((st = read_summary(p, s))) return st;
                const u64 used = p->hsum->pc[C_CURSOR], pool_used = p->hsum->dp_pool_used;
                if (used > cap || pool_used > pool) {  // grow and redo the stage (an overflowing wave
                    // stops the later ones, so the usage seen is a lower bound)
                    if (used > cap) cap = std::max<uint64_t>(2 * cap, used + used / 4 + 1024);
                    if (pool_used > pool) pool = std::max<uint64_t>(2 * pool, pool_used + pool_used / 4 + 1024);
                    uint32_t zero = 0;
                    if ((st = check_cuda(p, cudaMemcpyAsync(p->status_word(), &zero, sizeof(zero),
                                                            cudaMemcpyHostToDevice, s),
                                         "status reset")))
                        return st;
                    continue;
                }
                p->dp_pool_cap = int64_t(pool_used);
            }
            const u64* all_rows = &p->dsum()->counts[1];
            if ((st = check_cuda(p,
                                 row_scan(p, static_cast<const uint32_t*>(p->pc_rowlen.ptr), all_rows, n1cap,
                                          static_cast<int64_t*>(p->dstar_rowptr.ptr),
                                          static_cast<u64*>(p->minor_scan.ptr), s, &p->dsum()->dstar_nnz),
                                 "D* row scan")))
                return st;
            if (n1cap) {
                gather_rows<<<grid_cap(p, n1cap, 256), 256, 0, s>>>(
                    all_rows, n1cap, static_cast<const int64_t*>(p->pc_rowstart.ptr),
                    static_cast<const int64_t*>(p->dstar_rowptr.ptr), static_cast<const uint32_t*>(p->pc_col.ptr),
                    static_cast<const u64*>(p->pc_cnt.ptr), static_cast<uint32_t*>(p->dstar_col.ptr),
                    static_cast<u64*>(p->dstar_count.ptr), p->status_word());
                launched(p);
            }
            p->pc_staging_cap = int64_t(cap);
            return check_cuda(p, cudaGetLastError(), "gather launch");
        }
        return fail(p, MSC_ERR_CUDA, "internal: D* staging did not converge");
    }
    const int first_tier = std::max(0, std::min(2, int(p->opts.path_count_tier)));
    // tier-0 and tier-0b grids: persistent, as many CTAs as fit.  Tier 0 packs key and count into
    // one word when every junction and 2-saddle rank fits in 24 bits (the capacities bound them);
    // a row whose counts pass 255 then goes on to tier 0b, which keeps 32-bit counts.
    const bool pack = njcap < int64_t(0xFFFFFF) && n2cap < int64_t(0xFFFFFF);
    const size_t t0_smem = (pack ? sizeof(T0Warp<T0_F, T0_D, true>) : sizeof(T0Warp<T0_F, T0_D, false>)) * T0_WARPS;
    const size_t t0b_smem = sizeof(T0Warp<T0B_F, T0B_D, false>) * T0_WARPS;
    auto* k0 = pack ? rows_thread<T0_F, T0_LF, T0_D, T0_LD, true> : rows_thread<T0_F, T0_LF, T0_D, T0_LD, false>;
    auto* k0b = rows_thread<T0B_F, T0B_LF, T0B_D, T0B_LD, false>;
    if ((st = check_cuda(p, cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t0_smem)),
                         "cudaFuncSetAttribute(rows_thread)")) ||
        (st = check_cuda(p, cudaFuncSetAttribute(k0b, cudaFuncAttributeMaxDynamicSharedMemorySize, int(t0b_smem)),
                         "cudaFuncSetAttribute(rows_thread)")))
        return st;
    int per_sm = 0, per_sm_b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k0, T0_THREADS, t0_smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k0b, T0_THREADS, t0b_smem);
    const int t0_grid = int(std::max<int64_t>(
        1, std::min<int64_t>((n1cap + T0_THREADS - 1) / T0_THREADS, int64_t(std::max(1, per_sm)) * p->num_sms)));
    const int t0b_grid = int(std::max<int64_t>(
        1, std::min<int64_t>((n1cap + T0_THREADS - 1) / T0_THREADS, int64_t(std::max(1, per_sm_b)) * p->num_sms)));
    // staging capacity, including what tier-0 warps may leave unused at the end of their chunks;
    // a synchronised run grows it and reruns the stage on overflow, a replayed graph asks for a rerun
    const uint64_t slack = uint64_t(t0_grid) * T0_WARPS * (T0_OUT_CHUNK + 32 * T0_D) +
                           uint64_t(t0b_grid) * T0_WARPS * (T0_OUT_CHUNK + 32 * T0B_D);
    uint64_t cap = cap_mode ? uint64_t(p->caps.staging)
                            : uint64_t(std::max<int64_t>(p->dstar_nnz + p->dstar_nnz / 4, 8 * n1cap + 1024)) + slack;
    // a row never needs more slots than 2 x max(junctions, 2-saddles)
    const int lg_max = 1 + int(std::ceil(std::log2(double(std::max<int64_t>({njcap, n2cap, 64}) + 1))));
    uint32_t* lists[2] = {static_cast<uint32_t*>(p->pc_big.ptr), static_cast<uint32_t*>(p->pc_big.ptr) + n1c};
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((st = ensure(p, p->pc_col, sizeof(uint32_t) * cap))) return st;
        if ((st = ensure(p, p->pc_cnt, sizeof(u64) * cap))) return st;
        if ((st = ensure(p, p->dstar_col, sizeof(uint32_t) * cap))) return st;
        if ((st = ensure(p, p->dstar_count, sizeof(u64) * cap))) return st;
        if ((st = check_cuda(p, cudaMemsetAsync(ctr, 0, sizeof(u64) * PC_SLOTS, s), "memset counters"))) return st;
        PcArgs a{};
        a.n1_dev = &p->dsum()->counts[1];
        a.nj_dev = &p->dsum()->n_junctions;
        a.n1_cap = n1cap;
        a.nj_cap = njcap;
        a.tgt = static_cast<const uint32_t*>(p->trace.ptr);
        a.kinds = static_cast<const uint32_t*>(p->trace_kinds.ptr);
        a.out_col = static_cast<uint32_t*>(p->pc_col.ptr);
        a.out_cnt = static_cast<u64*>(p->pc_cnt.ptr);
        a.out_cap = cap;
        a.out_cursor = ctr + C_CURSOR;
        a.max_count = ctr + C_MAX;
        a.n_iter = ctr + C_ITER;
        a.n_entries = ctr + C_ENTRIES;
        a.row_start = static_cast<int64_t*>(p->pc_rowstart.ptr);
        a.row_len = static_cast<uint32_t*>(p->pc_rowlen.ptr);
        a.max_iter = p->opts.max_iterations;
        a.status = p->status_word();
        // each tier takes the rows the previous one deferred; tier 3 here means tier 0b
        auto launch = [&](int tier, const uint32_t* rows, const u64* nrows, uint32_t* defer, u64* defer_ctr, int lg,
                          bool last) {
            a.rows = rows;
            a.nrows_dev = nrows;
            a.deferred = defer;
            a.deferred_count = defer_ctr;
            a.retry_on_defer = last && cap_mode;
            msc_status e;
            if (tier != 2 && (e = check_cuda(p, cudaMemsetAsync(ctr + C_NEXT, 0, sizeof(u64), s), "memset"))) return e;
            if (tier == 0) {
                record_event(p, p->kev0, s);
                k0<<<t0_grid, T0_THREADS, t0_smem, s>>>(a, ctr + C_NEXT);
                record_event(p, p->kev1, s);
                launched(p);
            } else if (tier == 3) {
                k0b<<<t0b_grid, T0_THREADS, t0b_smem, s>>>(a, ctr + C_NEXT);
                launched(p);
            } else if (tier == 1) {
                rows_warp<<<std::max(1, p->num_sms) * 8, T1_WARPS * 32, 0, s>>>(a, ctr + C_NEXT);
                launched(p);
            } else {
                const int cap_t = 1 << lg;
                const int ctas = lg <= 14 ? 128 : lg <= 18 ? 64 : 2;
                const size_t slots = size_t(ctas) * 3 * size_t(cap_t);
                // every use leaves the tables empty, so they are initialised only when (re)allocated
                const bool fresh = p->pc_gk.bytes < sizeof(uint32_t) * slots;
                if ((e = ensure(p, p->pc_gk, sizeof(uint32_t) * slots))) return e;
                if ((e = ensure(p, p->pc_gv, sizeof(u64) * slots))) return e;
                if ((e = ensure(p, p->pc_gocc, sizeof(uint32_t) * size_t(ctas) * size_t(cap_t)))) return e;
                if (fresh) {
                    init_tables<<<1024, 256, 0, s>>>(static_cast<uint32_t*>(p->pc_gk.ptr),
                                                     static_cast<u64*>(p->pc_gv.ptr), p->pc_gk.bytes / sizeof(uint32_t));
                    launched(p);
                }
                rows_block<<<ctas, T2_THREADS, 0, s>>>(a, static_cast<uint32_t*>(p->pc_gk.ptr),
                                                      static_cast<u64*>(p->pc_gv.ptr),
                                                      static_cast<uint32_t*>(p->pc_gocc.ptr), cap_t, lg);
                launched(p);
            }
            return check_cuda(p, cudaGetLastError(), "path count launch");
        };
        const u64* all_rows = &p->dsum()->counts[1];
        int lg = std::min(14, lg_max);
        // after the last tier: the list (index) and counter of the rows still left
        int left_list = 1;
        u64* left_ctr = ctr + C_DEFER2;
        if (first_tier == 0) {
            if ((st = launch(0, nullptr, all_rows, lists[0], ctr + C_DEFER0, 0, false))) return st;
            if ((st = launch(3, lists[0], ctr + C_DEFER0, lists[1], ctr + C_DEFER1, 0, false))) return st;
            if ((st = launch(1, lists[1], ctr + C_DEFER1, lists[0], ctr + C_DEFER3, 0, false))) return st;
            if ((st = launch(2, lists[0], ctr + C_DEFER3, lists[1], ctr + C_DEFER2, lg, true))) return st;
        } else if (first_tier == 1) {
            if ((st = launch(1, nullptr, all_rows, lists[0], ctr + C_DEFER1, 0, false))) return st;
            if ((st = launch(2, lists[0], ctr + C_DEFER1, lists[1], ctr + C_DEFER2, lg, true))) return st;
        } else {
            if ((st = launch(2, nullptr, all_rows, lists[1], ctr + C_DEFER2, lg, true))) return st;
        }
        if (!cap_mode) {
            // rows that outgrow the tier-2 tables: bigger tables, on the host's watch
            if ((st = read_summary(p, s))) return st;
            if (p->hsum->pc[C_CURSOR] > cap) {  // staging overflow: grow and redo the stage
                cap = p->hsum->pc[C_CURSOR] + p->hsum->pc[C_CURSOR] / 4 + 1024 + slack;
                uint32_t zero = 0;
                if ((st = check_cuda(p, cudaMemcpyAsync(p->status_word(), &zero, sizeof(zero), cudaMemcpyHostToDevice, s),
                                     "status reset")))
                    return st;
                continue;
            }
            int in = left_list;
            u64* in_ctr = left_ctr;
            u64 left = p->hsum->pc[left_ctr - ctr];
            while (left > 0) {
                if (lg >= lg_max) return fail(p, MSC_ERR_CUDA, "internal: a path-count row does not fit");
                lg = std::min(lg + 4, lg_max);
                u64* out_ctr = in_ctr == ctr + C_DEFER2 ? ctr + C_DEFER1 : ctr + C_DEFER2;
                if ((st = check_cuda(p, cudaMemsetAsync(out_ctr, 0, sizeof(u64), s), "memset"))) return st;
                if ((st = launch(2, lists[in], in_ctr, lists[in ^ 1], out_ctr, lg, false))) return st;
                if ((st = read_summary(p, s))) return st;
                in ^= 1;
                in_ctr = out_ctr;
                left = p->hsum->pc[out_ctr - ctr];
            }
        }
        // D* row pointers (the scan also gives nnz), then the rows gathered into CSR
        if ((st = check_cuda(p,
                             row_scan(p, static_cast<const uint32_t*>(p->pc_rowlen.ptr), all_rows, n1cap,
                                      static_cast<int64_t*>(p->dstar_rowptr.ptr), static_cast<u64*>(p->minor_scan.ptr),
                                      s, &p->dsum()->dstar_nnz),
                             "D* row scan")))
            return st;
        if (n1cap) {
            gather_rows<<<grid_cap(p, n1cap, 256), 256, 0, s>>>(
                all_rows, n1cap, a.row_start, static_cast<const int64_t*>(p->dstar_rowptr.ptr), a.out_col, a.out_cnt,
                static_cast<uint32_t*>(p->dstar_col.ptr), static_cast<u64*>(p->dstar_count.ptr), p->status_word());
            launched(p);
        }
        p->pc_staging_cap = int64_t(cap);
        return check_cuda(p, cudaGetLastError(), "gather launch");
    }
    return fail(p, MSC_ERR_CUDA, "internal: D* staging did not converge");
}

}  // namespace msc

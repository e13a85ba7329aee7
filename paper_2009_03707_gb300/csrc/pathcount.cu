// (a6) Saddle-saddle path counting: D* = D + sum_{k>=0} A B^k B* (Sec. 3.3 "Path counting
// via matrix operations").
//
// The paper iterates A <- A B over the whole matrix (cuSPARSE SpGEMM), accumulating A* until
// the product is zero, then forms A* B* + D.  Row s of every product depends only on row s
// of A, so here the same iteration runs row by row (Gustavson's row-wise product): a group of
// threads owns one 1-saddle s and keeps
//   * the frontier A_k[s,:] as a hash table keyed by junction rank,
//   * the accumulator D*[s,:] as a hash table keyed by 2-saddle rank,
// and repeats "for each (j, c) in A_k[s,:]: every traced path j -> j' adds c to A_{k+1}[s,j'],
// every traced path j -> t adds c to D*[s,t]" until the frontier is empty.  The minor's
// adjacency is the 4-slot trace of each junction (minor.cu); a repeated destination is a
// repeated path, i.e. the multiplicity.  Counts are exact uint64; an add that wraps sets the
// overflow flag (the paper reports multiplicities near 1e10, beyond 32 bits).
//
// Tier 1: one warp per 1-saddle with 256-slot tables in shared memory; 1-saddles whose rows
// outgrow them are queued for tier 2: one CTA per 1-saddle with tables in global memory,
// sized up again (tier 3) for whatever still does not fit.  Each finished row is sorted by
// column and appended to a staging buffer; a scan of the row lengths and one gather give the
// CSR of D*.
#include "rowscan.cuh"

namespace msc {

namespace {

constexpr uint32_t EMPTY = 0xFFFFFFFFu;
constexpr int T1_WARPS = 4;
constexpr int T1_HASH = 256;  // slots per table (power of two)
constexpr int T1_LIST = T1_HASH / 2;
constexpr int T2_THREADS = 256;

struct Tables {
    uint32_t* fk;            // frontier hash keys (junction rank)
    unsigned long long* fv;  // frontier hash counts
    uint32_t* dk;            // D* row hash keys (2-saddle rank)
    unsigned long long* dv;  // D* row hash counts
    uint32_t* lk;            // current frontier list / sort buffer keys
    unsigned long long* lv;  // current frontier list / sort buffer counts
    int cap;                 // hash slots (power of two); the list holds cap/2
    int lg;                  // log2(cap)
    int* fsize;              // occupied frontier slots
    int* dsize;              // occupied D* slots
    int* lsize;              // list length
    int* bad;                // table overflow in this row
    unsigned long long* base;  // staging offset of the finished row
};

struct PcArgs {
    int64_t n1;
    const uint32_t* tgt;    // 4 destination ranks per source (1-saddles, then junctions)
    const uint8_t* kinds;   // 2 bits per slot: 1 junction, 2 2-saddle
    uint32_t* out_col;      // staging: columns of finished rows
    unsigned long long* out_cnt;
    uint64_t out_cap;
    unsigned long long* out_cursor;
    int64_t* row_start;
    uint32_t* row_len;
    uint32_t* big;          // 1-saddles deferred to the next tier
    unsigned long long* big_count;
    uint64_t big_cap;
    unsigned long long* next_source;
    unsigned long long* max_count;
    unsigned long long* n_iter;
    unsigned long long* n_entries;  // sum of frontier sizes (for the roofline's byte count)
    int64_t max_iter;
    uint32_t* status;
};

__device__ __forceinline__ uint32_t slot_of(uint32_t key, int lg) { return (key * 2654435761u) >> (32 - lg); }

// Adds val to key's entry; returns false if the table is over its load limit.
__device__ bool table_add(uint32_t* K, unsigned long long* V, int cap, int lg, int* size, uint32_t key,
                          unsigned long long val, uint32_t* status) {
    uint32_t h = slot_of(key, lg);
    for (int probe = 0; probe < cap; ++probe) {
        uint32_t k = K[h];
        if (k == EMPTY) {
            k = atomicCAS(&K[h], EMPTY, key);
            if (k == EMPTY) {
                if (atomicAdd(size, 1) >= cap / 2) return false;
                k = key;
            }
        }
        if (k == key) {
            unsigned long long old = atomicAdd(&V[h], val);
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

// Moves every occupied slot of a hash table into the list (lk, lv) and clears the table.
template <int G>
__device__ void drain(uint32_t* K, unsigned long long* V, const Tables& t, int r) {
    for (int i = r; i < t.cap; i += G) {
        const uint32_t k = K[i];
        if (k == EMPTY) continue;
        const int pos = atomicAdd(t.lsize, 1);
        if (pos < t.cap / 2) {
            t.lk[pos] = k;
            t.lv[pos] = V[i];
        } else {
            *t.bad = 1;
        }
        K[i] = EMPTY;
        V[i] = 0;
    }
}

// Row s of D*, computed by a group of G threads (rank r in the group).  Returns false if
// a table overflowed; the tables are left cleared either way.
template <int G>
__device__ bool count_row(const PcArgs& a, const Tables& t, int64_t s, int r) {
    if (r == 0) {
        *t.fsize = 0;
        *t.dsize = 0;
        *t.lsize = 0;
        *t.bad = 0;
    }
    group_sync<G>();
    // row s of A (the frontier A_0) and of D
    if (r < 4) {
        const uint32_t kind = (a.kinds[s] >> (2 * r)) & 3u;
        const uint32_t dst = a.tgt[s * 4 + r];
        bool ok = true;
        if (kind == 1) ok = table_add(t.fk, t.fv, t.cap, t.lg, t.fsize, dst, 1, a.status);
        if (kind == 2) ok = table_add(t.dk, t.dv, t.cap, t.lg, t.dsize, dst, 1, a.status);
        if (!ok) *t.bad = 1;
    }
    group_sync<G>();
    int64_t iter = 0;
    while (true) {
        drain<G>(t.fk, t.fv, t, r);  // A_k[s,:] -> list; frontier table cleared
        group_sync<G>();
        const int n = min(*t.lsize, t.cap / 2);
        const int bad = *t.bad;
        group_sync<G>();
        if (r == 0) {
            *t.lsize = 0;
            *t.fsize = 0;
        }
        group_sync<G>();
        if (n == 0 || bad) break;
        if (r == 0) atomicAdd(a.n_entries, (unsigned long long)n);
        if (++iter > a.max_iter) {
            if (r == 0) atomicOr(a.status, ST_ITER);
            break;
        }
        // A_{k+1}[s,:] += c B[j,:]  and  D*[s,:] += c B*[j,:]: one unit per traced path
        for (int i = r; i < n; i += G) {
            const int64_t j = a.n1 + int64_t(t.lk[i]);
            const unsigned long long c = t.lv[i];
            const uint32_t kinds = a.kinds[j];
            for (int k = 0; k < 4; ++k) {
                const uint32_t kind = (kinds >> (2 * k)) & 3u;
                if (!kind) continue;
                const uint32_t dst = a.tgt[j * 4 + k];
                const bool ok = kind == 1 ? table_add(t.fk, t.fv, t.cap, t.lg, t.fsize, dst, c, a.status)
                                          : table_add(t.dk, t.dv, t.cap, t.lg, t.dsize, dst, c, a.status);
                if (!ok) *t.bad = 1;
            }
        }
        group_sync<G>();
    }
    if (r == 0 && iter > 0) atomicMax(a.n_iter, (unsigned long long)iter);
    // D*[s,:] -> list (and drop frontier leftovers after an overflow)
    drain<G>(t.dk, t.dv, t, r);
    for (int i = r; i < t.cap; i += G)
        if (t.fk[i] != EMPTY) {
            t.fk[i] = EMPTY;
            t.fv[i] = 0;
        }
    group_sync<G>();
    const bool ok = *t.bad == 0;
    const int n = min(*t.lsize, t.cap / 2);
    group_sync<G>();
    if (!ok) return false;
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = n + r; i < P; i += G) {
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
                        const unsigned long long v = t.lv[i];
                        t.lv[i] = t.lv[l];
                        t.lv[l] = v;
                    }
                }
            }
            group_sync<G>();
        }
    if (r == 0) {
        const unsigned long long b = n ? atomicAdd(a.out_cursor, (unsigned long long)n) : 0ull;
        a.row_start[s] = int64_t(b);
        a.row_len[s] = uint32_t(n);
        *t.base = b;
    }
    group_sync<G>();
    const unsigned long long base = *t.base;
    unsigned long long mx = 0;
    for (int i = r; i < n; i += G) {
        if (base + i < a.out_cap) {
            a.out_col[base + i] = t.lk[i];
            a.out_cnt[base + i] = t.lv[i];
        } else {
            atomicOr(a.status, ST_CAPACITY);
        }
        mx = max(mx, t.lv[i]);
    }
    if (mx) atomicMax(a.max_count, mx);
    group_sync<G>();
    return true;
}

// Tier 1: warps pull 1-saddles from a shared counter.
__global__ void __launch_bounds__(T1_WARPS * 32) rows_warp(PcArgs a) {
    __shared__ uint32_t fk[T1_WARPS][T1_HASH], dk[T1_WARPS][T1_HASH], lk[T1_WARPS][T1_LIST];
    __shared__ unsigned long long fv[T1_WARPS][T1_HASH], dv[T1_WARPS][T1_HASH], lv[T1_WARPS][T1_LIST];
    __shared__ int counters[T1_WARPS][4];
    __shared__ unsigned long long bases[T1_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < T1_HASH; i += 32) {
        fk[w][i] = dk[w][i] = EMPTY;
        fv[w][i] = dv[w][i] = 0;
    }
    __syncwarp();
    Tables t{fk[w], fv[w], dk[w], dv[w], lk[w], lv[w], T1_HASH, 8, &counters[w][0], &counters[w][1], &counters[w][2],
             &counters[w][3], &bases[w]};
    while (true) {
        unsigned long long s = 0;
        if (lane == 0) s = atomicAdd(a.next_source, 1ull);
        s = __shfl_sync(0xFFFFFFFFu, s, 0);
        if (s >= (unsigned long long)a.n1) break;
        if (!count_row<32>(a, t, int64_t(s), lane) && lane == 0) {
            const unsigned long long pos = atomicAdd(a.big_count, 1ull);
            if (pos < a.big_cap) a.big[pos] = uint32_t(s);
            else atomicOr(a.status, ST_CAPACITY);
        }
    }
}

// Tiers 2 and 3: one CTA per deferred 1-saddle, tables in global memory (one set per CTA).
__global__ void __launch_bounds__(T2_THREADS) rows_block(PcArgs a, const uint32_t* __restrict__ list, int64_t n,
                                                         uint32_t* gk, unsigned long long* gv, int cap, int lg,
                                                         uint32_t* still_big, unsigned long long* still_count) {
    __shared__ int counters[4];
    __shared__ unsigned long long base;
    const size_t per = size_t(cap);
    uint32_t* fk = gk + size_t(blockIdx.x) * 3 * per;
    unsigned long long* fv = gv + size_t(blockIdx.x) * 3 * per;
    Tables t{fk, fv, fk + per, fv + per, fk + 2 * per, fv + 2 * per, cap, lg, &counters[0], &counters[1],
             &counters[2], &counters[3], &base};
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t s = list[i];
        if (!count_row<T2_THREADS>(a, t, s, threadIdx.x) && threadIdx.x == 0) {
            const unsigned long long pos = atomicAdd(still_count, 1ull);
            still_big[pos] = uint32_t(s);
        }
    }
}

__global__ void init_tables(uint32_t* k, unsigned long long* v, size_t n) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        k[i] = EMPTY;
        v[i] = 0;
    }
}

__global__ void gather_rows(int64_t n1, const int64_t* __restrict__ row_start, const int64_t* __restrict__ rowptr,
                            const uint32_t* __restrict__ in_col, const unsigned long long* __restrict__ in_cnt,
                            uint32_t* __restrict__ col, unsigned long long* __restrict__ cnt) {
    const int64_t s = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n1) return;
    const int64_t b = row_start[s], o = rowptr[s], len = rowptr[s + 1] - rowptr[s];
    for (int64_t i = 0; i < len; ++i) {
        col[o + i] = in_col[b + i];
        cnt[o + i] = in_cnt[b + i];
    }
}

}  // namespace

msc_status run_path_count(Plan* p, cudaStream_t s) {
    msc_status st;
    const int64_t n1 = p->counts[1], nj = p->n_junctions, n2 = p->counts[2];
    if ((st = ensure(p, p->dstar_rowptr, sizeof(int64_t) * size_t(n1 + 1)))) return st;
    if ((st = ensure(p, p->pc_rowstart, sizeof(int64_t) * size_t(n1 ? n1 : 1)))) return st;
    if ((st = ensure(p, p->pc_rowlen, sizeof(uint32_t) * size_t(n1 ? n1 : 1)))) return st;
    if ((st = ensure(p, p->pc_big, sizeof(uint32_t) * size_t(n1 ? n1 : 1) * 2))) return st;
    if ((st = ensure(p, p->pc_counters, sizeof(unsigned long long) * 8))) return st;
    if ((st = ensure(p, p->minor_scan, row_scan_scratch_bytes(n1)))) return st;
    auto* ctr = static_cast<unsigned long long*>(p->pc_counters.ptr);
    // staging capacity: grown and the stage re-run if a run overflows it
    uint64_t cap = uint64_t(std::max<int64_t>(p->dstar_nnz + p->dstar_nnz / 4, 8 * n1 + 1024));
    for (int attempt = 0; attempt < 8; ++attempt) {
        if ((st = ensure(p, p->pc_col, sizeof(uint32_t) * cap))) return st;
        if ((st = ensure(p, p->pc_cnt, sizeof(unsigned long long) * cap))) return st;
        if ((st = check_cuda(p, cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * 8, s), "memset counters")))
            return st;
        PcArgs a{};
        a.n1 = n1;
        a.tgt = static_cast<const uint32_t*>(p->trace.ptr);
        a.kinds = static_cast<const uint8_t*>(p->trace_kinds.ptr);
        a.out_col = static_cast<uint32_t*>(p->pc_col.ptr);
        a.out_cnt = static_cast<unsigned long long*>(p->pc_cnt.ptr);
        a.out_cap = cap;
        a.out_cursor = ctr + 0;
        a.next_source = ctr + 1;
        a.big_count = ctr + 2;
        a.max_count = ctr + 3;
        a.n_iter = ctr + 4;
        a.n_entries = ctr + 6;
        a.row_start = static_cast<int64_t*>(p->pc_rowstart.ptr);
        a.row_len = static_cast<uint32_t*>(p->pc_rowlen.ptr);
        a.big = static_cast<uint32_t*>(p->pc_big.ptr);
        a.big_cap = uint64_t(n1 ? n1 : 1);
        a.max_iter = p->opts.max_iterations;
        a.status = static_cast<uint32_t*>(p->status.ptr);
        if (n1) {
            const int grid = std::max(1, p->num_sms) * 4;
            cudaEventRecord(p->kev0, s);
            rows_warp<<<grid, T1_WARPS * 32, 0, s>>>(a);
            cudaEventRecord(p->kev1, s);
            launched(p);
            if ((st = check_cuda(p, cudaGetLastError(), "rows_warp launch"))) return st;
        }
        unsigned long long h[8];
        if ((st = check_cuda(p, cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s), "counter copy")))
            return st;
        if ((st = check_cuda(p, cudaStreamSynchronize(s), "path count sync"))) return st;
        if (n1) cudaEventElapsedTime(&p->stats.ms_rows_kernel, p->kev0, p->kev1);
        // deferred rows: CTAs with global tables, growing until every row fits
        int64_t nbig = int64_t(h[2]);
        uint32_t* list = static_cast<uint32_t*>(p->pc_big.ptr);
        uint32_t* next_list = list + (n1 ? n1 : 1);
        // a row never needs more slots than 2 x max(junctions, 2-saddles)
        const int lg_max = 1 + int(std::ceil(std::log2(double(std::max<int64_t>({nj, n2, 64}) + 1))));
        int lg = std::min(14, lg_max);
        while (nbig > 0) {
            const int cap_t = 1 << lg;
            const int ctas = int(std::min<int64_t>(nbig, lg <= 14 ? 1024 : lg <= 18 ? 64 : 2));
            const size_t slots = size_t(ctas) * 3 * size_t(cap_t);
            if ((st = ensure(p, p->pc_gk, sizeof(uint32_t) * slots))) return st;
            if ((st = ensure(p, p->pc_gv, sizeof(unsigned long long) * slots))) return st;
            init_tables<<<1024, 256, 0, s>>>(static_cast<uint32_t*>(p->pc_gk.ptr),
                                             static_cast<unsigned long long*>(p->pc_gv.ptr), slots);
            launched(p);
            if ((st = check_cuda(p, cudaMemsetAsync(ctr + 5, 0, sizeof(unsigned long long), s), "memset"))) return st;
            rows_block<<<ctas, T2_THREADS, 0, s>>>(a, list, nbig, static_cast<uint32_t*>(p->pc_gk.ptr),
                                                  static_cast<unsigned long long*>(p->pc_gv.ptr), cap_t, lg, next_list,
                                                  ctr + 5);
            launched(p);
            if ((st = check_cuda(p, cudaGetLastError(), "rows_block launch"))) return st;
            unsigned long long still = 0;
            if ((st = check_cuda(p, cudaMemcpyAsync(&still, ctr + 5, sizeof(still), cudaMemcpyDeviceToHost, s),
                                 "counter copy")))
                return st;
            if ((st = check_cuda(p, cudaStreamSynchronize(s), "path count sync"))) return st;
            if (still > 0 && lg >= lg_max) return fail(p, MSC_ERR_CUDA, "internal: a path-count row does not fit");
            std::swap(list, next_list);
            nbig = int64_t(still);
            lg = std::min(lg + 4, lg_max);
        }
        if ((st = check_cuda(p, cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s), "counter copy")))
            return st;
        if ((st = check_cuda(p, cudaStreamSynchronize(s), "path count sync"))) return st;
        if (h[0] > cap) {  // staging overflow: grow and redo the stage
            uint32_t zero = 0;
            if ((st = check_cuda(p, cudaMemcpyAsync(p->status.ptr, &zero, sizeof(zero), cudaMemcpyHostToDevice, s),
                                 "status reset")))
                return st;
            cap = h[0] + h[0] / 4 + 1024;
            continue;
        }
        const int64_t nnz = int64_t(h[0]);
        p->dstar_nnz = nnz;
        p->stats.nnz_Dstar = nnz;
        p->stats.max_path_count = h[3];
        p->stats.n_iter = int64_t(h[4]);
        p->stats.n_frontier_entries = int64_t(h[6]);
        if ((st = ensure(p, p->dstar_col, sizeof(uint32_t) * size_t(nnz ? nnz : 1)))) return st;
        if ((st = ensure(p, p->dstar_count, sizeof(unsigned long long) * size_t(nnz ? nnz : 1)))) return st;
        if ((st = check_cuda(p,
                             row_scan(p, a.row_len, n1, static_cast<int64_t*>(p->dstar_rowptr.ptr),
                                      static_cast<unsigned long long*>(p->minor_scan.ptr), s),
                             "D* row scan")))
            return st;
        if (n1) {
            gather_rows<<<int((n1 + 255) / 256), 256, 0, s>>>(
                n1, a.row_start, static_cast<const int64_t*>(p->dstar_rowptr.ptr), a.out_col, a.out_cnt,
                static_cast<uint32_t*>(p->dstar_col.ptr), static_cast<unsigned long long*>(p->dstar_count.ptr));
            launched(p);
        }
        return check_cuda(p, cudaGetLastError(), "gather launch");
    }
    return fail(p, MSC_ERR_CUDA, "internal: D* staging did not converge");
}

}  // namespace msc

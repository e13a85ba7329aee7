// Ordered bitmap compaction: the prefix-scan / stream-compaction primitives of Sec. 2.3,
// specialised to bitmaps of cells.
//
// A "sequence" is a logical array of 32-bit bitmap words visited in cell-id order.  Entry
// i in [0, 4*nz*ny*W) of a sequence decodes as (z, c, y, b, w) with
//     i = (((z*2 + c)*ny + y)*2 + b)*W + w,
// i.e. the refined-grid row (cz = 2z+c, cy = 2y+b) and the word w of x positions.  Cells of
// one dimension k in one refined row all have a = k-b-c, so walking i in order and the bits
// of each word upwards visits the k-cells in increasing cell id.  A Source maps (seq, i) to a
// bitmap word index (or -1 if the row holds no cells of that kind) and writes the ids.
//
// Three launches: per-block popcount sums, a per-sequence scan of those sums, and a final
// pass that scans inside each block, stores every word's exclusive prefix (the rank of its
// first set bit, so rank(cell) = prefix[word] + popc(word & below)) and writes the ids.
#pragma once

#include "msc_internal.cuh"

namespace msc {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

struct RowCoord {
    int z, c, y, b, w;
};

__host__ __device__ __forceinline__ RowCoord decode_row(const Geom& g, int64_t i64) {
    RowCoord r;
    const uint32_t i = uint32_t(i64);  // 4*nz*ny*W < 2^32 for every plan
    uint32_t q = g.div_W.div(i);
    r.w = int(i - q * uint32_t(g.W));
    r.b = int(q & 1u);
    q >>= 1;
    const uint32_t q2 = g.div_ny.div(q);
    r.y = int(q - q2 * uint32_t(g.ny));
    r.c = int(q2 & 1u);
    r.z = int(q2 >> 1);
    return r;
}

__host__ __device__ __forceinline__ int64_t seq_length(const Geom& g) { return int64_t(4) * g.nz * g.ny * g.W; }

// Critical cells: sequence k = dimension k over the per-slot bitmaps [slot][z][y][w]; the
// ids go to out[k].
struct CritSource {
    Geom g;
    const uint32_t* bits;
    uint32_t* prefix;
    uint32_t* out[4];
    uint64_t cap[4];
    uint32_t* status;
    __device__ int64_t word_index(int k, int64_t i) const {
        RowCoord r = decode_row(g, i);
        int a = k - r.b - r.c;
        if (a < 0 || a > 1) return -1;
        return g.slot_word(a + 2 * r.b + 4 * r.c, r.z, r.y, r.w);
    }
    __device__ void emit(int k, int64_t i, uint64_t pos, uint32_t word) const {
        RowCoord r = decode_row(g, i);
        int a = k - r.b - r.c;
        while (word) {
            int bit = __ffs(word) - 1;
            word &= word - 1;
            int x = r.w * 32 + bit;
            if (pos < cap[k]) out[k][pos] = g.cell_id(2 * x + a, 2 * r.y + r.b, 2 * r.z + r.c);
            else atomicOr(status, ST_CAPACITY);
            ++pos;
        }
    }
};

// 1-cells marked in a bitmap stored directly in the 1-cell row layout (a = 1-b-c): one
// sequence, word index = i, ids to out.
struct EdgeSource {
    Geom g;
    const uint32_t* bits;
    uint32_t* prefix;
    uint32_t* out;
    uint64_t cap;
    uint32_t* status;
    __device__ int64_t word_index(int, int64_t i) const {
        RowCoord r = decode_row(g, i);
        return (r.b & r.c) ? -1 : i;
    }
    __device__ void emit(int, int64_t i, uint64_t pos, uint32_t word) const {
        RowCoord r = decode_row(g, i);
        int a = 1 - r.b - r.c;
        while (word) {
            int bit = __ffs(word) - 1;
            word &= word - 1;
            int x = r.w * 32 + bit;
            if (pos < cap) out[pos] = g.cell_id(2 * x + a, 2 * r.y + r.b, 2 * r.z + r.c);
            else atomicOr(status, ST_CAPACITY);
            ++pos;
        }
    }
};

template <class Src>
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(Src src, int64_t len, int blocks_per_seq,
                                                                   unsigned long long* sums) {
    const int seq = blockIdx.x / blocks_per_seq;
    const int64_t base = int64_t(blockIdx.x % blocks_per_seq) * SCAN_CHUNK;
    unsigned long long acc = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + int64_t(j) * SCAN_THREADS + threadIdx.x;
        if (i < len) {
            int64_t wi = src.word_index(seq, i);
            if (wi >= 0) acc += __popc(src.bits[wi]);
        }
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    __shared__ unsigned long long warp_sums[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += warp_sums[w];
        sums[blockIdx.x] = t;
    }
}

// One block per sequence: exclusive scan of that sequence's block sums, in place; the
// sequence total goes to totals[seq].
static __global__ void __launch_bounds__(1024) scan_top_kernel(unsigned long long* sums, int blocks_per_seq,
                                                        unsigned long long* totals) {
    unsigned long long* s = sums + int64_t(blockIdx.x) * blocks_per_seq;
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < blocks_per_seq; base += blockDim.x) {
        int i = base + threadIdx.x;
        unsigned long long v = i < blocks_per_seq ? s[i] : 0;
        unsigned long long incl = v;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += n;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long wt = lane < int(blockDim.x >> 5) ? warp_tot[lane] : 0;
            unsigned long long wincl = wt;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, wincl, o);
                if (lane >= o) wincl += n;
            }
            if (lane < int(blockDim.x >> 5)) warp_tot[lane] = wincl - wt;  // exclusive per warp
        }
        __syncthreads();
        unsigned long long c = carry;
        if (i < blocks_per_seq) s[i] = c + warp_tot[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + warp_tot[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

template <class Src>
__global__ void __launch_bounds__(SCAN_THREADS) scan_emit_kernel(Src src, int64_t len, int blocks_per_seq,
                                                                 const unsigned long long* block_offsets) {
    const int seq = blockIdx.x / blocks_per_seq;
    const int64_t base = int64_t(blockIdx.x % blocks_per_seq) * SCAN_CHUNK + int64_t(threadIdx.x) * SCAN_ITEMS;
    int64_t widx[SCAN_ITEMS];
    uint32_t word[SCAN_ITEMS];
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + j;
        widx[j] = i < len ? src.word_index(seq, i) : -1;
        word[j] = widx[j] >= 0 ? src.bits[widx[j]] : 0u;
        acc += __popc(word[j]);
    }
    // block exclusive scan of the per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = acc;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += n;
    }
    __shared__ unsigned long long warp_tot[SCAN_THREADS / 32];
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long wt = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        unsigned long long wincl = wt;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, wincl, o);
            if (lane >= o) wincl += n;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wincl - wt;
    }
    __syncthreads();
    unsigned long long pos = block_offsets[blockIdx.x] + warp_tot[warp] + incl - acc;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (widx[j] < 0) continue;
        src.prefix[widx[j]] = uint32_t(pos);
        if (word[j]) src.emit(seq, base + j, pos, word[j]);
        pos += __popc(word[j]);
    }
}

// Host driver, phase 1: block sums, and per-sequence totals into d_totals[0..nseq) (device
// memory; no host synchronisation).
template <class Src>
msc_status compaction_sums(Plan* p, cudaStream_t s, const Src& src, int nseq, unsigned long long* d_totals) {
    const int64_t len = seq_length(p->g);
    const int bps = int((len + SCAN_CHUNK - 1) / SCAN_CHUNK);
    msc_status st;
    if ((st = ensure(p, p->scan_sums, sizeof(unsigned long long) * size_t(bps) * size_t(nseq)))) return st;
    auto* sums = static_cast<unsigned long long*>(p->scan_sums.ptr);
    scan_reduce_kernel<Src><<<bps * nseq, SCAN_THREADS, 0, s>>>(src, len, bps, sums);
    scan_top_kernel<<<nseq, 1024, 0, s>>>(sums, bps, d_totals);
    launched(p, 2);
    return check_cuda(p, cudaGetLastError(), "scan launch");
}

// Host driver, phase 2: prefixes and ids (the Src's output pointers must be sized by now).
template <class Src>
msc_status compaction_emit(Plan* p, cudaStream_t s, const Src& src, int nseq) {
    const int64_t len = seq_length(p->g);
    const int bps = int((len + SCAN_CHUNK - 1) / SCAN_CHUNK);
    auto* sums = static_cast<unsigned long long*>(p->scan_sums.ptr);
    scan_emit_kernel<Src><<<bps * nseq, SCAN_THREADS, 0, s>>>(src, len, bps, sums);
    launched(p);
    return check_cuda(p, cudaGetLastError(), "scan emit launch");
}

// Rank of a cell in an ordered compaction: prefix of its word plus the set bits below it.
__device__ __forceinline__ uint32_t bitmap_rank(const uint32_t* bits, const uint32_t* prefix, int64_t word_index,
                                                int bit) {
    return prefix[word_index] + __popc(bits[word_index] & ((1u << bit) - 1u));
}

}  // namespace msc

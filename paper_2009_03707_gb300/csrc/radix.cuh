// Stable least-significant-digit radix sort of (uint32 key, uint32 value) pairs, 8 bits a pass,
// as many passes as the largest key needs.  Each pass is three launches: per-tile digit
// histograms, one scan of all of them in (digit, tile) order, and a scatter in which every tile
// ranks its elements stably (equal digits keep their input order).  Used by the exports that
// regroup arcs by their other end (transpose.cu, graph.cu).
#pragma once

#include "rowscan.cuh"

namespace msc {

constexpr int RX_THREADS = 256;
constexpr int RX_ITEMS = 16;
constexpr int RX_TILE = RX_THREADS * RX_ITEMS;  // elements per tile, striped: item j of thread t
constexpr int RX_BINS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;

// Digit counts of one tile: hist[d * ntiles + tile].
static __global__ void __launch_bounds__(RX_THREADS) radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                                int ntiles, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[RX_BINS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = int64_t(blockIdx.x) * RX_TILE;
#pragma unroll 4
    for (int j = 0; j < RX_ITEMS; ++j) {
        const int64_t i = base + int64_t(j) * RX_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[int64_t(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: element i goes to offs[d * ntiles + tile] + (elements of digit d
// before it in the tile).  The tile is taken in RX_ITEMS rounds of RX_THREADS consecutive
// elements; within a round a warp ranks equal digits with a match mask, the warps are ordered by
// a per-digit prefix, and a running count carries the rounds.
static __global__ void __launch_bounds__(RX_THREADS) radix_scatter(const uint32_t* __restrict__ keys_in,
                                                                   const uint32_t* __restrict__ vals_in, int64_t n,
                                                                   int shift, int ntiles,
                                                                   const int64_t* __restrict__ offs,
                                                                   uint32_t* __restrict__ keys_out,
                                                                   uint32_t* __restrict__ vals_out) {
    __shared__ uint32_t wcnt[RX_WARPS][RX_BINS];
    __shared__ uint32_t run[RX_BINS];
    __shared__ int64_t base_of[RX_BINS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    run[t] = 0;
    base_of[t] = offs[int64_t(t) * ntiles + blockIdx.x];
    const int64_t tile = int64_t(blockIdx.x) * RX_TILE;
    const uint32_t lt = (1u << lane) - 1u;
    for (int j = 0; j < RX_ITEMS; ++j) {
#pragma unroll
        for (int w = 0; w < RX_WARPS; ++w) wcnt[w][t] = 0;
        __syncthreads();
        const int64_t i = tile + int64_t(j) * RX_THREADS + t;
        const bool live = i < n;
        const uint32_t key = live ? keys_in[i] : 0u;
        const uint32_t val = live ? vals_in[i] : 0u;
        const uint32_t d = live ? (key >> shift) & 0xFFu : uint32_t(RX_BINS);  // RX_BINS: no element
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, d);
        const uint32_t rank = __popc(peers & lt);
        if (live && rank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        {  // thread t: digit t's exclusive prefix over the warps, after the earlier rounds
            uint32_t acc = run[t];
#pragma unroll
            for (int w = 0; w < RX_WARPS; ++w) {
                const uint32_t c = wcnt[w][t];
                wcnt[w][t] = acc;
                acc += c;
            }
            run[t] = acc;
        }
        __syncthreads();
        if (live) {
            const int64_t pos = base_of[d] + wcnt[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

// Work space of radix_sort_pairs for n elements: digit histograms, their scan, scan scratch.
struct RadixSpace {
    uint32_t* hist;                // >= RX_BINS * ntiles
    int64_t* offs;                 // >= RX_BINS * ntiles + 1
    unsigned long long* scratch;   // row_scan scratch for RX_BINS * ntiles counts
};

inline int64_t radix_tiles(int64_t n) { return (n + RX_TILE - 1) / RX_TILE; }
inline size_t radix_hist_count(int64_t n) { return size_t(RX_BINS) * size_t(radix_tiles(n)); }

// Sorts keys[cur], vals[cur] (n pairs, keys <= max_key) stably by key, ping-ponging with the
// other buffer of each pair; *cur ends on the buffer holding the result.
inline cudaError_t radix_sort_pairs(Plan* p, uint32_t* keys[2], uint32_t* vals[2], int* cur, int64_t n,
                                    uint32_t max_key, const RadixSpace& ws, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t ntiles = radix_tiles(n);
    const int64_t nhist = int64_t(RX_BINS) * ntiles;
    for (int shift = 0; shift < 32 && (max_key >> shift) != 0; shift += 8) {
        radix_hist<<<unsigned(ntiles), RX_THREADS, 0, s>>>(keys[*cur], n, shift, int(ntiles), ws.hist);
        launched(p);
        cudaError_t e = row_scan(p, ws.hist, nullptr, nhist, ws.offs, ws.scratch, s);
        if (e != cudaSuccess) return e;
        radix_scatter<<<unsigned(ntiles), RX_THREADS, 0, s>>>(keys[*cur], vals[*cur], n, shift, int(ntiles), ws.offs,
                                                               keys[*cur ^ 1], vals[*cur ^ 1]);
        launched(p);
        *cur ^= 1;
    }
    return cudaGetLastError();
}

}  // namespace msc

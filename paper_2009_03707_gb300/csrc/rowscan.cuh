// Exclusive scan of uint32 row counts into int64 CSR row pointers (rowptr[n] = nnz), the
// prefix-sum primitive of Sec. 2.3 for CSR construction.  Three launches: block sums,
// a single-block scan of those sums, and the block-local scan plus offset.  The row count is
// either known on the host, or read on the device (n_dev, clamped to the capacity the grid was
// sized for), so that a pipeline can scan a row count it has not synchronised on.
#pragma once

#include "msc_internal.cuh"

namespace msc {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_CHUNK = RS_THREADS * RS_ITEMS;

__device__ __forceinline__ int64_t rows_of(const unsigned long long* n_dev, int64_t cap) {
    return n_dev ? int64_t(min((unsigned long long)cap, *n_dev)) : cap;
}

static __global__ void __launch_bounds__(RS_THREADS) rowscan_reduce(const uint32_t* __restrict__ cnt,
                                                                    const unsigned long long* n_dev, int64_t cap,
                                                                    unsigned long long* __restrict__ sums) {
    const int64_t n = rows_of(n_dev, cap);
    const int64_t base = int64_t(blockIdx.x) * RS_CHUNK;
    unsigned long long acc = 0;
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t i = base + int64_t(j) * RS_THREADS + threadIdx.x;
        if (i < n) acc += cnt[i];
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
    __shared__ unsigned long long ws[RS_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < RS_THREADS / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// single block of 1024 threads: exclusive scan of nb sums in place, total to *total
static __global__ void __launch_bounds__(1024) rowscan_top(unsigned long long* sums, int nb, long long* total) {
    __shared__ unsigned long long wt[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const unsigned long long v = i < nb ? sums[i] : 0;
        unsigned long long incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wt[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long a = wt[lane], ai = a;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, ai, o);
                if (lane >= o) ai += y;
            }
            wt[lane] = ai - a;
        }
        __syncthreads();
        const unsigned long long c = carry;
        if (i < nb) sums[i] = c + wt[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + wt[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = (long long)carry;
}

static __global__ void __launch_bounds__(RS_THREADS) rowscan_emit(const uint32_t* __restrict__ cnt,
                                                                  const unsigned long long* n_dev, int64_t cap,
                                                                  const unsigned long long* __restrict__ offs,
                                                                  int64_t* __restrict__ rowptr) {
    const int64_t n = rows_of(n_dev, cap);
    const int64_t base = int64_t(blockIdx.x) * RS_CHUNK + int64_t(threadIdx.x) * RS_ITEMS;
    uint32_t v[RS_ITEMS];
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        v[j] = (base + j < n) ? cnt[base + j] : 0u;
        acc += v[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = acc;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    __shared__ unsigned long long wt[RS_THREADS / 32];
    if (lane == 31) wt[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long a = lane < RS_THREADS / 32 ? wt[lane] : 0, ai = a;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, ai, o);
            if (lane >= o) ai += y;
        }
        if (lane < RS_THREADS / 32) wt[lane] = ai - a;
    }
    __syncthreads();
    unsigned long long pos = offs[blockIdx.x] + wt[warp] + incl - acc;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        if (base + j < n) rowptr[base + j] = (int64_t)pos;
        pos += v[j];
    }
}

static __global__ void rowscan_finish(int64_t* rowptr, const unsigned long long* n_dev, int64_t cap,
                                      const long long* total, unsigned long long* total_out) {
    rowptr[rows_of(n_dev, cap)] = *total;
    if (total_out) *total_out = (unsigned long long)*total;
}

// rowptr (n+1 int64) from cnt (n uint32), n = min(*n_dev, cap), or n = cap when n_dev is null;
// the total also goes to *total_out when given.  scratch holds >= ceil(cap/RS_CHUNK) + 2 uint64.
inline cudaError_t row_scan(Plan* p, const uint32_t* cnt, const unsigned long long* n_dev, int64_t cap,
                            int64_t* rowptr, unsigned long long* scratch, cudaStream_t s,
                            unsigned long long* total_out = nullptr) {
    const int nb = int((cap + RS_CHUNK - 1) / RS_CHUNK);
    long long* total = reinterpret_cast<long long*>(scratch + (nb > 0 ? nb : 1));
    if (nb > 0) {
        rowscan_reduce<<<nb, RS_THREADS, 0, s>>>(cnt, n_dev, cap, scratch);
        rowscan_top<<<1, 1024, 0, s>>>(scratch, nb, total);
        rowscan_emit<<<nb, RS_THREADS, 0, s>>>(cnt, n_dev, cap, scratch, rowptr);
        launched(p, 3);
    } else {
        cudaMemsetAsync(total, 0, sizeof(long long), s);
    }
    rowscan_finish<<<1, 1, 0, s>>>(rowptr, n_dev, cap, total, total_out);
    launched(p);
    return cudaGetLastError();
}

inline size_t row_scan_scratch_bytes(int64_t n) { return sizeof(unsigned long long) * size_t((n + RS_CHUNK - 1) / RS_CHUNK + 2); }

}  // namespace msc

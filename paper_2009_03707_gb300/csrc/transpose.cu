// Saddle-saddle arcs by 2-saddle: D* in compressed sparse column form.
//
// Sec. 3.5 "Data structure": the complex is queried in both directions -- the arcs that leave a
// 1-saddle (descending from a 2-saddle's point of view) and the arcs that reach a 2-saddle -- so
// every arc is kept twice.  The CSR of D* (pathcount.cu) lists each 1-saddle's 2-saddles; this is
// its transpose: for each 2-saddle (by rank in the 2-saddle list) the 1-saddles (by rank) with
// their path counts, sorted by 1-saddle rank.
//
// Built on request, host-synchronised, from the finished CSR:
//   1. column pointers: a count of every column and a scan;
//   2. a stable least-significant-digit radix sort of the entries by column, 8 bits a pass (as
//      many passes as the 2-saddle ranks need).  The entries start in row-major order, so a
//      stable sort by column leaves each column's rows ascending;
//   3. rows and counts gathered through the sorted entry indices.
// Each sort pass is three launches: per-tile digit histograms, one scan of all of them in
// (digit, tile) order, and a scatter in which each tile ranks its elements stably.
#include "radix.cuh"

namespace msc {

namespace {

// Row index of every CSR entry (the entries of row r are rowptr[r] .. rowptr[r+1]).
__global__ void __launch_bounds__(256) expand_rows(const int64_t* __restrict__ rowptr, int64_t nrows,
                                                   uint32_t* __restrict__ row_of) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < nrows; r += int64_t(gridDim.x) * blockDim.x)
        for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) row_of[e] = uint32_t(r);
}

// Entries per column, and the identity permutation the sort starts from.
__global__ void __launch_bounds__(256) count_cols(const uint32_t* __restrict__ col, int64_t nnz, int64_t ncols,
                                                  uint32_t* __restrict__ cnt, uint32_t* __restrict__ idx,
                                                  uint32_t* __restrict__ status) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t c = col[e];
        if (c < ncols) atomicAdd(&cnt[c], 1u);
        else atomicOr(status, ST_INTERNAL);
        idx[e] = uint32_t(e);
    }
}

__global__ void __launch_bounds__(256) gather_csc(const uint32_t* __restrict__ perm, int64_t nnz,
                                                  const uint32_t* __restrict__ row_of,
                                                  const unsigned long long* __restrict__ count_in,
                                                  uint32_t* __restrict__ row_out,
                                                  unsigned long long* __restrict__ count_out) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nnz; i += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t e = perm[i];
        row_out[i] = row_of[e];
        count_out[i] = count_in[e];
    }
}

int grid_of(const Plan* p, int64_t n) {
    const int64_t want = (n + 255) / 256;
    return int(std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(1, p->num_sms)) * 16)));
}

}  // namespace

msc_status build_dstar_csc(Plan* p, cudaStream_t s) {
    msc_status st;
    const int64_t n1 = p->counts[1], n2 = p->counts[2], nnz = p->dstar_nnz;
    if (nnz >= (int64_t(1) << 32)) return fail(p, MSC_ERR_TOO_LARGE, "D* has 2^32 or more entries");
    if ((st = ensure(p, p->csc_colptr, sizeof(int64_t) * size_t(n2 + 1)))) return st;
    if ((st = ensure(p, p->csc_row, sizeof(uint32_t) * size_t(nnz ? nnz : 1)))) return st;
    if ((st = ensure(p, p->csc_count, sizeof(unsigned long long) * size_t(nnz ? nnz : 1)))) return st;
    const int64_t nhist = int64_t(radix_hist_count(nnz));
    // work space: column counts, two key and two value arrays, the row of each entry, the digit
    // histograms and their scan
    const size_t scan_n = size_t(std::max<int64_t>(n2, nhist));
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) / 256 * 256;
        return at;
    };
    const size_t o_cnt = carve(sizeof(uint32_t) * size_t(std::max<int64_t>(n2, nhist)));
    const size_t o_k0 = carve(sizeof(uint32_t) * size_t(nnz)), o_k1 = carve(sizeof(uint32_t) * size_t(nnz));
    const size_t o_v0 = carve(sizeof(uint32_t) * size_t(nnz)), o_v1 = carve(sizeof(uint32_t) * size_t(nnz));
    const size_t o_row = carve(sizeof(uint32_t) * size_t(nnz));
    const size_t o_offs = carve(sizeof(int64_t) * size_t(nhist + 1));
    const size_t o_scr = carve(row_scan_scratch_bytes(int64_t(scan_n)));
    if ((st = ensure(p, p->csc_work, off))) return st;
    char* w = static_cast<char*>(p->csc_work.ptr);
    auto* cnt = reinterpret_cast<uint32_t*>(w + o_cnt);
    uint32_t* keys[2] = {reinterpret_cast<uint32_t*>(w + o_k0), reinterpret_cast<uint32_t*>(w + o_k1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(w + o_v0), reinterpret_cast<uint32_t*>(w + o_v1)};
    auto* row_of = reinterpret_cast<uint32_t*>(w + o_row);
    auto* offs = reinterpret_cast<int64_t*>(w + o_offs);
    auto* scratch = reinterpret_cast<unsigned long long*>(w + o_scr);
    auto* colptr = static_cast<int64_t*>(p->csc_colptr.ptr);
    const auto* col = static_cast<const uint32_t*>(p->dstar_col.ptr);
    // 1. column pointers
    if ((st = check_cuda(p, cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * size_t(n2 ? n2 : 1), s), "memset"))) return st;
    if (nnz) {
        count_cols<<<grid_of(p, nnz), 256, 0, s>>>(col, nnz, n2, cnt, vals[0], p->status_word());
        launched(p);
    }
    if ((st = check_cuda(p, row_scan(p, cnt, nullptr, n2, colptr, scratch, s), "column scan"))) return st;
    if (nnz == 0) return check_cuda(p, cudaGetLastError(), "csc launch");
    expand_rows<<<grid_of(p, n1), 256, 0, s>>>(static_cast<const int64_t*>(p->dstar_rowptr.ptr), n1, row_of);
    launched(p);
    if ((st = check_cuda(p, cudaMemcpyAsync(keys[0], col, sizeof(uint32_t) * size_t(nnz), cudaMemcpyDeviceToDevice, s),
                         "copy columns")))
        return st;
    // 2. stable sort by column, 8 bits a pass
    int cur = 0;
    const RadixSpace ws{cnt, offs, scratch};
    if ((st = check_cuda(p, radix_sort_pairs(p, keys, vals, &cur, nnz, uint32_t(std::max<int64_t>(n2 - 1, 0)), ws, s),
                         "column sort")))
        return st;
    // 3. rows and counts in column order
    gather_csc<<<grid_of(p, nnz), 256, 0, s>>>(vals[cur], nnz, row_of,
                                               static_cast<const unsigned long long*>(p->dstar_count.ptr),
                                               static_cast<uint32_t*>(p->csc_row.ptr),
                                               static_cast<unsigned long long*>(p->csc_count.ptr));
    launched(p);
    return check_cuda(p, cudaGetLastError(), "csc launch");
}

}  // namespace msc

// Internal definitions shared by the libmsc kernels and the C ABI (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/msc.h"
#include "geom.cuh"

namespace msc {

// ---- device status word (one per plan): bits OR-ed by kernels, read by the host ----------
enum StatusBit : uint32_t {
    ST_NAN = 1u << 0,        // the field holds a NaN
    ST_OVERFLOW = 1u << 1,   // a uint64 path count overflowed
    ST_CAPACITY = 1u << 2,   // a device buffer was too small (internal error)
    ST_ITER = 1u << 3,       // an iteration cap was reached
    ST_TIMEOUT = 1u << 4,    // a bounded spin wait gave up
    ST_INTERNAL = 1u << 5,   // an invariant was violated (a bounds check failed)
};

// ---- the plan ----------------------------------------------------------------------------
struct DeviceBuffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct Plan {
    Geom g;
    int device = 0;
    msc_opts opts{};
    std::string last_error;
    msc_stats stats{};
    int64_t peak_bytes = 0;
    int64_t live_bytes = 0;
    int num_sms = 0;

    // stage products and scratch (all grow-only, freed by msc_plan_destroy)
    DeviceBuffer words, status, crit_bits, crit_prefix, scan_sums, totals;
    DeviceBuffer cells[4];
    DeviceBuffer vmin, cmax, min_arcs, max_arcs, flag;
    DeviceBuffer visited, reach_tmp, reach_masks, reach_qdown, reach_flags, reach_count, node_info;
    DeviceBuffer junc_bits, junc_prefix, junc_cells;
    DeviceBuffer trace, trace_kinds, minor_rowcnt, minor_scan, minor_rowptr[4], minor_col[4], minor_mult[4];
    DeviceBuffer pc_rowstart, pc_rowlen, pc_big, pc_counters, pc_col, pc_cnt, pc_gk, pc_gv, pc_gocc;
    DeviceBuffer dstar_rowptr, dstar_col, dstar_count;

    template <class F>
    void for_each_buffer(F&& f) {
        DeviceBuffer* all[] = {&words, &status, &crit_bits, &crit_prefix, &scan_sums, &totals, &cells[0], &cells[1],
                               &cells[2], &cells[3], &vmin, &cmax, &min_arcs, &max_arcs, &flag, &visited, &node_info,
                               &reach_tmp, &reach_masks, &reach_qdown, &reach_flags, &reach_count, &junc_bits, &junc_prefix, &junc_cells, &trace,
                               &trace_kinds, &minor_rowcnt, &minor_scan, &minor_rowptr[0], &minor_rowptr[1],
                               &minor_rowptr[2], &minor_rowptr[3], &minor_col[0], &minor_col[1], &minor_col[2],
                               &minor_col[3], &minor_mult[0], &minor_mult[1], &minor_mult[2], &minor_mult[3],
                               &pc_rowstart, &pc_rowlen, &pc_big, &pc_counters, &pc_col, &pc_cnt, &pc_gk, &pc_gv, &pc_gocc,
                               &dstar_rowptr, &dstar_col, &dstar_count};
        for (DeviceBuffer* b : all) f(*b);
    }

    int64_t counts[4] = {0, 0, 0, 0};
    int64_t n_junctions = 0;
    int64_t minor_nnz[4] = {0, 0, 0, 0};
    int64_t minor_rows[4] = {0, 0, 0, 0};
    int64_t dstar_nnz = 0;
    // which stages are valid for the current field
    bool have_gradient = false, have_critical = false, have_extremum = false, have_reach = false,
         have_junctions = false, have_minor = false, have_dstar = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, kev0 = nullptr, kev1 = nullptr;  // stage / kernel timing
    // host-side fault injection (MSC_FAULT, read at plan creation; tests only): the failure is
    // made on the host -- a faked allocation failure, or a status bit raised as a kernel would
    int fault_kind = 0;  // 0 none, 1 alloc, 2 timeout (reachability), 3 overflow (path count)
    int64_t fault_at = 0, alloc_calls = 0;
};

// The trace of the DAG minor (minor.cu): for every 1-saddle (ranks 0..n1-1) then every junction
// (n1 + rank), 4 destination ranks, and a 32-bit word whose byte k is the kind of slot k:
// 0 none, 1 a junction, 2 a 2-saddle.
__host__ __device__ __forceinline__ uint32_t trace_kind(uint32_t kinds, int k) { return (kinds >> (8 * k)) & 0xFFu; }

// Counts one kernel launch of this plan (reported in msc_stats.n_launches).
inline void launched(Plan* p, int n = 1) { p->stats.n_launches += n; }

// Buffer helpers (api.cu): grow-only device allocations owned by the plan.
msc_status ensure(Plan* p, DeviceBuffer& b, size_t bytes);
msc_status fail(Plan* p, msc_status st, const std::string& msg);
msc_status check_cuda(Plan* p, cudaError_t e, const char* what);
msc_status check_status_word(Plan* p, cudaStream_t s);  // syncs, reads and clears the status word

// Stage launchers
msc_status run_gradient(Plan* p, const float* d_field, cudaStream_t s);
msc_status run_critical(Plan* p, cudaStream_t s);
msc_status run_extremum(Plan* p, cudaStream_t s);
msc_status run_reachability(Plan* p, cudaStream_t s);
msc_status run_junctions(Plan* p, cudaStream_t s);
msc_status run_minor(Plan* p, cudaStream_t s);
msc_status run_path_count(Plan* p, cudaStream_t s);

}  // namespace msc

// The opaque handle of the C ABI is the plan itself.
struct msc_plan_s : public msc::Plan {};

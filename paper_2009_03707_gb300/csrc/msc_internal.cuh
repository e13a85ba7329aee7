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
    ST_RETRY = 1u << 6,      // a replayed pipeline outgrew a capacity fixed at capture: rerun and re-capture
};

// A count produced earlier in the pass, against the capacity a launch was sized for.  When a count
// outgrows its capacity (possible only in a replayed graph) the pass is rerun, so every kernel
// that depends on counts must then do nothing at all -- ranks stored by earlier kernels may point
// past its buffers.  count_fits raises ST_RETRY and says no; pass_retrying sees an earlier one.
__device__ __forceinline__ bool pass_retrying(const uint32_t* status) {
    return (*reinterpret_cast<const volatile uint32_t*>(status) & ST_RETRY) != 0;
}
__device__ __forceinline__ bool count_fits(uint32_t* status, unsigned long long n, int64_t cap) {
    if (n <= (unsigned long long)cap) return true;
    if (threadIdx.x == 0) atomicOr(status, ST_RETRY);
    return false;
}

// ---- per-pass results the host needs, kept on the device and read back in one copy --------
// Path-count counter slots in Summary::pc.
enum PcCounter { PC_CURSOR = 0, PC_MAX = 1, PC_ITER = 2, PC_ENTRIES = 3, PC_DEFER0 = 4, PC_DEFER1 = 5, PC_NEXT = 6,
                 PC_DEFER2 = 7, PC_DEFER3 = 8, PC_SLOTS = 10 };
struct Summary {
    unsigned long long counts[4];     // critical cells per dimension
    unsigned long long n_junctions;
    unsigned long long reached;       // reachable 1-cells (the 1-saddles included)
    unsigned long long levels;        // non-empty BFS levels (level 0 = the 1-saddles)
    unsigned long long jump_rounds;   // pointer-jumping rounds
    unsigned long long sweep_iters;   // iterations of the reachability loop (two sweeps each)
    unsigned long long minor_nnz[4];  // distinct entries of A, B, B*, D
    unsigned long long pc[10];        // path-count counters (PcCounter)
    unsigned long long dstar_nnz;
    unsigned long long dp_wave_done;      // junction DP: junctions done in the current wave
    unsigned long long dp_pool_used;      // junction DP: J-row pool slots taken
    unsigned long long dp_junctions_done;
    unsigned long long dp_iters;          // iterations of the wave loop
    unsigned long long dp_long_n;         // junction DP: long merges handed to the warp kernel this wave
    unsigned int dp_wave;                 // the current wave
    unsigned int pad2;
    uint32_t loop_flag[4];            // "changed" flags of the iterative stages; [3] = continue (host loops)
    uint32_t status;                  // StatusBit word
    uint32_t pad;
    uint32_t jump_flag[2];            // pointer jumping's own "changed" flag and continue decision: that
                                      // stage runs beside the reachability loop in a replayed pass
    uint32_t pad3[2];
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

    // stage products and scratch (all grow-only, freed by msc_plan_destroy); `status` holds the
    // Summary (status word included)
    DeviceBuffer words, status, crit_bits, crit_prefix, scan_sums;
    DeviceBuffer cells[4];
    DeviceBuffer vmin, cmax, min_arcs, max_arcs, ext_lab_v, ext_lab_c;
    DeviceBuffer visited, reach_tmp, reach_masks, reach_qdown, reach_stamp, node_info;
    DeviceBuffer junc_bits, junc_prefix, junc_cells;
    DeviceBuffer trace, trace_kinds, minor_rowcnt, minor_scan, minor_rowptr[4], minor_col[4], minor_mult[4];
    DeviceBuffer pc_rowstart, pc_rowlen, pc_big, pc_col, pc_cnt, pc_gk, pc_gv, pc_gocc;
    DeviceBuffer dstar_rowptr, dstar_col, dstar_count;
    DeviceBuffer csc_colptr, csc_row, csc_count, csc_work;  // D* by 2-saddle (transpose.cu)
    DeviceBuffer graph_nodeptr, graph_adj, graph_mult, graph_work, graph_none;  // the 1-skeleton (graph.cu)
    DeviceBuffer geo_len, geo_off, geo_scan, geo_cells;  // cells along the saddle-extremum arcs (geometry.cu)
    DeviceBuffer ss_len, ss_off, ss_scan, ss_cells, ss_row;  // cells along the saddle-saddle arcs of count 1 (geometry.cu)
    // simplification (simplify.cu): node cells, values, alive (two copies), keys, per-node scratch,
    // row lengths, log positions, scan scratch, two CSRs, the log, the per-round host read-out
    DeviceBuffer simp_cell, simp_value, simp_alive, simp_keys, simp_node, simp_len, simp_pos, simp_scan;
    DeviceBuffer simp_ptr[2], simp_nbr[2], simp_mult[2], simp_log, simp_round;
    DeviceBuffer dp_pend, dp_in_cnt, dp_in_ptr, dp_in_idx, dp_j_off, dp_j_len, dp_pool_col, dp_pool_cnt, dp_long, dp_chunks;

    template <class F>
    void for_each_buffer(F&& f) {
        DeviceBuffer* all[] = {&words, &status, &crit_bits, &crit_prefix, &scan_sums, &cells[0], &cells[1], &cells[2],
                               &cells[3], &vmin, &cmax, &min_arcs, &max_arcs, &ext_lab_v, &ext_lab_c, &visited, &reach_tmp, &reach_masks,
                               &reach_qdown, &reach_stamp, &node_info, &junc_bits, &junc_prefix, &junc_cells, &trace, &trace_kinds,
                               &minor_rowcnt, &minor_scan, &minor_rowptr[0], &minor_rowptr[1], &minor_rowptr[2],
                               &minor_rowptr[3], &minor_col[0], &minor_col[1], &minor_col[2], &minor_col[3],
                               &minor_mult[0], &minor_mult[1], &minor_mult[2], &minor_mult[3], &pc_rowstart, &pc_rowlen,
                               &pc_big, &pc_col, &pc_cnt, &pc_gk, &pc_gv, &pc_gocc, &dstar_rowptr, &dstar_col,
                               &dstar_count, &dp_pend, &dp_in_cnt, &dp_in_ptr, &dp_in_idx, &dp_j_off,
                               &dp_j_len, &dp_pool_col, &dp_pool_cnt, &dp_long, &dp_chunks, &csc_colptr, &csc_row, &csc_count, &csc_work,
                               &graph_nodeptr, &graph_adj, &graph_mult, &graph_work, &graph_none,
                               &geo_len, &geo_off, &geo_scan, &geo_cells, &ss_len, &ss_off, &ss_scan, &ss_cells, &ss_row,
                               &simp_cell, &simp_value,
                               &simp_alive, &simp_keys, &simp_node, &simp_len, &simp_pos, &simp_scan,
                               &simp_ptr[0], &simp_ptr[1], &simp_nbr[0], &simp_nbr[1], &simp_mult[0],
                               &simp_mult[1], &simp_log, &simp_round};
        for (DeviceBuffer* b : all) f(*b);
    }

    Summary* dsum() const { return static_cast<Summary*>(status.ptr); }
    uint32_t* status_word() const { return &dsum()->status; }

    // Capacities of the count-dependent buffers, fixed when a pipeline graph is captured (from the
    // exact sizes of the last run with host synchronisation, plus headroom).  Kernels clamp to them
    // and raise ST_RETRY when a replay needs more.
    struct Caps {
        int64_t cells[4] = {0, 0, 0, 0};
        int64_t nj = 0;
        int64_t staging = 0;
        int64_t dp_pool = 0;
    } caps;
    bool capturing = false;          // enqueueing into a graph: no host synchronisation allowed
    cudaStream_t cap_stream = nullptr, body_stream = nullptr;  // private capture streams
    cudaStream_t side_stream = nullptr;                        // the extremum branch of a captured pass
    cudaStream_t side_body_stream = nullptr;                   // its loop body
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    const float* graph_field = nullptr;
    int64_t graph_static_launches = 0;  // kernels per replay outside the loops
    int64_t loop_body_launches[3] = {0, 0, 0};  // per iteration: pointer jumping, reachability, DP waves
    Summary* hsum = nullptr;          // pinned host mirror of the summary
    cudaEvent_t stage_ev[12] = {};    // start and end of stages 0..5 (read by msc_get_stats)
    uint32_t stage_recorded = 0;      // stages whose two events belong to the same pass
    bool caps_ready = false;          // a synchronised run has measured the sizes
    int64_t graph_replays = 0;
    int64_t capture_epoch = 0;        // bumped whenever the plan's graph is captured or dropped
    int grad_variant = -1;            // gradient tile variant (-1: not tuned yet)

    int64_t counts[4] = {0, 0, 0, 0};
    int64_t n_junctions = 0;
    int64_t minor_nnz[4] = {0, 0, 0, 0};
    int64_t minor_rows[4] = {0, 0, 0, 0};
    int64_t dstar_nnz = 0;
    int64_t pc_staging_cap = 0;  // staging slots of the last path-count run
    int64_t dp_pool_cap = 0;     // J-row pool slots of the last junction-DP run
    int pc_method_chosen = 0;    // path-count method once the first run has measured the minor (1, 2)
    int pc_method_used = 0;      // the method of the last run
    // which stages are valid for the current field
    bool have_gradient = false, have_critical = false, have_extremum = false, have_reach = false,
         have_junctions = false, have_trace = false, have_minor = false, have_dstar = false,
         have_dstar_csc = false, have_graph = false, have_geometry = false, have_ss_geometry = false,
         have_j = false;  // the junction-DP rows J of the current field (junction_dp.cu), whichever method ran
    int64_t ss_cells_n = 0;  // cells along all saddle-saddle arcs of count 1 (geometry.cu)
    int64_t graph_nodes = 0, graph_nadj = 0;
    int64_t geo_cells_n = 0;  // cells along all arcs (geometry.cu)
    // the last simplification (simplify.cu): which CSR copy holds it, its size, rounds, cancellations
    int simp_cur = 0;
    int64_t simp_nnz = 0, simp_rounds = 0, simp_cancelled = 0;
    cudaEvent_t kev0 = nullptr, kev1 = nullptr;  // around the tier-0 path-count kernel
    cudaEvent_t tev0 = nullptr, tev1 = nullptr;  // around the trace kernel
    cudaEvent_t gev0 = nullptr, gev1 = nullptr;  // around the lower-star kernel
    // a pass launched by msc_compute_async and not yet waited for: its summary copy ends at pend_ev
    cudaEvent_t pend_ev = nullptr;
    bool pending = false;
    const float* pending_field = nullptr;
    cudaStream_t pending_stream = nullptr;
    // host-side fault injection (MSC_FAULT, read at plan creation; tests only): the failure is
    // made on the host -- a faked allocation failure, or a status bit raised as a kernel would
    int fault_kind = 0;  // 0 none, 1 alloc, 2 timeout (reachability), 3 overflow (path count)
    int64_t fault_at = 0, alloc_calls = 0;
};

// The trace of the DAG minor (minor.cu): for every 1-saddle (ranks 0..n1-1) then every junction
// (n1 + rank), 4 destination ranks, and a 32-bit word whose byte k is the kind of slot k:
// 0 none, 1 a junction, 2 a 2-saddle.
__host__ __device__ __forceinline__ uint32_t trace_kind(uint32_t kinds, int k) { return (kinds >> (8 * k)) & 0xFFu; }

// Records a timing event on s; inside a capture it must be an external event-record node (a plain
// record there only orders captured work and is never recorded when the graph runs).
inline void record_event(const Plan* p, cudaEvent_t ev, cudaStream_t s) {
    if (!ev) return;  // a timing deliberately not taken
    if (p->capturing) cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else cudaEventRecord(ev, s);
}

// Counts one kernel launch of this plan (reported in msc_stats.n_launches).
inline void launched(Plan* p, int n = 1) { p->stats.n_launches += n; }

// Runs an iterative stage: body(stream, handle) enqueues one iteration and must end with a
// kernel that stores the continue decision in summary.loop_flag[3] (jump_flag[1] for pointer
// jumping, which = 0) and, when the handle is non-zero, sets the graph condition to it.  Host
// synchronised: a loop that reads the flag after every iteration.  Capturing: a conditional WHILE node whose body graph is captured from one
// call of body, so the loop runs on the device with no host round trip.
msc_status run_loop(Plan* p, cudaStream_t s, int which, int body_launches,
                    void (*body)(Plan*, cudaStream_t, cudaGraphConditionalHandle, void*), void* ctx);

// Buffer helpers (api.cu): grow-only device allocations owned by the plan.
msc_status ensure(Plan* p, DeviceBuffer& b, size_t bytes);
msc_status fail(Plan* p, msc_status st, const std::string& msg);
msc_status check_cuda(Plan* p, cudaError_t e, const char* what);
msc_status check_status_word(Plan* p, cudaStream_t s);  // syncs, reads and clears the status word
msc_status status_error(Plan* p, uint32_t word);        // the error a non-zero status word stands for

// Pipeline graphs (api.cu).  enqueue_pipeline issues every stage without host synchronisation
// (p->capturing set), the saddle-extremum stage on a branch of its own if `branch`; capture_graph
// records the plan's own graph; finish_replay takes a replay's
// summary (already in p->hsum): MSC_OK, MSC_NOT_READY (rerun synchronised) or the error;
// compute_synchronised runs a pass with host synchronisation and sets the capacities.
msc_status enqueue_pipeline(Plan* p, const float* d_field, cudaStream_t s, bool branch);
msc_status capture_graph(Plan* p, const float* d_field);
void destroy_graph(Plan* p);
msc_status finish_replay(Plan* p, cudaStream_t s);
msc_status compute_synchronised(Plan* p, const float* d_field, cudaStream_t s);
msc_status bind_device(Plan* p);
void invalidate(Plan* p);
inline bool graphs_enabled(const Plan* p) { return !(p->opts.flags & MSC_FLAG_NO_GRAPH) && p->fault_kind == 0; }
msc_status read_summary(Plan* p, cudaStream_t s);       // syncs; copies the summary to p->hsum

// Stage launchers
msc_status run_gradient(Plan* p, const float* d_field, cudaStream_t s);
msc_status run_critical(Plan* p, cudaStream_t s);
msc_status run_extremum(Plan* p, cudaStream_t s);
msc_status run_reachability(Plan* p, cudaStream_t s);
msc_status run_junctions(Plan* p, cudaStream_t s);
msc_status run_trace(Plan* p, cudaStream_t s);      // the minor's 4-slot trace (pipeline)
msc_status build_minor_csr(Plan* p, cudaStream_t s);  // CSR of A, B, B*, D (on request; syncs)
msc_status run_path_count(Plan* p, cudaStream_t s);
msc_status build_dstar_csc(Plan* p, cudaStream_t s);  // D* by 2-saddle (on request; syncs)
msc_status build_complex_graph(Plan* p, cudaStream_t s);  // the 1-skeleton adjacency (on request; syncs)
msc_status build_arc_geometry(Plan* p, cudaStream_t s);   // cells along the saddle-extremum arcs (on request; syncs)
msc_status build_ss_geometry(Plan* p, cudaStream_t s);    // cells along the saddle-saddle arcs of count 1 (needs J; syncs)
msc_status run_simplify(Plan* p, const float* d_field, double threshold, cudaStream_t s);  // (on request; syncs)
msc_status run_junction_dp(Plan* p, cudaStream_t s, uint64_t pool_cap, uint64_t out_cap);
int grid_cap(const Plan* p, int64_t threads, int block, int per_sm = 8);  // grid for a count-bounded loop

}  // namespace msc

// The opaque handle of the C ABI is the plan itself.
struct msc_plan_s : public msc::Plan {};

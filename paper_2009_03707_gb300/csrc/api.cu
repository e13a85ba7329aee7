// C ABI of libmsc (declared in include/msc.h): plans, device buffers, status reporting and
// the stage entry points.  Every stage's arithmetic runs in the kernels of the other
// translation units; this file only orders the launches and manages memory.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "msc_internal.cuh"
#include "scan.cuh"

namespace msc {

msc_status fail(Plan* p, msc_status st, const std::string& msg) {
    if (p) p->last_error = msg;
    return st;
}

msc_status check_cuda(Plan* p, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MSC_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(p, MSC_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    }
    return fail(p, MSC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

msc_status ensure(Plan* p, DeviceBuffer& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.ptr && b.bytes >= bytes) return MSC_OK;
    if (p->fault_kind == 1 && ++p->alloc_calls == p->fault_at)
        return fail(p, MSC_ERR_OOM, "injected allocation failure (MSC_FAULT)");
    if (b.ptr) {
        cudaFree(b.ptr);
        p->live_bytes -= int64_t(b.bytes);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    // grow with headroom so that repeated runs on similar fields do not reallocate
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&b.ptr, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        return fail(p, MSC_ERR_OOM, "device allocation of " + std::to_string(want) + " bytes failed");
    }
    b.bytes = want;
    p->live_bytes += int64_t(want);
    if (p->live_bytes > p->peak_bytes) p->peak_bytes = p->live_bytes;
    return MSC_OK;
}

msc_status check_status_word(Plan* p, cudaStream_t s) {
    uint32_t word = 0;
    msc_status st;
    if ((st = check_cuda(p, cudaMemcpyAsync(&word, p->status.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s),
                         "status copy")))
        return st;
    if ((st = check_cuda(p, cudaStreamSynchronize(s), "stream sync"))) return st;
    if (word == 0) return MSC_OK;
    if ((st = check_cuda(p, cudaMemsetAsync(p->status.ptr, 0, sizeof(uint32_t), s), "status clear"))) return st;
    if (word & ST_NAN) return fail(p, MSC_ERR_NAN, "the field holds a NaN");
    if (word & ST_OVERFLOW) return fail(p, MSC_ERR_OVERFLOW, "a saddle-saddle path count exceeds 2^64-1");
    if (word & ST_ITER) return fail(p, MSC_ERR_ITER_LIMIT, "an iterative stage reached its iteration cap");
    if (word & ST_TIMEOUT) return fail(p, MSC_ERR_TIMEOUT, "a bounded device wait gave up");
    if (word & ST_CAPACITY) return fail(p, MSC_ERR_CUDA, "internal: a device buffer was too small");
    return fail(p, MSC_ERR_CUDA, "internal: a device-side bounds check failed");
}

namespace {

// MSC_FAULT = alloc@k | timeout | overflow: host-side fault injection for tests.
void read_fault(Plan* p) {
    const char* f = std::getenv("MSC_FAULT");
    if (!f) return;
    if (!std::strncmp(f, "alloc@", 6)) {
        p->fault_kind = 1;
        p->fault_at = std::atoll(f + 6);
    } else if (!std::strcmp(f, "timeout")) {
        p->fault_kind = 2;
    } else if (!std::strcmp(f, "overflow")) {
        p->fault_kind = 3;
    }
}

// Raises a status bit on the device exactly as a kernel would (for injected faults).
void raise_status(Plan* p, uint32_t bit, cudaStream_t s) {
    uint32_t word = bit;
    cudaMemcpyAsync(p->status.ptr, &word, sizeof(word), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
}

struct StageTimer {
    Plan* p;
    cudaStream_t s;
    float* out;
    StageTimer(Plan* plan, cudaStream_t stream, float* dst) : p(plan), s(stream), out(dst) {
        cudaEventRecord(p->ev0, s);
    }
    void stop() {
        cudaEventRecord(p->ev1, s);
        if (cudaEventSynchronize(p->ev1) == cudaSuccess) cudaEventElapsedTime(out, p->ev0, p->ev1);
    }
};

msc_status bind_device(Plan* p) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(p, MSC_ERR_CUDA, "cudaGetDevice failed");
    if (cur != p->device) return check_cuda(p, cudaSetDevice(p->device), "cudaSetDevice");
    return MSC_OK;
}

void invalidate(Plan* p) {
    p->have_gradient = p->have_critical = p->have_extremum = p->have_reach = false;
    p->have_junctions = p->have_minor = p->have_dstar = false;
}

}  // namespace

msc_status run_critical(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    if ((st = ensure(p, p->crit_prefix, sizeof(uint32_t) * size_t(g.slot_words())))) return st;
    CritSource src{};
    src.g = g;
    src.bits = static_cast<const uint32_t*>(p->crit_bits.ptr);
    src.prefix = static_cast<uint32_t*>(p->crit_prefix.ptr);
    src.status = static_cast<uint32_t*>(p->status.ptr);
    unsigned long long tot[4] = {0, 0, 0, 0};
    if ((st = compaction_count(p, s, src, 4, tot))) return st;
    for (int k = 0; k < 4; ++k) {
        p->counts[k] = int64_t(tot[k]);
        if ((st = ensure(p, p->cells[k], sizeof(uint32_t) * size_t(tot[k] ? tot[k] : 1)))) return st;
        src.out[k] = static_cast<uint32_t*>(p->cells[k].ptr);
        src.cap[k] = tot[k];
    }
    return compaction_emit(p, s, src, 4);
}

}  // namespace msc

using msc::Plan;

// =========================================================================================
extern "C" {

msc_status msc_plan(const int64_t dims[3], const msc_opts* opts, msc_plan_t* out) {
    if (!dims || !out) return MSC_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < 3; ++i)
        if (dims[i] < 2 || dims[i] > (int64_t(1) << 30)) return MSC_ERR_ARG;
    const int64_t rx = 2 * dims[0] - 1, ry = 2 * dims[1] - 1, rz = 2 * dims[2] - 1;
    if (rx * ry > (int64_t(1) << 40) || double(rx) * double(ry) * double(rz) >= 4294967295.0) return MSC_ERR_TOO_LARGE;
    if (opts && opts->flags != 0) return MSC_ERR_ARG;
    msc_plan_s* p = new (std::nothrow) msc_plan_s();
    if (!p) return MSC_ERR_OOM;
    p->g.nx = int(dims[0]);
    p->g.ny = int(dims[1]);
    p->g.nz = int(dims[2]);
    p->g.finish();
    if (opts) p->opts = *opts;
    if (p->opts.max_iterations <= 0) p->opts.max_iterations = int64_t(1) << 20;
    msc::read_fault(p);
    msc_status st = msc::check_cuda(p, cudaGetDevice(&p->device), "cudaGetDevice");
    if (!st) st = msc::check_cuda(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device),
                                  "cudaDeviceGetAttribute");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->ev0), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->ev1), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->kev0), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->kev1), "cudaEventCreate");
    if (!st) st = msc::ensure(p, p->status, sizeof(uint32_t) * 4);
    if (!st) st = msc::check_cuda(p, cudaMemset(p->status.ptr, 0, sizeof(uint32_t) * 4), "cudaMemset(status)");
    if (st) {
        msc_plan_destroy(p);
        return st;
    }
    *out = p;
    return MSC_OK;
}

msc_status msc_plan_destroy(msc_plan_t plan) {
    if (!plan) return MSC_ERR_ARG;
    msc_plan_s* p = plan;
    p->for_each_buffer([](msc::DeviceBuffer& b) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    });
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->kev0) cudaEventDestroy(p->kev0);
    if (p->kev1) cudaEventDestroy(p->kev1);
    delete p;
    return MSC_OK;
}

const char* msc_last_error_string(msc_plan_t plan) {
    if (!plan) return "null plan";
    return plan->last_error.c_str();
}

msc_status msc_gradient(msc_plan_t plan, const float* d_field, msc_stream_t stream) {
    if (!plan || !d_field) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    msc::invalidate(p);
    p->stats.n_launches = 0;
    msc::StageTimer tm(p, s, &p->stats.ms_gradient);
    if ((st = msc::run_gradient(p, d_field, s))) return st;
    cudaEventRecord(p->ev1, s);  // stage time is read when the next stage synchronises
    p->have_gradient = true;
    return MSC_OK;
}

msc_status msc_gradient_words(msc_plan_t plan, const uint32_t** d_words) {
    if (!plan || !d_words) return MSC_ERR_ARG;
    if (!plan->have_gradient) return msc::fail(plan, MSC_ERR_STATE, "msc_gradient has not run");
    *d_words = static_cast<const uint32_t*>(plan->words.ptr);
    return MSC_OK;
}

static msc_status ensure_critical(Plan* p, cudaStream_t s) {
    if (!p->have_gradient) return msc::fail(p, MSC_ERR_STATE, "msc_gradient has not run");
    if (p->have_critical) return MSC_OK;
    msc_status st;
    // gradient time: ev0 was recorded before the gradient launch, ev1 after it
    if (cudaEventSynchronize(p->ev1) == cudaSuccess) cudaEventElapsedTime(&p->stats.ms_gradient, p->ev0, p->ev1);
    if ((st = msc::check_status_word(p, s))) return st;
    msc::StageTimer tm(p, s, &p->stats.ms_critical);
    if ((st = msc::run_critical(p, s))) return st;
    tm.stop();
    if ((st = msc::check_status_word(p, s))) return st;
    for (int k = 0; k < 4; ++k) p->stats.counts[k] = p->counts[k];
    p->have_critical = true;
    return MSC_OK;
}

msc_status msc_critical(msc_plan_t plan, msc_stream_t stream, int64_t counts[4], const uint32_t* d_cells[4]) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_critical(p, s))) return st;
    for (int k = 0; k < 4; ++k) {
        if (counts) counts[k] = p->counts[k];
        if (d_cells) d_cells[k] = static_cast<const uint32_t*>(p->cells[k].ptr);
    }
    return MSC_OK;
}

static msc_status ensure_extremum(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_critical(p, s))) return st;
    if (p->have_extremum) return MSC_OK;
    msc::StageTimer tm(p, s, &p->stats.ms_extremum);
    if ((st = msc::run_extremum(p, s))) return st;
    tm.stop();
    if ((st = msc::check_status_word(p, s))) return st;
    p->have_extremum = true;
    return MSC_OK;
}

msc_status msc_extremum_arcs(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_min_arcs,
                             const uint32_t** d_max_arcs, const uint32_t** d_vertex_min_label,
                             const uint32_t** d_cube_max_label) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_extremum(p, s))) return st;
    if (d_min_arcs) *d_min_arcs = static_cast<const uint32_t*>(p->min_arcs.ptr);
    if (d_max_arcs) *d_max_arcs = static_cast<const uint32_t*>(p->max_arcs.ptr);
    if (d_vertex_min_label) *d_vertex_min_label = static_cast<const uint32_t*>(p->vmin.ptr);
    if (d_cube_max_label) *d_cube_max_label = static_cast<const uint32_t*>(p->cmax.ptr);
    return MSC_OK;
}

static msc_status ensure_reach(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_critical(p, s))) return st;
    if (p->have_reach) return MSC_OK;
    msc::StageTimer tm(p, s, &p->stats.ms_reachability);
    if ((st = msc::run_reachability(p, s))) return st;
    tm.stop();
    if (p->fault_kind == 2) msc::raise_status(p, msc::ST_TIMEOUT, s);
    if ((st = msc::check_status_word(p, s))) return st;
    p->have_reach = true;
    return MSC_OK;
}

msc_status msc_reachability(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_visited, int64_t* n_words,
                            int64_t* n_levels) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_reach(p, s))) return st;
    if (d_visited) *d_visited = static_cast<const uint32_t*>(p->visited.ptr);
    if (n_words) *n_words = p->g.edge_words();
    if (n_levels) *n_levels = p->stats.n_bfs_levels;
    return MSC_OK;
}

static msc_status ensure_junctions(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_reach(p, s))) return st;
    if (p->have_junctions) return MSC_OK;
    float ms = 0;
    msc::StageTimer tm(p, s, &ms);
    if ((st = msc::run_junctions(p, s))) return st;
    tm.stop();
    p->stats.ms_minor = ms;
    if ((st = msc::check_status_word(p, s))) return st;
    p->have_junctions = true;
    return MSC_OK;
}

msc_status msc_junctions(msc_plan_t plan, msc_stream_t stream, const uint32_t** d_cells, int64_t* n) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_junctions(p, s))) return st;
    if (d_cells) *d_cells = static_cast<const uint32_t*>(p->junc_cells.ptr);
    if (n) *n = p->n_junctions;
    return MSC_OK;
}

static msc_status ensure_minor(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_junctions(p, s))) return st;
    if (p->have_minor) return MSC_OK;
    float ms = 0;
    msc::StageTimer tm(p, s, &ms);
    if ((st = msc::run_minor(p, s))) return st;
    tm.stop();
    p->stats.ms_minor += ms;
    if ((st = msc::check_status_word(p, s))) return st;
    p->have_minor = true;
    return MSC_OK;
}

msc_status msc_minor(msc_plan_t plan, msc_stream_t stream, int which, int64_t* rows, int64_t* nnz,
                     const int64_t** d_rowptr, const uint32_t** d_col, const uint32_t** d_mult) {
    if (!plan || which < 0 || which > 3) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_minor(p, s))) return st;
    if (rows) *rows = p->minor_rows[which];
    if (nnz) *nnz = p->minor_nnz[which];
    if (d_rowptr) *d_rowptr = static_cast<const int64_t*>(p->minor_rowptr[which].ptr);
    if (d_col) *d_col = static_cast<const uint32_t*>(p->minor_col[which].ptr);
    if (d_mult) *d_mult = static_cast<const uint32_t*>(p->minor_mult[which].ptr);
    return MSC_OK;
}

static msc_status ensure_dstar(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_minor(p, s))) return st;
    if (p->have_dstar) return MSC_OK;
    msc::StageTimer tm(p, s, &p->stats.ms_path_count);
    if ((st = msc::run_path_count(p, s))) return st;
    tm.stop();
    if (p->fault_kind == 3) msc::raise_status(p, msc::ST_OVERFLOW, s);
    if ((st = msc::check_status_word(p, s))) return st;
    p->have_dstar = true;
    return MSC_OK;
}

msc_status msc_saddle_arcs(msc_plan_t plan, msc_stream_t stream, int64_t* nnz, const int64_t** d_rowptr,
                           const uint32_t** d_col, const uint64_t** d_count) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_dstar(p, s))) return st;
    if (nnz) *nnz = p->dstar_nnz;
    if (d_rowptr) *d_rowptr = static_cast<const int64_t*>(p->dstar_rowptr.ptr);
    if (d_col) *d_col = static_cast<const uint32_t*>(p->dstar_col.ptr);
    if (d_count) *d_count = static_cast<const uint64_t*>(p->dstar_count.ptr);
    return MSC_OK;
}

msc_status msc_compute(msc_plan_t plan, const float* d_field, msc_stream_t stream) {
    if (!plan || !d_field) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc_gradient(plan, d_field, stream))) return st;
    if ((st = ensure_extremum(p, s))) return st;
    return ensure_dstar(p, s);
}

msc_status msc_get_stats(msc_plan_t plan, msc_stats* out) {
    if (!plan || !out) return MSC_ERR_ARG;
    plan->stats.peak_device_bytes = plan->peak_bytes;
    *out = plan->stats;
    return MSC_OK;
}

}  // extern "C"

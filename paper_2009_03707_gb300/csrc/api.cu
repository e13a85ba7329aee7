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

msc_status status_error(Plan* p, uint32_t word) {
    if (word & ST_NAN) return fail(p, MSC_ERR_NAN, "the field holds a NaN");
    if (word & ST_OVERFLOW) return fail(p, MSC_ERR_OVERFLOW, "a saddle-saddle path count exceeds 2^64-1");
    if (word & ST_ITER) return fail(p, MSC_ERR_ITER_LIMIT, "an iterative stage reached its iteration cap");
    if (word & ST_TIMEOUT) return fail(p, MSC_ERR_TIMEOUT, "a bounded device wait gave up");
    if (word & (ST_CAPACITY | ST_RETRY)) return fail(p, MSC_ERR_INTERNAL, "internal: a device buffer was too small");
    return fail(p, MSC_ERR_INTERNAL, "internal: a device-side invariant or bounds check failed");
}

msc_status check_status_word(Plan* p, cudaStream_t s) {
    uint32_t word = 0;
    msc_status st;
    if ((st = check_cuda(p, cudaMemcpyAsync(&word, p->status_word(), sizeof(uint32_t), cudaMemcpyDeviceToHost, s),
                         "status copy")))
        return st;
    if ((st = check_cuda(p, cudaStreamSynchronize(s), "stream sync"))) return st;
    if (word == 0) return MSC_OK;
    if ((st = check_cuda(p, cudaMemsetAsync(p->status_word(), 0, sizeof(uint32_t), s), "status clear"))) return st;
    return status_error(p, word);
}

msc_status read_summary(Plan* p, cudaStream_t s) {
    if (p->capturing) return fail(p, MSC_ERR_CUDA, "internal: host read during graph capture");
    msc_status st;
    if ((st = check_cuda(p, cudaMemcpyAsync(p->hsum, p->dsum(), sizeof(Summary), cudaMemcpyDeviceToHost, s),
                         "summary copy")))
        return st;
    return check_cuda(p, cudaStreamSynchronize(s), "stream sync");
}

__global__ void loop_arm(cudaGraphConditionalHandle h) { cudaGraphSetConditional(h, 1u); }

int grid_cap(const Plan* p, int64_t threads, int block, int per_sm) {
    const int64_t want = (threads + block - 1) / block;
    const int64_t cap = int64_t(p->num_sms > 0 ? p->num_sms : 148) * per_sm;
    return int(std::max<int64_t>(1, std::min(want, cap)));
}

msc_status run_loop(Plan* p, cudaStream_t s, int which, int body_launches,
                    void (*body)(Plan*, cudaStream_t, cudaGraphConditionalHandle, void*), void* ctx) {
    msc_status st;
    if (!p->capturing) {
        for (;;) {
            body(p, s, 0, ctx);
            launched(p, body_launches);
            uint32_t more = 0;
            if ((st = check_cuda(p, cudaGetLastError(), "loop launch"))) return st;
            const uint32_t* cont = which == 0 ? &p->dsum()->jump_flag[1] : &p->dsum()->loop_flag[3];
            if ((st = check_cuda(p, cudaMemcpyAsync(&more, cont, sizeof(more),
                                                    cudaMemcpyDeviceToHost, s),
                                 "loop flag copy")))
                return st;
            if ((st = check_cuda(p, cudaStreamSynchronize(s), "loop sync"))) return st;
            if (!more) return MSC_OK;  // the decision kernel also stops at the iteration cap
        }
    }
    // capturing: a conditional WHILE node after the work captured so far, its body captured on
    // the plan's second private stream.  The condition defaults to 0 at every launch and a
    // one-thread kernel just before the node sets it to 1: should the device-side setting ever
    // not take effect, the loop runs zero times (a wrong result the checks see), never forever.
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edata = nullptr;
    size_t nd = 0;
    if ((st = check_cuda(p, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edata, &nd), "capture info")))
        return st;
    cudaGraphConditionalHandle h;
    if ((st = check_cuda(p, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault), "conditional handle")))
        return st;
    loop_arm<<<1, 1, 0, s>>>(h);
    launched(p);
    if ((st = check_cuda(p, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edata, &nd), "capture info")))
        return st;
    std::vector<cudaGraphNode_t> dep(deps, deps + nd);
    std::vector<cudaGraphEdgeData> edge;
    if (edata) edge.assign(edata, edata + nd);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((st = check_cuda(p, cudaGraphAddNode(&node, g, dep.data(), edata ? edge.data() : nullptr, nd, &np),
                         "conditional node")))
        return st;
    cudaGraph_t body_graph = np.conditional.phGraph_out[0];
    cudaStream_t bs = s == p->side_stream ? p->side_body_stream : p->body_stream;  // the branch's priority
    if ((st = check_cuda(p, cudaStreamBeginCaptureToGraph(bs, body_graph, nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeRelaxed),
                         "body capture")))
        return st;
    body(p, bs, h, ctx);
    const cudaError_t e = cudaStreamEndCapture(bs, &body_graph);
    if ((st = check_cuda(p, e, "body capture end"))) return st;
    p->loop_body_launches[which] = body_launches;
    return check_cuda(p, cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                      "capture dependencies");
}

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
    cudaMemcpyAsync(p->status_word(), &word, sizeof(word), cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
}

// Stage k's device time is read from events recorded at its start and end, when the host next
// waits (msc_get_stats); recording costs nothing on the stream, and works inside a graph.
void stage_start(Plan* p, int k, cudaStream_t s) {
    record_event(p, p->stage_ev[2 * k], s);
    p->stage_recorded &= ~(1u << k);
}
void stage_end(Plan* p, int k, cudaStream_t s) {
    record_event(p, p->stage_ev[2 * k + 1], s);
    p->stage_recorded |= 1u << k;
}

msc_status settle(Plan* p);

// Every entry point starts here: the plan's device is made current, and a pass left in flight by
// msc_compute_async is waited for (its status is what this call returns if it failed).
msc_status bind_device(Plan* p) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return fail(p, MSC_ERR_CUDA, "cudaGetDevice failed");
    if (cur != p->device) {
        const msc_status st = check_cuda(p, cudaSetDevice(p->device), "cudaSetDevice");
        if (st) return st;
    }
    return p->pending ? settle(p) : MSC_OK;
}

void invalidate(Plan* p) {
    p->have_gradient = p->have_critical = p->have_extremum = p->have_reach = false;
    p->have_junctions = p->have_trace = p->have_minor = p->have_dstar = p->have_dstar_csc = p->have_graph = false;
    p->have_geometry = p->have_ss_geometry = p->have_j = false;
}

// Host mirrors and statistics from the summary last copied to p->hsum.
void absorb_summary(Plan* p) {
    const Summary& h = *p->hsum;
    for (int k = 0; k < 4; ++k) p->stats.counts[k] = p->counts[k] = int64_t(h.counts[k]);
    p->stats.n_junctions = p->n_junctions = int64_t(h.n_junctions);
    p->stats.n_reachable = int64_t(h.reached);
    p->stats.n_bfs_levels = int64_t(h.levels);
    p->stats.n_pointer_jumps = int64_t(h.jump_rounds);
    p->stats.nnz_A = int64_t(h.minor_nnz[0]);
    p->stats.nnz_B = int64_t(h.minor_nnz[1]);
    p->stats.nnz_Bstar = int64_t(h.minor_nnz[2]);
    p->stats.nnz_D = int64_t(h.minor_nnz[3]);
    p->stats.nnz_Dstar = p->dstar_nnz = int64_t(h.dstar_nnz);
    p->stats.max_path_count = h.pc[PC_MAX];
    p->stats.n_iter = int64_t(h.pc[PC_ITER]);
    p->stats.n_frontier_entries = int64_t(p->pc_method_used == 2 ? h.dp_pool_used : h.pc[PC_ENTRIES]);
    p->stats.path_count_method = p->pc_method_used;
}

// End of a stage run with host synchronisation: the summary, then its status word.
msc_status finish_stage(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = read_summary(p, s))) return st;
    const uint32_t word = p->hsum->status;
    if (word) {
        if ((st = check_cuda(p, cudaMemsetAsync(p->status_word(), 0, sizeof(uint32_t), s), "status clear"))) return st;
        return status_error(p, word);
    }
    absorb_summary(p);
    return MSC_OK;
}

msc_status run_critical(Plan* p, cudaStream_t s) {
    const Geom& g = p->g;
    msc_status st;
    if ((st = ensure(p, p->crit_prefix, sizeof(uint32_t) * size_t(g.slot_words())))) return st;
    CritSource src{};
    src.g = g;
    src.bits = static_cast<const uint32_t*>(p->crit_bits.ptr);
    src.prefix = static_cast<uint32_t*>(p->crit_prefix.ptr);
    src.status = p->status_word();
    if ((st = compaction_sums(p, s, src, 4, p->dsum()->counts))) return st;
    int64_t cap[4];
    if (p->capturing) {
        for (int k = 0; k < 4; ++k) cap[k] = p->caps.cells[k];
    } else {  // size the lists exactly
        if ((st = read_summary(p, s))) return st;
        for (int k = 0; k < 4; ++k) cap[k] = p->counts[k] = int64_t(p->hsum->counts[k]);
    }
    for (int k = 0; k < 4; ++k) {
        if ((st = ensure(p, p->cells[k], sizeof(uint32_t) * size_t(cap[k] ? cap[k] : 1)))) return st;
        src.out[k] = static_cast<uint32_t*>(p->cells[k].ptr);
        src.cap[k] = uint64_t(cap[k]);
    }
    return compaction_emit(p, s, src, 4);
}

// Every stage, enqueued without host synchronisation (the body of a captured graph).  The
// saddle-extremum stage needs only the gradient and the critical cells, and no later stage reads
// what it writes.  With `branch` it is a branch of its own, captured at the lowest stream
// priority beside the critical path (reachability, the minor and the path counts, whose
// latency-bound kernels leave room on the device), so it fills what they leave free.  The two
// branches share no buffer and no summary word but the status bits, which every kernel sets
// atomically.
msc_status enqueue_pipeline(Plan* p, const float* d_field, cudaStream_t s, bool branch) {
    msc_status st;
    if ((st = check_cuda(p, cudaMemsetAsync(p->dsum(), 0, sizeof(Summary), s), "summary clear"))) return st;
    stage_start(p, 0, s);
    if ((st = run_gradient(p, d_field, s))) return st;
    stage_end(p, 0, s);
    stage_start(p, 1, s);
    if ((st = run_critical(p, s))) return st;
    stage_end(p, 1, s);
    cudaStream_t side = s;
    if (branch) {
        side = p->side_stream;
        if ((st = check_cuda(p, cudaEventRecord(p->fork_ev, s), "fork")) ||
            (st = check_cuda(p, cudaStreamWaitEvent(side, p->fork_ev, 0), "fork")))
            return st;
    }
    stage_start(p, 2, side);
    if ((st = run_extremum(p, side))) return st;
    stage_end(p, 2, side);
    if (branch && (st = check_cuda(p, cudaEventRecord(p->join_ev, side), "join"))) return st;
    stage_start(p, 3, s);
    if ((st = run_reachability(p, s))) return st;
    stage_end(p, 3, s);
    stage_start(p, 4, s);
    if ((st = run_junctions(p, s))) return st;
    if ((st = run_trace(p, s))) return st;
    stage_end(p, 4, s);
    stage_start(p, 5, s);
    if ((st = run_path_count(p, s))) return st;
    stage_end(p, 5, s);
    return branch ? check_cuda(p, cudaStreamWaitEvent(s, p->join_ev, 0), "join") : MSC_OK;
}

void destroy_graph(Plan* p) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
    p->graph_field = nullptr;
    ++p->capture_epoch;
}

// Captures the pipeline for d_field.  The first capture only sizes the buffers for the
// capacities (a buffer that grows is reallocated, which must not happen between captured nodes)
// and is discarded; the second records the graph that is replayed.
msc_status capture_graph(Plan* p, const float* d_field) {
    destroy_graph(p);
    msc_status st = MSC_OK;
    const bool branch = !(p->opts.flags & MSC_FLAG_SERIAL_PASS);
    for (int pass = 0; pass < 2; ++pass) {
        p->capturing = true;
        p->stats.n_launches = 0;
        cudaError_t e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) st = enqueue_pipeline(p, d_field, p->cap_stream, branch);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(p->cap_stream, &g) : e;
        p->capturing = false;
        if (!st && e != cudaSuccess) st = check_cuda(p, e, "begin capture");
        if (!st && e2 != cudaSuccess) st = check_cuda(p, e2, "end capture");
        if (st) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st;
        }
        if (pass == 0) {
            cudaGraphDestroy(g);
            continue;
        }
        p->graph = g;
        p->graph_static_launches = p->stats.n_launches;
        if ((st = check_cuda(p, cudaGraphInstantiate(&p->graph_exec, g, branch ? cudaGraphInstantiateFlagUseNodePriority : 0), "graph instantiate"))) {
            destroy_graph(p);
            return st;
        }
    }
    p->graph_field = d_field;
    ++p->capture_epoch;
    return MSC_OK;
}

// Waits for the pass msc_compute_async launched and publishes it; a replay that outgrew the
// graph's capacities is run again synchronised, as msc_compute does.
msc_status compute_synchronised(Plan* p, const float* d_field, cudaStream_t s);
msc_status settle(Plan* p) {
    p->pending = false;
    msc_status st = check_cuda(p, cudaEventSynchronize(p->pend_ev), "wait for the pass");
    if (st) return st;
    st = finish_replay(p, p->pending_stream);
    if (st != MSC_NOT_READY) return st;
    return compute_synchronised(p, p->pending_field, p->pending_stream);
}

msc_status finish_replay(Plan* p, cudaStream_t s) {
    msc_status st;
    const uint32_t word = p->hsum->status;
    if (word) {
        if ((st = check_cuda(p, cudaMemsetAsync(p->status_word(), 0, sizeof(uint32_t), s), "status clear")))
            return st;
        if ((word & ST_RETRY) && !(word & ~(ST_RETRY | ST_CAPACITY))) {
            destroy_graph(p);
            return MSC_NOT_READY;
        }
        return status_error(p, word);
    }
    absorb_summary(p);
    p->stage_recorded = 0x3F;
    p->stats.n_launches = p->graph_static_launches + p->loop_body_launches[0] * int64_t(p->hsum->jump_rounds) +
                          p->loop_body_launches[1] * int64_t(p->hsum->sweep_iters) +
                          p->loop_body_launches[2] * int64_t(p->hsum->dp_iters);
    p->have_gradient = p->have_critical = p->have_extremum = p->have_reach = true;
    p->have_junctions = p->have_trace = p->have_dstar = true;
    ++p->graph_replays;
    return MSC_OK;
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
    if (opts && ((opts->flags & ~(MSC_FLAG_NO_GRAPH | MSC_FLAG_SERIAL_PASS)) || opts->gradient_tile < 0 || opts->gradient_tile > 9 ||
                 opts->path_count_method < 0 || opts->path_count_method > 2))
        return MSC_ERR_ARG;
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
    for (int i = 0; i < 12 && !st; ++i) st = msc::check_cuda(p, cudaEventCreate(&p->stage_ev[i]), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->kev0), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->kev1), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->tev0), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->tev1), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->gev0), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreate(&p->gev1), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreateWithFlags(&p->pend_ev, cudaEventDisableTiming), "cudaEventCreate");
    // the pass's critical path (capture and its loop bodies) at the highest priority, the extremum
    // branch at the lowest, so that the branch takes only what the critical path leaves free; a
    // replayed graph with the branch keeps these per-node priorities (one without it runs at the
    // priority of the stream it is launched into)
    int lo_prio = 0, hi_prio = 0;
    if (!st) st = msc::check_cuda(p, cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio), "cudaDeviceGetStreamPriorityRange");
    if (!st) st = msc::check_cuda(p, cudaStreamCreateWithPriority(&p->cap_stream, cudaStreamNonBlocking, hi_prio), "cudaStreamCreate");
    if (!st) st = msc::check_cuda(p, cudaStreamCreateWithPriority(&p->body_stream, cudaStreamNonBlocking, hi_prio), "cudaStreamCreate");
    if (!st) st = msc::check_cuda(p, cudaStreamCreateWithPriority(&p->side_stream, cudaStreamNonBlocking, lo_prio), "cudaStreamCreate");
    if (!st) st = msc::check_cuda(p, cudaStreamCreateWithPriority(&p->side_body_stream, cudaStreamNonBlocking, lo_prio), "cudaStreamCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming), "cudaEventCreate");
    if (!st) st = msc::check_cuda(p, cudaMallocHost(&p->hsum, sizeof(msc::Summary)), "cudaMallocHost");
    if (!st) st = msc::ensure(p, p->status, sizeof(msc::Summary));
    if (!st) st = msc::check_cuda(p, cudaMemset(p->status.ptr, 0, sizeof(msc::Summary)), "cudaMemset(summary)");
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
    if (p->pending) cudaEventSynchronize(p->pend_ev);  // the pass in flight still uses the buffers
    msc::destroy_graph(p);
    p->for_each_buffer([](msc::DeviceBuffer& b) {
        if (b.ptr) cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    });
    for (cudaEvent_t e : p->stage_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {p->kev0, p->kev1, p->tev0, p->tev1, p->gev0, p->gev1, p->pend_ev, p->fork_ev, p->join_ev})
        if (e) cudaEventDestroy(e);
    for (cudaStream_t t : {p->cap_stream, p->body_stream, p->side_stream, p->side_body_stream})
        if (t) cudaStreamDestroy(t);
    if (p->hsum) cudaFreeHost(p->hsum);
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
    p->stage_recorded = 0;
    if ((st = msc::check_cuda(p, cudaMemsetAsync(p->dsum(), 0, sizeof(msc::Summary), s), "summary clear"))) return st;
    msc::stage_start(p, 0, s);
    if ((st = msc::run_gradient(p, d_field, s))) return st;
    msc::stage_end(p, 0, s);
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
    if ((st = msc::finish_stage(p, s))) return st;  // a NaN in the field stops here
    msc::stage_start(p, 1, s);
    if ((st = msc::run_critical(p, s))) return st;
    msc::stage_end(p, 1, s);
    if ((st = msc::finish_stage(p, s))) return st;
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
    msc::stage_start(p, 2, s);
    if ((st = msc::run_extremum(p, s))) return st;
    msc::stage_end(p, 2, s);
    if ((st = msc::finish_stage(p, s))) return st;
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
    msc::stage_start(p, 3, s);
    if ((st = msc::run_reachability(p, s))) return st;
    msc::stage_end(p, 3, s);
    if (p->fault_kind == 2) msc::raise_status(p, msc::ST_TIMEOUT, s);
    if ((st = msc::finish_stage(p, s))) return st;
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
    msc::stage_start(p, 4, s);
    if ((st = msc::run_junctions(p, s))) return st;
    if ((st = msc::finish_stage(p, s))) return st;
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

static msc_status ensure_trace(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_junctions(p, s))) return st;
    if (p->have_trace) return MSC_OK;
    if ((st = msc::run_trace(p, s))) return st;
    msc::stage_end(p, 4, s);
    if ((st = msc::finish_stage(p, s))) return st;
    p->have_trace = true;
    return MSC_OK;
}

msc_status msc_minor(msc_plan_t plan, msc_stream_t stream, int which, int64_t* rows, int64_t* nnz,
                     const int64_t** d_rowptr, const uint32_t** d_col, const uint32_t** d_mult) {
    if (!plan || which < 0 || which > 3) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_trace(p, s))) return st;
    if (!p->have_minor) {
        if ((st = msc::build_minor_csr(p, s))) return st;
        if ((st = msc::finish_stage(p, s))) return st;
        p->have_minor = true;
    }
    if (rows) *rows = p->minor_rows[which];
    if (nnz) *nnz = p->minor_nnz[which];
    if (d_rowptr) *d_rowptr = static_cast<const int64_t*>(p->minor_rowptr[which].ptr);
    if (d_col) *d_col = static_cast<const uint32_t*>(p->minor_col[which].ptr);
    if (d_mult) *d_mult = static_cast<const uint32_t*>(p->minor_mult[which].ptr);
    return MSC_OK;
}

static msc_status ensure_dstar(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_trace(p, s))) return st;
    if (p->have_dstar) return MSC_OK;
    msc::stage_start(p, 5, s);
    if ((st = msc::run_path_count(p, s))) return st;
    msc::stage_end(p, 5, s);
    if (p->fault_kind == 3) msc::raise_status(p, msc::ST_OVERFLOW, s);
    if ((st = msc::finish_stage(p, s))) return st;
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

msc_status msc_saddle_arcs_csc(msc_plan_t plan, msc_stream_t stream, int64_t* nnz, const int64_t** d_colptr,
                               const uint32_t** d_row, const uint64_t** d_count) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_dstar(p, s))) return st;
    if (!p->have_dstar_csc) {
        if ((st = msc::build_dstar_csc(p, s))) return st;
        if ((st = msc::finish_stage(p, s))) return st;
        p->have_dstar_csc = true;
    }
    if (nnz) *nnz = p->dstar_nnz;
    if (d_colptr) *d_colptr = static_cast<const int64_t*>(p->csc_colptr.ptr);
    if (d_row) *d_row = static_cast<const uint32_t*>(p->csc_row.ptr);
    if (d_count) *d_count = static_cast<const uint64_t*>(p->csc_count.ptr);
    return MSC_OK;
}

static msc_status ensure_geometry(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_critical(p, s))) return st;
    if (p->have_geometry) return MSC_OK;
    if ((st = msc::build_arc_geometry(p, s))) return st;
    if ((st = msc::finish_stage(p, s))) return st;
    p->have_geometry = true;
    return MSC_OK;
}

msc_status msc_arc_geometry(msc_plan_t plan, msc_stream_t stream, int64_t* n_arcs, int64_t* n_cells,
                            const int64_t** d_offsets, const uint32_t** d_cells) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_geometry(p, s))) return st;
    if (n_arcs) *n_arcs = 2 * (p->counts[1] + p->counts[2]);
    if (n_cells) *n_cells = p->geo_cells_n;
    if (d_offsets) *d_offsets = static_cast<const int64_t*>(p->geo_off.ptr);
    if (d_cells) *d_cells = static_cast<const uint32_t*>(p->geo_cells.ptr);
    return MSC_OK;
}

// The cells of the saddle-saddle arcs of multiplicity 1 need the rows of J.  A pass that counted
// paths row by row has none, so the junction waves run once more for them (they give the same D*);
// the pass's summary, statistics and kernel timings are put back afterwards.
static msc_status ensure_ss_geometry(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_dstar(p, s))) return st;
    if (p->have_ss_geometry) return MSC_OK;
    if (!p->have_j && p->pc_method_used != 2) {
        if ((st = msc::read_summary(p, s))) return st;
        const msc::Summary saved = *p->hsum;
        const msc_stats stats = p->stats;
        const int32_t forced = p->opts.path_count_method;
        const int used = p->pc_method_used;
        cudaEvent_t k0 = p->kev0, k1 = p->kev1;
        p->kev0 = p->kev1 = nullptr;
        p->opts.path_count_method = 2;
        st = msc::run_path_count(p, s);
        if (st == MSC_OK) st = msc::finish_stage(p, s);
        p->opts.path_count_method = forced;
        p->pc_method_used = used;
        p->kev0 = k0;
        p->kev1 = k1;
        if (st == MSC_OK) {
            *p->hsum = saved;
            st = msc::check_cuda(p, cudaMemcpyAsync(p->dsum(), p->hsum, sizeof(msc::Summary), cudaMemcpyHostToDevice, s),
                                 "summary restore");
            if (st == MSC_OK) st = msc::check_cuda(p, cudaStreamSynchronize(s), "stream sync");
        }
        p->stats = stats;
        if (st) return st;
    }
    p->have_j = true;
    if ((st = msc::build_ss_geometry(p, s))) return st;
    if ((st = msc::finish_stage(p, s))) return st;
    p->have_ss_geometry = true;
    return MSC_OK;
}

msc_status msc_saddle_arc_geometry(msc_plan_t plan, msc_stream_t stream, int64_t* n_entries, int64_t* n_cells,
                                   const int64_t** d_offsets, const uint32_t** d_cells) {
    if (!plan) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_ss_geometry(p, s))) return st;
    if (n_entries) *n_entries = p->dstar_nnz;
    if (n_cells) *n_cells = p->ss_cells_n;
    if (d_offsets) *d_offsets = static_cast<const int64_t*>(p->ss_off.ptr);
    if (d_cells) *d_cells = static_cast<const uint32_t*>(p->ss_cells.ptr);
    return MSC_OK;
}

static msc_status ensure_graph(Plan* p, cudaStream_t s) {
    msc_status st;
    if ((st = ensure_extremum(p, s))) return st;
    if ((st = ensure_dstar(p, s))) return st;
    if (!p->have_dstar_csc) {
        if ((st = msc::build_dstar_csc(p, s))) return st;
        if ((st = msc::finish_stage(p, s))) return st;
        p->have_dstar_csc = true;
    }
    if (!p->have_graph) {
        if ((st = msc::build_complex_graph(p, s))) return st;
        if ((st = msc::finish_stage(p, s))) return st;
        p->have_graph = true;
    }
    return MSC_OK;
}

msc_status msc_simplify(msc_plan_t plan, msc_stream_t stream, const float* d_field, double threshold,
                        msc_simplified* out) {
    if (!plan || !d_field || !out || !(threshold >= 0.0)) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_graph(p, s))) return st;
    if ((st = msc::run_simplify(p, d_field, threshold, s))) return st;
    const int64_t n = p->graph_nodes;
    const int c = p->simp_cur;
    out->n_nodes = n;
    out->n_rounds = p->simp_rounds;
    out->n_cancelled = p->simp_cancelled;
    out->n_adj = p->simp_nnz;
    int64_t base[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) {
        base[k + 1] = base[k] + p->counts[k];
        out->counts[k] = 0;
    }
    const uint8_t* alive = static_cast<const uint8_t*>(p->simp_alive.ptr) + size_t(c) * size_t(n ? n : 1);
    if (n) {
        std::vector<uint8_t> h(static_cast<size_t>(n));
        if ((st = msc::check_cuda(p, cudaMemcpyAsync(h.data(), alive, size_t(n), cudaMemcpyDeviceToHost, s), "copy out")) ||
            (st = msc::check_cuda(p, cudaStreamSynchronize(s), "stream sync")))
            return st;
        for (int k = 0; k < 4; ++k)
            for (int64_t u = base[k]; u < base[k + 1]; ++u) out->counts[k] += h[size_t(u)];
    }
    out->d_alive = alive;
    out->d_nodeptr = static_cast<const int64_t*>(p->simp_ptr[c].ptr);
    out->d_adj = static_cast<const uint32_t*>(p->simp_nbr[c].ptr);
    out->d_mult = static_cast<const uint64_t*>(p->simp_mult[c].ptr);
    out->d_log = static_cast<const uint32_t*>(p->simp_log.ptr);
    return MSC_OK;
}

msc_status msc_complex_graph(msc_plan_t plan, msc_stream_t stream, int64_t* n_nodes, int64_t* n_adj,
                             int64_t* h_nodeptr, uint32_t* h_adj, uint64_t* h_mult) {
    if (!plan || !n_nodes || !n_adj) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if ((st = ensure_graph(p, s))) return st;
    const int64_t room = *n_adj;
    *n_nodes = p->graph_nodes;
    *n_adj = p->graph_nadj;
    if (!h_nodeptr) return MSC_OK;  // size query
    if (!h_adj || !h_mult) return MSC_ERR_ARG;
    if (room < p->graph_nadj) return MSC_ERR_CAPACITY;
    if ((st = msc::check_cuda(p, cudaMemcpyAsync(h_nodeptr, p->graph_nodeptr.ptr,
                                                 sizeof(int64_t) * size_t(p->graph_nodes + 1), cudaMemcpyDeviceToHost, s),
                              "graph copy")) ||
        (st = msc::check_cuda(p, cudaMemcpyAsync(h_adj, p->graph_adj.ptr, sizeof(uint32_t) * size_t(p->graph_nadj),
                                                 cudaMemcpyDeviceToHost, s),
                              "graph copy")) ||
        (st = msc::check_cuda(p, cudaMemcpyAsync(h_mult, p->graph_mult.ptr, sizeof(uint64_t) * size_t(p->graph_nadj),
                                                 cudaMemcpyDeviceToHost, s),
                              "graph copy")))
        return st;
    return msc::check_cuda(p, cudaStreamSynchronize(s), "stream sync");
}

// One pass as a replayed graph; MSC_NOT_READY asks the caller to run the pass synchronised
// (a capacity fixed at capture was too small).
static msc_status compute_graph(Plan* p, const float* d_field, cudaStream_t s) {
    msc_status st;
    if (!p->graph_exec || p->graph_field != d_field)
        if ((st = msc::capture_graph(p, d_field))) return st;
    msc::invalidate(p);
    p->stage_recorded = 0;
    if ((st = msc::check_cuda(p, cudaGraphLaunch(p->graph_exec, s), "graph launch"))) return st;
    if ((st = msc::read_summary(p, s))) return st;
    return msc::finish_replay(p, s);
}

}  // extern "C"

namespace msc {
// Minors at most this deep (iterations of the product loop) run the row-wise products when the
// method is automatic: on the 256^3 GRF (26 levels) they take 1.5 ms against 6 ms for the waves,
// on the 512^3 blob field (197 levels) 1.55 s against 24 ms.
constexpr int64_t kShallowMinor = 64;

// Every stage with host synchronisation and exact buffer sizes; the sizes plus headroom become
// the capacities of the next captured graph.
msc_status compute_synchronised(Plan* p, const float* d_field, cudaStream_t s) {
    msc_status st;
    if ((st = msc_gradient(static_cast<msc_plan_s*>(p), d_field, reinterpret_cast<msc_stream_t>(s)))) return st;
    if ((st = ensure_extremum(p, s))) return st;
    if ((st = ensure_dstar(p, s))) return st;
    auto room = [](int64_t n) { return n + n / 4 + 1024; };
    for (int k = 0; k < 4; ++k) p->caps.cells[k] = std::max(p->caps.cells[k], room(p->counts[k]));
    p->caps.nj = std::max(p->caps.nj, room(p->n_junctions));
    p->caps.staging = std::max<int64_t>(p->caps.staging, room(p->pc_staging_cap));
    p->caps.dp_pool = std::max<int64_t>(p->caps.dp_pool, room(p->dp_pool_cap));
    p->caps_ready = true;
    // automatic path-count method: the row-wise products re-expand the sub-DAG below every
    // 1-saddle, so their work grows with the depth of the minor, where the junction waves do every
    // junction once; on shallow minors the row-wise products are the faster of the two
    if (p->opts.path_count_method == 0 && p->pc_method_chosen == 0)
        p->pc_method_chosen = p->stats.n_iter <= kShallowMinor ? 1 : 2;
    destroy_graph(p);
    return MSC_OK;
}
}  // namespace msc

extern "C" {

msc_status msc_compute(msc_plan_t plan, const float* d_field, msc_stream_t stream) {
    if (!plan || !d_field) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    if (msc::graphs_enabled(p) && p->caps_ready) {
        st = compute_graph(p, d_field, s);
        if (st != MSC_NOT_READY) return st;
    }
    return msc::compute_synchronised(p, d_field, s);
}

msc_status msc_copy_to_host(msc_plan_t plan, msc_stream_t stream, int what, void* h_out, int64_t* bytes) {
    if (!plan || !bytes || what < MSC_OUT_CELLS0 || what > MSC_OUT_SS_ARC_CELLS) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;
    const void* src = nullptr;
    int64_t n = 0;  // bytes
    if (what <= MSC_OUT_CELLS3) {
        if ((st = ensure_critical(p, s))) return st;
        src = p->cells[what].ptr;
        n = int64_t(sizeof(uint32_t)) * p->counts[what];
    } else if (what <= MSC_OUT_CUBE_MAX) {
        if ((st = ensure_extremum(p, s))) return st;
        const int64_t nv = p->g.nverts;
        const msc::DeviceBuffer* b[4] = {&p->min_arcs, &p->max_arcs, &p->vmin, &p->cmax};
        const int64_t len[4] = {2 * p->counts[1], 2 * p->counts[2], nv, nv};
        src = b[what - MSC_OUT_MIN_ARCS]->ptr;
        n = int64_t(sizeof(uint32_t)) * len[what - MSC_OUT_MIN_ARCS];
    } else if (what >= MSC_OUT_SS_ARC_OFFSETS) {
        if ((st = ensure_ss_geometry(p, s))) return st;
        src = what == MSC_OUT_SS_ARC_OFFSETS ? p->ss_off.ptr : p->ss_cells.ptr;
        n = what == MSC_OUT_SS_ARC_OFFSETS ? int64_t(sizeof(int64_t)) * (p->dstar_nnz + 1)
                                           : int64_t(sizeof(uint32_t)) * p->ss_cells_n;
    } else if (what >= MSC_OUT_ARC_OFFSETS) {
        if ((st = ensure_geometry(p, s))) return st;
        const int64_t n_arcs = 2 * (p->counts[1] + p->counts[2]);
        src = what == MSC_OUT_ARC_OFFSETS ? p->geo_off.ptr : p->geo_cells.ptr;
        n = what == MSC_OUT_ARC_OFFSETS ? int64_t(sizeof(int64_t)) * (n_arcs + 1)
                                        : int64_t(sizeof(uint32_t)) * p->geo_cells_n;
    } else {
        if ((st = ensure_dstar(p, s))) return st;
        if (what == MSC_OUT_DSTAR_ROWPTR) {
            src = p->dstar_rowptr.ptr;
            n = int64_t(sizeof(int64_t)) * (p->counts[1] + 1);
        } else if (what == MSC_OUT_DSTAR_COL) {
            src = p->dstar_col.ptr;
            n = int64_t(sizeof(uint32_t)) * p->dstar_nnz;
        } else {
            src = p->dstar_count.ptr;
            n = int64_t(sizeof(uint64_t)) * p->dstar_nnz;
        }
    }
    const int64_t room = *bytes;
    *bytes = n;
    if (!h_out) return MSC_OK;
    if (room < n) return MSC_ERR_CAPACITY;
    if (n && (st = msc::check_cuda(p, cudaMemcpyAsync(h_out, src, size_t(n), cudaMemcpyDeviceToHost, s), "copy out")))
        return st;
    return msc::check_cuda(p, cudaStreamSynchronize(s), "stream sync");
}

msc_status msc_compute_async(msc_plan_t plan, const float* d_field, msc_stream_t stream) {
    if (!plan || !d_field) return MSC_ERR_ARG;
    Plan* p = plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    msc_status st;
    if ((st = msc::bind_device(p))) return st;  // also waits for a pass still in flight
    if (!msc::graphs_enabled(p) || !p->caps_ready) return msc::compute_synchronised(p, d_field, s);
    if (!p->graph_exec || p->graph_field != d_field)
        if ((st = msc::capture_graph(p, d_field))) return st;
    msc::invalidate(p);
    p->stage_recorded = 0;
    if ((st = msc::check_cuda(p, cudaGraphLaunch(p->graph_exec, s), "graph launch"))) return st;
    if ((st = msc::check_cuda(p, cudaMemcpyAsync(p->hsum, p->dsum(), sizeof(msc::Summary), cudaMemcpyDeviceToHost, s),
                              "summary copy")) ||
        (st = msc::check_cuda(p, cudaEventRecord(p->pend_ev, s), "event record")))
        return st;
    p->pending = true;
    p->pending_field = d_field;
    p->pending_stream = s;
    return MSC_OK;
}

msc_status msc_compute_wait(msc_plan_t plan) {
    if (!plan) return MSC_ERR_ARG;
    return msc::bind_device(plan);
}

msc_status msc_get_stats(msc_plan_t plan, msc_stats* out) {
    if (!plan || !out) return MSC_ERR_ARG;
    Plan* p = plan;
    if (p->pending) {
        const msc_status st = msc::bind_device(p);
        if (st) return st;
    }
    p->stats.peak_device_bytes = p->peak_bytes;
    float* dst[6] = {&p->stats.ms_gradient, &p->stats.ms_critical, &p->stats.ms_extremum,
                     &p->stats.ms_reachability, &p->stats.ms_minor, &p->stats.ms_path_count};
    for (int k = 0; k < 6; ++k)
        if ((p->stage_recorded >> k) & 1u && cudaEventSynchronize(p->stage_ev[2 * k + 1]) == cudaSuccess)
            cudaEventElapsedTime(dst[k], p->stage_ev[2 * k], p->stage_ev[2 * k + 1]);
    if (p->have_dstar && cudaEventSynchronize(p->kev1) == cudaSuccess)
        cudaEventElapsedTime(&p->stats.ms_rows_kernel, p->kev0, p->kev1);
    if (p->have_trace && cudaEventSynchronize(p->tev1) == cudaSuccess)
        cudaEventElapsedTime(&p->stats.ms_trace_kernel, p->tev0, p->tev1);
    if (p->have_gradient && cudaEventSynchronize(p->gev1) == cudaSuccess)
        cudaEventElapsedTime(&p->stats.ms_gradient_kernel, p->gev0, p->gev1);
    cudaGetLastError();
    *out = p->stats;
    return MSC_OK;
}

}  // extern "C"

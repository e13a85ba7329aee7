// Batching and serving runtime (host code): msc_batch_create / submit / poll / wait / destroy.
//
// The paper motivates fast MS-complex computation with time-varying data whose steps must be
// analysed within a budget (Sec. 1).  A small volume does not fill 152 SMs, so volumes run
// together:
//  * A submission whose plans have all run once (so their buffer sizes are known) becomes one
//    group job: the pipelines of all its volumes are captured as parallel branches of a single
//    CUDA graph, launched once -- one launch and one host wait for the whole batch.  The graph is
//    cached and replayed while the same plans and field pointers are submitted again.  A volume
//    that needs more room than its branch was captured with is rerun on its own.
//  * Otherwise every volume is a job of its own.  A pool of worker threads, each with its own
//    stream, takes jobs from a FIFO as soon as a worker is free, the volume's plan is not busy,
//    and the working-set estimate fits the HBM budget (continuous batching).
#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "msc_internal.cuh"

namespace {

struct Ticket {
    int remaining = 0;
    msc_status status = MSC_OK;
};

struct Job {
    msc_plan_t plan;
    const float* field;
    uint64_t ticket;
    cudaEvent_t ready;  // the submitting stream's position at submission
    int64_t footprint;
    std::vector<std::pair<msc_plan_t, const float*>> group;  // non-empty: a group job of these volumes
};

// A captured group: its volumes, the capture epoch of each plan when recorded, and the graph.
struct GroupGraph {
    std::vector<std::pair<msc_plan_t, const float*>> vols;
    std::vector<int64_t> epochs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int64_t footprint_of(msc_plan_t plan) {
    const msc::Plan* p = plan;
    return std::max<int64_t>(p->peak_bytes, int64_t(128) * p->g.nverts);
}

}  // namespace

struct msc_batch_s {
    int device = 0;
    int64_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::unordered_map<msc_plan_t, int> busy;  // plans with a job running
    uint64_t next_ticket = 1;
    int64_t in_flight = 0;
    int running = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::mutex graph_mu;                   // group graphs are captured and launched one at a time
    GroupGraph group;                      // the last captured group
    std::vector<cudaStream_t> branches;    // one capture stream per volume of a group
    std::vector<cudaEvent_t> joins;

    ~msc_batch_s() {
        drop_group();
        for (cudaStream_t t : branches) cudaStreamDestroy(t);
        for (cudaEvent_t e : joins) cudaEventDestroy(e);
    }

    void drop_group() {
        if (group.exec) cudaGraphExecDestroy(group.exec);
        if (group.graph) cudaGraphDestroy(group.graph);
        group = GroupGraph{};
    }

    bool group_current(const std::vector<std::pair<msc_plan_t, const float*>>& vols) const {
        if (!group.exec || group.vols != vols) return false;
        for (size_t i = 0; i < vols.size(); ++i)
            if (vols[i].first->capture_epoch != group.epochs[i]) return false;
        return true;
    }

    // Records the pipelines of all volumes as parallel branches of one graph, forked from and
    // joined into stream s.  Every plan is first captured on its own, which sizes its buffers
    // for its capacities (and leaves its own graph for single runs).
    msc_status capture_group(const std::vector<std::pair<msc_plan_t, const float*>>& vols, cudaStream_t s) {
        drop_group();
        msc_status st;
        for (auto& v : vols) {
            msc::Plan* p = v.first;
            if ((!p->graph_exec || p->graph_field != v.second) && (st = msc::capture_graph(p, v.second))) return st;
        }
        while (branches.size() < vols.size()) {
            cudaStream_t t;
            cudaEvent_t e;
            if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess) return MSC_ERR_CUDA;
            branches.push_back(t);
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return MSC_ERR_CUDA;
            joins.push_back(e);
        }
        cudaEvent_t fork = joins[0];
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return MSC_ERR_CUDA;
        st = MSC_OK;
        if (cudaEventRecord(fork, s) != cudaSuccess) st = MSC_ERR_CUDA;
        for (size_t i = 0; i < vols.size() && !st; ++i) {
            msc::Plan* p = vols[i].first;
            if (cudaStreamWaitEvent(branches[i], fork, 0) != cudaSuccess) {
                st = MSC_ERR_CUDA;
                break;
            }
            p->capturing = true;
            const int64_t launches = p->stats.n_launches;
            st = msc::enqueue_pipeline(p, vols[i].second, branches[i], false);  // the volumes fill the device
            p->capturing = false;
            p->stats.n_launches = launches;
            if (!st && (cudaEventRecord(joins[i], branches[i]) != cudaSuccess ||
                        cudaStreamWaitEvent(s, joins[i], 0) != cudaSuccess))
                st = MSC_ERR_CUDA;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st ? st : MSC_ERR_CUDA;
        }
        group.graph = g;
        if (cudaGraphInstantiate(&group.exec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            drop_group();
            return MSC_ERR_CUDA;
        }
        group.vols = vols;
        for (auto& v : vols) group.epochs.push_back(v.first->capture_epoch);
        return MSC_OK;
    }

    // One launch for the whole group on stream s, then every volume's summary in one wait.
    // Volumes that outgrew their capacities are rerun synchronised, on their own.
    msc_status run_group(const std::vector<std::pair<msc_plan_t, const float*>>& vols, cudaStream_t s) {
        std::lock_guard<std::mutex> lk(graph_mu);
        msc_status st;
        if (!group_current(vols) && (st = capture_group(vols, s))) return st;
        for (auto& v : vols) msc::invalidate(v.first);
        if (cudaGraphLaunch(group.exec, s) != cudaSuccess) return MSC_ERR_CUDA;
        for (auto& v : vols)
            if (cudaMemcpyAsync(v.first->hsum, v.first->dsum(), sizeof(msc::Summary), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess)
                return MSC_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return MSC_ERR_CUDA;
        msc_status first = MSC_OK;
        for (auto& v : vols) {
            st = msc::finish_replay(v.first, s);
            if (st == MSC_NOT_READY) {
                drop_group();
                st = msc::compute_synchronised(v.first, v.second, s);
            }
            if (st && !first) first = st;
        }
        return first;
    }

    // First queued job whose plan is idle and whose footprint is admissible (lock held).
    bool idle(const Job& j) const {
        if (busy.count(j.plan)) return false;
        for (auto& v : j.group)
            if (busy.count(v.first)) return false;
        return true;
    }

    bool pick(Job* out) {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            if (!idle(*it)) continue;
            const bool fits = budget <= 0 || running == 0 || in_flight + it->footprint <= budget;
            if (!fits) return false;  // FIFO admission: later jobs do not overtake a waiting one
            *out = *it;
            queue.erase(it);
            return true;
        }
        return false;
    }

    void worker() {
        cudaSetDevice(device);
        cudaStream_t s = nullptr;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        while (true) {
            Job job;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop ? queue.empty() : pick(&job); });
                if (stop && queue.empty()) break;
                busy[job.plan] = 1;
                for (auto& v : job.group) busy[v.first] = 1;
                in_flight += job.footprint;
                ++running;
            }
            msc_status st = MSC_OK;
            if (cudaStreamWaitEvent(s, job.ready, 0) != cudaSuccess) st = MSC_ERR_CUDA;
            if (st == MSC_OK && !job.group.empty()) st = run_group(job.group, s);
            else if (st == MSC_OK) st = msc_compute(job.plan, job.field, reinterpret_cast<msc_stream_t>(s));
            if (st == MSC_OK && cudaStreamSynchronize(s) != cudaSuccess) st = MSC_ERR_CUDA;
            cudaEventDestroy(job.ready);
            {
                std::lock_guard<std::mutex> lk(mu);
                for (auto& v : job.group) busy.erase(v.first);
                busy.erase(job.plan);
                in_flight -= job.footprint;
                --running;
                Ticket& t = tickets[job.ticket];
                if (st != MSC_OK && t.status == MSC_OK) t.status = st;
                t.remaining -= job.group.empty() ? 1 : int(job.group.size());
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
        cudaStreamDestroy(s);
    }
};

extern "C" {

msc_status msc_batch_create(int n_workers, int64_t hbm_budget_bytes, msc_batch_t* out) {
    if (!out || n_workers < 0 || n_workers > 256) return MSC_ERR_ARG;
    *out = nullptr;
    auto* b = new (std::nothrow) msc_batch_s();
    if (!b) return MSC_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return MSC_ERR_CUDA;
    }
    b->budget = hbm_budget_bytes;
    const int n = n_workers ? n_workers : 4;
    for (int i = 0; i < n; ++i) b->workers.emplace_back([b] { b->worker(); });
    *out = b;
    return MSC_OK;
}

msc_status msc_batch_destroy(msc_batch_t b) {
    if (!b) return MSC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
    }
    b->cv_work.notify_all();
    for (auto& t : b->workers) t.join();
    delete b;
    return MSC_OK;
}

msc_status msc_batch_submit(msc_batch_t b, msc_volume* vols, int n, msc_stream_t stream, uint64_t* ticket) {
    if (!b || !ticket || n < 0 || (n > 0 && !vols)) return MSC_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!vols[i].d_field) return MSC_ERR_ARG;
        if (vols[i].plan) {
            const msc::Geom& g = vols[i].plan->g;
            if (g.nx != vols[i].dims[0] || g.ny != vols[i].dims[1] || g.nz != vols[i].dims[2]) return MSC_ERR_ARG;
        }
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return MSC_ERR_CUDA;
    if (cur != b->device && cudaSetDevice(b->device) != cudaSuccess) return MSC_ERR_CUDA;
    std::vector<Job> jobs;
    for (int i = 0; i < n; ++i) {
        if (!vols[i].plan) {
            // the runtime keeps several passes in flight: each replays as one chain
            msc_opts o{};
            o.flags = MSC_FLAG_SERIAL_PASS;
            msc_status st = msc_plan(vols[i].dims, &o, &vols[i].plan);
            if (st) {
                for (auto& j : jobs) cudaEventDestroy(j.ready);
                return st;
            }
        }
        Job j{vols[i].plan, vols[i].d_field, 0, nullptr, footprint_of(vols[i].plan), {}};
        if (cudaEventCreateWithFlags(&j.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(j.ready, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
            for (auto& jj : jobs) cudaEventDestroy(jj.ready);
            return MSC_ERR_CUDA;
        }
        jobs.push_back(j);
    }
    // one group job when every volume's plan has run once, allows graphs, and appears once, and
    // the whole group fits the HBM budget
    bool group = n > 1;
    int64_t total = 0;
    std::unordered_map<msc_plan_t, int> seen;
    for (auto& j : jobs) {
        group = group && j.plan->caps_ready && msc::graphs_enabled(j.plan) && !seen[j.plan]++;
        total += j.footprint;
    }
    group = group && (b->budget <= 0 || total <= b->budget);
    if (group) {
        Job g{jobs[0].plan, nullptr, 0, jobs[0].ready, total, {}};
        for (size_t i = 1; i < jobs.size(); ++i) cudaEventDestroy(jobs[i].ready);
        for (auto& j : jobs) g.group.emplace_back(j.plan, j.field);
        jobs.assign(1, g);
    }
    {
        std::lock_guard<std::mutex> lk(b->mu);
        const uint64_t id = b->next_ticket++;
        b->tickets[id].remaining = n;
        for (auto& j : jobs) {
            j.ticket = id;
            b->queue.push_back(j);
        }
        *ticket = id;
    }
    b->cv_work.notify_all();
    if (cur != b->device) cudaSetDevice(cur);
    return MSC_OK;
}

msc_status msc_poll(msc_batch_t b, uint64_t ticket, int* done, int* status) {
    if (!b || !done) return MSC_ERR_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return MSC_ERR_ARG;
    *done = it->second.remaining == 0;
    if (status) *status = it->second.status;
    return MSC_OK;
}

msc_status msc_batch_wait(msc_batch_t b, uint64_t ticket, int* status) {
    if (!b) return MSC_ERR_ARG;
    std::unique_lock<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return MSC_ERR_ARG;
    b->cv_done.wait(lk, [&] { return it->second.remaining == 0; });
    if (status) *status = it->second.status;
    return MSC_OK;
}

}  // extern "C"

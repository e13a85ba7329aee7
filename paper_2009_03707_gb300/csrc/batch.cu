// Batching and serving runtime (host code): msc_batch_create / submit / poll / wait / destroy.
//
// The paper motivates fast MS-complex computation with time-varying data whose steps must be
// analysed within a budget (Sec. 1).  On one GB300 a single volume leaves the GPU idle during
// its host-side stage boundaries, and a small volume does not fill 152 SMs; running several
// volumes at once on separate streams keeps the device busy.  A batch is a pool of worker
// threads, each with its own stream; volumes wait in a FIFO and are started as soon as a worker
// is free, the volume's plan is not busy, and the working-set estimate fits the HBM budget.
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

    // First queued job whose plan is idle and whose footprint is admissible (lock held).
    bool pick(Job* out) {
        for (auto it = queue.begin(); it != queue.end(); ++it) {
            if (busy.count(it->plan)) continue;
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
                in_flight += job.footprint;
                ++running;
            }
            msc_status st = MSC_OK;
            if (cudaStreamWaitEvent(s, job.ready, 0) != cudaSuccess) st = MSC_ERR_CUDA;
            if (st == MSC_OK) st = msc_compute(job.plan, job.field, reinterpret_cast<msc_stream_t>(s));
            if (st == MSC_OK && cudaStreamSynchronize(s) != cudaSuccess) st = MSC_ERR_CUDA;
            cudaEventDestroy(job.ready);
            {
                std::lock_guard<std::mutex> lk(mu);
                busy.erase(job.plan);
                in_flight -= job.footprint;
                --running;
                Ticket& t = tickets[job.ticket];
                if (st != MSC_OK && t.status == MSC_OK) t.status = st;
                --t.remaining;
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
            msc_status st = msc_plan(vols[i].dims, nullptr, &vols[i].plan);
            if (st) {
                for (auto& j : jobs) cudaEventDestroy(j.ready);
                return st;
            }
        }
        Job j{vols[i].plan, vols[i].d_field, 0, nullptr, footprint_of(vols[i].plan)};
        if (cudaEventCreateWithFlags(&j.ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(j.ready, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) {
            for (auto& jj : jobs) cudaEventDestroy(jj.ready);
            return MSC_ERR_CUDA;
        }
        jobs.push_back(j);
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

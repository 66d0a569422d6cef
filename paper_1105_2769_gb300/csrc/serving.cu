// Serving engine: continuous batching of potential and force requests on one
// GPU (no counterpart in the paper).
//
// A request is admitted as soon as a slot is free and its estimated device
// footprint fits the HBM budget; each slot is a worker thread with its own
// context (scratch arena) and non-blocking stream, so admitted requests run
// concurrently on the device and a request that arrives while others run
// starts as soon as one finishes. Requests naming a system id keep that
// point set (and, for tree solves, its tree) resident on the device; later
// requests for the same id skip the copy and the build. Admission is FIFO
// with backfill: the oldest request has priority, and a younger one may start
// only if it fits beside the room held for the oldest.
//
// A resident system is published only with a CUDA event recorded after its
// upload and tree build on the creating slot's stream; every other slot
// makes its stream wait on that event before reading the system, so no slot
// reads points or a tree that are still being written. Evicted systems are
// taken off the table under the server lock and freed after it is released
// (freeing waits for the device), so submit, poll and the other slots never
// wait on device work through the lock.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mbm_internal.h"
#include "mbm_tree_api.h"

namespace {

using clk = std::chrono::steady_clock;

double ms_between(clk::time_point a, clk::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
    uint64_t ticket = 0;
    mbm_request req{};
    mbm_config cfg{};
    size_t est = 0;
    clk::time_point submitted;
};

struct Done {
    mbm_result res{};
    bool ready = false;
};

struct Resident {
    int64_t N = 0;
    double* X = nullptr;
    mbm_tree* tree = nullptr;
    cudaEvent_t ready = nullptr;  // recorded after the upload and the tree build
    size_t bytes = 0;
    int users = 0;
    uint64_t last_use = 0;
};

struct Worker {
    std::thread th;
    mbm_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    double* dX = nullptr;  // private input/output buffers (grown on demand)
    double* dOut = nullptr;
    size_t capX = 0, capOut = 0;
    unsigned long long* d_stamp = nullptr;  // device clock at a request's start and end
    unsigned long long* h_stamp = nullptr;  // pinned host copy
};

size_t estimate_bytes(const mbm_request& r, const mbm_config& c) {
    const size_t N = (size_t)r.N;
    const size_t io = N * 24 + N * (r.kind == MBM_REQ_FORCES ? 24 : 8);
    const int base = r.mode & 0xff;
    if (base != MBM_TREE) return io + N * 32 + 4096;
    return io + mbm_tree_solve_bytes(r.N, c, r.kind == MBM_REQ_FORCES) + (1 << 20);
}

}  // namespace

struct mbm_server {
    int device = 0;
    size_t budget = 0;
    size_t reserved = 0;        // admitted estimates + resident systems
    std::vector<Worker> workers;
    std::deque<Job> pending;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, Resident> resident;
    std::vector<Resident> evicted;  // off the table, not yet freed
    uint64_t next_ticket = 1, use_clock = 0;
    int64_t n_admitted = 0, n_rejected = 0, n_completed = 0;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
};

namespace {

void free_resident(Resident& r) {
    if (r.tree) mbm_tree_free(r.tree);
    if (r.X) cudaFree(r.X);
    if (r.ready) cudaEventDestroy(r.ready);
    r = Resident{};
}

// Take resident systems nobody uses off the table until `need` more bytes
// fit (LRU); the caller holds the lock, and they are freed after it is
// released (s->evicted).
void evict_for(mbm_server* s, size_t need) {
    while (s->budget && s->reserved + need > s->budget) {
        auto victim = s->resident.end();
        for (auto it = s->resident.begin(); it != s->resident.end(); ++it)
            if (it->second.users == 0 &&
                (victim == s->resident.end() || it->second.last_use < victim->second.last_use))
                victim = it;
        if (victim == s->resident.end()) return;
        s->reserved -= victim->second.bytes;
        s->evicted.push_back(victim->second);
        s->resident.erase(victim);
    }
}

// Pick the next job this worker may start (caller holds the lock).
bool take_job(mbm_server* s, Job& out) {
    if (s->pending.empty()) return false;
    const size_t room_head = s->pending.front().est;
    evict_for(s, room_head);
    if (!s->budget || s->reserved + room_head <= s->budget) {
        out = s->pending.front();
        s->pending.pop_front();
        s->reserved += out.est;
        return true;
    }
    for (auto it = s->pending.begin() + 1; it != s->pending.end(); ++it) {
        if (s->reserved + room_head + it->est <= s->budget) {
            out = *it;
            s->pending.erase(it);
            s->reserved += out.est;
            return true;
        }
    }
    return false;
}

mbm_status grow(double** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap) return MBM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    MBM_CUDA_TRY(cudaMalloc(p, bytes));
    *cap = bytes;
    return MBM_OK;
}

// Device clock (%globaltimer, ns) at this point of the stream's work.
__global__ void stamp_kernel(unsigned long long* t) {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

// Solve one request on this worker's stream with inputs X (and tree) in place.
mbm_status solve_job(Worker& w, const Job& job, const double* X, mbm_tree* tree, size_t ob) {
    const mbm_request& r = job.req;
    MBM_TRY(grow(&w.dOut, &w.capOut, ob));
    mbm_stream_t ms = reinterpret_cast<mbm_stream_t>(w.stream);
    stamp_kernel<<<1, 1, 0, w.stream>>>(w.d_stamp);
    mbm_status st;
    if (r.kind == MBM_REQ_FORCES)
        st = mbm_forces_ex(w.ctx, X, r.N, r.eps, r.alpha, r.mode, &job.cfg, tree, w.dOut, nullptr, ms);
    else st = mbm_potential_ex(w.ctx, X, r.N, r.eps, r.alpha, r.mode, &job.cfg, tree, w.dOut, nullptr, ms);
    stamp_kernel<<<1, 1, 0, w.stream>>>(w.d_stamp + 1);
    if (st != MBM_OK) return st;
    MBM_CUDA_TRY(cudaMemcpyAsync(w.h_stamp, w.d_stamp, 2 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, w.stream));
    MBM_CUDA_TRY(cudaMemcpyAsync(r.out_host, w.dOut, ob, cudaMemcpyDeviceToHost, w.stream));
    return MBM_OK;
}

mbm_status run_job(mbm_server* s, Worker& w, const Job& job, int slot, mbm_result& res) {
    const mbm_request& r = job.req;
    const size_t xb = (size_t)r.N * 24;
    const size_t ob = (size_t)r.N * (r.kind == MBM_REQ_FORCES ? 24 : 8);
    const bool tree_mode = (r.mode & 0xff) == MBM_TREE;
    res.slot = slot;
    w.h_stamp[0] = w.h_stamp[1] = 0;
    Resident* res_entry = nullptr;
    if (r.system_id) {
        std::unique_lock<std::mutex> lock(s->mu);
        auto it = s->resident.find(r.system_id);
        if (it != s->resident.end() && it->second.N == r.N) {
            res_entry = &it->second;
            res_entry->users++;
            res_entry->last_use = ++s->use_clock;
        }
    }
    mbm_status st = MBM_OK;
    if (res_entry) {
        // the creator's upload and build may still be running on its stream
        cudaError_t e = cudaStreamWaitEvent(w.stream, res_entry->ready, 0);
        st = e == cudaSuccess ? solve_job(w, job, res_entry->X, res_entry->tree, ob)
                              : mbm_cuda_fail(e, "cudaStreamWaitEvent(resident system)");
    } else if (r.system_id) {
        // first request for this system: make it resident
        double* dx = nullptr;
        mbm_tree* t = nullptr;
        cudaEvent_t ready = nullptr;
        cudaError_t e = cudaMalloc(&dx, xb);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dx, r.X_host, xb, cudaMemcpyHostToDevice, w.stream);
        if (e != cudaSuccess) st = mbm_cuda_fail(e, "upload of a resident system");
        if (st == MBM_OK && tree_mode && r.N >= 3)
            st = mbm_tree_build(w.ctx, dx, r.N, &job.cfg, w.stream, &t);
        if (st == MBM_OK) {
            e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventRecord(ready, w.stream);
            if (e != cudaSuccess) st = mbm_cuda_fail(e, "cudaEventRecord(resident system)");
        }
        if (st != MBM_OK) {
            cudaStreamSynchronize(w.stream);
            if (ready) cudaEventDestroy(ready);
            if (t) mbm_tree_free(t);
            if (dx) cudaFree(dx);
            return st;
        }
        bool shared = false;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            Resident ent;
            ent.N = r.N;
            ent.X = dx;
            ent.tree = t;
            ent.ready = ready;
            ent.bytes = xb + (t ? (size_t)r.N * 72 : 0);
            ent.users = 1;
            ent.last_use = ++s->use_clock;
            auto ins = s->resident.emplace(r.system_id, ent);
            if (ins.second) {
                s->reserved += ent.bytes;
                res_entry = &ins.first->second;
                shared = true;
            }
        }
        st = solve_job(w, job, dx, t, ob);
        if (!shared) {  // another slot made it resident meanwhile: ours stays private
            cudaStreamSynchronize(w.stream);
            cudaEventDestroy(ready);
            if (t) mbm_tree_free(t);
            cudaFree(dx);
        }
    } else {
        st = grow(&w.dX, &w.capX, xb);
        if (st == MBM_OK) {
            cudaError_t e = cudaMemcpyAsync(w.dX, r.X_host, xb, cudaMemcpyHostToDevice, w.stream);
            st = e == cudaSuccess ? solve_job(w, job, w.dX, nullptr, ob)
                                  : mbm_cuda_fail(e, "upload of a request");
        }
    }
    cudaError_t e = cudaStreamSynchronize(w.stream);
    if (e != cudaSuccess && st == MBM_OK) st = mbm_cuda_fail(e, "cudaStreamSynchronize");
    if (res_entry) {
        std::unique_lock<std::mutex> lock(s->mu);
        res_entry->users--;
    }
    if (st == MBM_OK) {
        res.dev_start_ns = (int64_t)w.h_stamp[0];
        res.dev_end_ns = (int64_t)w.h_stamp[1];
    }
    return st;
}

void worker_main(mbm_server* s, int slot) {
    Worker& w = s->workers[slot];
    cudaSetDevice(s->device);
    for (;;) {
        Job job;
        std::vector<Resident> dead;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->cv_work.wait(lock,
                            [&] { return s->stop || !s->evicted.empty() || take_job(s, job); });
            dead.swap(s->evicted);
            if (job.ticket != 0) s->n_admitted++;
        }
        for (auto& d : dead) free_resident(d);  // outside the lock
        if (job.ticket == 0) {
            if (s->stop) return;
            continue;
        }
        const clk::time_point t0 = clk::now();
        mbm_result res{};
        res.status = run_job(s, w, job, slot, res);
        const clk::time_point t1 = clk::now();
        res.queue_ms = ms_between(job.submitted, t0);
        res.compute_ms = ms_between(t0, t1);
        res.latency_ms = ms_between(job.submitted, t1);
        res.bytes_reserved = (int64_t)job.est;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            s->reserved -= job.est;
            Done& d = s->done[job.ticket];
            d.res = res;
            d.ready = true;
            s->n_completed++;
        }
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" mbm_status mbm_server_create(int device, size_t hbm_budget_bytes, int32_t slots,
                                        mbm_server** out) {
    if (!out) return mbm_fail(MBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 64) return mbm_fail(MBM_EINVAL, "slots must be in [1, 64]");
    mbm_server* s = new (std::nothrow) mbm_server();
    if (!s) return mbm_fail(MBM_ENOMEM, "host allocation failed");
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->workers.resize(slots);
    for (int i = 0; i < slots; ++i) {
        Worker& w = s->workers[i];
        mbm_status st = mbm_ctx_create(device, 0, &w.ctx);
        cudaError_t e = st == MBM_OK ? cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking)
                                     : cudaSuccess;
        if (st == MBM_OK && e == cudaSuccess)
            e = cudaMalloc(&w.d_stamp, 2 * sizeof(unsigned long long));
        if (st == MBM_OK && e == cudaSuccess)
            e = cudaMallocHost(&w.h_stamp, 2 * sizeof(unsigned long long));
        if (st != MBM_OK || e != cudaSuccess) {
            for (int j = 0; j <= i; ++j) {
                Worker& v = s->workers[j];
                if (v.d_stamp) cudaFree(v.d_stamp);
                if (v.h_stamp) cudaFreeHost(v.h_stamp);
                if (v.stream) cudaStreamDestroy(v.stream);
                if (v.ctx) mbm_ctx_destroy(v.ctx);
            }
            delete s;
            return st != MBM_OK ? st : mbm_cuda_fail(e, "cudaStreamCreate");
        }
    }
    for (int i = 0; i < slots; ++i) s->workers[i].th = std::thread(worker_main, s, i);
    *out = s;
    return MBM_OK;
}

extern "C" mbm_status mbm_server_destroy(mbm_server* s) {
    if (!s) return MBM_OK;
    {
        std::unique_lock<std::mutex> lock(s->mu);
        s->stop = true;
        s->pending.clear();
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers)
        if (w.th.joinable()) w.th.join();
    cudaSetDevice(s->device);
    for (auto& kv : s->resident) free_resident(kv.second);
    for (auto& d : s->evicted) free_resident(d);
    for (auto& w : s->workers) {
        if (w.dX) cudaFree(w.dX);
        if (w.dOut) cudaFree(w.dOut);
        if (w.d_stamp) cudaFree(w.d_stamp);
        if (w.h_stamp) cudaFreeHost(w.h_stamp);
        if (w.stream) cudaStreamDestroy(w.stream);
        if (w.ctx) mbm_ctx_destroy(w.ctx);
    }
    delete s;
    return MBM_OK;
}

extern "C" mbm_status mbm_submit(mbm_server* s, const mbm_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return mbm_fail(MBM_EINVAL, "NULL argument");
    if (req->N < 0 || (req->N > 0 && (!req->X_host || !req->out_host)))
        return mbm_fail(MBM_EINVAL, "bad request size or buffers");
    if (req->kind != MBM_REQ_POTENTIAL && req->kind != MBM_REQ_FORCES)
        return mbm_fail(MBM_EINVAL, "unknown request kind");
    Job job;
    job.req = *req;
    if (req->cfg) job.cfg = *req->cfg;
    else mbm_config_default(&job.cfg);
    job.req.cfg = nullptr;
    job.est = estimate_bytes(job.req, job.cfg);
    job.submitted = clk::now();
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->budget && job.est > s->budget) {
        s->n_rejected++;
        return mbm_fail(MBM_EBUDGET, "request's estimated footprint exceeds the server's budget");
    }
    job.ticket = s->next_ticket++;
    *ticket = job.ticket;
    s->done[job.ticket] = Done{};
    s->pending.push_back(job);
    lock.unlock();
    s->cv_work.notify_one();
    return MBM_OK;
}

extern "C" mbm_status mbm_poll(mbm_server* s, uint64_t ticket, mbm_result* res, int64_t timeout_us) {
    if (!s) return mbm_fail(MBM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return mbm_fail(MBM_EINVAL, "unknown ticket");
    if (!it->second.ready) {
        if (timeout_us == 0) return MBM_PENDING;
        auto pred = [&] { return s->done[ticket].ready; };
        if (timeout_us < 0) s->cv_done.wait(lock, pred);
        else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred))
            return MBM_ETIMEDOUT;
    }
    Done d = s->done[ticket];
    s->done.erase(ticket);
    if (res) *res = d.res;
    return MBM_OK;
}

extern "C" mbm_status mbm_server_stats(mbm_server* s, int64_t* admitted, int64_t* pending,
                                       int64_t* rejected, int64_t* completed, size_t* reserved) {
    if (!s) return mbm_fail(MBM_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    if (admitted) *admitted = s->n_admitted;
    if (pending) *pending = (int64_t)s->pending.size();
    if (rejected) *rejected = s->n_rejected;
    if (completed) *completed = s->n_completed;
    if (reserved) *reserved = s->reserved;
    return MBM_OK;
}

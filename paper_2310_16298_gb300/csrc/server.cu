// Serving loop: continuous batching of stencil solves.
//
// Requests (any 2D/3D problem the library accepts, each with its own step
// count) are queued by stencil_server_submit.  A worker thread admits them in
// arrival order while the HBM budget and the resident-slot limit allow,
// allocates their device state (one grid plus the plan, whose scratch grid is
// the second copy of the ping-pong: the request's grid is advanced in place),
// and keeps
// every resident request moving: each one advances by at most `quantum` time
// steps per issue on one of several CUDA streams, so the work of many
// requests overlaps on the device, and a request that arrives while others
// run is admitted as soon as memory and a slot free up.  A finished request's
// grid is copied back to host memory; its device state is released at once.
// The worker waits with cudaEventQuery and short sleeps: nothing spins on the
// device.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace stx;

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct Request {
    uint64_t id = 0;
    // problem
    int ndim = 2;
    int64_t shape[3] = {1, 1, 1};
    int r = 1;
    int kind = STENCIL_BOX;
    int dtype = STENCIL_F32;
    int bc = STENCIL_BC_DIRICHLET_ZERO;
    int impl = STENCIL_IMPL_AUTO;
    std::vector<double> cg;
    const void* h_in = nullptr;
    uint64_t seed = 0;
    double lo = 0.0, hi = 1.0;
    int64_t steps = 0;
    // state
    enum State { QUEUED, RESIDENT, DONE, FAILED } state = QUEUED;  // written under the server lock
    stencil_plan_t plan = nullptr;
    void* grid = nullptr;  // the request's field, advanced in place
    int64_t done_steps = 0;
    int stream = 0;
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    bool draining = false;  // the result copy has been queued
    size_t grid_bytes = 0;
    size_t charge = 0;  // budget charged while resident
    void* result = nullptr;  // pinned host copy of the final grid
    stencil_status error = STENCIL_OK;
    std::string message;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int used_impl = 0;
};

}  // namespace

struct stencil_server_s {
    int64_t budget = 0;
    int max_resident = 0;
    int quantum = 16;
    std::vector<cudaStream_t> streams;
    int device = 0;
    Clock::time_point t0;

    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;            // waiting for admission
    std::vector<std::shared_ptr<Request>> resident;        // worker-owned
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_id = 1;
    int64_t in_use = 0;
    bool stop = false;
    std::thread worker;
    // statistics
    int64_t admitted = 0, completed = 0, peak_resident = 0, peak_bytes = 0;
    std::atomic<int64_t> issued{0};
    // Finished plans are destroyed in groups (freeing a plan's scratch grid
    // synchronises the device); their memory stays charged until then.
    std::vector<std::pair<stencil_plan_t, int64_t>> graveyard;
};

namespace {

size_t dtype_size(int dtype) { return dtype == STENCIL_F64 ? 8 : 4; }

// Create the plan and device state of a request (worker thread).  The
// caller records the outcome in the request's state under the lock.
stencil_status admit(stencil_server_s* S, Request* q) {
    stencil_options o{};
    o.bc = q->bc;
    o.impl = q->impl;
    o.prec = STENCIL_PREC_NATIVE;
    stencil_status st = stencil_plan_create(&q->plan, q->ndim, q->shape, q->r, (stencil_kind)q->kind, q->cg.data(),
                                            (stencil_dtype)q->dtype, &o);
    if (st == STENCIL_OK) {
        q->used_impl = q->plan->impl;
        cudaStream_t s = S->streams[q->stream];
        cudaError_t e = cudaMallocAsync(&q->grid, q->grid_bytes, s);
        if (e == cudaSuccess) {
            if (q->h_in) {
                e = cudaMemcpyAsync(q->grid, q->h_in, q->grid_bytes, cudaMemcpyHostToDevice, s);
            } else {
                int64_t count = q->grid_bytes / dtype_size(q->dtype);
                e = fill_uniform(q->grid, q->dtype == STENCIL_F64, count, q->seed, 0, q->lo, q->hi, s);
            }
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(&q->result, q->grid_bytes);
        if (e != cudaSuccess) {
            st = STENCIL_ECUDA;
            q->message = std::string("admission: ") + cudaGetErrorString(e);
        }
    } else {
        q->message = last_error_string();
    }
    q->error = st;
    q->t_admit = seconds_since(S->t0);
    return st;
}

// Release a request's device state.  Returns the budget that can be given
// back now; the plan (and the rest of the charge) goes to the graveyard.
int64_t release(stencil_server_s* S, Request* q) {
    cudaStream_t s = S->streams[q->stream];
    if (q->grid) {
        cudaFreeAsync(q->grid, s);
        q->grid = nullptr;
    }
    if (q->ev) {
        cudaEventDestroy(q->ev);
        q->ev = nullptr;
    }
    const int64_t grids = (int64_t)q->grid_bytes;
    if (q->plan) {
        S->graveyard.emplace_back(q->plan, (int64_t)q->charge - grids);
        q->plan = nullptr;
        return grids;
    }
    return (int64_t)q->charge;
}

// Destroy graveyard plans (caller holds the lock).
void bury(stencil_server_s* S) {
    for (auto& g : S->graveyard) {
        stencil_plan_destroy(g.first);
        S->in_use -= g.second;
    }
    S->graveyard.clear();
}

void worker_loop(stencil_server_s* S) {
    cudaSetDevice(S->device);
    int rr = 0;
    for (;;) {
        // ---- admission (arrival order, while budget and slots allow)
        std::vector<std::shared_ptr<Request>> admitted;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->resident.empty() && S->queue.empty()) {
                if (!S->graveyard.empty()) bury(S);
                if (S->stop) return;
                S->cv.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            while (!S->queue.empty() && (int)S->resident.size() + (int)admitted.size() < S->max_resident) {
                auto q = S->queue.front();
                if (S->in_use + (int64_t)q->charge > S->budget && !S->graveyard.empty()) bury(S);
                if (S->in_use + (int64_t)q->charge > S->budget && !(S->resident.empty() && admitted.empty())) break;
                S->queue.pop_front();
                S->in_use += q->charge;
                S->peak_bytes = std::max(S->peak_bytes, S->in_use);
                q->stream = rr++ % (int)S->streams.size();
                admitted.push_back(q);
            }
        }
        for (auto& q : admitted) {
            const stencil_status st = admit(S, q.get());
            std::lock_guard<std::mutex> lk(S->mu);
            q->state = (st == STENCIL_OK) ? Request::RESIDENT : Request::FAILED;
            if (q->state == Request::FAILED) {
                S->in_use -= release(S, q.get());
                q->t_done = seconds_since(S->t0);
                S->cv.notify_all();
            } else {
                S->resident.push_back(q);
                ++S->admitted;
                S->peak_resident = std::max<int64_t>(S->peak_resident, (int64_t)S->resident.size());
            }
        }
        // ---- progress: issue the next quantum of every idle resident request
        bool progressed = !admitted.empty();
        std::vector<std::shared_ptr<Request>> finished;
        for (auto& q : S->resident) {
            if (q->in_flight) {
                cudaError_t e = cudaEventQuery(q->ev);
                if (e == cudaErrorNotReady) continue;
                q->in_flight = false;
                progressed = true;
                if (e != cudaSuccess) {
                    q->error = STENCIL_ECUDA;
                    q->message = std::string("request work: ") + cudaGetErrorString(e);
                    finished.push_back(q);
                    continue;
                }
                if (plan_error_status(q->plan, "request work") != STENCIL_OK) {
                    q->error = STENCIL_ECUDA;
                    q->message = last_error_string();
                    finished.push_back(q);
                    continue;
                }
                if (q->draining) {
                    finished.push_back(q);
                    continue;
                }
            }
            cudaStream_t s = S->streams[q->stream];
            if (q->done_steps < q->steps) {
                const int64_t k = std::min<int64_t>(S->quantum, q->steps - q->done_steps);
                stencil_status st = stencil_apply(q->plan, q->grid, q->grid, k, (stencil_stream_t)s);
                if (st != STENCIL_OK) {
                    q->error = st;
                    q->message = last_error_string();
                    finished.push_back(q);
                    continue;
                }
                q->done_steps += k;
                S->issued += 1;
            } else {
                // all steps issued: bring the result home
                cudaMemcpyAsync(q->result, q->grid, q->grid_bytes, cudaMemcpyDeviceToHost, s);
                q->draining = true;
            }
            cudaEventRecord(q->ev, s);
            q->in_flight = true;
            progressed = true;
        }
        if (!finished.empty()) {
            std::lock_guard<std::mutex> lk(S->mu);
            for (auto& q : finished) {
                if (q->in_flight) cudaEventSynchronize(q->ev);
                q->state = (q->error == STENCIL_OK) ? Request::DONE : Request::FAILED;
                S->in_use -= release(S, q.get());
                q->t_done = seconds_since(S->t0);
                ++S->completed;
                S->resident.erase(std::find(S->resident.begin(), S->resident.end(), q));
            }
            S->cv.notify_all();
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" stencil_status stencil_server_create(stencil_server_t* out, int64_t budget_bytes, int32_t max_resident,
                                                int32_t quantum_steps, int32_t nstreams) {
    if (!out) return fail(STENCIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (budget_bytes <= 0 || max_resident < 1 || quantum_steps < 1 || nstreams < 1 || nstreams > 64)
        return fail(STENCIL_EINVAL, "need budget > 0, max_resident >= 1, quantum >= 1, 1 <= nstreams <= 64");
    std::unique_ptr<stencil_server_s> S(new stencil_server_s);
    S->budget = budget_bytes;
    S->max_resident = max_resident;
    S->quantum = quantum_steps;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    for (int i = 0; i < nstreams; ++i) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto x : S->streams) cudaStreamDestroy(x);
            return cuda_fail(e, "cudaStreamCreate");
        }
        S->streams.push_back(s);
    }
    S->t0 = Clock::now();
    S->worker = std::thread(worker_loop, S.get());
    *out = S.release();
    return STENCIL_OK;
}

extern "C" stencil_status stencil_server_submit(stencil_server_t S, const stencil_request* rq, uint64_t* id) {
    if (!S || !rq || !id) return fail(STENCIL_EINVAL, "NULL argument");
    if (rq->ndim != 2 && rq->ndim != 3) return fail(STENCIL_EINVAL, "ndim must be 2 or 3");
    if (rq->radius < 1 || rq->radius > kMaxRadius) return fail(STENCIL_EINVAL, "radius must be in 1..4");
    if (!rq->coeffs) return fail(STENCIL_EINVAL, "coeffs is NULL");
    if (rq->steps < 0) return fail(STENCIL_EINVAL, "steps must be >= 0");
    if (rq->dtype != STENCIL_F32 && rq->dtype != STENCIL_F64) return fail(STENCIL_EINVAL, "bad dtype");
    auto q = std::make_shared<Request>();
    q->ndim = rq->ndim;
    int64_t pts = 1, nco = 1;
    for (int d = 0; d < rq->ndim; ++d) {
        if (rq->shape[d] < 2 * rq->radius + 1) return fail(STENCIL_EINVAL, "every extent must be at least 2*radius+1");
        q->shape[d] = rq->shape[d];
        pts *= rq->shape[d];
        nco *= 2 * rq->radius + 1;
    }
    q->r = rq->radius;
    q->kind = rq->kind;
    q->dtype = rq->dtype;
    q->bc = rq->bc;
    q->impl = rq->impl;
    q->cg.assign(rq->coeffs, rq->coeffs + nco);
    q->h_in = rq->h_in;
    q->seed = rq->seed;
    q->lo = rq->lo;
    q->hi = rq->hi;
    q->steps = rq->steps;
    q->grid_bytes = (size_t)pts * dtype_size(rq->dtype);
    // the request's grid, the plan's scratch grid, operands; plus a padded grid
    // when rows are not 16-byte multiples (the plan repacks for the tensor cores)
    q->charge = 2 * q->grid_bytes + (1 << 20);
    if ((q->shape[q->ndim - 1] * (int64_t)dtype_size(q->dtype)) % 16 != 0) q->charge += q->grid_bytes + (q->grid_bytes >> 2);
    if ((int64_t)q->charge > S->budget) return fail(STENCIL_ENOMEM, "request larger than the whole budget");
    std::lock_guard<std::mutex> lk(S->mu);
    q->id = S->next_id++;
    q->t_submit = seconds_since(S->t0);
    S->all[q->id] = q;
    S->queue.push_back(q);
    *id = q->id;
    S->cv.notify_all();
    return STENCIL_OK;
}

extern "C" stencil_status stencil_server_poll(stencil_server_t S, uint64_t id) {
    if (!S) return fail(STENCIL_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(STENCIL_EINVAL, "unknown request id");
    const Request* q = it->second.get();
    if (q->state == Request::DONE) return STENCIL_OK;
    if (q->state == Request::FAILED && q->t_done > 0) return fail(q->error, q->message);
    return STENCIL_ENOTREADY;
}

extern "C" stencil_status stencil_server_wait(stencil_server_t S, uint64_t id, int64_t timeout_ms) {
    if (!S) return fail(STENCIL_EINVAL, "NULL server");
    const auto t0 = Clock::now();
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        auto it = S->all.find(id);
        if (it == S->all.end()) return fail(STENCIL_EINVAL, "unknown request id");
        const Request* q = it->second.get();
        if (q->state == Request::DONE) return STENCIL_OK;
        if (q->state == Request::FAILED && q->t_done > 0) return fail(q->error, q->message);
        if (timeout_ms >= 0 && std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() >= timeout_ms)
            return fail(STENCIL_ETIMEDOUT, "request not finished");
        S->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

extern "C" stencil_status stencil_server_result(stencil_server_t S, uint64_t id, void* h_out,
                                                stencil_request_stats* stats) {
    if (!S) return fail(STENCIL_EINVAL, "NULL server");
    std::shared_ptr<Request> q;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->all.find(id);
        if (it == S->all.end()) return fail(STENCIL_EINVAL, "unknown request id");
        q = it->second;
        if (q->state != Request::DONE && !(q->state == Request::FAILED && q->t_done > 0))
            return fail(STENCIL_ENOTREADY, "request not finished");
        S->all.erase(it);
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->submit_s = q->t_submit;
        stats->admit_s = q->t_admit;
        stats->done_s = q->t_done;
        stats->impl = q->used_impl;
        stats->status = q->error;
        stats->updates = (int64_t)(q->grid_bytes / dtype_size(q->dtype)) * q->steps;
    }
    if (q->state == Request::FAILED) {
        if (q->result) cudaFreeHost(q->result);
        q->result = nullptr;
        return fail(q->error, q->message);
    }
    if (h_out) memcpy(h_out, q->result, q->grid_bytes);
    cudaFreeHost(q->result);
    q->result = nullptr;
    return STENCIL_OK;
}

extern "C" stencil_status stencil_server_stats(stencil_server_t S, stencil_server_stats_t* out) {
    if (!S || !out) return fail(STENCIL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->queued = (int64_t)S->queue.size();
    out->resident = (int64_t)S->resident.size();
    out->admitted = S->admitted;
    out->completed = S->completed;
    out->bytes_in_use = S->in_use;
    out->peak_bytes = S->peak_bytes;
    out->peak_resident = S->peak_resident;
    out->quanta_issued = S->issued.load();
    return STENCIL_OK;
}

extern "C" stencil_status stencil_server_destroy(stencil_server_t S) {
    if (!S) return STENCIL_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();  // the worker drains every admitted request first
    bury(S);
    for (auto& kv : S->all)
        if (kv.second->result) cudaFreeHost(kv.second->result);
    for (auto s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    delete S;
    return STENCIL_OK;
}

// Served stream of rBKI-TK requests: continuous batching with device-memory admission.
//
// One server owns, on one device:
//   * an arena of `mem_budget` bytes (one cudaMalloc at creation) from which every admitted
//     request's workspace (its Krylov basis, products, eigensolver scratch, ...) is carved;
//   * `wave_threads` wave workers, each a host thread with its own stream.  Requests that the
//     batched path takes (rbki_tucker_batched: BF16/FP16 products, I_n <= 256, ...) queue
//     for waves: a worker takes the longest FIFO prefix of that queue (at most `wave_max`
//     requests) whose workspaces fit in the arena together, runs them as one wave - one
//     launch per stage for all of them - and waits for the device.  Two workers keep one
//     wave on the GPU while the next is admitted and launched;
//   * `max_slots` slots, each a host thread with its own stream and its own per-mode
//     streams, for every other request (FP64 products, large tensors, flags): a slot takes
//     the oldest such request as soon as its workspace fits, runs Algorithms 1-2 on its
//     streams (rbki_tucker) and waits for the device.
// Requests that arrive while others run are admitted as workers and memory free up, and
// their kernels overlap on the GPU with the ones already there.
//
// Admission is FIFO per queue: a request that does not fit waits at the head of its queue
// until enough memory is released (no starvation of large requests).  A request whose
// workspace exceeds the whole budget is refused at submission (RBKI_E_NOMEM).
//
// The result of a request does not depend on what else runs: a wave item computes exactly
// what rbki_tucker_batched computes for it alone (per-item work queues and reductions of
// fixed order), and a slot request what rbki_tucker computes (fixed-order reductions,
// grids that depend only on the shape).
//
// Latency is measured on the host from rbki_submit to the moment the slot observes the
// request's last kernel complete.
#include <chrono>
#include <string>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan.h"

namespace rbki {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over [0, size) with coalescing; offsets 256-byte aligned.
class Arena {
public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_[*off] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                prev->second += len;
                return;
            }
        }
        free_[start] = len;
    }

private:
    std::map<size_t, size_t> free_, used_;
};

enum class State { QUEUED, RUNNING, DONE };

struct Request {
    uint64_t ticket = 0;
    rbki_tensor X{};
    rbki_params prm{};
    rbki_tucker_out out{};
    size_t ws_bytes = 0;
    State state = State::QUEUED;
    bool cancel = false;
    rbki_status result = RBKI_PENDING;
    double t_submit = 0, t_done = 0;
    cudaEvent_t ready = nullptr;   // recorded on the submitter's stream (or null)
    bool wave = false;             // served by the batched path
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaStream_t ms[RBKI_MAX_ORDER] = {nullptr};
};

}  // namespace
}  // namespace rbki

using namespace rbki;

struct rbki_server {
    int device = 0;
    size_t budget = 0;
    int nslots = 0;
    char* arena_base = nullptr;
    Arena* arena = nullptr;
    std::mutex mu;
    std::condition_variable cv_work;   // queue / memory changes (slots wait here)
    std::condition_variable cv_done;   // a request finished (drain waits here)
    std::deque<Request*> queue;                    // per-request path (slots)
    std::deque<Request*> wqueue;                   // batched path (wave workers)
    int wave_max = 0;
    std::vector<Slot> wslots;
    std::unordered_map<uint64_t, Request*> reqs;   // every request not yet retired by a poll
    uint64_t next_ticket = 1;
    int running = 0;
    bool stopping = false;
    std::vector<Slot> slots;
    std::vector<std::thread> workers;
};

namespace {

// Runs one admitted request on a slot; returns its status.
rbki_status run_request(rbki_server* s, Slot& slot, Request* r, size_t off) {
    Plan pl;
    RBKI_TRY(make_plan(&r->X, &r->prm, pl));
    carve(pl, s->arena_base + off);
    pl.xin = r->X.data;
    if (r->ready) RBKI_CUDA_TRY(cudaStreamWaitEvent(slot.st, r->ready, 0));
    rbki_status rs = run_tucker(pl, &r->out, slot.st, slot.ms);
    cudaError_t e = cudaStreamSynchronize(slot.st);
    if (rs < 0) return rs;
    if (e != cudaSuccess) return set_cuda_error(e, "server request");
    int32_t err = 0;
    e = cudaMemcpy(&err, pl.err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e, "server error word");
    if (err) return set_error(RBKI_E_TIMEOUT, "a bounded wait inside a kernel expired");
    return rs;
}

void slot_main(rbki_server* s, int id) {
    cudaSetDevice(s->device);
    Slot& slot = s->slots[id];
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        size_t off = 0;
        s->cv_work.wait(lk, [&] {
            return s->stopping || (!s->queue.empty() && s->arena->alloc(s->queue.front()->ws_bytes, &off));
        });
        if (s->stopping) return;
        Request* r = s->queue.front();
        s->queue.pop_front();
        r->state = State::RUNNING;
        ++s->running;
        lk.unlock();
        const rbki_status rs = run_request(s, slot, r, off);
        const double t = now_s();
        lk.lock();
        s->arena->release(off);
        --s->running;
        r->t_done = t;
        r->result = r->cancel ? RBKI_E_CANCELLED : rs;
        r->state = State::DONE;
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
}

// Admits the longest FIFO prefix of the wave queue (<= wave_max requests) whose workspaces fit
// in one arena block; returns the count (0: nothing fits yet) and the block's offset.
int admit_wave(rbki_server* s, size_t* off) {
    const int lim = std::min<int>((int)s->wqueue.size(), s->wave_max);
    std::vector<size_t> pre(lim + 1, 0);
    for (int k = 0; k < lim; ++k) pre[k + 1] = pre[k] + ((s->wqueue[k]->ws_bytes + 255) & ~(size_t)255);
    for (int k = lim; k >= 1; --k)
        if (s->arena->alloc(pre[k], off)) return k;
    return 0;
}

// Runs one admitted wave on a worker's stream; returns its status (shared by its requests).
rbki_status run_wave_requests(rbki_server* s, Slot& slot, const std::vector<Request*>& w, size_t off) {
    std::vector<rbki_tensor> X;
    std::vector<rbki_params> P;
    std::vector<rbki_tucker_out> O;
    size_t total = 0;
    for (Request* r : w) {
        if (r->ready) RBKI_CUDA_TRY(cudaStreamWaitEvent(slot.st, r->ready, 0));
        X.push_back(r->X);
        P.push_back(r->prm);
        O.push_back(r->out);
        total += (r->ws_bytes + 255) & ~(size_t)255;
    }
    rbki_status rs = rbki_tucker_batched((int32_t)w.size(), X.data(), P.data(), s->arena_base + off, total,
                                         O.data(), slot.st);
    cudaError_t e = cudaStreamSynchronize(slot.st);
    if (rs < 0) return rs;
    if (e != cudaSuccess) return set_cuda_error(e, "server wave");
    return rs;
}

// A wave item whose bounded wait expired (info[2N] != 0; requests without info cannot tell)
bool wave_item_timed_out(const Request* r) {
    if (!r->out.info) return false;
    int32_t e = 0;
    if (cudaMemcpy(&e, r->out.info + 2 * r->X.order, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    return e != 0;
}

void wave_main(rbki_server* s, int id) {
    cudaSetDevice(s->device);
    Slot& slot = s->wslots[id];
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        size_t off = 0;
        int k = 0;
        s->cv_work.wait(lk, [&] {
            if (s->stopping) return true;
            if (s->wqueue.empty()) return false;
            k = admit_wave(s, &off);
            return k > 0;
        });
        if (s->stopping) return;
        std::vector<Request*> w(s->wqueue.begin(), s->wqueue.begin() + k);
        s->wqueue.erase(s->wqueue.begin(), s->wqueue.begin() + k);
        for (Request* r : w) r->state = State::RUNNING;
        s->running += k;
        lk.unlock();
        const rbki_status rs = run_wave_requests(s, slot, w, off);
        std::vector<bool> timed_out(w.size(), false);
        if (rs >= 0)
            for (size_t i = 0; i < w.size(); ++i) timed_out[i] = wave_item_timed_out(w[i]);
        const double t = now_s();
        lk.lock();
        s->arena->release(off);
        s->running -= k;
        for (size_t i = 0; i < w.size(); ++i) {
            Request* r = w[i];
            r->t_done = t;
            r->result = r->cancel ? RBKI_E_CANCELLED : (timed_out[i] ? RBKI_E_TIMEOUT : rs);
            r->state = State::DONE;
        }
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

rbki_status rbki_server_create(int32_t device, size_t mem_budget, int32_t max_slots, rbki_server** out) {
    return rbki_server_create_ex(device, mem_budget, max_slots, RBKI_SERVER_WAVE_THREADS, RBKI_SERVER_WAVE_MAX, out);
}

rbki_status rbki_server_create_ex(int32_t device, size_t mem_budget, int32_t max_slots, int32_t wave_threads,
                                  int32_t wave_max, rbki_server** out) {
    if (!out) return set_error(RBKI_E_INVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 64) return set_error(RBKI_E_INVAL, "max_slots must be in [1, 64]");
    if (wave_threads < 0 || wave_threads > 8) return set_error(RBKI_E_INVAL, "wave_threads must be in [0, 8]");
    if (wave_threads > 0 && (wave_max < 1 || wave_max > 1024))
        return set_error(RBKI_E_INVAL, "wave_max must be in [1, 1024]");
    if (mem_budget < 4096) return set_error(RBKI_E_INVAL, "mem_budget too small");
    int ndev = 0;
    RBKI_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(RBKI_E_INVAL, "no such device");
    int prev = 0;
    RBKI_CUDA_TRY(cudaGetDevice(&prev));
    RBKI_CUDA_TRY(cudaSetDevice(device));
    rbki_server* s = new rbki_server();
    s->device = device;
    s->budget = mem_budget;
    s->nslots = max_slots;
    cudaError_t e = cudaMalloc(&s->arena_base, mem_budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        cudaSetDevice(prev);
        return set_error(RBKI_E_NOMEM, "server: cannot allocate mem_budget on the device");
    }
    s->arena = new Arena(mem_budget);
    s->wave_max = wave_threads > 0 ? wave_max : 0;
    s->slots.resize(max_slots);
    s->wslots.resize(wave_threads);
    for (auto& sl : s->slots) {
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        for (int n = 0; n < RBKI_MAX_ORDER && e == cudaSuccess; ++n)
            e = cudaStreamCreateWithFlags(&sl.ms[n], cudaStreamNonBlocking);
        if (e != cudaSuccess) break;
    }
    for (auto& sl : s->wslots) {
        if (e != cudaSuccess) break;
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
    }
    if (e != cudaSuccess) {
        rbki_server_destroy(s);
        cudaSetDevice(prev);
        return set_cuda_error(e, "server streams");
    }
    for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(slot_main, s, i);
    for (int i = 0; i < wave_threads; ++i) s->workers.emplace_back(wave_main, s, i);
    cudaSetDevice(prev);
    *out = s;
    return RBKI_OK;
}

rbki_status rbki_submit(rbki_server* s, const rbki_tensor* X, const rbki_params* prm, const rbki_tucker_out* out,
                        void* after_stream, uint64_t* ticket) {
    if (!s || !ticket) return set_error(RBKI_E_INVAL, "server / ticket is NULL");
    if (!out || !out->core) return set_error(RBKI_E_INVAL, "out->core is NULL");
    Plan pl;
    RBKI_TRY(make_plan(X, prm, pl));
    if (prm->flags & RBKI_FLAG_HOST_IO) return set_error(RBKI_E_UNSUPPORTED, "server requests use device buffers");
    for (int n = 0; n < pl.N; ++n)
        if (!out->factors[n]) return set_error(RBKI_E_INVAL, "out->factors[n] is NULL");
    size_t need = 0;
    bool wave = false;
    if (s->wave_max > 0) {
        // the batched path takes the request if rbki_tucker_batched supports it (its refusal
        // is not an error of this call: the message of the last error is put back)
        const std::string keep = rbki_last_error();
        wave = rbki_tucker_batched_workspace(1, X, prm, &need) == RBKI_OK;
        if (!wave) set_error(RBKI_OK, keep.c_str());
    }
    if (!wave) {
        carve(pl, nullptr);
        need = pl.ws_bytes;
    }
    if (need > s->budget) return set_error(RBKI_E_NOMEM, "request workspace exceeds the server budget");
    Request* r = new Request();
    r->wave = wave;
    if (after_stream) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s->device);
        cudaError_t e = cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(r->ready, (cudaStream_t)after_stream);
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            if (r->ready) cudaEventDestroy(r->ready);
            delete r;
            return set_cuda_error(e, "rbki_submit: event on after_stream");
        }
    }
    r->X = *X;
    r->prm = *prm;
    r->out = *out;
    r->ws_bytes = need;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            if (r->ready) cudaEventDestroy(r->ready);
            delete r;
            return set_error(RBKI_E_BUSY, "server is shutting down");
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        (r->wave ? s->wqueue : s->queue).push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_all();
    return RBKI_OK;
}

rbki_status rbki_poll(rbki_server* s, uint64_t ticket, rbki_status* result, double* latency_s) {
    if (!s) return set_error(RBKI_E_INVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(RBKI_E_NOTFOUND, "unknown or already retired ticket");
    Request* r = it->second;
    if (r->state != State::DONE) {
        if (result) *result = RBKI_PENDING;
        return RBKI_PENDING;
    }
    if (result) *result = r->result;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    s->reqs.erase(it);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
    return RBKI_OK;
}

rbki_status rbki_cancel(rbki_server* s, uint64_t ticket) {
    if (!s) return set_error(RBKI_E_INVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return set_error(RBKI_E_NOTFOUND, "unknown or already retired ticket");
        Request* r = it->second;
        if (r->state == State::QUEUED) {
            auto& dq = r->wave ? s->wqueue : s->queue;
            for (auto q = dq.begin(); q != dq.end(); ++q)
                if (*q == r) {
                    dq.erase(q);
                    break;
                }
            r->state = State::DONE;
            r->result = RBKI_E_CANCELLED;
            r->t_done = now_s();
        } else if (r->state == State::RUNNING) {
            r->cancel = true;   // its kernels finish; the result is reported as cancelled
        }
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    return RBKI_OK;
}

rbki_status rbki_server_drain(rbki_server* s, double timeout_s) {
    if (!s) return set_error(RBKI_E_INVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] { return s->queue.empty() && s->wqueue.empty() && s->running == 0; };
    if (timeout_s < 0) {
        s->cv_done.wait(lk, idle);
        return RBKI_OK;
    }
    if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), idle))
        return set_error(RBKI_E_TIMEOUT, "drain: requests still queued or running");
    return RBKI_OK;
}

rbki_status rbki_server_destroy(rbki_server* s) {
    if (!s) return set_error(RBKI_E_INVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (auto* dq : {&s->queue, &s->wqueue}) {
            for (Request* r : *dq) {
                r->state = State::DONE;
                r->result = RBKI_E_CANCELLED;
            }
            dq->clear();
        }
    }
    s->cv_work.notify_all();
    for (auto& w : s->workers) w.join();   // running requests finish first
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto* v : {&s->slots, &s->wslots})
        for (auto& sl : *v) {
            if (sl.st) cudaStreamDestroy(sl.st);
            for (auto m : sl.ms)
                if (m) cudaStreamDestroy(m);
        }
    if (s->arena_base) cudaFree(s->arena_base);
    cudaSetDevice(prev);
    for (auto& kv : s->reqs) {
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    delete s->arena;
    delete s;
    return RBKI_OK;
}

}  // extern "C"

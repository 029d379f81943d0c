// server.cpp -- continuous-batching serving loop for median-filter requests.
//
// Requests (2D images of any size, dtype and radius) are queued by
// hrm_submit.  A background thread admits them while their bytes fit the
// device-memory budget (the caller's arena) and fewer than max_inflight are
// admitted, then launches every admitted-but-unlaunched request as one wave:
// host inputs are copied into the arena, all requests of the wave run in one
// persistent batched kernel (hrm_filter_batch), host outputs are copied back,
// and a host callback marks the wave's requests done.  Waves alternate
// between two compute streams, so a request that arrives while earlier waves
// are on the GPU is admitted as memory frees up and its work overlaps theirs.
//
// Frame streams (requests naming a topology) keep their submission order:
// a wave holds at most one frame of each stream, and a wave that follows the
// stream's previous frame on the other compute stream waits for that wave.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/hrm.h"

namespace hrm {
int topology_device_of(const hrm_topology* t);  // api.cu
int fail(int code, const std::string& msg);     // api.cu: sets hrm_last_error, returns code
}
using hrm::fail;

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granules.
class Arena {
public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t n, size_t* off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

enum State { QUEUED, ADMITTED, RUNNING, DONE };

struct Req {
    uint64_t ticket = 0;
    hrm_request q{};
    State state = QUEUED;
    int status = HRM_OK;
    size_t budget = 0;              // bytes charged against the budget
    size_t off_in = 0, off_out = 0; // arena offsets of host-buffer copies
    bool has_in = false, has_out = false;
    Clock::time_point t_submit, t_done;
};

struct Wave;

}  // namespace

struct hrm_server {
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    Arena alloc{0};
    int max_inflight = 0, max_queue = 0;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;
    std::vector<Req*> admitted;
    std::unordered_map<uint64_t, Req*> live;
    std::unordered_map<uint64_t, double> retired_latency;
    std::deque<uint64_t> retired_order;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread th;
    cudaStream_t s_copy = nullptr, s_comp[2] = {nullptr, nullptr};
    cudaEvent_t wave_end[2] = {nullptr, nullptr};  // end of the last wave on each compute stream
    std::unordered_map<hrm_topology*, int> topo_stream;  // compute stream of a topology's last frame
    int parity = 0;
    int inflight = 0;
    size_t resident = 0, high_water = 0;
    uint64_t submitted = 0, admitted_n = 0, completed = 0, rejected = 0, waves = 0;
};

namespace {

struct Wave {
    hrm_server* s;
    std::vector<Req*> reqs;
};

size_t elem_size(int dtype) { return dtype == HRM_U16 ? 2 : 1; }

void CUDART_CB wave_done(void* p) {
    Wave* w = (Wave*)p;
    hrm_server* s = w->s;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto now = Clock::now();
        for (Req* r : w->reqs) {
            r->state = DONE;
            r->t_done = now;
            if (r->has_in) s->alloc.release(r->off_in, r->budget / 2);
            if (r->has_out) s->alloc.release(r->off_out, r->budget / 2);
            s->resident -= r->budget;
            s->inflight--;
            s->completed++;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    delete w;
}

// Launch every admitted request as one wave (called without the lock held).
void launch_wave(hrm_server* s, std::vector<Req*>& batch) {
    const int mine = s->parity;
    cudaStream_t cs = s->s_comp[mine];
    s->parity ^= 1;
    std::vector<hrm_job> jobs;
    jobs.reserve(batch.size());
    cudaError_t e = cudaSuccess;
    bool copied = false;
    // a frame whose stream last ran on the other compute stream reads the
    // topology that wave rewrites: wait for it
    bool wait_other = false;
    for (Req* r : batch) {
        if (!r->q.topo) continue;
        auto it = s->topo_stream.find(r->q.topo);
        if (it != s->topo_stream.end() && it->second != mine) wait_other = true;
        s->topo_stream[r->q.topo] = mine;
    }
    if (wait_other) e = cudaStreamWaitEvent(cs, s->wave_end[mine ^ 1], 0);
    for (Req* r : batch) {
        const hrm_request& q = r->q;
        const size_t es = elem_size(q.dtype), row = (size_t)q.width * es;
        hrm_job j{};
        j.dtype = q.dtype;
        j.dims = 2;
        j.width = q.width;
        j.height = q.height;
        j.depth = 1;
        j.radius = q.radius;
        j.rank = -1;
        j.flags = q.flags;
        j.topo = q.topo;
        if (r->has_in) {
            j.src = s->arena + r->off_in;
            j.src_pitch = row;
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(s->arena + r->off_in, row, q.src, q.src_pitch, row, q.height,
                                      cudaMemcpyHostToDevice, s->s_copy);
            copied = true;
        } else {
            j.src = q.src;
            j.src_pitch = q.src_pitch;
        }
        if (r->has_out) {
            j.dst = s->arena + r->off_out;
            j.dst_pitch = row;
        } else {
            j.dst = q.dst;
            j.dst_pitch = q.dst_pitch;
        }
        jobs.push_back(j);
    }
    cudaEvent_t ev = nullptr;
    if (copied && e == cudaSuccess) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, s->s_copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
    }
    int rc = e == cudaSuccess ? hrm_filter_batch(jobs.data(), (int)jobs.size(), cs) : HRM_ECUDA;
    for (size_t i = 0; rc == HRM_OK && i < batch.size(); ++i) {
        Req* r = batch[i];
        if (!r->has_out) continue;
        const size_t row = (size_t)r->q.width * elem_size(r->q.dtype);
        e = cudaMemcpy2DAsync(r->q.dst, r->q.dst_pitch, s->arena + r->off_out, row, row, r->q.height,
                              cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) rc = HRM_ECUDA;
    }
    if (ev) cudaEventDestroy(ev);  // safe: destruction is deferred until the event completes
    if (rc == HRM_OK && cudaEventRecord(s->wave_end[mine], cs) != cudaSuccess) rc = HRM_ECUDA;
    Wave* w = new Wave{s, batch};
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Req* r : batch) {
            r->state = RUNNING;
            if (rc != HRM_OK) r->status = rc;
        }
        s->waves++;
    }
    if (cudaLaunchHostFunc(cs, wave_done, w) != cudaSuccess) {
        cudaStreamSynchronize(cs);
        wave_done(w);
    }
}

void server_loop(hrm_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // admission: by memory budget and in-flight slots, in arrival order
        while (!s->queue.empty() && s->inflight < s->max_inflight) {
            Req* r = s->queue.front();
            const hrm_request& q = r->q;
            const size_t bytes = (size_t)q.width * q.height * elem_size(q.dtype);
            bool ok = true;
            if (s->resident + 2 * bytes > s->arena_bytes) ok = false;
            if (ok && q.src_on_host) {
                ok = s->alloc.alloc(bytes, &r->off_in);
                r->has_in = ok;
            }
            if (ok && q.dst_on_host) {
                ok = s->alloc.alloc(bytes, &r->off_out);
                r->has_out = ok;
                if (!ok && r->has_in) {
                    s->alloc.release(r->off_in, bytes);
                    r->has_in = false;
                }
            }
            if (!ok) break;  // wait for memory to free up (no reordering: large requests do not starve)
            r->budget = 2 * bytes;
            s->resident += r->budget;
            s->high_water = std::max(s->high_water, s->resident);
            s->inflight++;
            s->admitted_n++;
            r->state = ADMITTED;
            s->queue.pop_front();
            s->admitted.push_back(r);
        }
        if (!s->admitted.empty()) {
            // one frame per stream and wave; later frames wait for the next wave
            std::vector<Req*> batch, later;
            std::unordered_set<hrm_topology*> frames;
            for (Req* r : s->admitted) {
                if (r->q.topo && !frames.insert(r->q.topo).second) later.push_back(r);
                else batch.push_back(r);
            }
            s->admitted.swap(later);
            lk.unlock();
            launch_wave(s, batch);
            lk.lock();
            continue;
        }
        if (s->stop) break;
        s->cv_work.wait(lk);
    }
}

}  // namespace

extern "C" {

int hrm_server_create(void* arena_dev_ptr, size_t arena_bytes, int max_inflight, int max_queue,
                      hrm_server** out) {
    if (!out) return fail(HRM_EINVAL, "hrm_server_create: null output pointer");
    if (!arena_dev_ptr || arena_bytes == 0) return fail(HRM_EINVAL, "hrm_server_create: empty arena");
    if (max_inflight <= 0 || max_queue < 0)
        return fail(HRM_EINVAL, "hrm_server_create: max_inflight must be > 0 and max_queue >= 0");
    auto* s = new hrm_server();
    s->arena = (unsigned char*)arena_dev_ptr;
    s->arena_bytes = arena_bytes;
    s->alloc = Arena(arena_bytes);
    s->max_inflight = max_inflight;
    s->max_queue = max_queue ? max_queue : 4096;
    cudaGetDevice(&s->device);
    if (cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->s_comp[0], cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->s_comp[1], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->wave_end[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->wave_end[1], cudaEventDisableTiming) != cudaSuccess) {
        for (cudaStream_t st : {s->s_copy, s->s_comp[0], s->s_comp[1]})
            if (st) cudaStreamDestroy(st);
        for (cudaEvent_t ev : s->wave_end)
            if (ev) cudaEventDestroy(ev);
        delete s;
        const cudaError_t e = cudaGetLastError();
        return fail(HRM_ECUDA, std::string("hrm_server_create: stream or event creation failed: ") +
                                   cudaGetErrorString(e));
    }
    s->th = std::thread(server_loop, s);
    *out = s;
    return HRM_OK;
}

int hrm_submit(hrm_server* s, const hrm_request* q, uint64_t* ticket) {
    if (!s || !q || !ticket) return fail(HRM_EINVAL, "hrm_submit: null server, request or ticket pointer");
    const size_t es = (q->dtype == HRM_U16) ? 2 : 1;
    const bool bad = (q->dtype != HRM_U8 && q->dtype != HRM_U16) || q->width <= 0 || q->height <= 0 ||
                     q->radius < 0 || q->radius > HRM_MAX_RADIUS_2D || (q->flags & ~(unsigned)HRM_ADAPTIVE) ||
                     !q->src || !q->dst || q->src_pitch < (size_t)q->width * es ||
                     q->dst_pitch < (size_t)q->width * es ||
                     (q->topo && (q->flags || hrm::topology_device_of(q->topo) != s->device));
    std::lock_guard<std::mutex> lk(s->mu);
    if (bad) {
        s->rejected++;
        return fail(HRM_EINVAL, "hrm_submit: malformed request (dtype, size, radius, flags, pointers, pitches "
                                "or topology)");
    }
    if (2 * (size_t)q->width * q->height * es > s->arena_bytes) {
        s->rejected++;
        return fail(HRM_EINVAL, "hrm_submit: the request's input and output never fit the arena");
    }
    if ((int)s->queue.size() >= s->max_queue) return fail(HRM_EAGAIN, "hrm_submit: submit queue full");
    Req* r = new Req();
    r->ticket = s->next_ticket++;
    r->q = *q;
    r->t_submit = Clock::now();
    s->live[r->ticket] = r;
    s->queue.push_back(r);
    s->submitted++;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return HRM_OK;
}

static int retire(hrm_server* s, Req* r) {
    const int st = r->status;
    const double us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
    s->retired_latency[r->ticket] = us;
    s->retired_order.push_back(r->ticket);
    while (s->retired_order.size() > 1000000) {
        s->retired_latency.erase(s->retired_order.front());
        s->retired_order.pop_front();
    }
    s->live.erase(r->ticket);
    delete r;
    return st;
}

int hrm_poll(hrm_server* s, uint64_t ticket, int timeout_us) {
    if (!s) return fail(HRM_EINVAL, "hrm_poll: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->live.find(ticket);
    if (it == s->live.end()) return fail(HRM_EINVAL, "hrm_poll: unknown or retired ticket");
    Req* r = it->second;
    if (r->state != DONE) {
        if (timeout_us == 0) return fail(HRM_EAGAIN, "hrm_poll: request still pending");
        auto pred = [&] { return r->state == DONE; };
        if (timeout_us < 0) s->cv_done.wait(lk, pred);
        else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
            return fail(HRM_ETIMEDOUT, "hrm_poll: request still pending after the timeout");
    }
    const int st = retire(s, r);
    if (st == HRM_ECANCELED) return fail(st, "hrm_poll: request cancelled (server destroyed)");
    if (st != HRM_OK) return fail(st, "hrm_poll: the request's wave failed with status " + std::to_string(st));
    return st;
}

double hrm_ticket_latency_us(hrm_server* s, uint64_t ticket) {
    if (!s) return -1.0;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->retired_latency.find(ticket);
    return it == s->retired_latency.end() ? -1.0 : it->second;
}

int hrm_server_stats_get(hrm_server* s, hrm_server_stats* o) {
    if (!s || !o) return fail(HRM_EINVAL, "hrm_server_stats_get: null server or output pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    o->submitted = s->submitted;
    o->admitted = s->admitted_n;
    o->completed = s->completed;
    o->rejected = s->rejected;
    o->waves = s->waves;
    o->bytes_resident = s->resident;
    o->bytes_high_water = s->high_water;
    o->arena_bytes = s->arena_bytes;
    o->inflight = s->inflight;
    o->queued = (int)s->queue.size();
    return HRM_OK;
}

int hrm_server_destroy(hrm_server* s) {
    if (!s) return HRM_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Req* r : s->queue) {  // never admitted: cancelled
            r->state = DONE;
            r->status = HRM_ECANCELED;
            r->t_done = Clock::now();
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaStreamSynchronize(s->s_copy);
    cudaStreamSynchronize(s->s_comp[0]);
    cudaStreamSynchronize(s->s_comp[1]);
    cudaStreamDestroy(s->s_copy);
    cudaStreamDestroy(s->s_comp[0]);
    cudaStreamDestroy(s->s_comp[1]);
    cudaEventDestroy(s->wave_end[0]);
    cudaEventDestroy(s->wave_end[1]);
    for (auto& kv : s->live) delete kv.second;
    delete s;
    return HRM_OK;
}

}  // extern "C"

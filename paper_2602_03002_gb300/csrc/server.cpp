// server.cpp -- continuous-batching render server (rpl_server_* in include/rpl.h).
//
// Trainers submit render requests (a view, a step, pose and depth buffers) from any thread.  A
// worker thread admits waiting requests in arrival order whenever a stream slot is free, skipping
// (without reordering) requests whose view already has work on the GPU or whose host-buffer
// staging does not fit the device budget, fuses the admitted ones into one launch -- one prep
// launch per request, then one render launch over the tiles of all of them -- and completes them
// when the launch's event has passed.  Batches on different slots overlap on the device, so
// requests that arrive while others run are admitted as soon as a slot and memory free up.
// Inside a fused launch the requests are ordered by size, smallest first, and a request whose
// buffers are on the device completes as soon as its own tiles are done: the kernel counts them off
// and raises a flag in host-mapped memory that the worker polls, so a small request fused with a
// large one does not wait for the large one.
// The slots' streams are non-blocking, so at submit time the server records an event on the legacy
// default stream and the request's launch waits for it: the request sees the poses and output
// memory as work already queued on that stream left them (a producer kernel, a caching allocator
// handing the memory out again).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/rpl.h"
#include "render.h"
#include "scene_access.h"

using namespace rpl;

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kAlign = 256;

size_t round_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over the byte range [0, size) of the staging arena.
class Arena {
public:
    void reset(size_t size) {
        free_.clear();
        if (size) free_[0] = size;
        used_ = 0;
    }
    bool alloc(size_t n, size_t *off) {
        n = round_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, start = it->first + n;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += n;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round_up(n);
        used_ -= n;
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
    size_t used() const { return used_; }

private:
    std::map<size_t, size_t> free_;   // offset -> length of free ranges
    size_t used_ = 0;
};

constexpr size_t kNone = ~(size_t)0;

struct Request {
    uint64_t id = 0;
    rpl_view *view = nullptr;
    const float *poses = nullptr;
    void *out = nullptr;
    int64_t step = 0, env_offset = 0;
    bool poses_host = false, out_host = false;
    size_t pose_bytes = 0, out_bytes = 0, pose_off = kNone, out_off = kNone;
    Clock::time_point t_submit, t_done;
    rpl_status status = RPL_OK;
    std::string err;
    bool done = false, cancelled = false;
    bool early = false;   // completes by its own flag inside the fused launch
    bool waiting = false; // a thread is blocked in rpl_server_wait on it (it then owns the deletion)
    cudaEvent_t ready = nullptr;   // recorded on the legacy default stream at submit (borrowed from the pool)
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    RenderParams *h_params = nullptr;   // pinned
    int64_t *h_prefix = nullptr;        // pinned
    RenderParams *d_params = nullptr;
    int64_t *d_prefix = nullptr;
    int32_t *h_flags = nullptr;         // pinned, mapped: per-request completion flags
    int32_t *d_flags = nullptr;         // device address of h_flags
    int32_t *h_remaining = nullptr;     // pinned: tiles per request
    int32_t *d_remaining = nullptr;     // device: tiles still running per request
    bool busy = false;
    std::vector<Request *> reqs;
};

}  // namespace

struct rpl_server {
    rpl_scene *scene = nullptr;
    int device = 0;
    int bvh_kind = RPL_BVH2;
    rpl_server_opts opts{};
    unsigned char *arena_dev = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> tickets;
    std::unordered_map<rpl_view *, int64_t> last_submitted;
    std::unordered_set<rpl_view *> on_gpu;   // views with a request in a busy slot
    uint64_t next_id = 1;
    bool stop = false;
    int inflight = 0;
    rpl_server_stats stats{};
    bool registered = false;   // counted as a user of the scene
    std::thread worker;
    std::mutex ev_mu;                     // guards the event pool (taken without mu)
    std::vector<cudaEvent_t> ev_all, ev_free;
};

namespace {

// Borrows an event from the server's pool (creating one if the pool is empty); the caller has set
// the server's device.
cudaError_t take_event(rpl_server *sv, cudaEvent_t *ev) {
    std::lock_guard<std::mutex> lk(sv->ev_mu);
    if (!sv->ev_free.empty()) {
        *ev = sv->ev_free.back();
        sv->ev_free.pop_back();
        return cudaSuccess;
    }
    cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) sv->ev_all.push_back(*ev);
    return e;
}

// Returns a request's event to the pool once a wait on it has been queued (a later record does not
// change what that wait waits for).
void give_event(rpl_server *sv, Request *r) {
    if (!r->ready) return;
    std::lock_guard<std::mutex> lk(sv->ev_mu);
    sv->ev_free.push_back(r->ready);
    r->ready = nullptr;
}

// Fills slot s with the admitted batch and launches it (called without the server lock).
void launch_batch(rpl_server *sv, Slot &s) {
    nvtxRangePushA("rpl_server_batch");
    cudaStream_t st = s.stream;
    const int n = (int)s.reqs.size();
    for (int i = 0; i < n; ++i) {   // after the work queued on the legacy default stream before submit
        Request *r = s.reqs[i];
        if (!r->ready) continue;
        const cudaError_t e = cudaStreamWaitEvent(st, r->ready, 0);
        give_event(sv, r);
        if (e != cudaSuccess) {
            r->status = RPL_ERR_CUDA;
            r->err = cudaGetErrorString(e);
        }
    }
    std::vector<RenderParams> prm(n);
    std::vector<int64_t> tiles(n, 0);
    for (int i = 0; i < n; ++i) {
        Request *r = s.reqs[i];
        if (r->status != RPL_OK) continue;
        const float *pd = r->poses_host ? reinterpret_cast<const float *>(sv->arena_dev + r->pose_off) : r->poses;
        void *od = r->out_host ? (void *)(sv->arena_dev + r->out_off) : r->out;
        if (r->poses_host) {
            cudaError_t e = cudaMemcpyAsync(const_cast<float *>(pd), r->poses, r->pose_bytes, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) {
                r->status = RPL_ERR_CUDA;
                r->err = cudaGetErrorString(e);
                continue;
            }
        }
        int64_t warps = 0;
        rpl_status stt = view_prepare(r->view, pd, r->step, r->env_offset, od, st, &prm[i], &warps);
        if (stt != RPL_OK) {
            r->status = stt;
            r->err = rpl_last_error();
            continue;
        }
        view_commit(r->view, r->step, st);
        tiles[i] = warps;
    }
    // smallest requests first: the launch's warps run roughly in order, so they finish early
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return tiles[a] < tiles[b]; });
    std::vector<Request *> sorted(n);
    int64_t total = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        Request *r = s.reqs[i];
        sorted[k] = r;
        s.h_params[k] = prm[i];
        s.h_prefix[k] = total;
        total += tiles[i];
        // a request with device buffers and no downsampled camera completes by its own flag
        r->early = r->status == RPL_OK && !r->out_host && prm[i].raw_per_env == 0 && tiles[i] > 0;
        s.h_flags[k] = 0;
        s.h_remaining[k] = (int32_t)tiles[i];
        s.h_params[k].done_counter = r->early ? s.d_remaining + k : nullptr;
        s.h_params[k].done_flag = r->early ? s.d_flags + k : nullptr;
    }
    s.reqs = sorted;
    s.h_prefix[n] = total;
    cudaError_t e = cudaMemcpyAsync(s.d_params, s.h_params, (size_t)n * sizeof(RenderParams), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.d_prefix, s.h_prefix, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s.d_remaining, s.h_remaining, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_render_multi(s.d_params, s.d_prefix, n, total, sv->bvh_kind, sv->opts.min_blocks,
                                sv->opts.persistent != 0, st);
    for (int i = 0; i < n && e == cudaSuccess; ++i)   // downsampled cameras of a request: average + sensor
        if (s.reqs[i]->status == RPL_OK && s.h_params[i].raw_per_env > 0) e = launch_downsample(s.h_params[i], st);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        Request *r = s.reqs[i];
        if (r->out_host && r->status == RPL_OK)
            e = cudaMemcpyAsync(r->out, sv->arena_dev + r->out_off, r->out_bytes, cudaMemcpyDeviceToHost, st);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i)   // rpl_sync / rpl_view_destroy of a view wait for this
        if (s.reqs[i]->status == RPL_OK) view_mark_done(s.reqs[i]->view, st);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, st);
    if (e != cudaSuccess) {
        for (Request *r : s.reqs) {
            r->early = false;   // completes with the batch, carrying the error
            if (r->status == RPL_OK) {
                r->status = RPL_ERR_CUDA;
                r->err = cudaGetErrorString(e);
            }
        }
        cudaStreamSynchronize(st);   // let anything that did launch finish before the slot is reused
        cudaGetLastError();
        cudaEventRecord(s.done, st);
    }
    nvtxRangePop();
}

void release_staging(rpl_server *sv, Request *r) {
    if (r->pose_off != kNone) sv->arena.release(r->pose_off, r->pose_bytes);
    if (r->out_off != kNone) sv->arena.release(r->out_off, r->out_bytes);
    r->pose_off = r->out_off = kNone;
}

// Marks r done (lock held); a cancelled request is forgotten right away.
void finish(rpl_server *sv, Request *r, Clock::time_point now) {
    r->done = true;
    r->t_done = now;
    if (r->status == RPL_OK)
        sv->stats.completed++;
    else
        sv->stats.failed++;
    if (r->cancelled && !r->waiting) {   // a waiter, woken by cv_done, deletes it instead
        sv->tickets.erase(r->id);
        delete r;
    }
}

// Completes the requests whose own flag is up and the batches whose event has passed (lock held).
// An early-completed request leaves the slot's list (its caller may free it once waited for).
void poll_slots(rpl_server *sv) {
    bool any = false;
    for (Slot &s : sv->slots) {
        if (!s.busy) continue;
        for (size_t k = 0; k < s.reqs.size(); ++k) {
            Request *r = s.reqs[k];
            if (!r || !r->early || r->cancelled) continue;
            if (*reinterpret_cast<volatile int32_t *>(s.h_flags + k) == 0) continue;
            sv->on_gpu.erase(r->view);   // its tiles are done: the view may take its next request
            release_staging(sv, r);      // staged poses were consumed by the prep kernel
            finish(sv, r, Clock::now());
            s.reqs[k] = nullptr;
            any = true;
        }
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        const Clock::time_point now = Clock::now();
        for (Request *r : s.reqs) {
            if (!r) continue;
            if (q != cudaSuccess && r->status == RPL_OK) {
                r->status = RPL_ERR_CUDA;
                r->err = cudaGetErrorString(q);
            }
            release_staging(sv, r);
            sv->on_gpu.erase(r->view);
            finish(sv, r, now);
        }
        if (q != cudaSuccess) cudaGetLastError();
        s.reqs.clear();
        s.busy = false;
        sv->inflight--;
        any = true;
    }
    if (any) sv->cv_done.notify_all();
}

void worker_main(rpl_server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        poll_slots(sv);
        if (sv->stop) {
            // fail what never reached the GPU, then drain the slots
            const Clock::time_point now = Clock::now();
            while (!sv->queue.empty()) {
                Request *r = sv->queue.front();
                sv->queue.pop_front();
                r->status = RPL_ERR_INVALID_ARG;
                r->err = "rpl_server: the server was destroyed before the request was admitted";
                finish(sv, r, now);
            }
            sv->cv_done.notify_all();
            if (sv->inflight == 0) break;
            sv->cv_work.wait_for(lk, std::chrono::microseconds(100));
            continue;
        }
        int free_slot = -1;
        for (size_t i = 0; i < sv->slots.size(); ++i)
            if (!sv->slots[i].busy) {
                free_slot = (int)i;
                break;
            }
        if (free_slot >= 0 && !sv->queue.empty()) {
            Slot &s = sv->slots[free_slot];
            std::unordered_set<rpl_view *> blocked;   // views whose earlier request waits: keep their order
            for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)s.reqs.size() < sv->opts.max_batch;) {
                Request *r = *it;
                if (blocked.count(r->view) || sv->on_gpu.count(r->view)) {
                    blocked.insert(r->view);
                    ++it;
                    continue;
                }
                bool ok = true;
                if (r->poses_host && !sv->arena.alloc(r->pose_bytes, &r->pose_off)) ok = false;
                if (ok && r->out_host && !sv->arena.alloc(r->out_bytes, &r->out_off)) ok = false;
                if (!ok) {
                    release_staging(sv, r);
                    blocked.insert(r->view);
                    ++it;
                    continue;
                }
                sv->on_gpu.insert(r->view);
                s.reqs.push_back(r);
                it = sv->queue.erase(it);
            }
            if (!s.reqs.empty()) {
                s.busy = true;
                sv->inflight++;
                sv->stats.batches++;
                sv->stats.fused_requests += s.reqs.size();
                sv->stats.max_batch_seen = std::max(sv->stats.max_batch_seen, (int32_t)s.reqs.size());
                sv->stats.max_inflight_batches_seen = std::max(sv->stats.max_inflight_batches_seen, (int32_t)sv->inflight);
                sv->stats.staging_peak_bytes = std::max(sv->stats.staging_peak_bytes, (int64_t)sv->arena.used());
                lk.unlock();
                launch_batch(sv, s);
                lk.lock();
                continue;
            }
        }
        if (sv->inflight > 0)
            sv->cv_work.wait_for(lk, std::chrono::microseconds(100));   // poll the busy slots' events
        else
            sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
    }
}

rpl_status server_fail(rpl_status st, const std::string &msg) { return set_error(st, msg.c_str()); }

}  // namespace

extern "C" {

RPL_API rpl_status rpl_server_create(rpl_scene_t scene, const rpl_server_opts *opts, rpl_server_t *out) {
    if (!out) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_create: out is NULL");
    *out = nullptr;
    SceneInputs si;
    if (!scene_inputs(scene, &si))
        return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_create: scene is NULL or not frozen (create a view first)");
    rpl_server_opts o{};
    if (opts) o = *opts;
    if (o.max_batch == 0) o.max_batch = 32;
    if (o.n_streams == 0) o.n_streams = 2;
    if (o.staging_bytes == 0) o.staging_bytes = (int64_t)256 << 20;
    if (o.min_blocks == 0) o.min_blocks = 8;
    if (o.max_batch < 1 || o.max_batch > 64 || o.n_streams < 1 || o.n_streams > 8 || o.staging_bytes < 0 ||
        (o.min_blocks != 8 && o.min_blocks != 10 && o.min_blocks != 12))
        return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_create: max_batch 1..64, n_streams 1..8, "
                                                "staging_bytes >= 0, min_blocks 8, 10 or 12");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(si.device);
    rpl_server *sv = new (std::nothrow) rpl_server();
    if (!sv) return server_fail(RPL_ERR_OUT_OF_MEMORY, "rpl_server_create: host allocation");
    sv->scene = scene;
    sv->device = si.device;
    sv->bvh_kind = si.bvh_kind;
    sv->opts = o;
    cudaError_t e = cudaMalloc(&sv->arena_dev, std::max<size_t>((size_t)o.staging_bytes, kAlign));
    sv->arena.reset((size_t)o.staging_bytes);
    sv->slots.resize(o.n_streams);
    for (Slot &s : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaHostAlloc(&s.h_params, o.max_batch * sizeof(RenderParams), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&s.h_prefix, (o.max_batch + 1) * sizeof(int64_t), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_params, o.max_batch * sizeof(RenderParams));
        if (e == cudaSuccess) e = cudaMalloc(&s.d_prefix, (o.max_batch + 1) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaHostAlloc(&s.h_flags, o.max_batch * sizeof(int32_t), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&s.d_flags, s.h_flags, 0);
        if (e == cudaSuccess) e = cudaHostAlloc(&s.h_remaining, o.max_batch * sizeof(int32_t), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaMalloc(&s.d_remaining, o.max_batch * sizeof(int32_t));
    }
    if (e != cudaSuccess) {
        rpl_server_destroy(sv);
        if (prev >= 0) cudaSetDevice(prev);
        return server_fail(e == cudaErrorMemoryAllocation ? RPL_ERR_OUT_OF_MEMORY : RPL_ERR_CUDA,
                           std::string("rpl_server_create: ") + cudaGetErrorString(e));
    }
    scene_add_server(scene);
    sv->registered = true;
    sv->worker = std::thread(worker_main, sv);
    if (prev >= 0) cudaSetDevice(prev);
    *out = sv;
    return RPL_OK;
}

RPL_API rpl_status rpl_server_submit(rpl_server_t sv, rpl_view_t view, const float *poses, int64_t step,
                                     int64_t env_offset, void *out, uint64_t *ticket) {
    if (!sv || !view || !ticket) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_submit: NULL argument");
    if (view_scene(view) != sv->scene)
        return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_submit: the view belongs to another scene");
    rpl_status st = view_validate(view, poses, env_offset, out);
    if (st != RPL_OK) return st;
    Request *r = new (std::nothrow) Request();
    if (!r) return server_fail(RPL_ERR_OUT_OF_MEMORY, "rpl_server_submit: host allocation");
    r->view = view;
    r->poses = poses;
    r->out = out;
    r->step = step;
    r->env_offset = env_offset;
    r->pose_bytes = view_pose_bytes(view);
    r->out_bytes = view_out_bytes(view);
    {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(sv->device);
        r->poses_host = view_envs(view) > 0 && !pointer_on_device(poses, sv->device);
        r->out_host = view_envs(view) > 0 && !pointer_on_device(out, sv->device);
        cudaError_t e = cudaSuccess;
        if (view_envs(view) > 0) {
            e = take_event(sv, &r->ready);
            if (e == cudaSuccess) e = cudaEventRecord(r->ready, cudaStreamLegacy);
        }
        if (prev >= 0) cudaSetDevice(prev);
        if (e != cudaSuccess) {
            give_event(sv, r);
            delete r;
            return server_fail(RPL_ERR_CUDA, std::string("rpl_server_submit: ") + cudaGetErrorString(e));
        }
    }
    const size_t staging = (r->poses_host ? round_up(r->pose_bytes) : 0) + (r->out_host ? round_up(r->out_bytes) : 0);
    if (staging > (size_t)sv->opts.staging_bytes) {
        give_event(sv, r);
        delete r;
        return server_fail(RPL_ERR_CAPACITY, "rpl_server_submit: the request's host-buffer staging exceeds the "
                                             "server's whole staging budget");
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            give_event(sv, r);
            delete r;
            return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_submit: the server is stopping");
        }
        auto it = sv->last_submitted.find(view);
        const bool order_ok = it != sv->last_submitted.end() ? (step == it->second || step == it->second + 1)
                                                             : view_step_allowed(view, step);
        if (!order_ok) {
            give_event(sv, r);
            delete r;
            return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_submit: a view's steps must advance by 0 or 1");
        }
        r->id = sv->next_id++;
        sv->last_submitted[view] = step;
        sv->stats.submitted++;
        sv->tickets[r->id] = r;
        if (view_envs(view) == 0) {
            finish(sv, r, Clock::now());   // nothing to render
        } else {
            sv->queue.push_back(r);
        }
        *ticket = r->id;
    }
    sv->cv_work.notify_one();
    return RPL_OK;
}

RPL_API rpl_status rpl_server_wait(rpl_server_t sv, uint64_t ticket, int32_t timeout_ms, double *latency_s) {
    if (!sv) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_wait: server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end() || it->second->cancelled)
        return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_wait: unknown ticket");
    Request *r = it->second;
    if (r->waiting) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_wait: another thread waits on this ticket");
    r->waiting = true;
    auto pred = [&] { return r->done; };
    bool done = true;
    if (timeout_ms < 0)
        sv->cv_done.wait(lk, pred);
    else
        done = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred);
    r->waiting = false;
    if (r->cancelled) {
        // cancelled by another thread while this one waited: forget it once it has rendered
        if (r->done) {
            sv->tickets.erase(r->id);
            delete r;
        }
        return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_wait: the request was cancelled");
    }
    if (!done) return server_fail(RPL_ERR_TIMEOUT, "rpl_server_wait: the request is still pending");
    const rpl_status st = r->status;
    const std::string err = r->err;
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    sv->tickets.erase(r->id);
    delete r;
    if (st != RPL_OK) return server_fail(st, err);
    return RPL_OK;
}

RPL_API rpl_status rpl_server_cancel(rpl_server_t sv, uint64_t ticket) {
    if (!sv) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_cancel: server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_cancel: unknown ticket");
    Request *r = it->second;
    sv->stats.cancelled++;
    if (r->done) {
        sv->tickets.erase(it);
        delete r;
    } else {
        r->cancelled = true;   // it still renders (the view's step sequence stays whole), then is forgotten
    }
    return RPL_OK;
}

RPL_API rpl_status rpl_server_stats_get(rpl_server_t sv, rpl_server_stats *stats) {
    if (!sv || !stats) return server_fail(RPL_ERR_INVALID_ARG, "rpl_server_stats_get: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *stats = sv->stats;
    return RPL_OK;
}

RPL_API void rpl_server_destroy(rpl_server_t sv) {
    if (!sv) return;
    if (sv->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stop = true;
        }
        sv->cv_work.notify_all();
        sv->worker.join();
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(sv->device);
    for (Slot &s : sv->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_params) cudaFreeHost(s.h_params);
        if (s.h_prefix) cudaFreeHost(s.h_prefix);
        if (s.d_params) cudaFree(s.d_params);
        if (s.d_prefix) cudaFree(s.d_prefix);
        if (s.h_flags) cudaFreeHost(s.h_flags);
        if (s.h_remaining) cudaFreeHost(s.h_remaining);
        if (s.d_remaining) cudaFree(s.d_remaining);
    }
    if (sv->arena_dev) cudaFree(sv->arena_dev);
    for (auto &kv : sv->tickets) delete kv.second;
    for (cudaEvent_t ev : sv->ev_all) cudaEventDestroy(ev);
    if (prev >= 0) cudaSetDevice(prev);
    rpl_scene *scene = sv->registered ? sv->scene : nullptr;
    delete sv;
    if (scene) scene_remove_server(scene);
}

}  // extern "C"

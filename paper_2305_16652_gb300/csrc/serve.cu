// Serving loop: ray-query requests from many clients against resident
// scenes, run with continuous admission on one GPU.
//
// Each request names a resident scene (its BVH and cut stay on the device)
// and brings n rays in host memory.  A dispatcher thread owned by the server
// admits queued requests in arrival order whenever an execution slot is free
// and the request's device memory fits the budget.  An admitted request gets
// its buffers from a stream-ordered memory pool and its whole life is queued
// on its slot's stream: copy in, encode, sort, trace through the sorted ids
// (the reordering pipeline of Sec. 5), copy out, release.  Requests that
// arrive while others are running therefore start at once and their work
// overlaps on the device.  A host callback queued behind each request wakes
// the dispatcher, which confirms completion with the slot's event; latency
// runs from submission to that completion.
//
// Results do not depend on the mix: a request's kernels read only its own
// buffers, its slot's error word and the read-only scene data.
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

#include "hcc_internal.cuh"

namespace hcc {
// Device views of the opaque handles (hcc_api.cu).
void bvh_view(const hcc_bvh *b, SceneDesc *out, int *layout, int *device);
void cut_view(const hcc_cut *c, const float4 **boxes, uint32_t *on_device, int *device);
}  // namespace hcc

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    uint32_t scene = 0;
    int any_hit = 0;
    const float *org = nullptr, *dir = nullptr;
    uint64_t n = 0;
    hcc_hit *hits = nullptr;
    uint64_t bytes = 0;  // budget charge
    Clock::time_point submitted, finished;
    hcc_status status = HCC_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *d_err = nullptr;  // error word (16-byte allocation; the second half is the trace's slot counter)
    uint32_t *h_err = nullptr;  // page-locked copy of d_err, written by the request's last copy
    Request *req = nullptr;     // running request, nullptr = free
    hcc_server *owner = nullptr;
};

}  // namespace

struct hcc_server {
    int device = 0;
    int layout = 0;
    hcc_method method = HCC_METHOD_HCC;
    uint32_t key_bits = 32;
    std::vector<hcc::SceneDesc> scenes;
    std::vector<const float4 *> cut_boxes;
    std::vector<uint32_t> cut_used;
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;

    std::mutex mu;  // guards everything below
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request> reqs;  // element addresses stay valid across inserts
    uint64_t next_ticket = 1;
    uint64_t budget = 0, in_use = 0;
    hcc_server_stats stats{};
    uint64_t wakeups = 0;  // bumped by submissions, completions and stop
    bool stop = false;
    std::thread worker;
};

namespace {

uint64_t key_size(uint32_t key_bits) { return key_bits > 32 ? 8 : 4; }

// Pool bytes of one request (each allocation rounded up to 512 bytes).
uint64_t request_bytes(const hcc_server *s, uint64_t n) {
    auto r = [](uint64_t b) { return (b + 511) & ~uint64_t(511); };
    uint64_t b = r(n * 32) + r(n * sizeof(hcc_hit));
    if (s->method != HCC_METHOD_NOSORT)
        b += r(n * key_size(s->key_bits)) + r(n * 4) + r(hcc::sort_scratch_bytes(n, s->key_bits));
    return b;
}

// Runs on a CUDA callback thread once a request's stream has passed its last
// copy; makes no CUDA call.
void CUDART_CB on_request_done(void *p) {
    Slot *sl = static_cast<Slot *>(p);
    hcc_server *s = sl->owner;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        ++s->wakeups;
    }
    s->cv_work.notify_one();
}

// Queues a request's whole life on its slot's stream.  Runs on the
// dispatcher without the lock (a copy from pageable memory may block).
hcc_status launch_request(hcc_server *s, const Request &r, Slot &sl) {
    cudaStream_t st = sl.stream;
    const uint64_t n = r.n;
    const bool sorts = s->method != HCC_METHOD_NOSORT;
    void *d_rays = nullptr, *d_hits = nullptr, *d_keys = nullptr, *d_perm = nullptr, *d_scratch = nullptr;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, s->pool, st);
    };
    alloc(&d_rays, n * 32);
    alloc(&d_hits, n * sizeof(hcc_hit));
    if (sorts) {
        alloc(&d_keys, n * key_size(s->key_bits));
        alloc(&d_perm, n * 4);
        alloc(&d_scratch, hcc::sort_scratch_bytes(n, s->key_bits));
    }
    float4 *org = static_cast<float4 *>(d_rays);
    float4 *dir = org + n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(org, r.org, n * 16, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dir, r.dir, n * 16, cudaMemcpyHostToDevice, st);
    const hcc::SceneDesc &sc = s->scenes[r.scene];
    hcc::TraceArgs a;
    a.nodes = sc.nodes;
    a.layout = s->layout;
    a.tris = sc.tris;
    a.root_ref = sc.root_ref;
    a.org = org;
    a.dir = dir;
    a.n = n;
    a.hits = static_cast<int4 *>(d_hits);
    a.err = sl.d_err;
    // closest hit: persistent trace with ray replacement; any hit: one thread per ray
    a.work = r.any_hit ? nullptr : reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(sl.d_err) + 8);
    if (e == cudaSuccess && sorts) {
        uint32_t *perm = static_cast<uint32_t *>(d_perm);
        switch (s->method) {
        case HCC_METHOD_HCC:
            e = hcc::launch_encode_hcc(st, org, dir, n, 1, s->cut_boxes[r.scene],
                                       std::min(s->cut_used[r.scene], s->key_bits), s->key_bits, d_keys);
            break;
        case HCC_METHOD_TWOPOINT:
            e = hcc::launch_encode_twopoint(st, org, dir, n, 1, sc.lo, sc.ext, sc.L, s->key_bits, d_keys);
            break;
        case HCC_METHOD_ORIGIN:
            e = hcc::launch_encode_origin(st, org, n, 1, sc.lo, sc.ext, s->key_bits, d_keys);
            break;
        default:
            e = hcc::launch_encode_origin_dir(st, org, dir, n, 1, sc.lo, sc.ext, s->key_bits, d_keys);
            break;
        }
        if (e == cudaSuccess) e = hcc::launch_sort(st, d_keys, s->key_bits, n, perm, d_scratch, sl.d_err);
        a.gather = perm;  // trace fetches ray perm[j] and writes its hit back to perm[j]
        a.scatter = perm;
    }
    if (e == cudaSuccess) e = hcc::launch_trace(st, a, r.any_hit);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.hits, d_hits, n * sizeof(hcc_hit), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_err, sl.d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.d_err, 0, sizeof(uint32_t), st);
    for (void *p : {d_rays, d_hits, d_keys, d_perm, d_scratch})
        if (p) cudaFreeAsync(p, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
    if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_request_done, &sl);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(st);
        cudaMemset(sl.d_err, 0, sizeof(uint32_t));
        return e == cudaErrorMemoryAllocation ? HCC_ERR_OOM : HCC_ERR_CUDA;
    }
    return HCC_OK;
}

// Marks a request finished (lock held).
void finish(hcc_server *s, Request *r, hcc_status st) {
    r->status = st;
    r->finished = Clock::now();
    r->done = true;
    s->in_use -= r->bytes;
    if (st == HCC_OK) {
        ++s->stats.completed;
        s->stats.rays += r->n;
    } else {
        ++s->stats.failed;
    }
}

void dispatcher(hcc_server *s) {
    cudaSetDevice(s->device);
    std::vector<std::pair<Request *, Slot *>> admit;
    std::unique_lock<std::mutex> lock(s->mu);
    for (;;) {
        const uint64_t seen = s->wakeups;
        bool finished_any = false;
        for (Slot &sl : s->slots) {
            if (!sl.req || cudaEventQuery(sl.done) == cudaErrorNotReady) continue;
            const uint32_t err = *sl.h_err;
            hcc_status st = HCC_OK;
            if (err & hcc::ERR_STACK)
                st = HCC_ERR_STACK_OVERFLOW;
            else if (err & hcc::ERR_TIMEOUT)
                st = HCC_ERR_TIMEOUT;
            else if (err)
                st = HCC_ERR_INVALID_ARG;
            finish(s, sl.req, st);
            sl.req = nullptr;
            finished_any = true;
        }
        // Admit in arrival order: the head waits for memory rather than being overtaken.
        admit.clear();
        uint32_t running = 0;
        for (Slot &sl : s->slots) running += sl.req != nullptr;
        while (!s->queue.empty()) {
            Request *r = s->queue.front();
            if (running > 0 && s->in_use + r->bytes > s->budget) break;
            Slot *slot = nullptr;
            for (Slot &sl : s->slots)
                if (!sl.req) {
                    slot = &sl;
                    break;
                }
            if (!slot) break;
            s->queue.pop_front();
            s->in_use += r->bytes;
            s->stats.peak_bytes = std::max(s->stats.peak_bytes, s->in_use);
            slot->req = r;
            ++running;
            admit.emplace_back(r, slot);
        }
        s->stats.max_in_flight = std::max(s->stats.max_in_flight, running);
        if (!admit.empty()) {
            lock.unlock();
            std::vector<hcc_status> res(admit.size());
            for (size_t i = 0; i < admit.size(); ++i) {
                *admit[i].second->h_err = 0;
                res[i] = launch_request(s, *admit[i].first, *admit[i].second);
            }
            lock.lock();
            for (size_t i = 0; i < admit.size(); ++i)
                if (res[i] != HCC_OK) {
                    finish(s, admit[i].first, res[i]);
                    admit[i].second->req = nullptr;
                    finished_any = true;
                }
        }
        if (finished_any) s->cv_done.notify_all();
        running = 0;
        for (Slot &sl : s->slots) running += sl.req != nullptr;
        if (s->stop && running == 0 && s->queue.empty()) break;
        // Sleep until a submission, a completion callback or stop; the time
        // limit only bounds the wait should a callback never run.
        if (running > 0)
            s->cv_work.wait_for(lock, std::chrono::milliseconds(2), [&] { return s->wakeups != seen; });
        else if (s->queue.empty() && !s->stop)
            s->cv_work.wait(lock, [&] { return s->wakeups != seen; });
    }
}

}  // namespace

extern "C" {

hcc_status hcc_server_create(int device, uint32_t num_scenes, const hcc_bvh *const *bvhs, const hcc_cut *const *cuts,
                             const hcc_server_config *cfg, hcc_server **out) {
    if (!out) return HCC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!bvhs || !cfg || num_scenes == 0) return HCC_ERR_INVALID_ARG;
    if (cfg->slots == 0 || cfg->slots > 64) return HCC_ERR_INVALID_ARG;
    if (cfg->method != HCC_METHOD_NOSORT && cfg->method != HCC_METHOD_HCC && cfg->method != HCC_METHOD_TWOPOINT &&
        cfg->method != HCC_METHOD_ORIGIN && cfg->method != HCC_METHOD_ORIGIN_DIR)
        return HCC_ERR_INVALID_ARG;
    if (cfg->method != HCC_METHOD_NOSORT && (cfg->key_bits < 1 || cfg->key_bits > 64)) return HCC_ERR_INVALID_ARG;
    if (cfg->method == HCC_METHOD_HCC && !cuts) return HCC_ERR_INVALID_ARG;
    hcc_server *s = new (std::nothrow) hcc_server;
    if (!s) return HCC_ERR_OOM;
    s->device = device;
    s->method = cfg->method;
    s->key_bits = cfg->method == HCC_METHOD_NOSORT ? 32 : cfg->key_bits;
    s->scenes.resize(num_scenes);
    s->cut_boxes.assign(num_scenes, nullptr);
    s->cut_used.assign(num_scenes, 0);
    for (uint32_t k = 0; k < num_scenes; ++k) {
        int layout = 0, dev = 0;
        bool ok = bvhs[k] != nullptr;
        if (ok) {
            hcc::bvh_view(bvhs[k], &s->scenes[k], &layout, &dev);
            if (k == 0) s->layout = layout;
            ok = layout == s->layout && dev == device;
        }
        if (ok && cfg->method == HCC_METHOD_HCC) {
            ok = cuts[k] != nullptr;
            if (ok) {
                hcc::cut_view(cuts[k], &s->cut_boxes[k], &s->cut_used[k], &dev);
                ok = dev == device;
            }
        }
        if (!ok) {
            delete s;
            return HCC_ERR_INVALID_ARG;
        }
    }
    int prev = -1;
    cudaGetDevice(&prev);
    auto fail = [&](hcc_status st) {
        cudaGetLastError();
        hcc_server_destroy(s);
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    };
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return HCC_ERR_INVALID_ARG;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(HCC_ERR_CUDA);
    s->budget = cfg->hbm_budget ? cfg->hbm_budget : (uint64_t)(0.9 * (double)free_b);
    s->stats.budget = s->budget;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
        s->pool = nullptr;
        return fail(HCC_ERR_CUDA);
    }
    uint64_t keep = UINT64_MAX;  // released request buffers stay in the pool
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    s->slots.resize(cfg->slots);
    for (Slot &sl : s->slots) {
        sl.owner = s;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) sl.stream = nullptr;
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) sl.done = nullptr;
        if (cudaMalloc(&sl.d_err, 16) != cudaSuccess) sl.d_err = nullptr;
        if (cudaMallocHost(&sl.h_err, sizeof(uint32_t)) != cudaSuccess) sl.h_err = nullptr;
        if (!sl.stream || !sl.done || !sl.d_err || !sl.h_err) return fail(HCC_ERR_CUDA);
        if (cudaMemset(sl.d_err, 0, sizeof(uint32_t)) != cudaSuccess) return fail(HCC_ERR_CUDA);
        *sl.h_err = 0;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(HCC_ERR_CUDA);
    try {
        s->worker = std::thread(dispatcher, s);
    } catch (...) {
        return fail(HCC_ERR_OOM);
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = s;
    return HCC_OK;
}

hcc_status hcc_server_submit(hcc_server *s, uint32_t scene, const float *org_tmin, const float *dir_tmax, uint64_t n,
                             int any_hit, hcc_hit *hits, uint64_t *ticket) {
    if (!s || !ticket) return HCC_ERR_INVALID_ARG;
    *ticket = 0;
    if (scene >= s->scenes.size() || n == 0 || n > HCC_MAX_SORT_N) return HCC_ERR_INVALID_ARG;
    if (!org_tmin || !dir_tmax || !hits) return HCC_ERR_INVALID_ARG;
    const uint64_t bytes = request_bytes(s, n);
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) return HCC_ERR_INVALID_ARG;
    if (bytes > s->budget) return HCC_ERR_OOM;
    const uint64_t t = s->next_ticket++;
    Request &r = s->reqs[t];
    r.ticket = t;
    r.scene = scene;
    r.any_hit = any_hit ? 1 : 0;
    r.org = org_tmin;
    r.dir = dir_tmax;
    r.n = n;
    r.hits = hits;
    r.bytes = bytes;
    r.submitted = Clock::now();
    s->queue.push_back(&r);
    *ticket = t;
    ++s->wakeups;
    s->cv_work.notify_one();
    return HCC_OK;
}

hcc_status hcc_server_query(hcc_server *s, uint64_t ticket, int *done) {
    if (!s || !done) return HCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HCC_ERR_INVALID_ARG;
    *done = it->second.done ? 1 : 0;
    return HCC_OK;
}

hcc_status hcc_server_wait(hcc_server *s, uint64_t ticket, double *latency_ms) {
    if (!s) return HCC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HCC_ERR_INVALID_ARG;
    Request *r = &it->second;
    s->cv_done.wait(lock, [&] { return r->done; });
    const hcc_status st = r->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->finished - r->submitted).count();
    s->reqs.erase(it);
    return st;
}

hcc_status hcc_server_stats_get(hcc_server *s, hcc_server_stats *out) {
    if (!s || !out) return HCC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->queued = (uint32_t)s->queue.size();
    return HCC_OK;
}

hcc_status hcc_server_request_bytes(const hcc_server *s, uint64_t n, uint64_t *bytes) {
    if (!s || !bytes || n > HCC_MAX_SORT_N) return HCC_ERR_INVALID_ARG;
    *bytes = request_bytes(s, n);
    return HCC_OK;
}

hcc_status hcc_server_destroy(hcc_server *s) {
    if (!s) return HCC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        ++s->wakeups;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.d_err) cudaFree(sl.d_err);
        if (sl.h_err) cudaFreeHost(sl.h_err);
    }
    if (s->pool) cudaMemPoolDestroy(s->pool);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
    return HCC_OK;
}

}  // extern "C"

// Serving loop: filter requests as they arrive, with continuous batching.
//
// In the paper's read mapper integration the filter receives candidate pairs
// as the mapper produces them and returns one bit per pair (Sec. 3.6,
// Table 15).  Here requests (pairs of mixed lengths and thresholds) arrive at
// any time from any host thread, and a dispatcher thread admits them in
// arrival order by device memory:
//  - A worker is a batch object (one CUDA graph per run) with its own stream
//    and staging buffers, sized for a capacity class of 4096 x 2^k pairs.
//    A request runs on the smallest free worker that holds it; when there is
//    none, a worker of the request's class is made if its bytes fit in the
//    memory budget next to everything already held (idle workers are
//    released, least recently used first, to make room).  Otherwise the
//    request waits until a running one finishes.  So a request holds device
//    memory in proportion to its own size (at most about twice its need),
//    and the number of requests on the GPU at once follows from the budget.
//  - A request's round trip (copies in, the batch's graph, copies out) is
//    queued on its worker's stream, so requests admitted while others are
//    running overlap with them on the device.  Events around it give each
//    request's GPU start and end, so that the overlap can be measured.
//  - Reference texts (a reference genome, say) can be made resident once;
//    a request then sends only its reads and the offsets of its candidate
//    reference segments in that text.  Results can also stay in device
//    memory (the caller's buffers), for a consumer on the GPU.
// Host waits have deadlines and return SHOUJI_ETIMEOUT when they pass.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "shouji_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr size_t kMinClass = 4096;  // pairs of the smallest worker class

struct Request {
    uint64_t id = 0;
    shouji_server_request r;        // the caller's description
    Clock::time_point t_submit, t_done;
    double gpu_t0 = -1.0, gpu_t1 = -1.0;  // seconds since the server's base event
    shouji_status status = SHOUJI_OK;
    bool done = false;
};

struct Worker {
    size_t cap = 0;
    uint64_t bytes = 0;
    shouji_batch *batch = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr, t0 = nullptr, t1 = nullptr;
    uint8_t *reads = nullptr, *refs = nullptr;
    uint64_t *ref_off = nullptr;
    uint16_t *lens = nullptr;
    uint8_t *E = nullptr;
    uint32_t *accept = nullptr;
    uint8_t *count = nullptr;
    // pinned host staging of the results, for callers whose host buffers are
    // not pinned (a copy into pageable memory would block the dispatcher
    // until the request is done, and requests would no longer overlap)
    uint32_t *h_accept = nullptr;
    uint8_t *h_count = nullptr;
    bool staged = false;             // the running request's results go through them
    Request *req = nullptr;
    uint64_t last_use = 0;
};

struct Reference {
    uint8_t *text = nullptr;
    uint64_t bytes = 0;
};

}  // namespace

struct shouji_server {
    int device = 0;
    size_t max_req = 0;
    uint32_t max_m = 0;
    uint64_t max_stride = 0;
    int e_min = 0, e_max = 0, with_n = 0;
    std::string tune_cache;
    bool has_cache = false;
    int max_workers = 0;
    uint64_t budget = 0, used = 0, peak_used = 0, ref_bytes = 0;
    uint64_t admitted = 0, made = 0, released = 0, use_clock = 0;
    int busy = 0, peak_busy = 0;
    cudaEvent_t base = nullptr;
    std::vector<Worker *> workers;
    std::vector<Reference> refs;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> requests;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread dispatcher;
    bool stop = false;
    uint64_t next_id = 1;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

// Capacity of the class that holds n pairs: 4096 x 2^k, at most max_req.
size_t class_of(const shouji_server *sv, size_t n)
{
    size_t c = kMinClass;
    while (c < n)
        c <<= 1;
    return c < sv->max_req ? c : sv->max_req;
}

// Device bytes of a worker of capacity cap: its batch object and staging.
uint64_t worker_bytes(const shouji_server *sv, size_t cap)
{
    const uint64_t staging = 2 * (uint64_t)cap * sv->max_stride + sizeof(uint64_t) * cap +
                             sizeof(uint16_t) * cap + cap + (cap + 31) / 32 * sizeof(uint32_t) + cap;
    // (the pinned host staging of the results is host memory: not counted)
    return shouji_batch_device_bytes(cap, sv->max_m, sv->e_min, sv->e_max, sv->with_n) + staging;
}

void free_worker(Worker *w)
{
    if (w->batch)
        shouji_batch_destroy(w->batch);
    for (cudaEvent_t ev : {w->done, w->t0, w->t1})
        if (ev)
            cudaEventDestroy(ev);
    if (w->stream)
        cudaStreamDestroy(w->stream);
    cudaFree(w->reads);
    cudaFree(w->refs);
    cudaFree(w->ref_off);
    cudaFree(w->lens);
    cudaFree(w->E);
    cudaFree(w->accept);
    cudaFree(w->count);
    if (w->h_accept)
        cudaFreeHost(w->h_accept);
    if (w->h_count)
        cudaFreeHost(w->h_count);
    delete w;
}

// Whether host memory at p is pinned (page-locked or registered).
bool is_pinned(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// A worker for requests of up to cap pairs, or null when the device could
// not provide it.
Worker *make_worker(shouji_server *sv, size_t cap)
{
    Worker *w = new (std::nothrow) Worker;
    if (!w)
        return nullptr;
    w->cap = cap;
    w->bytes = worker_bytes(sv, cap);
    const shouji_status st = shouji_batch_create(cap, sv->max_m, sv->e_min, sv->e_max, sv->with_n,
                                                 sv->has_cache ? sv->tune_cache.c_str() : nullptr,
                                                 &w->batch);
    bool ok = st == SHOUJI_OK &&
              cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&w->t0) == cudaSuccess && cudaEventCreate(&w->t1) == cudaSuccess &&
              cudaMalloc(&w->reads, cap * sv->max_stride) == cudaSuccess &&
              cudaMalloc(&w->refs, cap * sv->max_stride) == cudaSuccess &&
              cudaMalloc(&w->ref_off, cap * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&w->lens, cap * sizeof(uint16_t)) == cudaSuccess &&
              cudaMalloc(&w->E, cap) == cudaSuccess &&
              cudaMalloc(&w->accept, (cap + 31) / 32 * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&w->count, cap) == cudaSuccess &&
              cudaMallocHost(&w->h_accept, (cap + 31) / 32 * sizeof(uint32_t)) == cudaSuccess &&
              cudaMallocHost(&w->h_count, cap) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_worker(w);
        return nullptr;
    }
    return w;
}

// Enqueue a request's whole round trip on its worker's stream.
shouji_status launch(shouji_server *sv, Worker &w, Request *q)
{
    const shouji_server_request &r = q->r;
    const bool dev_out = (r.flags & SHOUJI_SERVE_DEVICE_RESULTS) != 0;
    const bool at = r.refs == nullptr;
    cudaError_t e;
    const size_t in_bytes = r.n_pairs * r.stride;
#define TRY(x)                                   \
    do {                                         \
        if ((e = (x)) != cudaSuccess)            \
            return shouji::cuda_status(e);       \
    } while (0)
    TRY(cudaEventRecord(w.t0, w.stream));
    TRY(cudaMemcpyAsync(w.reads, r.reads, in_bytes, cudaMemcpyHostToDevice, w.stream));
    if (at)
        TRY(cudaMemcpyAsync(w.ref_off, r.ref_offsets, r.n_pairs * sizeof(uint64_t),
                            cudaMemcpyHostToDevice, w.stream));
    else
        TRY(cudaMemcpyAsync(w.refs, r.refs, in_bytes, cudaMemcpyHostToDevice, w.stream));
    TRY(cudaMemcpyAsync(w.lens, r.lens, r.n_pairs * sizeof(uint16_t), cudaMemcpyHostToDevice,
                        w.stream));
    TRY(cudaMemcpyAsync(w.E, r.E_per_pair, r.n_pairs, cudaMemcpyHostToDevice, w.stream));
    uint32_t *acc = dev_out ? r.accept : w.accept;
    uint8_t *cnt = dev_out ? r.count : (r.count ? w.count : nullptr);
    shouji_status st;
    if (at)
        st = shouji_batch_run_at(w.batch, w.reads, r.stride, sv->refs[r.ref_id].text, w.ref_off,
                                 w.lens, w.E, r.n_pairs, acc, cnt, w.stream);
    else
        st = shouji_batch_run(w.batch, w.reads, w.refs, r.stride, w.lens, w.E, r.n_pairs, acc,
                              cnt, w.stream);
    if (st)
        return st;
    w.staged = false;
    if (!dev_out) {
        w.staged = !is_pinned(r.accept) || (r.count && !is_pinned(r.count));
        TRY(cudaMemcpyAsync(w.staged ? w.h_accept : r.accept, w.accept,
                            (r.n_pairs + 31) / 32 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                            w.stream));
        if (r.count)
            TRY(cudaMemcpyAsync(w.staged ? w.h_count : r.count, w.count, r.n_pairs,
                                cudaMemcpyDeviceToHost, w.stream));
    }
    TRY(cudaEventRecord(w.t1, w.stream));
    TRY(cudaEventRecord(w.done, w.stream));
#undef TRY
    return SHOUJI_OK;
}

void finish(shouji_server *sv, Request *r, shouji_status st)
{
    r->status = st;
    r->t_done = Clock::now();
    r->done = true;
    sv->cv_done.notify_all();
}

void note_used(shouji_server *sv)
{
    if (sv->used > sv->peak_used)
        sv->peak_used = sv->used;
}

// A free worker for the queue's first request, made (releasing idle workers
// to make room) when none is free and the budget allows; null when the
// request must wait for a running one.  *fail is set when it can never run.
Worker *place(shouji_server *sv, Request *q, shouji_status *fail)
{
    const size_t n = q->r.n_pairs;
    Worker *best = nullptr;
    for (Worker *w : sv->workers)
        if (!w->req && w->cap >= n && (!best || w->cap < best->cap))
            best = w;
    const size_t cap = class_of(sv, n);
    if (best && best->cap <= 2 * cap)
        return best;
    const uint64_t need = worker_bytes(sv, cap);
    const bool fits = sv->used + need <= sv->budget && (int)sv->workers.size() < sv->max_workers;
    if (best && !fits)  // a larger free worker, rather than releasing others
        return best;
    // release idle workers, least recently used first, until the new one fits
    while (sv->used + need > sv->budget || (int)sv->workers.size() >= sv->max_workers) {
        Worker *lru = nullptr;
        size_t at = 0;
        for (size_t i = 0; i < sv->workers.size(); ++i) {
            Worker *w = sv->workers[i];
            if (!w->req && w != best && (!lru || w->last_use < lru->last_use)) {
                lru = w;
                at = i;
            }
        }
        if (!lru)
            break;
        sv->workers.erase(sv->workers.begin() + (long)at);
        sv->used -= lru->bytes;
        ++sv->released;
        free_worker(lru);
    }
    if (sv->used + need <= sv->budget && (int)sv->workers.size() < sv->max_workers) {
        Worker *w = make_worker(sv, cap);
        if (w) {
            sv->workers.push_back(w);
            sv->used += w->bytes;
            ++sv->made;
            note_used(sv);
            return w;
        }
    }
    if (best)  // a larger free worker, rather than waiting
        return best;
    if (sv->busy == 0)  // nothing will free up: the request cannot run
        *fail = SHOUJI_ENOMEM;
    return nullptr;
}

void dispatch_loop(shouji_server *sv)
{
    DeviceGuard g(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // completions
        for (Worker *w : sv->workers) {
            if (!w->req)
                continue;
            const cudaError_t q = cudaEventQuery(w->done);
            if (q == cudaErrorNotReady)
                continue;
            float a = 0.f, b = 0.f;
            if (q == cudaSuccess && cudaEventElapsedTime(&a, sv->base, w->t0) == cudaSuccess &&
                cudaEventElapsedTime(&b, sv->base, w->t1) == cudaSuccess) {
                w->req->gpu_t0 = a * 1e-3;
                w->req->gpu_t1 = b * 1e-3;
            }
            if (q == cudaSuccess && w->staged) {
                const shouji_server_request &r = w->req->r;
                memcpy(r.accept, w->h_accept, (r.n_pairs + 31) / 32 * sizeof(uint32_t));
                if (r.count)
                    memcpy(r.count, w->h_count, r.n_pairs);
            }
            finish(sv, w->req, q == cudaSuccess ? SHOUJI_OK : shouji::cuda_status(q));
            w->req = nullptr;
            --sv->busy;
        }
        // admissions, in arrival order, while memory and workers allow
        while (!sv->queue.empty()) {
            Request *q = sv->queue.front();
            shouji_status fail = SHOUJI_OK;
            Worker *w = place(sv, q, &fail);
            if (!w) {
                if (fail) {
                    sv->queue.pop_front();
                    finish(sv, q, fail);
                    continue;
                }
                break;
            }
            sv->queue.pop_front();
            const shouji_status st = launch(sv, *w, q);
            if (st) {
                cudaStreamSynchronize(w->stream);
                finish(sv, q, st);
                continue;
            }
            w->req = q;
            w->last_use = ++sv->use_clock;
            ++sv->admitted;
            if (++sv->busy > sv->peak_busy)
                sv->peak_busy = sv->busy;
        }
        if (sv->stop && sv->busy == 0 && sv->queue.empty())
            return;
        if (sv->busy == 0 && sv->queue.empty()) {
            sv->cv_work.wait(lk);
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

shouji_status check_request(const shouji_server *sv, const shouji_server_request &r)
{
    if (r.n_pairs == 0 || r.n_pairs > sv->max_req || r.stride == 0 || r.stride > sv->max_stride ||
        !r.reads || !r.lens || !r.E_per_pair || !r.accept)
        return SHOUJI_EINVAL;
    if (r.flags & ~SHOUJI_SERVE_DEVICE_RESULTS)
        return SHOUJI_EINVAL;
    if (!r.refs) {
        if (!r.ref_offsets || r.ref_id >= sv->refs.size())
            return SHOUJI_EINVAL;
        // every segment read must lie inside the resident text (lengths past
        // max_m are rejected by the batch without being read)
        const uint64_t size = sv->refs[r.ref_id].bytes;
        for (size_t i = 0; i < r.n_pairs; ++i) {
            const uint64_t len = r.lens[i] < sv->max_m ? r.lens[i] : sv->max_m;
            if (r.ref_offsets[i] > size || size - r.ref_offsets[i] < len)
                return SHOUJI_EINVAL;
        }
    }
    return SHOUJI_OK;
}

}  // namespace

extern "C" {

shouji_status shouji_server_create(size_t max_request_pairs, uint32_t max_m, uint64_t max_stride,
                                   int e_min, int e_max, int with_n, size_t memory_budget,
                                   int max_slots, const char *tune_cache, shouji_server **out)
{
    if (!out || max_request_pairs == 0 || max_request_pairs >= ((size_t)1 << 31) ||
        max_stride < max_m || max_slots < 1 || max_m < 1 || max_m > SHOUJI_MAX_M || e_min < 0 ||
        e_max > SHOUJI_MAX_E || e_min > e_max)
        return SHOUJI_EINVAL;
    *out = nullptr;
    shouji_server *sv = new (std::nothrow) shouji_server;
    if (!sv)
        return SHOUJI_ENOMEM;
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e) {
        delete sv;
        return shouji::cuda_status(e);
    }
    sv->max_req = max_request_pairs;
    sv->max_m = max_m;
    sv->max_stride = max_stride;
    sv->e_min = e_min;
    sv->e_max = e_max;
    sv->with_n = with_n ? 1 : 0;
    sv->has_cache = tune_cache != nullptr;
    if (tune_cache)
        sv->tune_cache = tune_cache;
    sv->max_workers = max_slots;
    sv->budget = memory_budget;
    // every admissible request must be able to run alone
    if (worker_bytes(sv, class_of(sv, max_request_pairs)) > memory_budget) {
        delete sv;
        return SHOUJI_ENOMEM;
    }
    if ((e = cudaEventCreate(&sv->base)) || (e = cudaEventRecord(sv->base, 0)) ||
        (e = cudaEventSynchronize(sv->base))) {
        if (sv->base)
            cudaEventDestroy(sv->base);
        delete sv;
        return shouji::cuda_status(e);
    }
    sv->dispatcher = std::thread(dispatch_loop, sv);
    *out = sv;
    return SHOUJI_OK;
}

shouji_status shouji_server_info(shouji_server *sv, int *slots, uint64_t *bytes_per_slot)
{
    if (!sv)
        return SHOUJI_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (slots)
        *slots = (int)sv->workers.size();
    if (bytes_per_slot)
        *bytes_per_slot = worker_bytes(sv, class_of(sv, sv->max_req));
    return SHOUJI_OK;
}

shouji_status shouji_server_stats_read(shouji_server *sv, shouji_server_stats *out)
{
    if (!sv || !out)
        return SHOUJI_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    out->budget_bytes = sv->budget;
    out->used_bytes = sv->used;
    out->peak_used_bytes = sv->peak_used;
    out->reference_bytes = sv->ref_bytes;
    out->workers = (int)sv->workers.size();
    out->busy_workers = sv->busy;
    out->peak_busy_workers = sv->peak_busy;
    out->queued = (int)sv->queue.size();
    out->admitted = sv->admitted;
    out->workers_made = sv->made;
    out->workers_released = sv->released;
    return SHOUJI_OK;
}

shouji_status shouji_server_add_reference(shouji_server *sv, const uint8_t *text, uint64_t bytes,
                                          uint32_t *ref_id)
{
    if (!sv || !text || bytes == 0 || !ref_id)
        return SHOUJI_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    // the reference must leave room for one worker of the largest class
    if (sv->ref_bytes + bytes + worker_bytes(sv, class_of(sv, sv->max_req)) > sv->budget)
        return SHOUJI_ENOMEM;
    // make room among idle workers if the budget is taken
    while (sv->used + bytes > sv->budget) {
        Worker *lru = nullptr;
        size_t at = 0;
        for (size_t i = 0; i < sv->workers.size(); ++i)
            if (!sv->workers[i]->req && (!lru || sv->workers[i]->last_use < lru->last_use)) {
                lru = sv->workers[i];
                at = i;
            }
        if (!lru)
            return SHOUJI_ENOMEM;
        sv->workers.erase(sv->workers.begin() + (long)at);
        sv->used -= lru->bytes;
        ++sv->released;
        free_worker(lru);
    }
    DeviceGuard g(sv->device);
    Reference ref;
    cudaError_t e = cudaMalloc(&ref.text, bytes);
    if (e) {
        cudaGetLastError();
        return SHOUJI_ENOMEM;
    }
    if ((e = cudaMemcpy(ref.text, text, bytes, cudaMemcpyHostToDevice))) {
        cudaFree(ref.text);
        return shouji::cuda_status(e);
    }
    ref.bytes = bytes;
    sv->refs.push_back(ref);
    sv->ref_bytes += bytes;
    sv->used += bytes;
    note_used(sv);
    *ref_id = (uint32_t)(sv->refs.size() - 1);
    return SHOUJI_OK;
}

shouji_status shouji_server_submit_request(shouji_server *sv, const shouji_server_request *req,
                                           uint64_t *request_id)
{
    if (!sv || !req || !request_id)
        return SHOUJI_EINVAL;
    Request *q = new (std::nothrow) Request;
    if (!q)
        return SHOUJI_ENOMEM;
    q->r = *req;
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const shouji_status st = check_request(sv, q->r);
        if (st || sv->stop) {
            delete q;
            return st ? st : SHOUJI_EINVAL;
        }
        q->id = sv->next_id++;
        sv->requests[q->id] = q;
        sv->queue.push_back(q);
    }
    sv->cv_work.notify_one();
    *request_id = q->id;
    return SHOUJI_OK;
}

shouji_status shouji_server_submit(shouji_server *sv, const uint8_t *reads, const uint8_t *refs,
                                   uint64_t stride, const uint16_t *lens,
                                   const uint8_t *E_per_pair, size_t n_pairs, uint32_t *accept,
                                   uint8_t *count, uint64_t *request_id)
{
    if (!refs)
        return SHOUJI_EINVAL;
    shouji_server_request r = {};
    r.reads = reads;
    r.refs = refs;
    r.stride = stride;
    r.lens = lens;
    r.E_per_pair = E_per_pair;
    r.n_pairs = n_pairs;
    r.accept = accept;
    r.count = count;
    return shouji_server_submit_request(sv, &r, request_id);
}

shouji_status shouji_server_wait_timed(shouji_server *sv, uint64_t request_id, double timeout_s,
                                       double *times)
{
    if (!sv)
        return SHOUJI_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->requests.find(request_id);
    if (it == sv->requests.end())
        return SHOUJI_EINVAL;
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    while (!r->done) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
            return SHOUJI_ETIMEOUT;
    }
    if (times) {
        times[0] = std::chrono::duration<double>(r->t_done - r->t_submit).count();
        times[1] = r->gpu_t0;
        times[2] = r->gpu_t1;
    }
    const shouji_status st = r->status;
    sv->requests.erase(it);
    delete r;
    return st;
}

shouji_status shouji_server_wait(shouji_server *sv, uint64_t request_id, double timeout_s,
                                 double *latency_s)
{
    double t[3] = {-1.0, -1.0, -1.0};
    const shouji_status st = shouji_server_wait_timed(sv, request_id, timeout_s, t);
    if (latency_s && t[0] >= 0)
        *latency_s = t[0];
    return st;
}

void shouji_server_destroy(shouji_server *sv)
{
    if (!sv)
        return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->dispatcher.joinable())
        sv->dispatcher.join();
    DeviceGuard g(sv->device);
    for (Worker *w : sv->workers)
        free_worker(w);
    for (Reference &r : sv->refs)
        cudaFree(r.text);
    if (sv->base)
        cudaEventDestroy(sv->base);
    for (auto &kv : sv->requests)
        delete kv.second;
    delete sv;
}

}  // extern "C"

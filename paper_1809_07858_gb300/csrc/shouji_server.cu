// Serving loop: filter requests as they arrive, with continuous batching.
//
// In the paper's read mapper integration the filter receives candidate pairs
// as the mapper produces them and returns one bit per pair (Sec. 3.6,
// Table 15).  Here requests (host buffers of pairs of mixed lengths and
// thresholds) arrive at any time from any host thread.  A dispatcher thread
// admits them in arrival order into slots: a slot is a batch object (one
// CUDA graph) with its own stream and device buffers, and the number of
// slots is bounded by the device-memory budget given at creation.  An
// admitted request is copied in, filtered and copied out on its slot's
// stream, so requests admitted while others are on the GPU run concurrently
// with them; when a slot's completion event fires, the request is finished
// and the slot takes the next queued request.  Host waits have deadlines and
// return SHOUJI_ETIMEOUT when they pass.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "shouji_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    const uint8_t *reads = nullptr, *refs = nullptr;
    uint64_t stride = 0;
    const uint16_t *lens = nullptr;
    const uint8_t *E = nullptr;
    size_t n = 0;
    uint32_t *accept = nullptr;
    uint8_t *count = nullptr;
    Clock::time_point t_submit, t_done;
    shouji_status status = SHOUJI_OK;
    bool done = false;
};

struct Slot {
    shouji_batch *batch = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *reads = nullptr, *refs = nullptr;
    uint16_t *lens = nullptr;
    uint8_t *E = nullptr;
    uint32_t *accept = nullptr;
    uint8_t *count = nullptr;
    Request *req = nullptr;
};

}  // namespace

struct shouji_server {
    int device = 0;
    size_t max_req = 0;
    uint64_t max_stride = 0;
    uint64_t bytes_per_slot = 0;
    std::vector<Slot> slots;
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

void free_slot(Slot &s)
{
    if (s.batch)
        shouji_batch_destroy(s.batch);
    if (s.stream)
        cudaStreamDestroy(s.stream);
    if (s.done)
        cudaEventDestroy(s.done);
    cudaFree(s.reads);
    cudaFree(s.refs);
    cudaFree(s.lens);
    cudaFree(s.E);
    cudaFree(s.accept);
    cudaFree(s.count);
    s = Slot();
}

shouji_status make_slot(shouji_server *sv, Slot &s, uint32_t max_m, int e_min, int e_max,
                        int with_n, const char *tune_cache)
{
    const size_t n = sv->max_req;
    shouji_status st = shouji_batch_create(n, max_m, e_min, e_max, with_n, tune_cache, &s.batch);
    if (st)
        return st;
    bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&s.reads, n * sv->max_stride) == cudaSuccess &&
              cudaMalloc(&s.refs, n * sv->max_stride) == cudaSuccess &&
              cudaMalloc(&s.lens, n * sizeof(uint16_t)) == cudaSuccess &&
              cudaMalloc(&s.E, n) == cudaSuccess &&
              cudaMalloc(&s.accept, (n + 31) / 32 * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&s.count, n) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_slot(s);
        return SHOUJI_ENOMEM;
    }
    return SHOUJI_OK;
}

// Enqueue a request's whole round trip on its slot's stream.
shouji_status launch(Slot &s, Request *r)
{
    cudaError_t e;
    const size_t in_bytes = r->n * r->stride;
#define TRY(x)                                   \
    do {                                         \
        if ((e = (x)) != cudaSuccess)            \
            return shouji::cuda_status(e);       \
    } while (0)
    TRY(cudaMemcpyAsync(s.reads, r->reads, in_bytes, cudaMemcpyHostToDevice, s.stream));
    TRY(cudaMemcpyAsync(s.refs, r->refs, in_bytes, cudaMemcpyHostToDevice, s.stream));
    TRY(cudaMemcpyAsync(s.lens, r->lens, r->n * sizeof(uint16_t), cudaMemcpyHostToDevice, s.stream));
    TRY(cudaMemcpyAsync(s.E, r->E, r->n, cudaMemcpyHostToDevice, s.stream));
    shouji_status st = shouji_batch_run(s.batch, s.reads, s.refs, r->stride, s.lens, s.E, r->n,
                                        s.accept, r->count ? s.count : nullptr, s.stream);
    if (st)
        return st;
    TRY(cudaMemcpyAsync(r->accept, s.accept, (r->n + 31) / 32 * sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, s.stream));
    if (r->count)
        TRY(cudaMemcpyAsync(r->count, s.count, r->n, cudaMemcpyDeviceToHost, s.stream));
    TRY(cudaEventRecord(s.done, s.stream));
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

void dispatch_loop(shouji_server *sv)
{
    DeviceGuard g(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool busy = false;
        // completions
        for (Slot &s : sv->slots) {
            if (!s.req)
                continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            finish(sv, s.req, q == cudaSuccess ? SHOUJI_OK : shouji::cuda_status(q));
            s.req = nullptr;
        }
        // admissions, in arrival order, while slots are free
        for (Slot &s : sv->slots) {
            if (s.req || sv->queue.empty())
                continue;
            Request *r = sv->queue.front();
            sv->queue.pop_front();
            const shouji_status st = launch(s, r);
            if (st) {
                cudaStreamSynchronize(s.stream);
                finish(sv, r, st);
            } else {
                s.req = r;
                busy = true;
            }
        }
        if (sv->stop && !busy && sv->queue.empty())
            return;
        if (!busy && sv->queue.empty()) {
            sv->cv_work.wait(lk);
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

shouji_status shouji_server_create(size_t max_request_pairs, uint32_t max_m, uint64_t max_stride,
                                   int e_min, int e_max, int with_n, size_t memory_budget,
                                   int max_slots, const char *tune_cache, shouji_server **out)
{
    if (!out || max_request_pairs == 0 || max_stride < max_m || max_slots < 1 ||
        max_m < 1 || max_m > SHOUJI_MAX_M || e_min < 0 || e_max > SHOUJI_MAX_E || e_min > e_max)
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
    sv->max_stride = max_stride;
    // The first slot measures what one slot costs; the budget decides how
    // many more are made.
    size_t free0 = 0, free1 = 0, total = 0;
    cudaMemGetInfo(&free0, &total);
    sv->slots.emplace_back();
    shouji_status st = make_slot(sv, sv->slots.back(), max_m, e_min, e_max, with_n, tune_cache);
    if (st) {
        sv->slots.clear();
        delete sv;
        return st;
    }
    cudaMemGetInfo(&free1, &total);
    sv->bytes_per_slot = free0 > free1 ? free0 - free1 : 1;
    if (sv->bytes_per_slot > memory_budget) {
        free_slot(sv->slots.back());
        delete sv;
        return SHOUJI_ENOMEM;
    }
    const size_t fit = memory_budget / sv->bytes_per_slot;
    const int want = (int)(fit < (size_t)max_slots ? fit : (size_t)max_slots);
    while ((int)sv->slots.size() < want) {
        sv->slots.emplace_back();
        if (make_slot(sv, sv->slots.back(), max_m, e_min, e_max, with_n, tune_cache)) {
            sv->slots.pop_back();
            break;
        }
    }
    sv->dispatcher = std::thread(dispatch_loop, sv);
    *out = sv;
    return SHOUJI_OK;
}

shouji_status shouji_server_info(shouji_server *sv, int *slots, uint64_t *bytes_per_slot)
{
    if (!sv)
        return SHOUJI_EINVAL;
    if (slots)
        *slots = (int)sv->slots.size();
    if (bytes_per_slot)
        *bytes_per_slot = sv->bytes_per_slot;
    return SHOUJI_OK;
}

shouji_status shouji_server_submit(shouji_server *sv, const uint8_t *reads, const uint8_t *refs,
                                   uint64_t stride, const uint16_t *lens,
                                   const uint8_t *E_per_pair, size_t n_pairs, uint32_t *accept,
                                   uint8_t *count, uint64_t *request_id)
{
    if (!sv || !request_id || n_pairs == 0 || n_pairs > sv->max_req || stride > sv->max_stride ||
        stride == 0 || !reads || !refs || !lens || !E_per_pair || !accept)
        return SHOUJI_EINVAL;
    Request *r = new (std::nothrow) Request;
    if (!r)
        return SHOUJI_ENOMEM;
    r->reads = reads;
    r->refs = refs;
    r->stride = stride;
    r->lens = lens;
    r->E = E_per_pair;
    r->n = n_pairs;
    r->accept = accept;
    r->count = count;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            return SHOUJI_EINVAL;
        }
        r->id = sv->next_id++;
        sv->requests[r->id] = r;
        sv->queue.push_back(r);
    }
    sv->cv_work.notify_one();
    *request_id = r->id;
    return SHOUJI_OK;
}

shouji_status shouji_server_wait(shouji_server *sv, uint64_t request_id, double timeout_s,
                                 double *latency_s)
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
    if (latency_s)
        *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    const shouji_status st = r->status;
    sv->requests.erase(it);
    delete r;
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
    for (Slot &s : sv->slots)
        free_slot(s);
    for (auto &kv : sv->requests)
        delete kv.second;
    delete sv;
}

}  // extern "C"

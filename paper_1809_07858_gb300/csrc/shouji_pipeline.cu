// Host pipeline: the whole filter for pairs held in host memory.
//
// The paper's accelerator streams pairs from the host over PCIe to its
// filtering units and returns one bit per pair in input order (Sec. 2.3,
// Sec. 3.3).  On a GB300 the link is NVLink-C2C to the Grace host; the
// pipeline cuts the batch into chunks and alternates two CUDA streams, so the
// host-to-device copy of one chunk overlaps the pack / filter / compaction of
// the previous one:
//   H2D reads, refs -> shouji_pack x2 -> shouji_filter -> D2H accept (+count)
//                                                     -> compaction (+indices)
// shouji_pipeline_run_packed takes pairs the caller already holds in the
// packed 2-bit layout (2 bits per base instead of 8), copies those words and
// filters them, so that it moves a quarter of the bytes over the host link.
// Survivor indices of successive chunks are appended to one device array in
// input order (the compaction of chunk k waits for that of chunk k-1 through
// an event, and carries the running total on the device), and copied back
// once at the end.  All device memory is allocated by shouji_pipeline_create.
#include <stdlib.h>
#include <string.h>

#include "shouji_internal.cuh"

struct shouji_pipeline {
    int device;
    uint32_t m;
    size_t chunk;      // pairs per chunk, multiple of 1024
    size_t max_pairs;  // capacity of the survivor index array
    int with_n;
    cudaStream_t st[2];
    cudaEvent_t ev_compact;
    uint8_t *d_reads[2], *d_refs[2];
    uint32_t *d_pr[2], *d_pt[2], *d_nr[2], *d_nt[2];
    uint32_t *d_acc[2];
    uint8_t *d_cnt[2];
    void *d_ws[2];
    uint32_t *d_idx;
    uint32_t *d_total;
    unsigned int *d_nflag;  // per stream: a pack without N masks read an 'N'

    uint32_t *h_total;  // pinned
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

void release(shouji_pipeline *p)
{
    if (!p)
        return;
    DeviceGuard g(p->device);
    for (int s = 0; s < 2; ++s) {
        cudaFree(p->d_reads[s]);
        cudaFree(p->d_refs[s]);
        cudaFree(p->d_pr[s]);
        cudaFree(p->d_pt[s]);
        cudaFree(p->d_nr[s]);
        cudaFree(p->d_nt[s]);
        cudaFree(p->d_acc[s]);
        cudaFree(p->d_cnt[s]);
        cudaFree(p->d_ws[s]);
        if (p->st[s])
            cudaStreamDestroy(p->st[s]);
    }
    cudaFree(p->d_idx);
    cudaFree(p->d_total);
    cudaFree(p->d_nflag);
    if (p->h_total)
        cudaFreeHost(p->h_total);
    if (p->ev_compact)
        cudaEventDestroy(p->ev_compact);
    free(p);
}

}  // namespace

using namespace shouji;

extern "C" {

shouji_status shouji_pipeline_create(uint32_t m, size_t chunk_pairs, size_t max_pairs,
                                     int with_n, shouji_pipeline **out)
{
    if (!out || m < 1 || m > SHOUJI_MAX_M || chunk_pairs == 0 ||
        max_pairs >= ((size_t)1 << 32))
        return SHOUJI_EINVAL;
    *out = nullptr;
    shouji_pipeline *p = (shouji_pipeline *)calloc(1, sizeof(shouji_pipeline));
    if (!p)
        return SHOUJI_ENOMEM;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        free(p);
        return cuda_status(e);
    }
    p->m = m;
    p->chunk = (chunk_pairs + kTile - 1) / kTile * kTile;
    p->max_pairs = max_pairs;
    p->with_n = with_n ? 1 : 0;
    const size_t ascii = p->chunk * m;
    const size_t packed = shouji_packed_words(p->chunk, m) * 4;
    const size_t nmask = shouji_nmask_words(p->chunk, m) * 4;
    const size_t words = groups_of(p->chunk) * 4;
    const size_t ws = compact_workspace_bytes(p->chunk);
    bool ok = true;
    for (int s = 0; s < 2 && ok; ++s) {
        ok = ok && cudaStreamCreateWithFlags(&p->st[s], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_reads[s], ascii) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_refs[s], ascii) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_pr[s], packed) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_pt[s], packed) == cudaSuccess;
        if (p->with_n) {
            ok = ok && cudaMalloc(&p->d_nr[s], nmask) == cudaSuccess;
            ok = ok && cudaMalloc(&p->d_nt[s], nmask) == cudaSuccess;
        }
        ok = ok && cudaMalloc(&p->d_acc[s], words) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_cnt[s], p->chunk) == cudaSuccess;
        ok = ok && cudaMalloc(&p->d_ws[s], ws) == cudaSuccess;
    }
    if (ok && max_pairs)
        ok = cudaMalloc(&p->d_idx, max_pairs * sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&p->d_total, sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaMalloc(&p->d_nflag, 2 * sizeof(unsigned int)) == cudaSuccess;
    ok = ok && cudaMallocHost(&p->h_total, sizeof(uint32_t)) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&p->ev_compact, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();  // clear the sticky-free allocation error
        release(p);
        return SHOUJI_ENOMEM;
    }
    *out = p;
    return SHOUJI_OK;
}

void shouji_pipeline_destroy(shouji_pipeline *p) { release(p); }

}  // extern "C"

namespace {

// Runs a batch chunk by chunk on the two streams.  stage(slot, base, nc, s,
// args) enqueues on stream s whatever puts the nc pairs from pair `base` on
// the device in the packed layout (the slot's buffers), and sets the
// filter's input pointers in args; the filter, the copies back and the
// compaction follow.  check_n: report an 'N' read without N masks.
template <class Stage>
shouji_status run_chunks(shouji_pipeline *p, size_t n_pairs, int E, uint32_t *accept,
                         uint8_t *count, uint32_t *idx, uint64_t *n_accepted, bool check_n,
                         Stage stage)
{
    if (n_pairs == 0) {
        if (n_accepted)
            *n_accepted = 0;
        return SHOUJI_OK;
    }
    if (idx && n_pairs > p->max_pairs)
        return SHOUJI_EINVAL;
    DeviceGuard g(p->device);
    const bool want_idx = idx != nullptr;
    cudaError_t e = cudaSuccess;
#define SHOUJI_TRY(x)                          \
    do {                                       \
        e = (x);                               \
        if (e != cudaSuccess)                  \
            return cuda_status(e);             \
    } while (0)
    if (want_idx) {
        SHOUJI_TRY(cudaMemsetAsync(p->d_total, 0, sizeof(uint32_t), p->st[0]));
        SHOUJI_TRY(cudaEventRecord(p->ev_compact, p->st[0]));
    }
    for (int k = 0; k < 2; ++k)
        SHOUJI_TRY(cudaMemsetAsync(p->d_nflag + k, 0, sizeof(unsigned int), p->st[k]));
    int slot = 0;
    for (size_t base = 0; base < n_pairs; base += p->chunk, slot ^= 1) {
        cudaStream_t s = p->st[slot];
        const size_t nc = (n_pairs - base < p->chunk) ? n_pairs - base : p->chunk;
        FilterArgs a;
        SHOUJI_TRY(stage(slot, base, nc, s, a));
        a.E_per_pair = nullptr;
        a.accept = p->d_acc[slot];
        a.count = count ? p->d_cnt[slot] : nullptr;
        a.vectors = nullptr;
        a.n_pairs = nc;
        a.m = (int)p->m;
        SHOUJI_TRY(launch_filter(a, E, s));
        SHOUJI_TRY(cudaMemcpyAsync(accept + base / 32, p->d_acc[slot], groups_of(nc) * 4,
                                   cudaMemcpyDeviceToHost, s));
        if (count)
            SHOUJI_TRY(cudaMemcpyAsync(count + base, p->d_cnt[slot], nc, cudaMemcpyDeviceToHost, s));
        if (want_idx) {
            SHOUJI_TRY(cudaStreamWaitEvent(s, p->ev_compact, 0));
            SHOUJI_TRY(launch_compact_append(p->d_acc[slot], nc, (uint32_t)base, p->d_idx,
                                             p->d_total, 1, p->d_ws[slot], s));
            SHOUJI_TRY(cudaEventRecord(p->ev_compact, s));
        }
    }
    SHOUJI_TRY(cudaStreamSynchronize(p->st[0]));
    SHOUJI_TRY(cudaStreamSynchronize(p->st[1]));
    uint64_t total = 0;
    if (want_idx) {
        SHOUJI_TRY(cudaMemcpyAsync(p->h_total, p->d_total, sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, p->st[0]));
        SHOUJI_TRY(cudaStreamSynchronize(p->st[0]));
        total = *p->h_total;
        if (total)
            SHOUJI_TRY(cudaMemcpyAsync(idx, p->d_idx, total * sizeof(uint32_t),
                                       cudaMemcpyDeviceToHost, p->st[0]));
        SHOUJI_TRY(cudaStreamSynchronize(p->st[0]));
    } else if (n_accepted) {
        const size_t words = groups_of(n_pairs);
        for (size_t w = 0; w < words; ++w)
            total += (uint64_t)__builtin_popcount(accept[w]);
    }
    unsigned int nflag[2] = {0, 0};
    if (check_n)
        SHOUJI_TRY(cudaMemcpy(nflag, p->d_nflag, sizeof nflag, cudaMemcpyDeviceToHost));
    const bool unmasked_n = nflag[0] || nflag[1];
#undef SHOUJI_TRY
    if (n_accepted)
        *n_accepted = total;
    // Results are complete either way; without N masks an 'N' was read as 'G'.
    return unmasked_n ? SHOUJI_EINVAL : SHOUJI_OK;
}

}  // namespace

extern "C" {

shouji_status shouji_pipeline_run(shouji_pipeline *p, const uint8_t *reads, const uint8_t *refs,
                                  uint64_t stride, size_t n_pairs, int E, uint32_t *accept,
                                  uint8_t *count, uint32_t *idx, uint64_t *n_accepted)
{
    if (!p || E < 0 || E > SHOUJI_MAX_E || stride < p->m)
        return SHOUJI_EINVAL;
    if (n_pairs && (!reads || !refs || !accept))
        return SHOUJI_EINVAL;
    const uint32_t m = p->m;
    auto stage = [&](int slot, size_t base, size_t nc, cudaStream_t s, FilterArgs &a) {
        cudaError_t e;
        if (stride == m) {
            e = cudaMemcpyAsync(p->d_reads[slot], reads + base * m, nc * m,
                                cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p->d_refs[slot], refs + base * m, nc * m,
                                    cudaMemcpyHostToDevice, s);
        } else {
            e = cudaMemcpy2DAsync(p->d_reads[slot], m, reads + base * stride, stride, m, nc,
                                  cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(p->d_refs[slot], m, refs + base * stride, stride, m, nc,
                                      cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess)
            e = launch_pack(p->d_reads[slot], m, nc, (int)m, p->d_pr[slot],
                            p->with_n ? p->d_nr[slot] : nullptr, s, p->d_nflag + slot);
        if (e == cudaSuccess)
            e = launch_pack(p->d_refs[slot], m, nc, (int)m, p->d_pt[slot],
                            p->with_n ? p->d_nt[slot] : nullptr, s, p->d_nflag + slot);
        a.reads = reinterpret_cast<const uint2 *>(p->d_pr[slot]);
        a.refs = reinterpret_cast<const uint2 *>(p->d_pt[slot]);
        a.reads_n = p->with_n ? p->d_nr[slot] : nullptr;
        a.refs_n = p->with_n ? p->d_nt[slot] : nullptr;
        return e;
    };
    return run_chunks(p, n_pairs, E, accept, count, idx, n_accepted, !p->with_n, stage);
}

shouji_status shouji_pipeline_run_packed(shouji_pipeline *p, const uint32_t *reads,
                                         const uint32_t *refs, const uint32_t *reads_n,
                                         const uint32_t *refs_n, size_t n_pairs, int E,
                                         uint32_t *accept, uint8_t *count, uint32_t *idx,
                                         uint64_t *n_accepted)
{
    if (!p || E < 0 || E > SHOUJI_MAX_E || (!reads_n) != (!refs_n) || (reads_n && !p->with_n))
        return SHOUJI_EINVAL;
    if (n_pairs && (!reads || !refs || !accept))
        return SHOUJI_EINVAL;
    const uint32_t m = p->m;
    const bool masks = reads_n != nullptr;
    auto stage = [&](int slot, size_t base, size_t nc, cudaStream_t s, FilterArgs &a) {
        // a chunk starts on a tile (the chunk size is a multiple of 1024), so
        // its packed words and masks are contiguous in the caller's arrays
        const size_t w0 = shouji_packed_words(base, m), wn = shouji_packed_words(nc, m);
        cudaError_t e = cudaMemcpyAsync(p->d_pr[slot], reads + w0, wn * 4,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->d_pt[slot], refs + w0, wn * 4, cudaMemcpyHostToDevice, s);
        if (masks) {
            const size_t n0 = shouji_nmask_words(base, m), nn = shouji_nmask_words(nc, m);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p->d_nr[slot], reads_n + n0, nn * 4,
                                    cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p->d_nt[slot], refs_n + n0, nn * 4,
                                    cudaMemcpyHostToDevice, s);
        }
        a.reads = reinterpret_cast<const uint2 *>(p->d_pr[slot]);
        a.refs = reinterpret_cast<const uint2 *>(p->d_pt[slot]);
        a.reads_n = masks ? p->d_nr[slot] : nullptr;
        a.refs_n = masks ? p->d_nt[slot] : nullptr;
        return e;
    };
    return run_chunks(p, n_pairs, E, accept, count, idx, n_accepted, false, stage);
}

}  // extern "C"

// The C ABI of libshouji.so (declared in include/shouji.h): argument checks,
// status codes and dispatch to the kernels.  Nothing here computes a result.
#include "shouji_internal.cuh"

namespace shouji {

static thread_local int g_last_cuda_error = 0;

shouji_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return SHOUJI_OK;
    g_last_cuda_error = (int)e;
    return SHOUJI_ECUDA;
}

cudaError_t take_unmasked_n(uint32_t *seen)
{
    *seen = 0;
    cudaError_t e = cudaDeviceSynchronize();
    uint32_t a = 0, b = 0, c = 0;
    if (e == cudaSuccess)
        e = take_pack_unmasked_n(&a);
    if (e == cudaSuccess)
        e = take_fused_unmasked_n(&b);
    if (e == cudaSuccess)
        e = take_batch_unmasked_n(&c);
    *seen = a | b | c;
    return e;
}

namespace {

using LaunchFn = cudaError_t (*)(const FilterArgs &, cudaStream_t);


constexpr LaunchFn kFilter[SHOUJI_MAX_E + 1] = {
    &launch_filter_E<0>,  &launch_filter_E<1>,  &launch_filter_E<2>,  &launch_filter_E<3>,
    &launch_filter_E<4>,  &launch_filter_E<5>,  &launch_filter_E<6>,  &launch_filter_E<7>,
    &launch_filter_E<8>,  &launch_filter_E<9>,  &launch_filter_E<10>, &launch_filter_E<11>,
    &launch_filter_E<12>, &launch_filter_E<13>, &launch_filter_E<14>, &launch_filter_E<15>,
    &launch_filter_E<16>, &launch_filter_E<17>, &launch_filter_E<18>, &launch_filter_E<19>,
    &launch_filter_E<20>, &launch_filter_E<21>, &launch_filter_E<22>, &launch_filter_E<23>,
    &launch_filter_E<24>, &launch_filter_E<25>, &launch_filter_E<26>, &launch_filter_E<27>,
    &launch_filter_E<28>, &launch_filter_E<29>, &launch_filter_E<30>, &launch_filter_E<31>,
};

}  // namespace

cudaError_t launch_filter(const FilterArgs &a, int E, cudaStream_t s)
{
    return kFilter[E](a, s);
}

}  // namespace shouji

using namespace shouji;

extern "C" {

const char *shouji_status_string(shouji_status s)
{
    switch (s) {
    case SHOUJI_OK: return "SHOUJI_OK";
    case SHOUJI_EINVAL: return "SHOUJI_EINVAL: invalid argument";
    case SHOUJI_ENOMEM: return "SHOUJI_ENOMEM: allocation failed";
    case SHOUJI_ECUDA: return "SHOUJI_ECUDA: CUDA call failed";
    case SHOUJI_ETIMEOUT: return "SHOUJI_ETIMEOUT: deadline passed";
    }
    return "SHOUJI: unknown status";
}

int shouji_last_cuda_error(void) { return g_last_cuda_error; }

size_t shouji_packed_words(size_t n, uint32_t m) { return tiles_of(n) * (size_t)m * 64; }

size_t shouji_nmask_words(size_t n, uint32_t m) { return tiles_of(n) * (size_t)m * 32; }

shouji_status shouji_pack(const uint8_t *seqs, uint64_t stride, size_t n, uint32_t m,
                          uint32_t *packed, uint32_t *nmask, void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || stride < m)
        return SHOUJI_EINVAL;
    if (n == 0)
        return SHOUJI_OK;
    if (!seqs || !packed)
        return SHOUJI_EINVAL;
    return cuda_status(launch_pack(seqs, stride, n, (int)m, packed, nmask, (cudaStream_t)stream));
}

shouji_status shouji_wait_failures(uint32_t *count)
{
    if (!count)
        return SHOUJI_EINVAL;
    return cuda_status(take_wait_failures(count));
}

shouji_status shouji_selftest_pack_wait(uint32_t *failures)
{
    if (!failures)
        return SHOUJI_EINVAL;
    return cuda_status(selftest_pack_wait(failures));
}

shouji_status shouji_unmasked_n(int *seen)
{
    if (!seen)
        return SHOUJI_EINVAL;
    uint32_t v = 0;
    const cudaError_t e = take_unmasked_n(&v);
    *seen = v ? 1 : 0;
    if (e != cudaSuccess)
        return cuda_status(e);
    return v ? SHOUJI_EINVAL : SHOUJI_OK;
}

shouji_status shouji_alu_probe(int op, double *lane_ops_per_sm_clock)
{
    if (!lane_ops_per_sm_clock || op < SHOUJI_PROBE_LOP3 || op > SHOUJI_PROBE_LOP3_IMAD)
        return SHOUJI_EINVAL;
    return cuda_status(alu_probe(op, lane_ops_per_sm_clock));
}

shouji_status shouji_filter(const uint32_t *reads, const uint32_t *refs,
                            const uint32_t *reads_nmask, const uint32_t *refs_nmask,
                            uint32_t m, size_t n_pairs, int E, const uint8_t *E_per_pair,
                            uint32_t *out_accept, uint8_t *out_count, uint32_t *out_vectors,
                            void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    if ((reads_nmask == nullptr) != (refs_nmask == nullptr))
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!reads || !refs || !out_accept)
        return SHOUJI_EINVAL;
    if ((uintptr_t)reads % 8 || (uintptr_t)refs % 8)
        return SHOUJI_EINVAL;
    FilterArgs a;
    a.reads = reinterpret_cast<const uint2 *>(reads);
    a.refs = reinterpret_cast<const uint2 *>(refs);
    a.reads_n = reads_nmask;
    a.refs_n = refs_nmask;
    a.E_per_pair = E_per_pair;
    a.accept = out_accept;
    a.count = out_count;
    a.vectors = out_vectors;
    a.n_pairs = n_pairs;
    a.m = (int)m;
    return cuda_status(launch_filter(a, E, (cudaStream_t)stream));
}

shouji_status shouji_pack_filter(const uint8_t *reads, const uint8_t *refs, uint64_t stride,
                                 size_t n_pairs, uint32_t m, int E, uint32_t *packed_reads,
                                 uint32_t *packed_refs, uint32_t *out_accept, uint8_t *out_count,
                                 void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || stride < m || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!reads || !refs || !packed_reads || !packed_refs || !out_accept)
        return SHOUJI_EINVAL;
    if ((uintptr_t)packed_reads % 8 || (uintptr_t)packed_refs % 8)
        return SHOUJI_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (stride == m && (uintptr_t)reads % 16 == 0 && (uintptr_t)refs % 16 == 0 &&
        pack_filter_fusable((int)m, E)) {
        const cudaError_t f = launch_pack_filter(reads, refs, n_pairs, (int)m, E, packed_reads,
                                                 packed_refs, out_accept, out_count, s);
        if (f != cudaErrorNotSupported)
            return cuda_status(f);
    }
    cudaError_t e = launch_pack(reads, stride, n_pairs, (int)m, packed_reads, nullptr, s);
    if (e == cudaSuccess)
        e = launch_pack(refs, stride, n_pairs, (int)m, packed_refs, nullptr, s);
    if (e != cudaSuccess)
        return cuda_status(e);
    FilterArgs a;
    a.reads = reinterpret_cast<const uint2 *>(packed_reads);
    a.refs = reinterpret_cast<const uint2 *>(packed_refs);
    a.reads_n = a.refs_n = nullptr;
    a.E_per_pair = nullptr;
    a.accept = out_accept;
    a.count = out_count;
    a.vectors = nullptr;
    a.n_pairs = n_pairs;
    a.m = (int)m;
    return cuda_status(launch_filter(a, E, s));
}

namespace {

// Whether shouji_pack_filter_results runs the fused kernel for these
// arguments, and the workspace bytes it needs: the per-CTA rings of both
// sides if so, else both full packed arrays for the separate launches.
cudaError_t results_plan(const uint8_t *reads, const uint8_t *refs, uint64_t stride,
                         size_t n_pairs, uint32_t m, int E, bool *fused, size_t *bytes)
{
    *fused = false;
    *bytes = 0;
    if (n_pairs == 0)
        return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (stride == m && reads && refs && (uintptr_t)reads % 16 == 0 && (uintptr_t)refs % 16 == 0)
        e = pack_filter_kernel_applies((int)m, E, fused);
    if (e != cudaSuccess)
        return e;
    if (*fused) {
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        *bytes = 2 * pack_filter_ring_words(n_pairs, (int)m, sms) * 4;
    } else {
        *bytes = 2 * shouji_packed_words(n_pairs, m) * 4;
    }
    return cudaSuccess;
}

}  // namespace

shouji_status shouji_pack_filter_workspace_size(const uint8_t *reads, const uint8_t *refs,
                                                uint64_t stride, size_t n_pairs, uint32_t m,
                                                int E, size_t *bytes)
{
    if (!bytes)
        return SHOUJI_EINVAL;
    *bytes = 0;
    if (m < 1 || m > SHOUJI_MAX_M || stride < m || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    bool fused = false;
    return cuda_status(results_plan(reads, refs, stride, n_pairs, m, E, &fused, bytes));
}

shouji_status shouji_pack_filter_results(const uint8_t *reads, const uint8_t *refs,
                                         uint64_t stride, size_t n_pairs, uint32_t m, int E,
                                         void *workspace, size_t workspace_bytes,
                                         uint32_t *out_accept, uint8_t *out_count, void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || stride < m || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!reads || !refs || !workspace || !out_accept || (uintptr_t)workspace % 16)
        return SHOUJI_EINVAL;
    bool fused = false;
    size_t need = 0;
    const cudaError_t e = results_plan(reads, refs, stride, n_pairs, m, E, &fused, &need);
    if (e != cudaSuccess)
        return cuda_status(e);
    if (workspace_bytes < need)
        return SHOUJI_EINVAL;
    uint32_t *side_r = static_cast<uint32_t *>(workspace);
    uint32_t *side_t = side_r + need / 8;   // the two halves of the workspace
    if (fused) {
        const cudaError_t f = launch_pack_filter(reads, refs, n_pairs, (int)m, E, side_r, side_t,
                                                 out_accept, out_count, (cudaStream_t)stream,
                                                 true);
        if (f != cudaErrorNotSupported)
            return cuda_status(f);
        return SHOUJI_ECUDA;  // the kernel applied a moment ago
    }
    return shouji_pack_filter(reads, refs, stride, n_pairs, m, E, side_r, side_t, out_accept,
                              out_count, stream);
}

shouji_status shouji_pack_filter_fused(const uint8_t *reads, const uint8_t *refs,
                                       uint64_t stride, uint32_t m, int E, int *fused)
{
    if (!fused)
        return SHOUJI_EINVAL;
    *fused = 0;
    if (m < 1 || m > SHOUJI_MAX_M || stride < m || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    if (stride != m || (uintptr_t)reads % 16 || (uintptr_t)refs % 16 || !reads || !refs)
        return SHOUJI_OK;
    bool applies = false;
    const shouji_status st = cuda_status(pack_filter_kernel_applies((int)m, E, &applies));
    *fused = applies ? 1 : 0;
    return st;
}

size_t shouji_compact_workspace_size(size_t n_pairs)
{
    return n_pairs ? compact_workspace_bytes(n_pairs) : 0;
}

shouji_status shouji_compact(const uint32_t *accept, size_t n_pairs, uint32_t *out_idx,
                             uint32_t *out_n, void *workspace, size_t workspace_bytes,
                             void *stream)
{
    if (n_pairs >= ((size_t)1 << 32))
        return SHOUJI_EINVAL;
    if (n_pairs == 0) {
        if (out_n)
            return cuda_status(cudaMemsetAsync(out_n, 0, sizeof(uint32_t), (cudaStream_t)stream));
        return SHOUJI_OK;
    }
    if (!accept || !out_idx || !out_n || !workspace)
        return SHOUJI_EINVAL;
    if (workspace_bytes < compact_workspace_bytes(n_pairs) || (uintptr_t)workspace % 16)
        return SHOUJI_EINVAL;
    return cuda_status(launch_compact(accept, n_pairs, out_idx, out_n, workspace,
                                      (cudaStream_t)stream));
}

}  // extern "C"

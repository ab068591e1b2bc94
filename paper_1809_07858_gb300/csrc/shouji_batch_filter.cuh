// Persistent filter of one threshold class of a bucketed batch: the per-group
// filter core of shouji_filter.cuh applied to every group of the buckets of
// one threshold E, with the packed base of each group looked up in the
// bucket tables.
#pragma once

#include "shouji_filter.cuh"
#include "shouji_batch.cuh"


namespace shouji {
namespace batch {

template <int E, int U, bool WITH_N>
__global__ void __launch_bounds__(filt::kThreads, filt::min_blocks<E>())
batch_filter_kernel(FilterParams p)
{
    const Tables *T = p.tables;
    const uint32_t G = T->ec_groups[E];
    if (G == 0)
        return;
    const uint32_t first = T->ec_first[E];
    const uint32_t nb = T->ec_count[E];
    // this threshold's buckets, cached in shared memory (at most 255)
    __shared__ uint32_t s_gstart[kMaxM], s_m[kMaxM], s_slot[kMaxM], s_rel0[kMaxM];
    __shared__ uint64_t s_poff[kMaxM];
    for (uint32_t i = threadIdx.x; i < nb; i += blockDim.x) {
        const uint32_t b = first + i, mc = T->bk_mc[b];
        s_gstart[i] = T->bk_gstart[b];
        s_m[i] = T->bk_m[b];
        s_slot[i] = T->bk_slot[b];
        s_rel0[i] = T->bk_slot[b] - T->mc_slot[mc];   // bucket start inside its m-class
        s_poff[i] = T->mc_poff[mc];
    }
    __syncthreads();
    // group g -> (m, first slot, packed base) of its bucket
    auto locate = [&](uint32_t g, int &m, uint32_t &slot0, size_t &base) {
        uint32_t lo = 0, hi = nb;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_gstart[mid] <= g)
                lo = mid;
            else
                hi = mid;
        }
        m = (int)s_m[lo];
        const uint32_t off = 32u * (g - s_gstart[lo]);
        slot0 = s_slot[lo] + off;
        const uint32_t rel = s_rel0[lo] + off;
        base = s_poff[lo] + (size_t)(rel / kTile) * m * kLanes + (rel % kTile) / 32;
    };
    auto run_group = [&](uint32_t g) {
        int m;
        uint32_t slot0;
        size_t base;
        locate(g, m, slot0, base);
        filt::View v;
        v.rd = p.preads + base;
        v.rf = p.prefs + base;
        v.rdn = WITH_N ? p.nreads + base : nullptr;
        v.rfn = WITH_N ? p.nrefs + base : nullptr;
        v.vec = nullptr;
        v.m = m;
        uint32_t inactive[E + 1];
#pragma unroll
        for (int j = 0; j <= E; ++j)
            inactive[j] = 0u;
        uint32_t C[8];
        filt::filter_group<E, U, WITH_N ? 1 : 0>(v, inactive, C);
        uint32_t cw[8];
        filt::counts_to_bytes(C, cw);
        uint4 *dst = reinterpret_cast<uint4 *>(p.count_slot + slot0);
        dst[0] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
        dst[1] = make_uint4(cw[4], cw[5], cw[6], cw[7]);
    };
    if (p.schedule == 2) {
        __shared__ uint32_t s_base;
        for (;;) {
            if (threadIdx.x == 0)
                s_base = atomicAdd(&p.work[E], blockDim.x);
            __syncthreads();
            const uint32_t base = s_base;
            __syncthreads();
            if (base >= G)
                break;
            if (base + threadIdx.x < G)
                run_group(base + threadIdx.x);
        }
        return;
    }
    uint32_t g, gend, gstep;
    if (p.schedule == 0) {
        g = blockIdx.x * blockDim.x + threadIdx.x;
        gstep = gridDim.x * blockDim.x;
        gend = G;
    } else {
        // a contiguous, block-aligned range of groups per CTA
        const uint32_t per = (G + gridDim.x - 1) / gridDim.x;
        const uint32_t per_r = (per + blockDim.x - 1) / blockDim.x * blockDim.x;
        g = blockIdx.x * per_r + threadIdx.x;
        gend = min(G, (blockIdx.x + 1) * per_r);
        gstep = blockDim.x;
    }
    for (; g < gend; g += gstep)
        run_group(g);
}

template <int E>
cudaError_t launch_filter_E(const FilterParams &p, int threads, int ctas, cudaStream_t s)
{
    if constexpr (E <= kMaxE8) {
        if (p.u == 8) {
            if (p.nreads)
                batch_filter_kernel<E, 8, true><<<ctas, threads, 0, s>>>(p);
            else
                batch_filter_kernel<E, 8, false><<<ctas, threads, 0, s>>>(p);
            return cudaGetLastError();
        }
    }
    if (p.nreads)
        batch_filter_kernel<E, SHOUJI_FILTER_U, true><<<ctas, threads, 0, s>>>(p);
    else
        batch_filter_kernel<E, SHOUJI_FILTER_U, false><<<ctas, threads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace batch
}  // namespace shouji

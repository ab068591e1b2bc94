// shouji_alu_probe: issue rate of the integer instructions the filter and
// the pack are built from, in lane-operations per SM clock.
//
// The roofline of the bit-sliced filter is set by the integer pipes, not by
// a vendor figure: the peak that the filter's algorithmic lane-ops are
// divided by is the rate measured here (LOP3) times the SM count and the
// maximum SM clock.  Each thread of one 1024-thread CTA per SM runs 8
// independent dependency chains of one instruction kind; the CTA counts its
// own SM cycles with clock64 around the loop, so the rate does not depend on
// the clock the GPU happens to run at.  Each chain step takes operands that
// no other step of the chain uses, so the compiler cannot merge two logic
// steps into one LOP3 or fold the chain.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

template <int OP>
__device__ __forceinline__ uint32_t step(uint32_t x, uint32_t p, uint32_t q)
{
    uint32_t y;
    if constexpr (OP == SHOUJI_PROBE_LOP3) {
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(y) : "r"(x), "r"(p), "r"(q));
    } else if constexpr (OP == SHOUJI_PROBE_SHF) {
        asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(y) : "r"(x), "r"(p), "r"(q));
    } else if constexpr (OP == SHOUJI_PROBE_PRMT) {
        asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(y) : "r"(x), "r"(p), "r"(q));
    } else if constexpr (OP == SHOUJI_PROBE_IADD3) {
        asm volatile("add.u32 %0, %1, %2;\n\tadd.u32 %0, %0, %3;" : "=r"(y) : "r"(x), "r"(p), "r"(q));
    } else if constexpr (OP == SHOUJI_PROBE_IMAD) {
        asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(y) : "r"(x), "r"(p), "r"(q));
    } else {
        asm volatile("popc.b32 %0, %1;" : "=r"(y) : "r"(x));
    }
    return y;
}

// Chains 0..3 use OP_A and 4..7 use OP_B (the same kind for a plain probe).
template <int OP_A, int OP_B>
__global__ void __launch_bounds__(kProbeThreads, 1)
probe_kernel(uint32_t seed, int iters, uint32_t *sink, unsigned long long *cycles)
{
    uint32_t x[kChains], p[kChains][2], q[kChains][2];
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
        x[i] = seed * (2u * threadIdx.x + 1u) + 0x9E3779B9u * (uint32_t)i;
        p[i][0] = (seed ^ (0x85EBCA6Bu * (uint32_t)(i + 1))) | 1u;
        p[i][1] = (seed ^ (0xC2B2AE35u * (uint32_t)(i + 3))) | 1u;
        q[i][0] = seed + 0x27D4EB2Fu * (uint32_t)(i + 5);
        q[i][1] = seed + 0x165667B1u * (uint32_t)(i + 7);
    }
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) {
                if (i < kChains / 2)
                    x[i] = step<OP_A>(x[i], p[i][u & 1], q[i][u & 1]);
                else
                    x[i] = step<OP_B>(x[i], p[i][u & 1], q[i][u & 1]);
            }
        }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i)
        acc ^= x[i];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

template <int A, int B>
cudaError_t run_probe(int sms, int iters, uint32_t *sink, unsigned long long *cycles)
{
    probe_kernel<A, B><<<sms, kProbeThreads>>>(0x2545F491u, iters, sink, cycles);
    return cudaGetLastError();
}

}  // namespace

cudaError_t alu_probe(int op, double *rate)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    uint32_t *sink = nullptr;
    unsigned long long *cycles = nullptr;
    if ((e = cudaMalloc(&sink, (size_t)sms * kProbeThreads * sizeof(uint32_t))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&cycles, (size_t)sms * sizeof(unsigned long long))) != cudaSuccess) {
        cudaFree(sink);
        return e;
    }
    const int iters = 2048;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
        switch (op) {
        case SHOUJI_PROBE_LOP3: e = run_probe<SHOUJI_PROBE_LOP3, SHOUJI_PROBE_LOP3>(sms, iters, sink, cycles); break;
        case SHOUJI_PROBE_SHF: e = run_probe<SHOUJI_PROBE_SHF, SHOUJI_PROBE_SHF>(sms, iters, sink, cycles); break;
        case SHOUJI_PROBE_PRMT: e = run_probe<SHOUJI_PROBE_PRMT, SHOUJI_PROBE_PRMT>(sms, iters, sink, cycles); break;
        case SHOUJI_PROBE_IADD3: e = run_probe<SHOUJI_PROBE_IADD3, SHOUJI_PROBE_IADD3>(sms, iters, sink, cycles); break;
        case SHOUJI_PROBE_IMAD: e = run_probe<SHOUJI_PROBE_IMAD, SHOUJI_PROBE_IMAD>(sms, iters, sink, cycles); break;
        case SHOUJI_PROBE_POPC: e = run_probe<SHOUJI_PROBE_POPC, SHOUJI_PROBE_POPC>(sms, iters, sink, cycles); break;
        default: e = run_probe<SHOUJI_PROBE_LOP3, SHOUJI_PROBE_IMAD>(sms, iters, sink, cycles); break;
        }
        if (e == cudaSuccess)
            e = cudaDeviceSynchronize();
    }
    unsigned long long *h = nullptr;
    if (e == cudaSuccess) {
        h = new unsigned long long[sms];
        e = cudaMemcpy(h, cycles, (size_t)sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) {
        // median over the SMs of lane-ops per cycle
        double *r = new double[sms];
        const double ops = (double)kProbeThreads * kChains * kUnroll * iters;
        for (int i = 0; i < sms; ++i)
            r[i] = h[i] ? ops / (double)h[i] : 0.0;
        for (int i = 1; i < sms; ++i)
            for (int j = i; j > 0 && r[j - 1] > r[j]; --j) {
                const double t = r[j];
                r[j] = r[j - 1];
                r[j - 1] = t;
            }
        *rate = r[sms / 2];
        delete[] r;
    }
    delete[] h;
    cudaFree(sink);
    cudaFree(cycles);
    return e;
}

}  // namespace shouji

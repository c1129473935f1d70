// probe.cu -- memory-operation rate probes used as roofline denominators.
#include <stdint.h>

#include "asyrk_probe.h"
#include "common.cuh"

namespace asyrk {

// cheap per-thread generator for probe addresses (xorshift32)
__device__ __forceinline__ unsigned xs32(unsigned &s)
{
    s ^= s << 13;
    s ^= s >> 17;
    s ^= s << 5;
    return s;
}

// Each thread issues P independent operations per loop trip so that the probe
// is limited by the memory system, not by the latency of one thread's chain.
constexpr int P = 8;

template <int KIND>
__global__ void __launch_bounds__(256) k_probe(float *a, unsigned n, long long ops, float *sink)
{
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned s = 0x9E3779B9u ^ (unsigned)(tid * 2654435761ull) ^ 0x85EBCA6Bu;
    if (s == 0) s = 1;
    float acc = 0.f;
    if (KIND == ASYRK_PROBE_STREAM) {
        const float4 *v = reinterpret_cast<const float4 *>(a);
        const long long n4 = ops / 4;
        for (long long k = tid; k < n4; k += nth) {
            const float4 t = __ldcs(v + k);
            acc += t.x + t.y + t.z + t.w;
        }
    } else {
        // ops counts single operations (pairs for GATHER_RED)
        for (long long k = tid * P; k < ops; k += nth * P) {
            unsigned idx[P];
#pragma unroll
            for (int q = 0; q < P; ++q) idx[q] = __umulhi(xs32(s), n);
            if (KIND == ASYRK_PROBE_RED_F32) {
#pragma unroll
                for (int q = 0; q < P; ++q)
                    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(a + idx[q]),
                                 "f"(1e-30f)
                                 : "memory");
            } else {
                float g[P];
#pragma unroll
                for (int q = 0; q < P; ++q) g[q] = __ldcg(a + idx[q]);
                float r = 0.f;
#pragma unroll
                for (int q = 0; q < P; ++q) r += g[q];
                if (KIND == ASYRK_PROBE_GATHER_F32) {
                    acc += r;
                } else {  // the projection's pattern: reduce, then update the same entries
                    const float sc = 1e-30f * r;
#pragma unroll
                    for (int q = 0; q < P; ++q)
                        asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(a + idx[q]),
                                     "f"(sc)
                                     : "memory");
                }
            }
        }
    }
    if (acc == 12345.678f) *sink = acc;  // keep the loads
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_probe(int kind, int64_t n, int64_t ops, float *ms)
{
    if (kind < 0 || kind > 3 || n < 1 || ops < 1 || !ms || n > 0xffffffffLL)
        return set_error(ASYRK_EINVAL, "bad probe arguments");
    if (kind == ASYRK_PROBE_STREAM && ops > n) return set_error(ASYRK_EINVAL, "ops > n");
    float *a = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    ASYRK_CK(cudaGetDevice(&dev));
    ASYRK_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ASYRK_CK(cudaMalloc((void **)&a, (size_t)n * sizeof(float)));
    cudaError_t e = cudaMalloc((void **)&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(a, 0, (size_t)n * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned grid = (unsigned)sms * 8;
    for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {  // first launch warms up
        e = cudaEventRecord(e0, 0);
        switch (kind) {
        case 0: k_probe<0><<<grid, 256>>>(a, (unsigned)n, ops, sink); break;
        case 1: k_probe<1><<<grid, 256>>>(a, (unsigned)n, ops, sink); break;
        case 2: k_probe<2><<<grid, 256>>>(a, (unsigned)n, ops, sink); break;
        default: k_probe<3><<<grid, 256>>>(a, (unsigned)n, ops, sink); break;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    }
    cudaFree(a);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "probe", __FILE__, __LINE__);
    return ASYRK_OK;
}

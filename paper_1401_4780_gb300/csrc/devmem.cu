// devmem.cu -- the per-device memory pool of problem handles (devmem.cuh).
#include <mutex>

#include "common.cuh"
#include "devmem.cuh"

namespace asyrk {

namespace {

constexpr int MAX_DEVICES = 64;
// memory the pool keeps after frees: 1/8 of the device's, at most 16 GiB
constexpr unsigned long long KEEP_MAX = 16ULL << 30;

std::mutex g_mu;
cudaMemPool_t g_pool[MAX_DEVICES];

int pool_for_current(cudaMemPool_t *out)
{
    int dev = 0;
    ASYRK_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(ASYRK_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        ASYRK_CK(cudaMemPoolCreate(&pool, &props));
        size_t free_b = 0, total_b = 0;
        unsigned long long keep = KEEP_MAX;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && total_b / 8 < keep) keep = total_b / 8;
        (void)cudaGetLastError();
        cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return cuda_fail(e, "cudaMemPoolSetAttribute", __FILE__, __LINE__);
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return ASYRK_OK;
}

}  // namespace

int devmem_alloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    int st = pool_for_current(&pool);
    if (st != ASYRK_OK) return st;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? ASYRK_ENOMEM : ASYRK_ECUDA,
                         "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return ASYRK_OK;
}

void devmem_free(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

}  // namespace asyrk

using namespace asyrk;

extern "C" int asyrk_trim_memory(void)
{
    int dev = 0;
    ASYRK_CK(cudaGetDevice(&dev));
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (dev >= 0 && dev < MAX_DEVICES) pool = g_pool[dev];
    }
    if (!pool) return ASYRK_OK;
    ASYRK_CK(cudaDeviceSynchronize());
    ASYRK_CK(cudaMemPoolTrimTo(pool, 0));
    return ASYRK_OK;
}

// partition.cu -- SM partitions through green contexts (driver API, reached
// through the runtime's entry-point query so that the library needs no link
// against the driver library).
#include <cuda.h>
#include <string.h>

#include "partition.cuh"

namespace asyrk {

namespace {

typedef CUresult (*GetDevResourceFn)(CUdevice, CUdevResource *, CUdevResourceType);
typedef CUresult (*SmSplitFn)(CUdevResource *, unsigned int *, const CUdevResource *,
                              CUdevResource *, unsigned int, unsigned int);
typedef CUresult (*GenerateDescFn)(CUdevResourceDesc *, CUdevResource *, unsigned int);
typedef CUresult (*GreenCtxCreateFn)(CUgreenCtx *, CUdevResourceDesc, CUdevice, unsigned int);
typedef CUresult (*GreenCtxStreamCreateFn)(CUstream *, CUgreenCtx, unsigned int, int);
typedef CUresult (*GreenCtxDestroyFn)(CUgreenCtx);

void *entry(const char *name)
{
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &f, 13000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return f;
}

}  // namespace

void sm_partition_destroy(SmPartition *p)
{
    if (!p) return;
    for (int g = 0; g < 2; ++g)
        if (p->stream[g]) cudaStreamDestroy(p->stream[g]);
    auto destroy = (GreenCtxDestroyFn)entry("cuGreenCtxDestroy");
    for (int g = 0; g < 2; ++g)
        if (p->ctx[g] && destroy) destroy((CUgreenCtx)p->ctx[g]);
    *p = SmPartition();
}

bool sm_partition_add_stream(const SmPartition &p, int g, cudaStream_t *s)
{
    *s = nullptr;
    auto screate = (GreenCtxStreamCreateFn)entry("cuGreenCtxStreamCreate");
    if (!screate || g < 0 || g > 1 || !p.ctx[g]) return false;
    CUstream cs = nullptr;
    if (screate(&cs, (CUgreenCtx)p.ctx[g], CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
        (void)cudaGetLastError();
        return false;
    }
    *s = (cudaStream_t)cs;
    return true;
}

bool sm_partition_create(int dev, int first, SmPartition *out)
{
    *out = SmPartition();
    auto get_res = (GetDevResourceFn)entry("cuDeviceGetDevResource");
    auto split = (SmSplitFn)entry("cuDevSmResourceSplitByCount");
    auto gen = (GenerateDescFn)entry("cuDevResourceGenerateDesc");
    auto create = (GreenCtxCreateFn)entry("cuGreenCtxCreate");
    auto screate = (GreenCtxStreamCreateFn)entry("cuGreenCtxStreamCreate");
    if (!get_res || !split || !gen || !create || !screate || first < 1) return false;
    CUdevResource all, grp, rest;
    memset(&all, 0, sizeof all);
    memset(&grp, 0, sizeof grp);
    memset(&rest, 0, sizeof rest);
    if (get_res((CUdevice)dev, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return false;
    unsigned groups = 1;
    if (split(&grp, &groups, &all, &rest, 0, (unsigned)first) != CUDA_SUCCESS || groups != 1 ||
        grp.sm.smCount == 0 || rest.sm.smCount == 0)
        return false;
    CUdevResourceDesc d0 = nullptr, d1 = nullptr;
    if (gen(&d0, &grp, 1) != CUDA_SUCCESS || gen(&d1, &rest, 1) != CUDA_SUCCESS) return false;
    SmPartition p;
    CUgreenCtx c0 = nullptr, c1 = nullptr;
    CUstream s0 = nullptr, s1 = nullptr;
    bool ok = create(&c0, d0, (CUdevice)dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS;
    p.ctx[0] = c0;
    ok = ok && create(&c1, d1, (CUdevice)dev, CU_GREEN_CTX_DEFAULT_STREAM) == CUDA_SUCCESS;
    p.ctx[1] = c1;
    // group 0's stream at the highest priority: where the groups share a
    // hardware queue, its launches go first
    int lo_prio = 0, hi_prio = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio) != cudaSuccess) {
        (void)cudaGetLastError();
        hi_prio = 0;
    }
    ok = ok && screate(&s0, c0, CU_STREAM_NON_BLOCKING, hi_prio) == CUDA_SUCCESS;
    p.stream[0] = (cudaStream_t)s0;
    ok = ok && screate(&s1, c1, CU_STREAM_NON_BLOCKING, 0) == CUDA_SUCCESS;
    p.stream[1] = (cudaStream_t)s1;
    if (!ok) {
        sm_partition_destroy(&p);
        (void)cudaGetLastError();
        return false;
    }
    p.sms[0] = (int)grp.sm.smCount;
    p.sms[1] = (int)rest.sm.smCount;
    *out = p;
    return true;
}

}  // namespace asyrk

// partition.cuh -- a split of the GPU's SMs into two disjoint groups, each
// with its own stream: kernels launched on a group's stream run on that
// group's SMs only (green contexts of the CUDA driver, which share the primary
// context's memory and differ from it only in the SMs they may use).
#pragma once

#include <cuda_runtime.h>

namespace asyrk {

struct SmPartition {
    void *ctx[2] = {nullptr, nullptr};            // CUgreenCtx of each group
    cudaStream_t stream[2] = {nullptr, nullptr};  // a non-blocking stream in each group
                                                  // (group 0's at the highest priority)
    int sms[2] = {0, 0};                          // SMs of each group
};

// Split the SMs of device `dev` so that group 0 gets at least `first` SMs
// (rounded up to the driver's granularity) and group 1 the rest.  Returns
// false, holding nothing, when the driver offers no such split (then the
// caller runs without one); errors of the driver are cleared.
bool sm_partition_create(int dev, int first, SmPartition *out);
// Another non-blocking stream in group g (the caller destroys it before the
// partition); false when the driver refuses.
bool sm_partition_add_stream(const SmPartition &p, int g, cudaStream_t *s);
void sm_partition_destroy(SmPartition *p);

}  // namespace asyrk

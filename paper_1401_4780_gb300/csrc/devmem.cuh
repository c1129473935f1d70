// devmem.cuh -- device memory of problem handles.
//
// Every problem's device arrays, its set-up temporaries and its solve
// workspace come from one stream-ordered memory pool per device.  The pool
// keeps what asyrk_destroy frees, up to a fixed share of the device's memory,
// so a problem created after another was destroyed reuses that memory instead
// of asking the driver again (a cudaMalloc of a large buffer costs about a
// millisecond, a cudaFree as much); asyrk_trim_memory hands it back.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace asyrk {

// bytes on the current device, ordered on stream s (usable by other streams
// once s has reached this point); ASYRK_OK, ENOMEM or ECUDA (with the message set)
int devmem_alloc(void **p, size_t bytes, cudaStream_t s);
// back to the pool, ordered on s: work on other streams that uses p must have
// finished (the callers synchronise the device first)
void devmem_free(void *p, cudaStream_t s);

template <typename T>
int devmem_alloc_n(T **p, size_t count, cudaStream_t s)
{
    return devmem_alloc(reinterpret_cast<void **>(p), (count ? count : 1) * sizeof(T), s);
}

}  // namespace asyrk

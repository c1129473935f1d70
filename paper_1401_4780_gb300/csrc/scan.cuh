// scan.cuh -- device-wide exclusive prefix sum of int64 (scan.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace asyrk {

// out[0..count) = exclusive prefix sum of in[0..count) (int64, exact); *total =
// the sum (a device address, written on the stream); tmp holds
// scan_tmp_count(count) entries.  in and out may not overlap.
int exclusive_scan(const int64_t *in, int64_t *out, int64_t count, int64_t *tmp, int64_t *total,
                   cudaStream_t s);
int64_t scan_tmp_count(int64_t count);

}  // namespace asyrk
